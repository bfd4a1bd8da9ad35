"""Definitional brute-force clusterizer for tiny modules (test infrastructure only).

A third statement of the three-threshold rule (arXiv 2101.11489, section 2), written
as a predicate over intervals rather than a left-to-right scan, so that it shares
no control flow with ``sst_oracle.c``:

  [l, r] is a candidate  <=>  l and r are active,
                              every two successive active strips in [l, r] are linked,
                              the active strip before l (if any) is not linked to l,
                              the active strip after r (if any) is not linked to r;
  a candidate is a cluster when it holds a seed and passes the cluster threshold.

Every interval of the module is tested, O(n^3) in pure Python: use it only on
modules of a handful of strips.  Binary32 arithmetic goes through numpy float32
scalars (one IEEE rounding per operation).
"""
from __future__ import annotations

import numpy as np

f32 = np.float32


def _active(adc, noise, bad, t):
    return (not bad) and f32(adc) > f32(f32(t) * f32(noise))


def _linked(a, b, bad, max_holes, max_bad):
    # Split the open gap (a, b) into maximal runs of equal bad-ness and bound each.
    gap = [bool(bad[t]) for t in range(a + 1, b)]
    i = 0
    while i < len(gap):
        j = i
        while j < len(gap) and gap[j] == gap[i]:
            j += 1
        run = j - i
        if gap[i] and run > max_bad:
            return False
        if (not gap[i]) and run > max_holes:
            return False
        i = j
    return True


def _corrected(adc, gain):
    if adc >= 254:
        return int(adc)
    c = int(f32(f32(adc) / f32(gain)) + f32(0.5))
    return 254 if c > 253 else c


def cluster_module(adc, noise, bad, gain, p) -> list[tuple[int, int, int, float]]:
    """Returns [(first, width, charge, barycenter)] in strip order."""
    n = len(adc)
    act = [_active(adc[i], noise[i], bad[i], p.t_channel) for i in range(n)]
    seed = [_active(adc[i], noise[i], bad[i], p.t_seed) for i in range(n)]
    actives = [i for i in range(n) if act[i]]

    def lk(a, b):
        return _linked(a, b, bad, p.max_seq_holes, p.max_seq_bad)

    out = []
    for l in range(n):
        for r in range(l, n):
            if not (act[l] and act[r]):
                continue
            inside = [i for i in actives if l <= i <= r]
            if not all(lk(inside[k], inside[k + 1]) for k in range(len(inside) - 1)):
                continue
            before = [i for i in actives if i < l]
            after = [i for i in actives if i > r]
            if before and lk(before[-1], l):
                continue
            if after and lk(r, after[0]):
                continue
            if not any(seed[i] for i in inside):
                continue
            s_raw = sum(int(adc[i]) for i in inside)
            n2 = f32(0.0)
            for i in inside:
                n2 = f32(n2 + f32(f32(noise[i]) * f32(noise[i])))
            if not (f32(s_raw) > f32(f32(p.t_cluster) * np.sqrt(n2, dtype=np.float32))):
                continue
            lo, hi = l, r
            k = 0
            while k < p.max_adj_bad and lo - 1 >= 0 and bad[lo - 1]:
                lo -= 1
                k += 1
            k = 0
            while k < p.max_adj_bad and hi + 1 < n and bad[hi + 1]:
                hi += 1
                k += 1
            qs = [_corrected(int(adc[i]), gain[i]) for i in inside]
            charge = sum(qs)
            moment = sum((i - lo) * q for i, q in zip(inside, qs))
            w = hi - lo + 1
            if charge == 0:
                bary = f32(f32(lo) + f32(f32(0.5) * f32(w)))
            else:
                bary = f32(f32(f32(lo) + f32(0.5)) + f32(f32(moment) / f32(charge)))
            out.append((lo, w, charge, float(bary)))
    out.sort()
    return out
