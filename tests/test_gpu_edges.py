"""GPU parity at the edges of the method, against the oracle.

arXiv 2101.11489 section 2: a strip is active / a seed when its S/N is *larger
than* the channel / seed threshold, and a candidate is a cluster when its charge is
larger than the cluster threshold.  Random events reach the strict boundaries only
by chance, so these tests build them on purpose and run them through the per-event
path (sst_unpack + sst_cluster) and the batched path (sst_batch, both work-item
widths):
  - every pattern of 7 strip states over modules of 1 to 5 strips, packed as FED
    data, under three sets of hole / bad-strip limits;
  - ADC values one below, at and one above the channel and seed limits for noises
    whose threshold products are exact binary32 integers, and cluster sums equal to
    t_cluster x sqrt(sum noise^2) exactly;
  - the gain-corrected charge of every ADC 1..253 under many gains, including gains
    whose binary32 reciprocal does not reproduce the quotient's rounding for every
    ADC (the library then divides), checked strip by strip through the amplitudes;
  - valid payloads the canonical packers never write: runs across strip 128,
    touching runs, widths up to 255.
"""
import itertools

import numpy as np
import pytest

import eventgen as eg
import oracle as orc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_11489_gb300 as sst  # noqa: E402
import _fedbuild as fb  # noqa: E402
from _gpu_util import Gpu, assert_clusters_equal, assert_digis_equal, orc_params  # noqa: E402

f32 = np.float32
STATES = [(0, 0), (6, 0), (10, 0), (14, 0), (40, 0), (0, 1), (40, 1)]  # (ADC, bad) at noise 4
PARAMS = {"default": sst.params(),
          "h1b0a1": sst.params(max_seq_holes=1, max_seq_bad=0, max_adj_bad=1),
          "h2b2a1": sst.params(max_seq_holes=2, max_seq_bad=2, max_adj_bad=1)}


def check_both_paths(g, raw, fl, n_feds):
    """Per event and batched (work items of 2 and of 1 FE units) against the oracle."""
    od, oc, ost = g.oracle(raw, fl, n_feds)
    dh, ch = g.event(raw, fl, n_feds)
    assert_digis_equal(dh, od)
    assert {k: dh[k] for k in ost} == ost
    assert_clusters_equal(ch, oc)
    keep = sst.sst_get_tune(g.ctx)
    try:
        for units in (2, 1):
            sst.sst_set_tune(g.ctx, units_per_warp=units)
            (st, cl), = g.batch([(raw, fl)])
            assert st == ost
            assert_clusters_equal(cl, oc)
    finally:
        sst.sst_set_tune(g.ctx, **keep)
    return oc


def pattern_event(n_feds):
    """Every pattern of the 7 states over 1..5 strips, 28 patterns per channel, 9
    strips apart (the 4+ empty good strips between them link nothing under these
    limits); noise 4 everywhere, random gains per APV."""
    n = n_feds * 96 * 256
    adc = np.zeros(n, np.uint8)
    bad = np.zeros(n, np.uint8)
    slot = 0
    for width in range(1, 6):
        for states in itertools.product(STATES, repeat=width):
            ch, k = divmod(slot, 28)
            s0 = ch * 256 + (251 if k == 27 else 9 * k)  # the channel's last pattern ends at strip 255
            for i, (a, b) in enumerate(states):
                adc[s0 + i], bad[s0 + i] = a, b
            slot += 1
    assert slot <= n_feds * 96 * 28
    noise = np.full(n, 4.0, f32)
    gain = np.random.default_rng(3).uniform(0.8, 1.2, n // 128).astype(f32)
    raw, fl = eg.pack_event(adc, adc > 0, n_feds)
    return raw, fl, noise, gain, bad


@pytest.mark.parametrize("which", list(PARAMS))
def test_every_small_module_pattern(which):
    n_feds = 8
    raw, fl, noise, gain, bad = pattern_event(n_feds)
    g = Gpu(noise, gain, bad, PARAMS[which])
    try:
        oc = check_both_paths(g, raw, fl, n_feds)
        assert oc["det"].size > 3000
    finally:
        g.close()


# Noises whose products with 2 (channel) and 3 (seed) are exact in binary32, some
# integers (ties) and some not.
TIE_NOISES = [0.5, 1.25, 2.5, 3.0, 3.5, 4.0, 5.0, 6.0, 4.5, 3.75]


def tie_event(n_feds):
    """Channel c tests noise TIE_NOISES[c % 10]: strips 4 m hold single test strips
    next to a strong seed (active or not: width 2 or 1), the rest of the channel
    lone test strips (seed or not: a cluster or none, with t_cluster 0); plus
    cluster-threshold ties on channels >= 40: sums equal to 5 sqrt(N2) and one
    more."""
    n = n_feds * 96 * 256
    adc = np.zeros(n, np.uint8)
    noise = np.full(n, 4.0, f32)
    for c in range(40):
        nz = f32(TIE_NOISES[c % len(TIE_NOISES)])
        base = c * 256
        noise[base:base + 256] = nz
        pc, ps = int(np.floor(f32(2) * nz)), int(np.floor(f32(3) * nz))
        vals = [v for p in (pc, ps) for v in (p - 1, p, p + 1) if 0 < v < 254]
        for m, v in enumerate(vals):
            s = base + 8 * m
            adc[s], adc[s + 1] = v, 250  # test strip, then a strong seed
            adc[base + 128 + 8 * m] = v  # a lone test strip
    # cluster threshold 5 x sqrt(sum noise^2) met exactly: (noises, ADCs at the tie)
    ties = [((4.0,), (20,)), ((5.0,), (25,)), ((6.0,), (30,)), ((3.0, 4.0), (12, 13)), ((4.0, 3.0), (13, 12)),
            ((2.0, 3.0, 6.0), (8, 8, 19)), ((6.0, 3.0, 2.0), (19, 8, 8))]
    c = 40
    for nzs, vals in ties:
        for extra in (0, 1):  # at the tie (rejected) and one count above (kept)
            base = c * 256
            for rep in range(20):
                s = base + 12 * rep
                for i, (nz, v) in enumerate(zip(nzs, vals)):
                    noise[s + i] = nz
                    adc[s + i] = v + (extra if i == len(vals) - 1 else 0)
            c += 1
    bad = np.zeros(n, np.uint8)
    gain = np.ones(n // 128, f32)
    raw, fl = eg.pack_event(adc, adc > 0, n_feds)
    return raw, fl, noise, gain, bad


def test_threshold_ties_default_cluster_threshold():
    n_feds = 1
    raw, fl, noise, gain, bad = tie_event(n_feds)
    g = Gpu(noise, gain, bad, sst.params())
    try:
        oc = check_both_paths(g, raw, fl, n_feds)
        # cluster-threshold ties: each tie channel pair is (rejected, kept)
        kept = np.bincount(oc["det"], minlength=96)
        for k in range(7):
            assert kept[40 + 2 * k] == 0 and kept[41 + 2 * k] == 20, k
    finally:
        g.close()


def test_threshold_ties_no_cluster_threshold():
    n_feds = 1
    raw, fl, noise, gain, bad = tie_event(n_feds)
    g = Gpu(noise, gain, bad, sst.params(t_cluster=0.0))
    try:
        oc = check_both_paths(g, raw, fl, n_feds)
        # a lone strip is a cluster exactly when its ADC exceeds 3 x noise
        for c in range(40):
            nz = f32(TIE_NOISES[c % len(TIE_NOISES)])
            lone = oc["first"][(oc["det"] == c) & (oc["first"] >= 128)]
            for s in lone.tolist():
                m = (s - 128) // 8
                pc, ps = int(np.floor(f32(2) * nz)), int(np.floor(f32(3) * nz))
                vals = [v for p in (pc, ps) for v in (p - 1, p, p + 1) if 0 < v < 254]
                assert f32(vals[m]) > f32(3) * nz
    finally:
        g.close()


def charge(adc, g, mul):
    x = (adc.astype(f32) * g) if mul else (adc.astype(f32) / g)
    y = (x + f32(0.5)).astype(f32)
    return np.where(y >= f32(254), 254, np.floor(y)).astype(np.int64)


def uncertified_gains(n_want, seed):
    """Gains for which no multiplier within 4 ulp of the binary32 reciprocal gives
    the quotient's charge (ADC / gain + 1/2, truncated, binary32) for every ADC
    1..253: the library divides for these."""
    rng = np.random.default_rng(seed)
    a = np.arange(1, 254, dtype=f32)[None, :]
    found = []
    while len(found) < n_want:
        g = rng.uniform(0.5, 2.0, 20000).astype(f32)[:, None]
        want = charge(a, g, False)
        r = (f32(1) / g).astype(f32)
        ok = np.zeros(g.shape[0], bool)
        up = dn = r
        cands = [r]
        for _ in range(4):
            up, dn = np.nextafter(up, f32(np.inf)), np.nextafter(dn, f32(0))
            cands += [up, dn]
        for m in cands:
            ok |= (charge(a, m, True) == want).all(axis=1)
        found += g[~ok, 0].tolist()
    return np.array(found[:n_want], f32)


def test_gain_corrected_charge_of_every_adc():
    """All 256 strips of 64 channels active with ADCs cycling 1..253; each channel's
    two APVs get random gains or gains without a certified multiplier.  The
    amplitudes give every strip's gain-corrected charge."""
    n_feds = 1
    n = n_feds * 96 * 256
    adc = np.zeros(n, np.uint8)
    adc[:64 * 256] = 1 + (np.arange(64 * 256) * 7) % 253
    noise = np.full(n, 0.25, f32)
    gain = np.random.default_rng(8).uniform(0.5, 2.0, n // 128).astype(f32)
    ug = uncertified_gains(6, 21)
    gain[:ug.size] = ug
    gain[ug.size:2 * ug.size] = np.array([0.8, 1.0, 1.2, 0.5, 2.0, 0.75], f32)[:ug.size]
    bad = np.zeros(n, np.uint8)
    raw, fl = eg.pack_event(adc, adc > 0, n_feds)
    g = Gpu(noise, gain, bad, sst.params())
    try:
        od, oc, ost = g.oracle(raw, fl, n_feds)
        af, amp = orc.cluster_amplitudes(od, oc, noise, gain, bad, orc_params(g.params))
        e = eg.Event(raw, fl, n_feds, 0.0, int(np.count_nonzero(adc)))
        rt = torch.from_numpy(raw).cuda()
        ft = torch.from_numpy(fl.view(np.int32)).cuda()
        d = sst.DigiBuffers.alloc(e.nbytes, n_feds)
        cb = sst.ClusterBuffers.alloc(e.nbytes // 2 + 1, amp_capacity=4 * e.nbytes)
        drec = d.record()
        sst.sst_unpack(g.ctx, rt, ft, n_feds, drec)
        sst.sst_cluster(g.ctx, drec, n_feds, cb.record())
        torch.cuda.synchronize()
        dh = d.to_host()
        ch = cb.to_host(0, dh["n_clusters"])
        assert dh["n_clusters"] == ost["n_clusters"] == 64
        assert_clusters_equal({k: ch[k] for k in ("det", "first", "width", "charge", "barycenter")}, oc)
        got = cb.amplitudes()[:amp.size]
        assert np.array_equal(got, amp)
        assert amp.size == 64 * 256
        # and the amplitudes are the quotient's charge, strip by strip
        s = np.arange(64 * 256)
        assert np.array_equal(amp.astype(np.int64), charge(adc[s], gain[s // 128], False))
    finally:
        g.close()


@pytest.mark.parametrize("which", ["default", "h2b2a1"])
def test_valid_non_canonical_payloads(which):
    n_feds = 4
    feds = fb.non_canonical_feds(np.random.default_rng(17), n_feds)
    raw, fl = fb.event(feds)
    calib = eg.make_calibration(n_feds, 5, 0.02)
    g = Gpu(calib.noise, calib.gain, calib.bad, PARAMS[which])
    try:
        od, _, _ = g.oracle(raw, fl, n_feds)
        strips, adcs = fb.expected_digis(feds)
        assert np.array_equal(od["strip"], strips) and np.array_equal(od["adc"], adcs)
        oc = check_both_paths(g, raw, fl, n_feds)
        assert oc["det"].size > 50
    finally:
        g.close()
