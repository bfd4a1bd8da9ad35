"""Pins of the oracle's local cluster positions (synthetic pitch per module).

arXiv 2101.11489 section 4: clusters become hits with positions for the track
finder.  Reading: local x = (barycenter - 128) * pitch[det] in binary32, origin at
the module centre.  Pinned by what that definition fixes without re-evaluating
it: zero at the centre, sign, exactness where both operations are exact (pitch 1,
power-of-two pitches, barycenters with few significant bits), linearity in the
pitch for power-of-two factors, and the per-module pitch lookup.
"""
import numpy as np

import oracle as orc


def test_centre_is_zero_and_sign_follows_the_side():
    x = orc.local_x(np.array([0, 0, 0], np.uint32), np.array([128.0, 127.5, 128.5], np.float32),
                    np.array([0.0122], np.float32))
    assert x[0] == 0.0 and x[1] < 0 < x[2] and x[1] == -x[2]


def test_exact_where_both_operations_are_exact():
    # barycenters on a 1/64 grid within [64, 256): b - 128 is exact; pitch 1 and 2^-7
    b = (np.arange(64 * 64, 256 * 64, 37) / 64.0).astype(np.float32)
    det = np.zeros(b.size, np.uint32)
    assert np.array_equal(orc.local_x(det, b, np.array([1.0], np.float32)), (b.astype(np.float64) - 128).astype(np.float32))
    x = orc.local_x(det, b, np.array([2.0 ** -7], np.float32))
    assert np.array_equal(x.astype(np.float64), (b.astype(np.float64) - 128) * 2.0 ** -7)


def test_power_of_two_pitch_scales_exactly_and_each_module_uses_its_pitch():
    rng = np.random.default_rng(7)
    b = rng.uniform(0, 256, 1000).astype(np.float32)
    det = rng.integers(0, 3, 1000).astype(np.uint32)
    pitch = np.array([0.0080, 0.0122, 0.0183], np.float32)
    x1 = orc.local_x(det, b, pitch)
    x2 = orc.local_x(det, b, pitch * np.float32(4))
    assert np.array_equal(x2, x1 * np.float32(4))
    for m in range(3):
        sel = det == m
        assert np.array_equal(orc.local_x(np.zeros(sel.sum(), np.uint32), b[sel], pitch[m:m + 1]), x1[sel])
    # within one rounding of the exact value (two binary32 operations)
    exact = (b.astype(np.float64) - 128) * pitch[det].astype(np.float64)
    assert np.all(np.abs(x1 - exact) <= 2.5 * np.spacing(np.abs(exact).astype(np.float32)) + 1e-12)
