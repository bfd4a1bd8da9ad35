"""Pins of the oracle's optional per-strip cluster amplitudes.

arXiv 2101.11489 section 2: a kept cluster reports its boundaries, its centroid and
optionally its ADC values.  Reading: the amplitude of each strip of the cluster is
its gain-corrected charge when the strip is active and 0 otherwise (a hole, a bad
strip inside, or a bad strip the cluster was widened over).  Pinned against what
the definition fixes independently of the amplitude code: one amplitude per strip
of the width, the amplitudes add up to the cluster charge (pinned separately), a
hand-built module, and zeros exactly at the strips that cannot be active.
"""
import numpy as np

import eventgen as eg
import oracle as orc
from oracle import Params

PER_FED = 96 * 256


def one_fed(strips: dict, bad=(), noise=4.0, gain=1.0):
    """Digis and calibration of one FED with the given {global strip: adc}."""
    noise_a = np.full(PER_FED, noise, np.float32)
    bad_a = np.zeros(PER_FED, np.uint8)
    bad_a[list(bad)] = 1
    gain_a = np.full(PER_FED // 128, gain, np.float32)
    keys = sorted(strips)
    strip = np.array(keys, np.uint32)
    adc = np.array([strips[k] for k in keys], np.uint8)
    chan_off = np.searchsorted(strip, np.arange(97) * 256).astype(np.uint32)
    return {"strip": strip, "adc": adc, "chan_off": chan_off}, noise_a, gain_a, bad_a


def run(digis, noise, gain, bad, p):
    c = orc.cluster_event(digis, 1, noise, gain, bad, p)
    af, amp = orc.cluster_amplitudes(digis, c, noise, gain, bad, p)
    return c, af, amp


def test_hand_built_module_with_a_bad_strip_inside():
    # channel 3: seed 30 at strip 10, bad strip 11, active 20 at strip 12 (noise 4:
    # active > 8, seed > 12); max_seq_bad 1 links 10 and 12 over the bad strip
    g0 = 3 * 256
    d, n, gn, b = one_fed({g0 + 10: 30, g0 + 12: 20}, bad=[g0 + 11])
    c, af, amp = run(d, n, gn, b, Params())
    assert c["det"].tolist() == [3] and c["first"].tolist() == [10] and c["width"].tolist() == [3]
    assert af.tolist() == [0]
    assert amp.tolist() == [30, 0, 20]  # gain 1: corrected charge = ADC


def test_widening_over_an_adjacent_bad_strip_adds_a_zero():
    g0 = 5 * 256
    d, n, gn, b = one_fed({g0 + 40: 50, g0 + 41: 10}, bad=[g0 + 39])
    c, af, amp = run(d, n, gn, b, Params(max_adj_bad=1))
    assert c["first"].tolist() == [39] and c["width"].tolist() == [3]
    assert amp.tolist() == [0, 50, 10]


def test_holes_inside_a_cluster_are_zero_and_gain_is_applied():
    # max_seq_holes 1: strips 100 and 102 are linked over the unrecorded strip 101;
    # gain 0.8: 40 / 0.8 = 50, 12 / 0.8 = 15
    g0 = 0
    d, n, gn, b = one_fed({g0 + 100: 40, g0 + 102: 12}, gain=0.8)
    c, af, amp = run(d, n, gn, b, Params(max_seq_holes=1))
    assert c["first"].tolist() == [100] and c["width"].tolist() == [3]
    assert amp.tolist() == [50, 0, 15]
    assert int(c["charge"][0]) == 65


def test_several_clusters_are_back_to_back():
    g0 = 7 * 256
    d, n, gn, b = one_fed({g0 + 1: 30, g0 + 2: 25, g0 + 50: 40, 8 * 256 + 3: 60})
    c, af, amp = run(d, n, gn, b, Params())
    assert c["det"].tolist() == [7, 7, 8]
    assert c["width"].tolist() == [2, 1, 1]
    assert af.tolist() == [0, 2, 3]
    assert amp.tolist() == [30, 25, 40, 60]


def check_event_properties(w, calib, event, p):
    e = eg.make_event(w, calib, event)
    d, c = orc.process_event(e.raw, e.fed_len, w.n_feds, calib.noise, calib.gain, calib.bad, p)
    af, amp = orc.cluster_amplitudes(d, c, calib.noise, calib.gain, calib.bad, p)
    width = c["width"].astype(np.int64)
    assert amp.size == width.sum()
    assert np.array_equal(af.astype(np.int64), np.concatenate([[0], np.cumsum(width)[:-1]]))
    seg = np.repeat(np.arange(width.size), width)
    assert np.array_equal(np.bincount(seg, weights=amp, minlength=width.size).astype(np.int64),
                          c["charge"].astype(np.int64))
    # strips that cannot be active (bad, or not recorded) have amplitude 0
    g = (c["det"].astype(np.int64) * 256)[seg] + (c["first"].astype(np.int64)[seg] +
                                                 (np.arange(amp.size) - af.astype(np.int64)[seg]))
    recorded = np.isin(g, d["strip"].astype(np.int64))
    dead = (calib.bad[g] != 0) | ~recorded
    assert (amp[dead] == 0).all()
    return amp.size


def test_event_amplitudes_add_up_to_the_charge_and_vanish_where_inactive():
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
    assert check_event_properties(w, calib, 0, Params()) > 1000


def test_event_amplitudes_with_holes_and_widening():
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(w.n_feds, w.seed, 0.02)
    assert check_event_properties(w, calib, 1, Params(max_seq_holes=1, max_seq_bad=2, max_adj_bad=1)) > 1000
