"""Sanity of the seeded synthetic events (shapes and orders of magnitude only).

The paper's sample has about 800,000 recorded strips and 150,000 seed strips per
event on the full CMS strip tracker (arXiv 2101.11489 section 2); the synthetic
full-detector events must be of the same order.  Nothing here checks the method.
"""
import numpy as np

import eventgen as eg


def test_keyed_generator_is_reproducible_per_event():
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
    a = eg.make_event(w, calib, 3)
    b = eg.make_event(w, calib, 3)
    c = eg.make_event(w, calib, 4)
    assert np.array_equal(a.raw, b.raw) and np.array_equal(a.fed_len, b.fed_len)
    assert not np.array_equal(a.raw[:2000], c.raw[:2000])


def test_small_event_statistics():
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
    n = w.n_feds * 96 * 256
    assert calib.noise.dtype == np.float32 and calib.noise.min() >= 3 and calib.noise.max() <= 6
    assert 0.8 <= calib.gain.min() and calib.gain.max() <= 1.2 and calib.gain.size == n // 128
    assert 0.0005 < calib.bad.mean() < 0.002
    adc, rec = eg.make_event_strips(w, calib, 0)
    occ = rec.mean()
    # 1% signal strips plus about 2.3% noise strips above 2 sigma
    assert 0.025 < occ < 0.045
    assert (adc[rec == 0] == 0).all()
    e = eg.make_event(w, calib, 0)
    assert e.raw.size == int(e.fed_len.sum()) and all(x % 16 == 0 for x in e.fed_len)


def test_batch_layout():
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
    evs = [eg.make_event(w, calib, i, occupancy=0.005 * (i + 1)) for i in range(3)]
    b = eg.make_batch(evs)
    assert b.event_off.tolist() == [0, evs[0].nbytes, evs[0].nbytes + evs[1].nbytes, b.raw.size]
    assert b.fed_len.size == 3 * w.n_feds
    assert all(int(o) % 16 == 0 for o in b.event_off)


def test_fed_skew_variant_spreads_fed_payloads_eightfold():
    """The batched configuration says FED payloads differ up to 8x; with the stated
    noise model they differ far less, so the stress variant skews the FEDs'
    occupancies (measured here on four events; the plain workload for contrast)."""
    def spread(wid):
        w = eg.WORKLOADS[wid]
        calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
        fl = np.array([eg.make_event(w, calib, e).fed_len for e in range(4)]).astype(float) - 32
        return (fl.max(axis=1) / fl.min(axis=1)).max(), fl.max() / fl.min()
    within, across = spread(5)
    assert within >= 8.0 and across >= 8.0
    within2, across2 = spread(2)
    assert across2 < 2.0
