"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Digis, channel statuses, event statuses and cluster det / first / width / charge
must match bit for bit; barycenters within 1e-6 strip (the same binary32
expression is evaluated on both sides, so they are expected to be equal).
Method: arXiv 2101.11489 section 2 (unpack, three-threshold clustering) and
section 3 (many events per launch).
"""
import numpy as np
import pytest

import eventgen as eg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_11489_gb300 as sst  # noqa: E402
from _gpu_util import Gpu, assert_clusters_equal, assert_digis_equal  # noqa: E402


@pytest.fixture(scope="module")
def w0():
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
    g = Gpu(calib.noise, calib.gain, calib.bad)
    yield w, calib, g
    g.close()


def check_event(g, raw, fl, n_feds, **kw):
    dh, ch = g.event(raw, fl, n_feds, **kw)
    od, oc, ost = g.oracle(raw, fl, n_feds)
    assert_digis_equal(dh, od)
    assert_clusters_equal(ch, oc)
    for k in ("n_digi", "n_clusters", "flags", "n_bad_channels"):
        assert dh[k] == ost[k], k
    return dh, ch, oc


def test_small_event_parity(w0):
    w, calib, g = w0
    e = eg.make_event(w, calib, 0)
    dh, ch, oc = check_event(g, e.raw, e.fed_len, w.n_feds)
    assert oc["det"].size > 1000


@pytest.mark.parametrize("event", [1, 2, 3])
def test_small_event_parity_more_events(w0, event):
    w, calib, g = w0
    e = eg.make_event(w, calib, event, occupancy=0.004 * event)
    check_event(g, e.raw, e.fed_len, w.n_feds)


@pytest.mark.parametrize("occ", [0.0, 0.2, 0.6])
def test_occupancy_extremes_and_tile_chunking(w0, occ):
    # 20% and 60% signal occupancy put several thousand digis in one FED: more
    # than one tile (chunked clustering) and FED records above the staging buffer
    w, calib, g = w0
    e = eg.make_event(w, calib, 7, n_feds=4, occupancy=occ)
    check_event(g, e.raw, e.fed_len, 4)


def test_absent_feds_and_subset(w0):
    w, calib, g = w0
    e = eg.make_event(w, calib, 11, n_feds=6)
    # drop FEDs 1 and 4 (fed_len 0, records removed)
    offs = np.concatenate([[0], np.cumsum(e.fed_len)]).astype(np.int64)
    keep = [0, 2, 3, 5]
    raw = np.concatenate([e.raw[offs[f]:offs[f + 1]] for f in keep])
    fl = e.fed_len.copy()
    fl[[1, 4]] = 0
    check_event(g, raw, fl, 6)


def test_single_fed_and_empty_channels(w0):
    w, calib, g = w0
    n = 96 * 256
    adc = np.zeros(n, np.uint8)
    rec = np.zeros(n, np.uint8)
    raw, fl = eg.pack_event(adc, rec, 1)
    dh, ch, oc = check_event(g, raw, fl, 1)
    assert dh["n_digi"] == 0 and oc["det"].size == 0


def test_full_channels_and_alternating_runs(w0):
    w, calib, g = w0
    n = 2 * 96 * 256
    r = np.random.default_rng(5)
    adc = r.integers(0, 256, n).astype(np.uint8)
    rec = np.zeros(n, np.uint8)
    rec[0:256] = 1                      # channel 0 fully recorded
    rec[256:512:2] = 1                  # channel 1: 128 runs of width 1
    rec[96 * 256 + 3 * 256:96 * 256 + 4 * 256] = 1
    rec[5000:5400] = (r.random(400) < 0.5)
    adc = np.where(rec != 0, adc, 0).astype(np.uint8)
    raw, fl = eg.pack_event(adc, rec, 2)
    check_event(g, raw, fl, 2)


def test_full_detector_event_parity():
    w = eg.WORKLOADS[1]
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
    g = Gpu(calib.noise, calib.gain, calib.bad)
    try:
        e = eg.make_event(w, calib, 0)
        dh, ch, oc = check_event(g, e.raw, e.fed_len, w.n_feds)
        assert dh["n_digi"] > 300_000 and oc["det"].size > 40_000
    finally:
        g.close()


def check_params(params, p_bad, occupancy):
    """Per-event and batched paths against the oracle under one parameter set."""
    w = eg.Workload("variant", 3, 1, ("fixed", occupancy), (1, 12), p_bad, 77, overlap=True, sat_frac=0.05)
    calib = eg.make_calibration(3, 77, p_bad)
    g = Gpu(calib.noise, calib.gain, calib.bad, sst.params(**params))
    try:
        evs = [eg.make_event(w, calib, ev) for ev in range(3)]
        for e in evs:
            check_event(g, e.raw, e.fed_len, 3)
        for e, (st, cl) in zip(evs, g.batch([(e.raw, e.fed_len) for e in evs])):
            _, oc, ost = g.oracle(e.raw, e.fed_len, 3)
            assert st == ost
            assert_clusters_equal(cl, oc)
    finally:
        g.close()


@pytest.mark.parametrize("params", [
    dict(), dict(max_seq_bad=0), dict(max_seq_holes=1), dict(max_seq_holes=2, max_seq_bad=2, max_adj_bad=1),
    dict(t_channel=2.5, t_seed=4.0, t_cluster=3.0), dict(t_cluster=0.0)])
def test_parameter_variants(params):
    check_params(params, 0.03, 0.05)


@pytest.mark.parametrize("holes,bad", [(0, 0), (0, 3), (3, 0), (1, 1), (2, 3), (5, 4), (255, 255)])
def test_gap_rules_on_a_dense_bad_strip_map(holes, bad):
    """Hole / bad-strip linking where a third of the strips are bad, so that gaps
    alternate between runs of bad strips and holes of every length."""
    check_params(dict(max_seq_holes=holes, max_seq_bad=bad, max_adj_bad=1), 0.33, 0.08)


def test_batch_equals_per_event(w0):
    w, calib, g = w0
    evs = [eg.make_event(w, calib, 20 + i, occupancy=0.003 * (i + 1)) for i in range(5)]
    out = g.batch([(e.raw, e.fed_len) for e in evs])
    for e, (st, cl) in zip(evs, out):
        od, oc, ost = g.oracle(e.raw, e.fed_len, w.n_feds)
        assert st == ost
        assert_clusters_equal(cl, oc)


def test_batch_launch_shapes_give_identical_results(w0):
    """Every knob of the batched kernel (block, CTAs per SM, FE units per work
    item) gives the same statuses and clusters as the default shape."""
    w, calib, g = w0
    evs = [eg.make_event(w, calib, 40 + i, occupancy=0.01 * (i + 1)) for i in range(3)]
    keep = sst.sst_get_tune(g.ctx)
    ref = g.batch([(e.raw, e.fed_len) for e in evs])
    for block, cps, units in [(128, 4, 1), (128, 2, 2), (256, 3, 1), (256, 8, 2), (256, 1, 1)]:
        sst.sst_set_tune(g.ctx, block=block, ctas_per_sm=cps, units_per_warp=units)
        got = g.batch([(e.raw, e.fed_len) for e in evs])
        for (s0, c0), (s1, c1) in zip(ref, got):
            assert s0 == s1
            for k in c0:
                assert np.array_equal(c0[k], c1[k])
    sst.sst_set_tune(g.ctx, **keep)


def _as_set(c):
    return set(zip(c["det"].tolist(), c["first"].tolist(), c["width"].tolist(), c["charge"].tolist()))


def test_cluster_capacity_overflow_is_flagged_and_bounded(w0):
    w, calib, g = w0
    e = eg.make_event(w, calib, 3)
    od, oc, ost = g.oracle(e.raw, e.fed_len, w.n_feds)
    cap = oc["det"].size // 3
    dh, ch = g.event(e.raw, e.fed_len, w.n_feds, clu_cap=cap)
    assert dh["flags"] & sst.SST_EV_CLUSTER_CAPACITY
    assert dh["n_clusters"] <= cap and ch["det"].size == dh["n_clusters"]
    key = ch["det"].astype(np.int64) * 256 + ch["first"]
    assert np.all(np.diff(key) > 0)  # still sorted
    assert _as_set(ch) <= _as_set(oc)  # a subset of the true clusters
    # the batched path flags the same event the same way (a sorted subset of its
    # clusters, those of whole work items) and leaves the events around it intact,
    # one of them with exactly the capacity it needs
    other = eg.make_event(w, calib, 5)
    _, oc2, ost2 = g.oracle(other.raw, other.fed_len, w.n_feds)
    out = g.batch([(other.raw, other.fed_len), (e.raw, e.fed_len), (other.raw, other.fed_len)],
                  clu_caps=[oc2["det"].size, cap, oc2["det"].size + 5])
    st, cl = out[1]
    assert st["flags"] & sst.SST_EV_CLUSTER_CAPACITY and st["n_clusters"] <= cap
    key = cl["det"].astype(np.int64) * 256 + cl["first"]
    assert np.all(np.diff(key) > 0)
    assert _as_set(cl) <= _as_set(oc)
    for st2, cl2 in (out[0], out[2]):
        assert st2 == ost2
        assert_clusters_equal(cl2, oc2)


def test_digi_capacity_overflow_is_flagged_and_bounded(w0):
    w, calib, g = w0
    e = eg.make_event(w, calib, 4)
    od, oc, ost = g.oracle(e.raw, e.fed_len, w.n_feds)
    cap = od["strip"].size // 2
    dh, ch = g.event(e.raw, e.fed_len, w.n_feds, digi_cap=cap)
    assert dh["flags"] & sst.SST_EV_DIGI_CAPACITY
    assert dh["n_digi"] == cap
    assert np.array_equal(dh["strip"], od["strip"][:cap])
    assert np.all(dh["chan_off"] <= cap)
