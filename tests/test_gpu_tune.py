"""The autotuner's knobs on the GPU (arXiv 2101.11489 section 3: throughput from
tuning how much work is in flight).

Each knob of the batched path changes the launch it is meant to change (grid,
threads per CTA, shared memory, work items per FED, host chunks), every shape the
autotuner sweeps gives bit-identical statuses and clusters that match the oracle,
including corrupt and chunked work items, and the autotuners keep a shape from
their sweep.
"""
import numpy as np
import pytest

import eventgen as eg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_11489_gb300 as sst  # noqa: E402
from _gpu_util import Gpu, assert_clusters_equal  # noqa: E402
from test_gpu_corrupt import corruptions  # noqa: E402

N_FEDS = 4
SWEEP = [(b, u, p) for b in (128, 256) for u in (1, 2) for p in (2, 3, 4, 6, 8)]


@pytest.fixture(scope="module")
def g4():
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(N_FEDS, w.seed, w.p_bad)
    g = Gpu(calib.noise, calib.gain, calib.bad)
    yield w, calib, g
    g.close()


def mixed_events(w, calib):
    """Ordinary events, one so dense that work items exceed the on-chip tile and
    take the chunked path, and one corrupt event of every kind."""
    evs = [eg.make_event(w, calib, 70 + i, occupancy=o, n_feds=N_FEDS) for i, o in enumerate((0.005, 0.03, 0.3))]
    out = [(e.raw, e.fed_len) for e in evs]
    base = evs[1]
    out += [(r, f) for _, r, f in corruptions(base.raw, base.fed_len)][:6]
    return out


def test_each_knob_changes_the_launch(g4):
    _, _, g = g4
    keep = sst.sst_get_tune(g.ctx)
    try:
        def info(**kn):
            sst.sst_set_tune(g.ctx, **kn)
            return sst.sst_get_launch_info(g.ctx, 64, 440)
        a = info(block=256, ctas_per_sm=4, units_per_warp=2, host_chunk_events=32)
        b = info(block=128, ctas_per_sm=4, units_per_warp=2, host_chunk_events=32)
        assert (a["block"], b["block"]) == (256, 128) and a["smem_bytes"] == 2 * b["smem_bytes"]
        c = info(block=256, ctas_per_sm=2, units_per_warp=2, host_chunk_events=32)
        assert c["grid"] == a["grid"] // 2
        d = info(block=256, ctas_per_sm=4, units_per_warp=1, host_chunk_events=32)
        assert (a["items_per_fed"], d["items_per_fed"]) == (4, 8) and d["smem_bytes"] < a["smem_bytes"]
        e = info(block=256, ctas_per_sm=4, units_per_warp=2, host_chunk_events=8)
        assert (a["host_chunks"], e["host_chunks"]) == (2, 8)
    finally:
        sst.sst_set_tune(g.ctx, **keep)


def test_every_swept_shape_gives_identical_results(g4):
    w, calib, g = g4
    evs = mixed_events(w, calib)
    keep = sst.sst_get_tune(g.ctx)
    ref = g.batch(evs)
    for (r, f), (st, cl) in zip(evs, ref):
        _, oc, ost = g.oracle(r, f, N_FEDS)
        assert st == ost
        assert_clusters_equal(cl, oc)
    try:
        for block, units, cps in SWEEP:
            sst.sst_set_tune(g.ctx, block=block, units_per_warp=units, ctas_per_sm=cps)
            got = g.batch(evs)
            for (s0, c0), (s1, c1) in zip(ref, got):
                assert s0 == s1, (block, units, cps)
                for k in c0:
                    assert np.array_equal(c0[k], c1[k]), (block, units, cps, k)
    finally:
        sst.sst_set_tune(g.ctx, **keep)


def test_autotune_keeps_a_swept_shape(g4):
    w, calib, g = g4
    evs = [eg.make_event(w, calib, 90 + i, n_feds=N_FEDS) for i in range(8)]
    n = len(evs)
    sizes = [e.raw.size for e in evs]
    eoff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    coff = np.concatenate([[0], np.cumsum([s // 2 + 1 for s in sizes])]).astype(np.int64)
    raw = torch.from_numpy(np.concatenate([e.raw for e in evs])).cuda()
    fl = torch.from_numpy(np.concatenate([e.fed_len for e in evs]).astype(np.uint32).view(np.int32)).cuda()
    eo, co = torch.from_numpy(eoff).cuda(), torch.from_numpy(coff).cuda()
    cb = sst.ClusterBuffers.alloc(int(coff[-1]))
    st = torch.zeros(n * 4, dtype=torch.int32, device="cuda")
    keep = sst.sst_get_tune(g.ctx)
    try:
        best, us = sst.sst_autotune(g.ctx, raw, eo, fl, n, N_FEDS, co, cb.record(), st)
        assert (best["block"], best["units_per_warp"], best["ctas_per_sm"]) in SWEEP and us > 0
        assert sst.sst_get_tune(g.ctx) == best
        sst.sst_batch(g.ctx, raw, eo, fl, n, N_FEDS, co, cb.record(), st)
        torch.cuda.synchronize()
        sth = st.cpu().numpy().view(np.uint32).reshape(n, 4)
        for i, e in enumerate(evs):
            _, oc, ost = g.oracle(e.raw, e.fed_len, N_FEDS)
            assert int(sth[i, 1]) == ost["n_clusters"]
            assert_clusters_equal(cb.to_host(int(coff[i]), int(sth[i, 1])), oc)
    finally:
        sst.sst_set_tune(g.ctx, **keep)


def test_autotune_host_picks_a_batch_depth(g4):
    w, calib, g = g4
    evs = [eg.make_event(w, calib, 110 + i, n_feds=N_FEDS) for i in range(24)]
    b = eg.make_batch(evs)
    n = len(evs)
    cap = int(sum(e.nbytes // 2 + 1 for e in evs))
    out = sst.HostClusters.alloc(cap)
    ef = np.zeros(n + 1, np.uint64)
    sth = np.zeros((n, 4), np.uint32)
    keep = sst.sst_get_tune(g.ctx)
    try:
        best, us = sst.sst_autotune_host(g.ctx, b.raw, b.event_off, b.fed_len, n, N_FEDS, out, ef, sth)
        assert best in (0, 4, 8, 16) and us > 0
        assert sst.sst_get_tune(g.ctx)["host_chunk_events"] == best
        sst.sst_batch_host(g.ctx, b.raw, b.event_off, b.fed_len, n, N_FEDS, out, ef, sth)
        for i, e in enumerate(evs):
            _, oc, ost = g.oracle(e.raw, e.fed_len, N_FEDS)
            assert int(sth[i, 1]) == ost["n_clusters"]
            assert_clusters_equal(out.view(int(ef[i]), int(sth[i, 1])), oc)
    finally:
        sst.sst_set_tune(g.ctx, **keep)


@pytest.mark.parametrize("n_small", [40, 2])
def test_oversized_items_first_equal_the_oracle(g4, n_small):
    """Work items too large for the staging buffer are listed by the prologue and
    taken first; with few of them (one dense event among 40, under 1 in 32 of the
    items) the staged items keep their shared-memory code, with many (one among 2)
    every item takes the in-place code.  Both batches equal the oracle event by
    event, in every shape the autotuner sweeps over the work-item width."""
    w, calib, g = g4
    evs = [eg.make_event(w, calib, 400 + i, occupancy=0.004 + 0.002 * (i % 3), n_feds=N_FEDS) for i in range(n_small)]
    dense = eg.make_event(w, calib, 499, occupancy=0.3, n_feds=N_FEDS)
    events = [(e.raw, e.fed_len) for e in evs[: n_small // 2]] + [(dense.raw, dense.fed_len)] + \
             [(e.raw, e.fed_len) for e in evs[n_small // 2:]]
    keep = sst.sst_get_tune(g.ctx)
    try:
        for units in (2, 1):
            sst.sst_set_tune(g.ctx, units_per_warp=units)
            got = g.batch(events)
            for (r, f), (st, cl) in zip(events, got):
                _, oc, ost = g.oracle(r, f, N_FEDS)
                assert st == ost, units
                assert_clusters_equal(cl, oc)
    finally:
        sst.sst_set_tune(g.ctx, **keep)
