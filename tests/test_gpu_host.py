"""sst_batch_host (events and results in host memory, copies overlapped with the
kernels over chunks of events) against the oracle and against sst_batch.

Batches are long enough to be cut into more chunks than the pipeline has slots,
with a ragged last chunk, so that every slot is reused.  Clusters, statuses and
the packed event starts must equal the oracle's event by event.
arXiv 2101.11489 section 3: many events per launch, transfers overlapped with
computation on CUDA streams.
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


@pytest.fixture(scope="module")
def w0():
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
    g = Gpu(calib.noise, calib.gain, calib.bad)
    yield w, calib, g
    g.close()


def _arena(events, prefix=0):
    sizes = [e.nbytes for e in events]
    eoff = np.zeros(len(events) + 1, np.uint64)
    eoff[0] = prefix
    eoff[1:] = prefix + np.cumsum(sizes)
    raw = np.concatenate([np.full(prefix, 0xEE, np.uint8)] + [e.raw for e in events])
    fl = np.concatenate([e.fed_len for e in events]).astype(np.uint32)
    return raw, eoff, fl


def _run(g, events, cap=None, prefix=0, pinned=False):
    raw, eoff, fl = _arena(events, prefix)
    n = len(events)
    total_cap = sum(e.nbytes // 2 + 1 for e in events) if cap is None else cap
    out = sst.HostClusters.alloc(total_cap, pinned=pinned)
    first = np.zeros(n + 1, np.uint64)
    status = np.zeros((n, 4), np.uint32)
    sst.sst_batch_host(g.ctx, raw, eoff, fl, n, g.n_feds, out, first, status)
    return out, first, status


def _status(row):
    return {"n_digi": int(row[0]), "n_clusters": int(row[1]), "flags": int(row[2]), "n_bad_channels": int(row[3])}


def test_host_batch_equals_oracle(w0):
    w, calib, g = w0
    # 11 events: chunks of 3, 3, 3, 2 over three pipeline slots
    events = [eg.make_event(w, calib, 300 + i, occupancy=0.002 + 0.004 * (i % 7)) for i in range(11)]
    out, first, status = _run(g, events)
    pos = 0
    for k, e in enumerate(events):
        _, oc, ost = g.oracle(e.raw, e.fed_len, w.n_feds)
        st = _status(status[k])
        assert st == ost, k
        assert int(first[k]) == pos
        assert_clusters_equal(out.view(pos, st["n_clusters"]), oc)
        pos += st["n_clusters"]
    assert int(first[-1]) == pos


def test_host_batch_equals_device_batch_pinned_with_offset(w0):
    w, calib, g = w0
    events = [eg.make_event(w, calib, 400 + i, occupancy=0.01 + 0.01 * (i % 3)) for i in range(6)]
    out, first, status = _run(g, events, prefix=48, pinned=True)
    ref = g.batch([(e.raw, e.fed_len) for e in events])
    for k, (st, cl) in enumerate(ref):
        assert _status(status[k]) == st
        got = out.view(int(first[k]), st["n_clusters"])
        for key in cl:
            assert np.array_equal(got[key], cl[key]), key


def test_host_batch_capacity_cut_is_flagged(w0):
    w, calib, g = w0
    events = [eg.make_event(w, calib, 500 + i, occupancy=0.02) for i in range(5)]
    full_out, full_first, full_status = _run(g, events)
    total = int(full_first[-1])
    cap = total // 2 + 7
    out, first, status = _run(g, events, cap=cap)
    assert int(first[-1]) == cap
    assert np.array_equal(out.det[:cap], full_out.det[:cap])
    assert np.array_equal(out.barycenter[:cap], full_out.barycenter[:cap])
    for k in range(len(events)):
        a, n_full = int(full_first[k]), int(full_status[k, 1])
        cut = a + n_full > cap
        assert bool(status[k, 2] & sst.SST_EV_CLUSTER_CAPACITY) == cut
        assert int(status[k, 1]) == (max(0, min(n_full, cap - a)) if cut else n_full)
        assert int(first[k]) == min(a, cap)


def test_host_batch_arena_growth_and_single_event(w0):
    w, calib, g = w0
    small = [eg.make_event(w, calib, 600, occupancy=0.003)]
    big = [eg.make_event(w, calib, 601 + i, occupancy=0.04) for i in range(9)]
    for events in (small, big, small):
        out, first, status = _run(g, events)
        pos = 0
        for k, e in enumerate(events):
            _, oc, ost = g.oracle(e.raw, e.fed_len, w.n_feds)
            assert _status(status[k]) == ost
            assert_clusters_equal(out.view(pos, ost["n_clusters"]), oc)
            pos += ost["n_clusters"]


def test_host_batch_rejects_decreasing_offsets(w0):
    w, calib, g = w0
    e = eg.make_event(w, calib, 700)
    raw, eoff, fl = _arena([e, e])
    eoff[1] = eoff[2] + 16
    out = sst.HostClusters.alloc(16)
    with pytest.raises(sst.SstError):
        sst.sst_batch_host(g.ctx, np.concatenate([raw, np.zeros(32, np.uint8)]), eoff, fl, 2, g.n_feds, out,
                           np.zeros(3, np.uint64), np.zeros((2, 4), np.uint32))


def test_submitted_batches_overlap_and_each_equals_the_oracle(w0):
    """Three batches queued back to back (the second larger, so the arenas grow
    between batches), waited in reverse order; each equals the oracle."""
    w, calib, g = w0
    sets = [[eg.make_event(w, calib, 800 + 10 * b + i, occupancy=0.003 + 0.01 * b) for i in range(n)]
            for b, n in enumerate((5, 9, 3))]
    pending = []
    for events in sets:
        raw, eoff, fl = _arena(events)
        out = sst.HostClusters.alloc(sum(e.nbytes // 2 + 1 for e in events), pinned=True)
        first = np.zeros(len(events) + 1, np.uint64)
        status = np.zeros((len(events), 4), np.uint32)
        t = sst.sst_batch_host_submit(g.ctx, raw, eoff, fl, len(events), g.n_feds, out, first, status)
        pending.append((t, events, raw, eoff, fl, out, first, status))
    for t, events, raw, eoff, fl, out, first, status in reversed(pending):
        sst.sst_batch_host_wait(g.ctx, t)
        pos = 0
        for k, e in enumerate(events):
            _, oc, ost = g.oracle(e.raw, e.fed_len, w.n_feds)
            assert _status(status[k]) == ost
            assert int(first[k]) == pos
            assert_clusters_equal(out.view(pos, ost["n_clusters"]), oc)
            pos += ost["n_clusters"]
        assert int(first[-1]) == pos
    with pytest.raises(sst.SstError):
        sst.sst_batch_host_wait(g.ctx, pending[0][0])  # already released
