"""Served path (continuous batching behind sst_submit / sst_poll) against the oracle.

Events of uneven occupancy are submitted one at a time while earlier ones are on
the GPU; the server batches whatever is pending whenever a batch slot frees up.
Every event's clusters and status must equal the oracle's, whether the event was
processed alone or in the mix (nothing in the method depends on the batch).
arXiv 2101.11489 section 3: many events processed concurrently on one GPU.
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
def served():
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
    g = Gpu(calib.noise, calib.gain, calib.bad)
    sst.sst_server_start(g.ctx, 256 << 20, 6, 2, 32, w.n_feds)
    yield w, calib, g
    sst.sst_server_stop(g.ctx)
    g.close()


def _poll(g, ticket, cap):
    code, info, cl = sst.sst_poll(g.ctx, ticket, -1, cap)
    assert code == sst.SST_OK
    st = {"n_digi": info.status.n_digi, "n_clusters": info.status.n_clusters, "flags": info.status.flags,
          "n_bad_channels": info.status.n_bad_channels}
    assert info.t_done_us >= info.t_submit_us
    return st, cl


def test_alone_and_in_the_mix_equal_the_oracle(served):
    w, calib, g = served
    events = [eg.make_event(w, calib, 100 + i, occupancy=0.002 + 0.003 * (i % 9)) for i in range(30)]
    # alone: submit, wait, next
    alone = []
    for e in events[:5]:
        code, t = sst.sst_submit(g.ctx, e.raw, e.fed_len)
        assert code == sst.SST_OK
        alone.append(_poll(g, t, e.nbytes))
    # mix: submit everything while earlier events are in flight; when the server
    # is full, poll the oldest outstanding event; poll the rest newest first
    results, outstanding = {}, []
    for k, e in enumerate(events):
        while True:
            code, t = sst.sst_submit(g.ctx, e.raw, e.fed_len)
            if code == sst.SST_OK:
                outstanding.append((k, t))
                break
            assert code in (sst.SST_ERR_BUSY, sst.SST_ERR_BUDGET)
            kk, tt = outstanding.pop(0)
            results[kk] = _poll(g, tt, events[kk].nbytes)
    for kk, tt in reversed(outstanding):
        results[kk] = _poll(g, tt, events[kk].nbytes)
    tickets = results
    for k, e in enumerate(events):
        od, oc, ost = g.oracle(e.raw, e.fed_len, w.n_feds)
        st, cl = tickets[k]
        assert st == ost, k
        assert_clusters_equal(cl, oc)
        if k < 5:
            assert alone[k][0] == st
            for key in cl:
                assert np.array_equal(alone[k][1][key], cl[key])


def test_admission_limits(served):
    w, calib, g = served
    e = eg.make_event(w, calib, 7)
    big = np.zeros(16 << 20, np.uint8)  # more than a batch slot's raw arena
    code, _ = sst.sst_submit(g.ctx, big, e.fed_len)
    assert code == sst.SST_ERR_TOO_LARGE
    tickets = []
    busy = False
    for _ in range(40):
        code, t = sst.sst_submit(g.ctx, e.raw, e.fed_len)
        if code == sst.SST_ERR_BUSY:
            busy = True
            break
        assert code in (sst.SST_OK, sst.SST_ERR_BUDGET)
        if code == sst.SST_OK:
            tickets.append(t)
    assert busy  # 32 request slots
    for t in tickets:
        assert sst.sst_poll(g.ctx, t, -1, 0)[0] == sst.SST_OK
    with pytest.raises(sst.SstError):
        sst.sst_poll(g.ctx, 123456789, 0, 0)


def test_zero_copy_submission_equals_the_oracle():
    """With zero_copy the server reads each event from the caller's (pinned)
    buffer, which the caller keeps until the event is polled."""
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
    g = Gpu(calib.noise, calib.gain, calib.bad)
    sst.sst_server_start(g.ctx, 256 << 20, 4, 2, 64, w.n_feds, zero_copy=True)
    try:
        events = [eg.make_event(w, calib, 900 + i, occupancy=0.002 + 0.004 * (i % 5)) for i in range(12)]
        pinned = [torch.from_numpy(e.raw).pin_memory() for e in events]  # lent to the server until polled
        tickets = []
        for e, p in zip(events, pinned):
            code, t = sst.sst_submit(g.ctx, p.numpy(), e.fed_len)
            assert code == sst.SST_OK
            tickets.append(t)
        for e, t in zip(events, tickets):
            st, cl = _poll(g, t, e.nbytes)
            _, oc, ost = g.oracle(e.raw, e.fed_len, w.n_feds)
            assert st == ost
            assert_clusters_equal(cl, oc)
    finally:
        sst.sst_server_stop(g.ctx)
        g.close()
