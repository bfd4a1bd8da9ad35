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


def test_in_place_submission_equals_the_oracle():
    """In place (zero_copy 2) the kernels read each event straight from the
    caller's pinned buffer, whose bytes sit at scattered host addresses; every
    event equals the oracle.  Buffers that are pageable or not 16-byte aligned are
    refused at submission (nothing is read from them)."""
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
    g = Gpu(calib.noise, calib.gain, calib.bad)
    sst.sst_server_start(g.ctx, 256 << 20, 5, 2, 64, w.n_feds, zero_copy="in_place")
    try:
        events = [eg.make_event(w, calib, 950 + i, occupancy=0.002 + 0.004 * (i % 5)) for i in range(14)]
        pinned = [torch.from_numpy(e.raw).pin_memory() for e in events]  # lent until polled
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
        e = events[0]
        with pytest.raises(sst.SstError) as ei:  # pageable
            sst.sst_submit(g.ctx, e.raw.copy(), e.fed_len)
        assert ei.value.code == sst.SST_ERR_INVALID_ARG
        big = torch.empty(e.raw.size + 16, dtype=torch.uint8).pin_memory()
        big[1:1 + e.raw.size] = torch.from_numpy(e.raw)
        with pytest.raises(sst.SstError) as ei:  # pinned, but not 16-byte aligned
            sst.sst_submit(g.ctx, big.numpy()[1:1 + e.raw.size], e.fed_len)
        assert ei.value.code == sst.SST_ERR_INVALID_ARG
    finally:
        sst.sst_server_stop(g.ctx)
        g.close()


def test_budget_full_then_poll_then_resubmit():
    """Admission by memory: with a small budget the host pool of admitted events
    fills, sst_submit answers BUDGET, and after one poll the same event is admitted."""
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
    g = Gpu(calib.noise, calib.gain, calib.bad)
    try:
        sst.sst_server_start(g.ctx, 64 << 20, 4, 1, 4096, w.n_feds)
        e = eg.make_event(w, calib, 7, occupancy=0.02)
        tickets = []
        for _ in range(4096):
            code, t = sst.sst_submit(g.ctx, e.raw, e.fed_len)
            if code != sst.SST_OK:
                break
            tickets.append(t)
        assert code == sst.SST_ERR_BUDGET and len(tickets) >= 2
        st, _ = _poll(g, tickets.pop(0), 0)
        code, t = sst.sst_submit(g.ctx, e.raw, e.fed_len)
        assert code == sst.SST_OK
        tickets.append(t)
        _, oc, ost = g.oracle(e.raw, e.fed_len, w.n_feds)
        assert st == ost
        for t in tickets:
            st, cl = _poll(g, t, e.nbytes)
            assert st == ost
            assert_clusters_equal(cl, oc)
        big = np.zeros(64 << 20, np.uint8)  # larger than a batch slot's raw arena: never admissible
        code, _ = sst.sst_submit(g.ctx, big, e.fed_len)
        assert code == sst.SST_ERR_TOO_LARGE
    finally:
        sst.sst_server_stop(g.ctx)
        g.close()


def test_stop_while_other_threads_submit_and_poll():
    """sst_server_stop is safe while other threads are inside sst_submit / sst_poll:
    every call returns OK, a refusal, or STATE once the server is gone."""
    import threading
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
    g = Gpu(calib.noise, calib.gain, calib.bad)
    e = eg.make_event(w, calib, 8, occupancy=0.01)
    seen = []
    try:
        sst.sst_server_start(g.ctx, 256 << 20, 4, 2, 64, w.n_feds)

        def client():
            for _ in range(400):
                try:
                    code, t = sst.sst_submit(g.ctx, e.raw, e.fed_len)
                    if code == sst.SST_OK:
                        code = sst.sst_poll(g.ctx, t, -1, 0)[0]
                except sst.SstError as ex:  # the binding raises the codes it does not return
                    code = ex.code
                seen.append(code)
                if code == sst.SST_ERR_STATE:
                    return

        th = [threading.Thread(target=client) for _ in range(4)]
        for t in th:
            t.start()
        import time
        time.sleep(0.05)
        sst.sst_server_stop(g.ctx)
        for t in th:
            t.join(timeout=60)
            assert not t.is_alive()
        assert set(seen) <= {sst.SST_OK, sst.SST_ERR_BUSY, sst.SST_ERR_BUDGET, sst.SST_ERR_STATE}
        assert sst.SST_OK in seen
        with pytest.raises(sst.SstError) as ei:
            sst.sst_submit(g.ctx, e.raw, e.fed_len)
        assert ei.value.code == sst.SST_ERR_STATE
    finally:
        sst.sst_server_stop(g.ctx)
        g.close()


@pytest.mark.parametrize("zero_copy", [True, "in_place"])
def test_native_client_saturating_and_poisson(zero_copy):
    """The native load generator (sst_serve_load) drives the server through the
    public calls from its own threads (lent buffers copied, or read in place):
    every request is collected, latencies are ordered, and an offered rate well
    below capacity is what comes out."""
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
    g = Gpu(calib.noise, calib.gain, calib.bad)
    try:
        sst.sst_server_start(g.ctx, 512 << 20, 16, 3, 256, w.n_feds, zero_copy=zero_copy)
        pinned = [torch.from_numpy(eg.make_event(w, calib, 200 + i).raw).pin_memory() for i in range(8)]
        evs = [(p.numpy(), eg.make_event(w, calib, 200 + i).fed_len) for i, p in enumerate(pinned)]
        sat = sst.sst_serve_load(g.ctx, evs, 2000, 0.0, submitters=4, pollers=2)
        assert sat["requests"] == 2000 and sat["throughput"] > 1000
        assert 0 < sat["p50_us"] <= sat["p99_us"] <= sat["max_us"]
        rate = 0.2 * sat["throughput"]
        r = sst.sst_serve_load(g.ctx, evs, 1000, rate, submitters=4, pollers=2, seed=3, latencies=True)
        assert r["requests"] == 1000 and abs(r["throughput"] - rate) < 0.25 * rate
        lat = r["latency_us"]
        assert lat.size == 1000 and (lat > 0).all()
        assert abs(np.percentile(lat, 99) - r["p99_us"]) <= 1e-6 * r["p99_us"] + 1.0
    finally:
        sst.sst_server_stop(g.ctx)
        g.close()


def test_a_ticket_is_collected_once_by_racing_pollers(served):
    """Several threads poll the same tickets at once: for each ticket exactly one
    gets OK with the oracle's clusters, every other one INVALID_ARG (the result
    is handed out once; the copy out runs outside the server's lock)."""
    import threading
    w, calib, g = served
    events = [eg.make_event(w, calib, 300 + i, occupancy=0.01) for i in range(6)]
    tickets = []
    for e in events:
        code, t = sst.sst_submit(g.ctx, e.raw, e.fed_len)
        assert code == sst.SST_OK
        tickets.append(t)
    got = {t: [] for t in tickets}

    def poller(t, cap):
        try:
            code, info, cl = sst.sst_poll(g.ctx, t, -1, cap)
            got[t].append((code, info.status.n_clusters, cl))
        except sst.SstError as ex:
            got[t].append((ex.code, None, None))

    th = [threading.Thread(target=poller, args=(t, e.nbytes)) for t, e in zip(tickets, events) for _ in range(3)]
    for x in th:
        x.start()
    for x in th:
        x.join(timeout=60)
        assert not x.is_alive()
    for t, e in zip(tickets, events):
        codes = sorted(c for c, _, _ in got[t])
        assert codes == [sst.SST_OK, sst.SST_ERR_INVALID_ARG, sst.SST_ERR_INVALID_ARG], codes
        _, n, cl = next(x for x in got[t] if x[0] == sst.SST_OK)
        _, oc, ost = g.oracle(e.raw, e.fed_len, w.n_feds)
        assert n == ost["n_clusters"]
        assert_clusters_equal(cl, oc)
