"""Parity at full size on the workloads the throughput figures are quoted on.

The smaller parity tests exercise every code path on inputs the oracle finishes
in seconds; these run the full-detector configurations (440 FEDs x 96 channels x
256 strips) through the same entry points and launch shapes the benchmark times,
and compare with the oracle event by event (arXiv 2101.11489 sections 2 and 3:
the per-event form, many events per launch, and events served as they arrive):

* the single full-detector event, through the host-buffer batch;
* 64 events of occupancy U[0.5%, 4%] in one batched launch with the autotuned
  shape: every event;
* 256 events at 5% occupancy, widths 1-12, 2% bad and 3% saturated strips in one
  launch: a sample of 16 events spread over the batch;
* 64 events of the served mix (lognormal occupancy) submitted to a server with
  the benchmark's options: every event.

Events are generated and the oracle run in a process pool (spawn).
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import eventgen as eg
import oracle as orc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_11489_gb300 as sst  # noqa: E402
from _gpu_util import Gpu, assert_clusters_equal  # noqa: E402

_W = None
_CAL = None


def _init(wid):
    global _W, _CAL
    _W = eg.WORKLOADS[wid]
    _CAL = eg.make_calibration(_W.n_feds, _W.seed, _W.p_bad)


def _gen(ev):
    e = eg.make_event(_W, _CAL, ev)
    return e.raw, e.fed_len


def _oracle(args):
    raw, fl = args
    d, c = orc.process_event(raw, fl, _W.n_feds, _CAL.noise, _CAL.gain, _CAL.bad, orc.Params())
    flags, nbad = orc.event_status(d["chan_status"])
    return c, {"n_digi": int(d["strip"].size), "n_clusters": int(c["det"].size), "flags": flags,
               "n_bad_channels": nbad}


class Workload:
    """Events of one workload and the oracle's answers, computed in a pool."""

    def __init__(self, wid, n_events):
        self.w = eg.WORKLOADS[wid]
        self.calib = eg.make_calibration(self.w.n_feds, self.w.seed, self.w.p_bad)
        self.pool = mp.get_context("spawn").Pool(os.cpu_count() or 1, initializer=_init, initargs=(wid,))
        self.events = self.pool.map(_gen, range(n_events), chunksize=1)

    def oracle(self, idx):
        return self.pool.map(_oracle, [self.events[i] for i in idx], chunksize=1)

    def close(self):
        self.pool.terminate()


def batch_launch(g, events, autotune):
    n = len(events)
    sizes = [r.size for r, _ in events]
    eoff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    coff = np.concatenate([[0], np.cumsum([s // 2 + 1 for s in sizes])]).astype(np.int64)
    raw = torch.from_numpy(np.concatenate([r for r, _ in events])).cuda()
    fl = torch.from_numpy(np.concatenate([f for _, f in events]).astype(np.uint32).view(np.int32)).cuda()
    eo, co = torch.from_numpy(eoff).cuda(), torch.from_numpy(coff).cuda()
    cb = sst.ClusterBuffers.alloc(int(coff[-1]))
    st = torch.zeros(n * 4, dtype=torch.int32, device="cuda")
    if autotune:
        sst.sst_autotune(g.ctx, raw, eo, fl, n, g.n_feds, co, cb.record(), st)
    sst.sst_batch(g.ctx, raw, eo, fl, n, g.n_feds, co, cb.record(), st)
    torch.cuda.synchronize()
    sth = st.cpu().numpy().view(np.uint32).reshape(n, 4)
    return sth, cb, coff


def status_dict(row):
    return {"n_digi": int(row[0]), "n_clusters": int(row[1]), "flags": int(row[2]), "n_bad_channels": int(row[3])}


def test_single_full_event_through_the_host_batch():
    wl = Workload(1, 1)
    try:
        g = Gpu(wl.calib.noise, wl.calib.gain, wl.calib.bad)
        raw, fl = wl.events[0]
        out = sst.HostClusters.alloc(raw.size // 2 + 1)
        first = np.zeros(2, np.uint64)
        status = np.zeros((1, 4), np.uint32)
        sst.sst_batch_host(g.ctx, raw, np.array([0, raw.size], np.uint64), fl.astype(np.uint32), 1, g.n_feds, out,
                           first, status)
        (oc, ost), = wl.oracle([0])
        assert status_dict(status[0]) == ost
        assert ost["n_clusters"] > 40000
        assert_clusters_equal(out.view(0, ost["n_clusters"]), oc)
        g.close()
    finally:
        wl.close()


def test_batch64_every_event_in_the_benchmarked_launch():
    wl = Workload(2, 64)
    try:
        g = Gpu(wl.calib.noise, wl.calib.gain, wl.calib.bad)
        sth, cb, coff = batch_launch(g, wl.events, autotune=True)
        res = wl.oracle(range(64))
        for k, (oc, ost) in enumerate(res):
            assert status_dict(sth[k]) == ost, k
            assert_clusters_equal(cb.to_host(int(coff[k]), int(sth[k, 1])), oc)
        g.close()
    finally:
        wl.close()


def test_batch256_high_occupancy_sampled():
    wl = Workload(3, 256)
    try:
        g = Gpu(wl.calib.noise, wl.calib.gain, wl.calib.bad)
        sth, cb, coff = batch_launch(g, wl.events, autotune=False)
        idx = sorted(set(range(0, 256, 17)) | {255})
        res = wl.oracle(idx)
        for k, (oc, ost) in zip(idx, res):
            assert status_dict(sth[k]) == ost, k
            assert_clusters_equal(cb.to_host(int(coff[k]), int(sth[k, 1])), oc)
        # every event of the batch ran: digis and clusters are counted for all of them
        assert (sth[:, 0] > 0).all() and (sth[:, 1] > 0).all() and (sth[:, 2] == 0).all()
        g.close()
    finally:
        wl.close()


def test_served_mix_every_event_with_the_benchmark_options():
    wl = Workload(4, 64)
    try:
        g = Gpu(wl.calib.noise, wl.calib.gain, wl.calib.bad)
        sst.sst_server_start(g.ctx, 8 << 30, 64, 3, 4096, g.n_feds)
        try:
            tickets = []
            for raw, fl in wl.events:
                code, t = sst.sst_submit(g.ctx, raw, fl)
                assert code == sst.SST_OK
                tickets.append(t)
            res = wl.oracle(range(64))
            for (raw, _), t, (oc, ost) in zip(wl.events, tickets, res):
                code, info, cl = sst.sst_poll(g.ctx, t, -1, raw.size // 2 + 1)
                assert code == sst.SST_OK
                assert status_dict([info.status.n_digi, info.status.n_clusters, info.status.flags,
                                    info.status.n_bad_channels]) == ost
                assert_clusters_equal(cl, oc)
        finally:
            sst.sst_server_stop(g.ctx)
        g.close()
    finally:
        wl.close()


def test_batch64_fed_skew_variant_sampled():
    """The batched configuration with FED payloads differing about 8x (the FED-skew
    stress variant): a sample of the events, both work-item widths."""
    wl = Workload(5, 16)
    try:
        g = Gpu(wl.calib.noise, wl.calib.gain, wl.calib.bad)
        res = wl.oracle(range(16))
        for units in (2, 1):
            sst.sst_set_tune(g.ctx, units_per_warp=units)
            sth, cb, coff = batch_launch(g, wl.events, autotune=False)
            for k, (oc, ost) in enumerate(res):
                assert status_dict(sth[k]) == ost, k
                assert_clusters_equal(cb.to_host(int(coff[k]), int(sth[k, 1])), oc)
        g.close()
    finally:
        wl.close()
