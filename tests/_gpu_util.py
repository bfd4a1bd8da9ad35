"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and the
oracle on the same seeded inputs, and compare element by element."""
from __future__ import annotations

import numpy as np

import oracle as orc
import paper_2101_11489_gb300 as sst

BARY_TOL = 1e-6  # strip units; digis, statuses, det/first/width/charge are compared exactly


def orc_params(p: sst.sst_params) -> orc.Params:
    return orc.Params(p.t_channel, p.t_seed, p.t_cluster, p.max_seq_holes, p.max_seq_bad, p.max_adj_bad)


class Gpu:
    """One library context with calibration, on cuda:0."""

    def __init__(self, calib_noise, calib_gain, calib_bad, params: sst.sst_params | None = None):
        import torch
        self.torch = torch
        self.params = params or sst.params()
        self.n_feds = calib_noise.size // (96 * 256)
        self.ctx = sst.sst_create(0, self.n_feds)
        sst.sst_calib_upload(self.ctx, calib_noise, calib_gain, calib_bad, self.params)
        self.noise, self.gain, self.bad = calib_noise, calib_gain, calib_bad

    def close(self):
        if self.ctx:
            sst.sst_destroy(self.ctx)
            self.ctx = None

    def event(self, raw: np.ndarray, fed_len: np.ndarray, n_feds: int, digi_cap=None, clu_cap=None):
        torch = self.torch
        raw_t = torch.from_numpy(np.ascontiguousarray(raw, np.uint8)).cuda()
        fl_t = torch.from_numpy(np.ascontiguousarray(fed_len, np.uint32).view(np.int32)).cuda()
        dcap = max(int(raw.size), 1) if digi_cap is None else digi_cap
        ccap = max(int(raw.size) // 2 + 1, 1) if clu_cap is None else clu_cap
        d = sst.DigiBuffers.alloc(dcap, n_feds)
        c = sst.ClusterBuffers.alloc(ccap)
        drec = d.record()
        sst.sst_unpack(self.ctx, raw_t, fl_t, n_feds, drec)
        sst.sst_cluster(self.ctx, drec, n_feds, c.record())
        torch.cuda.synchronize()
        dh = d.to_host()
        ch = c.to_host(0, min(dh["n_clusters"], ccap))
        return dh, ch

    def batch(self, events, clu_caps=None):
        """events: list of (raw, fed_len) with the same n_feds.  Returns per-event
        (status dict, clusters dict)."""
        torch = self.torch
        n_feds = events[0][1].size
        sizes = [int(r.size) for r, _ in events]
        eoff = np.zeros(len(events) + 1, np.uint64)
        eoff[1:] = np.cumsum(sizes)
        caps = [max(s // 2 + 1, 1) for s in sizes] if clu_caps is None else clu_caps
        coff = np.zeros(len(events) + 1, np.uint64)
        coff[1:] = np.cumsum(caps)
        raw = np.concatenate([r for r, _ in events]) if sum(sizes) else np.zeros(16, np.uint8)
        fl = np.concatenate([f for _, f in events]).astype(np.uint32)
        raw_t = torch.from_numpy(raw).cuda()
        eoff_t = torch.from_numpy(eoff.view(np.int64)).cuda()
        fl_t = torch.from_numpy(fl.view(np.int32)).cuda()
        coff_t = torch.from_numpy(coff.view(np.int64)).cuda()
        c = sst.ClusterBuffers.alloc(int(coff[-1]))
        st = torch.zeros(len(events) * 4, dtype=torch.int32, device="cuda")
        sst.sst_batch(self.ctx, raw_t, eoff_t, fl_t, len(events), n_feds, coff_t, c.record(), st)
        torch.cuda.synchronize()
        sth = st.cpu().numpy().view(np.uint32).reshape(-1, 4)
        out = []
        for e in range(len(events)):
            s = {"n_digi": int(sth[e, 0]), "n_clusters": int(sth[e, 1]), "flags": int(sth[e, 2]),
                 "n_bad_channels": int(sth[e, 3])}
            out.append((s, c.to_host(int(coff[e]), min(s["n_clusters"], caps[e]))))
        return out

    def oracle(self, raw, fed_len, n_feds):
        d, c = orc.process_event(raw, fed_len, n_feds, self.noise, self.gain, self.bad, orc_params(self.params))
        flags, nbad = orc.event_status(d["chan_status"])
        return d, c, {"n_digi": int(d["strip"].size), "n_clusters": int(c["det"].size), "flags": flags,
                      "n_bad_channels": nbad}


def assert_digis_equal(g: dict, o: dict):
    assert g["n_digi"] == o["strip"].size
    assert np.array_equal(g["strip"], o["strip"])
    assert np.array_equal(g["adc"], o["adc"])
    assert np.array_equal(g["chan_off"], o["chan_off"])
    assert np.array_equal(g["chan_status"], o["chan_status"])


def assert_clusters_equal(g: dict, o: dict):
    n = o["det"].size
    assert g["det"].size == n, (g["det"].size, n)
    for k in ("det", "first", "width", "charge"):
        assert np.array_equal(g[k], o[k]), k
    assert np.all(np.abs(g["barycenter"].astype(np.float64) - o["barycenter"].astype(np.float64)) <= BARY_TOL)
