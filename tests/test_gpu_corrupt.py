"""Corrupt raw data on the GPU against the oracle.

Data errors are reported, never fatal: every corrupt channel (bad packet code, run
out of range, overlapping runs, truncated record), every FE unit whose channel
lengths do not chain up, and every FED whose header does not match gets its
status bit, yields no digis, and leaves every other channel alone (the readings
of arXiv 2101.11489 section 2's data format in include/sst.h).  The batched
kernel handles two adjacent FE units per warp, so corruption is placed in the
first and in the second unit of a pair; each corrupt event goes through the
per-event path and the batched path, alone and mixed with the others.
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

N_FEDS = 4


def channel_record_pos(raw, fed_start, ch):
    fe_len = [int(raw[fed_start + 16 + 2 * u]) | (int(raw[fed_start + 17 + 2 * u]) << 8) for u in range(8)]
    u, k = divmod(ch, 12)
    p = fed_start + 32 + sum((l + 7) // 8 * 8 for l in fe_len[:u])
    for _ in range(k):
        p += int(raw[p]) | (int(raw[p + 1]) << 8)
    return p


def runs_of(raw, p):
    ln = int(raw[p]) | (int(raw[p + 1]) << 8)
    out, q = [], p + 3
    while q < p + ln:
        out.append((q, int(raw[q]), int(raw[q + 1])))
        q += 2 + int(raw[q + 1])
    return out


def channel_with(raw, fed_start, channels, cond):
    for ch in channels:
        p = channel_record_pos(raw, fed_start, ch)
        rs = runs_of(raw, p)
        if cond(rs):
            return p, rs
    raise AssertionError("no suitable channel")


def corruptions(raw, fl):
    """(name, raw, fed_len) variants of one event, each with one kind of error."""
    f1 = int(fl[0])  # FED 1 starts here
    out = []
    r = raw.copy()
    p, _ = channel_with(raw, 0, range(0, 12), lambda rs: len(rs) >= 1)  # FE unit 0: first of a pair
    r[p + 2] = 0x11
    out.append(("bad code, first unit of a pair", r, fl))
    r = raw.copy()
    p, _ = channel_with(raw, 0, range(12, 24), lambda rs: len(rs) >= 1)  # FE unit 1: second of the pair
    r[p + 2] = 0x11
    out.append(("bad code, second unit of a pair", r, fl))
    r = raw.copy()
    _, rs = channel_with(raw, f1, range(24, 48), lambda rs: len(rs) >= 1)
    r[rs[0][0] + 1] = 0
    out.append(("zero-width run", r, fl))
    r = raw.copy()
    _, rs = channel_with(raw, f1, range(48, 96), lambda rs: len(rs) >= 2)
    r[rs[1][0]] = rs[0][1]
    out.append(("overlapping runs", r, fl))
    r = raw.copy()
    _, rs = channel_with(raw, 0, range(60, 96), lambda rs: len(rs) >= 1 and rs[-1][1] + rs[-1][2] < 256)
    r[rs[-1][0] + 1] = rs[-1][2] + 1
    out.append(("truncated run", r, fl))
    r = raw.copy()
    p = channel_record_pos(raw, 0, 3 * 12 + 2)  # FE unit 3: second of pair (2, 3)
    r[p] = (int(raw[p]) + 1) & 0xFF
    out.append(("framing, second unit of a pair", r, fl))
    r = raw.copy()
    p = channel_record_pos(raw, f1, 4 * 12 + 5)  # FE unit 4: first of pair (4, 5)
    r[p], r[p + 1] = 2, 0
    out.append(("framing, first unit of a pair", r, fl))
    r = raw.copy()
    r[f1 + 4] ^= 1  # FED 1's id
    out.append(("FED header", r, fl))
    r = raw.copy()
    v = (int(r[16]) | (int(r[17]) << 8)) + 16
    r[16], r[17] = v & 0xFF, v >> 8
    out.append(("FE length inconsistent with FED length", r, fl))
    fl2 = fl.copy()
    fl2[1] = 16
    keep = np.concatenate([raw[:f1 + 16], raw[int(fl[0]) + int(fl[1]):]])
    out.append(("FED length too short for a header", keep, fl2))
    return out


@pytest.fixture(scope="module")
def setup():
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(N_FEDS, w.seed, 0.01)
    g = Gpu(calib.noise, calib.gain, calib.bad)
    e = eg.make_event(w, calib, 2, n_feds=N_FEDS, occupancy=0.03)
    yield g, e
    g.close()


def test_each_corruption_per_event_and_batched(setup):
    g, e = setup
    variants = corruptions(e.raw, e.fed_len)
    for name, raw, fl in variants:
        od, oc, ost = g.oracle(raw, fl, N_FEDS)
        assert ost["flags"] != 0, name
        dh, ch = g.event(raw, fl, N_FEDS)
        assert dh["flags"] == ost["flags"] and dh["n_bad_channels"] == ost["n_bad_channels"], name
        assert_digis_equal(dh, od)
        assert_clusters_equal(ch, oc)
        (st, cl), = g.batch([(raw, fl)])
        assert st == ost, name
        assert_clusters_equal(cl, oc)


def test_corrupt_events_mixed_in_one_batch(setup):
    g, e = setup
    variants = corruptions(e.raw, e.fed_len)
    batch = [(e.raw, e.fed_len)] + [(r, f) for _, r, f in variants] + [(e.raw, e.fed_len)]
    out = g.batch(batch)
    for (raw, fl), (st, cl) in zip(batch, out):
        _, oc, ost = g.oracle(raw, fl, N_FEDS)
        assert st == ost
        assert_clusters_equal(cl, oc)


def test_corrupt_events_through_host_batches(setup):
    """The same mix through sst_batch_host: statuses are copied back on their own
    stream and must still match event by event."""
    g, e = setup
    events = [(e.raw, e.fed_len)] + [(r, f) for _, r, f in corruptions(e.raw, e.fed_len)]
    raw = np.concatenate([r for r, _ in events])
    eoff = np.zeros(len(events) + 1, np.uint64)
    eoff[1:] = np.cumsum([r.size for r, _ in events])
    fl = np.concatenate([f for _, f in events]).astype(np.uint32)
    out = sst.HostClusters.alloc(int(raw.size // 2 + len(events)), pinned=True)
    first = np.zeros(len(events) + 1, np.uint64)
    status = np.zeros((len(events), 4), np.uint32)
    sst.sst_batch_host(g.ctx, raw, eoff, fl, len(events), N_FEDS, out, first, status)
    for k, (r, f) in enumerate(events):
        _, oc, ost = g.oracle(r, f, N_FEDS)
        assert {"n_digi": int(status[k, 0]), "n_clusters": int(status[k, 1]), "flags": int(status[k, 2]),
                "n_bad_channels": int(status[k, 3])} == ost, k
        assert_clusters_equal(out.view(int(first[k]), ost["n_clusters"]), oc)
