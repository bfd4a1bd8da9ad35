"""Optional per-strip cluster amplitudes on the GPU against the oracle.

arXiv 2101.11489 section 2: a kept cluster reports its boundaries, centroid and
optionally its ADC values (here: the gain-corrected charge of every strip of the
cluster, 0 for holes and bad strips).  Clusters, amplitude offsets and amplitudes
are compared exactly, per event and batched, with the default and the gap-rule
parameter sets, on FE units small enough for one tile and on chunked ones, and
with an amplitude capacity too small for the event.
"""
import numpy as np
import pytest

import eventgen as eg
import oracle as orc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_11489_gb300 as sst  # noqa: E402
from _gpu_util import Gpu, assert_clusters_equal, orc_params  # noqa: E402

GAPS = sst.params(max_seq_holes=1, max_seq_bad=2, max_adj_bad=1)


def oracle_amps(g, e, n_feds):
    d, c, st = g.oracle(e.raw, e.fed_len, n_feds)
    af, amp = orc.cluster_amplitudes(d, c, g.noise, g.gain, g.bad, orc_params(g.params))
    return c, st, af, amp


def event_with_amps(g, e, n_feds, amp_cap=None):
    raw = torch.from_numpy(e.raw).cuda()
    fl = torch.from_numpy(e.fed_len.view(np.int32)).cuda()
    d = sst.DigiBuffers.alloc(max(e.nbytes, 1), n_feds)
    cap = e.nbytes // 2 + 1
    cb = sst.ClusterBuffers.alloc(cap, amp_capacity=amp_cap or 4 * e.nbytes)
    drec = d.record()
    sst.sst_unpack(g.ctx, raw, fl, n_feds, drec)
    sst.sst_cluster(g.ctx, drec, n_feds, cb.record())
    torch.cuda.synchronize()
    dh = d.to_host()
    return dh, cb.to_host(0, dh["n_clusters"]), cb.amplitudes()


def check_against_oracle(c_gpu, amp_gpu, c_orc, af_orc, amp_orc, base=0):
    assert_clusters_equal({k: c_gpu[k] for k in ("det", "first", "width", "charge", "barycenter")}, c_orc)
    assert np.array_equal(c_gpu["amp_first"].astype(np.int64) - base, af_orc.astype(np.int64))
    assert np.array_equal(amp_gpu[base:base + amp_orc.size], amp_orc)


@pytest.fixture(scope="module")
def w0():
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(w.n_feds, w.seed, 0.02)  # 2% bad strips: widening and bad gaps happen
    gd = Gpu(calib.noise, calib.gain, calib.bad)
    gg = Gpu(calib.noise, calib.gain, calib.bad, GAPS)
    yield w, calib, gd, gg
    gd.close()
    gg.close()


@pytest.mark.parametrize("which", ["default", "gaps"])
@pytest.mark.parametrize("occ", [0.01, 0.2])
def test_per_event_amplitudes_equal_the_oracle(w0, which, occ):
    w, calib, gd, gg = w0
    g = gd if which == "default" else gg
    e = eg.make_event(w, calib, 11, occupancy=occ)
    c_orc, st_orc, af, amp = oracle_amps(g, e, w.n_feds)
    dh, ch, ah = event_with_amps(g, e, w.n_feds)
    assert dh["n_clusters"] == st_orc["n_clusters"] and dh["flags"] == st_orc["flags"]
    assert amp.size > 1000
    check_against_oracle(ch, ah, c_orc, af, amp)


@pytest.mark.parametrize("which", ["default", "gaps"])
def test_batch_amplitudes_equal_the_oracle(w0, which):
    w, calib, gd, gg = w0
    g = gd if which == "default" else gg
    events = [eg.make_event(w, calib, 20 + i, occupancy=0.005 + 0.02 * (i % 4)) for i in range(6)]
    n = len(events)
    sizes = [e.nbytes for e in events]
    eoff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    coff = np.concatenate([[0], np.cumsum([s // 2 + 1 for s in sizes])]).astype(np.int64)
    aoff = np.concatenate([[0], np.cumsum([4 * s for s in sizes])]).astype(np.int64)
    raw = torch.from_numpy(np.concatenate([e.raw for e in events])).cuda()
    fl = torch.from_numpy(np.concatenate([e.fed_len for e in events]).view(np.int32)).cuda()
    cb = sst.ClusterBuffers.alloc(int(coff[-1]), amp_capacity=int(aoff[-1]))
    cb.amp_off = torch.from_numpy(aoff).cuda()
    st = torch.zeros(n * 4, dtype=torch.int32, device="cuda")
    sst.sst_batch(g.ctx, raw, torch.from_numpy(eoff).cuda(), fl, n, w.n_feds, torch.from_numpy(coff).cuda(),
                  cb.record(), st)
    torch.cuda.synchronize()
    sth = st.cpu().numpy().view(np.uint32).reshape(n, 4)
    amp_all = cb.amplitudes()
    for k, e in enumerate(events):
        c_orc, st_orc, af, amp = oracle_amps(g, e, w.n_feds)
        assert int(sth[k, 1]) == st_orc["n_clusters"] and int(sth[k, 2]) == st_orc["flags"]
        ch = cb.to_host(int(coff[k]), int(sth[k, 1]))
        check_against_oracle(ch, amp_all, c_orc, af, amp, base=int(aoff[k]))


def test_amplitude_capacity_overflow_is_flagged_and_leaves_clusters_whole(w0):
    w, calib, gd, _ = w0
    e = eg.make_event(w, calib, 31, occupancy=0.02)
    c_orc, st_orc, af, amp = oracle_amps(gd, e, w.n_feds)
    cap = amp.size // 3
    dh, ch, ah = event_with_amps(gd, e, w.n_feds, amp_cap=cap)
    assert dh["flags"] & sst.SST_EV_AMP_CAPACITY
    assert dh["n_clusters"] == st_orc["n_clusters"]
    assert_clusters_equal({k: ch[k] for k in ("det", "first", "width", "charge", "barycenter")}, c_orc)
    kept = ch["amp_first"] != sst.NO_AMP
    assert 0 < kept.sum() < kept.size
    width = c_orc["width"].astype(np.int64)
    stored = 0
    for k in np.flatnonzero(kept):
        a = int(ch["amp_first"][k])
        assert a + width[k] <= cap
        assert np.array_equal(ah[a:a + width[k]], amp[af[k]:af[k] + width[k]])
        stored += width[k]
    assert stored <= cap


@pytest.mark.parametrize("chunk", [2, 0])
def test_host_batch_amplitudes_equal_the_oracle(w0, chunk):
    """sst_batch_host with amplitudes: events in host memory, processed in chunks
    (2 events per chunk, or the default plan), each chunk's amp_first made absolute
    and its amplitude slices copied back; every event equals the oracle."""
    w, calib, gd, gg = w0
    events = [eg.make_event(w, calib, 50 + i, occupancy=0.005 + 0.02 * (i % 4)) for i in range(7)]
    n = len(events)
    sizes = [e.nbytes for e in events]
    eoff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    aoff = np.concatenate([[0], np.cumsum([4 * s for s in sizes])]).astype(np.uint64)
    raw = np.concatenate([e.raw for e in events])
    fl = np.concatenate([e.fed_len for e in events]).astype(np.uint32)
    out = sst.HostClusters.alloc(int(sum(s // 2 + 1 for s in sizes)), amp_off=aoff)
    ef = np.zeros(n + 1, np.uint64)
    sth = np.zeros((n, 4), np.uint32)
    keep = sst.sst_get_tune(gd.ctx)
    try:
        sst.sst_set_tune(gd.ctx, host_chunk_events=chunk)
        sst.sst_batch_host(gd.ctx, raw, eoff, fl, n, w.n_feds, out, ef, sth)
    finally:
        sst.sst_set_tune(gd.ctx, **keep)
    for k, e in enumerate(events):
        c_orc, st_orc, af, amp = oracle_amps(gd, e, w.n_feds)
        assert int(sth[k, 1]) == st_orc["n_clusters"] and int(sth[k, 2]) == st_orc["flags"]
        ch = out.view(int(ef[k]), int(sth[k, 1]))
        check_against_oracle(ch, out.amp, c_orc, af, amp, base=int(aoff[k]))


def test_host_batch_rejects_inconsistent_amplitude_slices(w0):
    w, calib, gd, _ = w0
    e = eg.make_event(w, calib, 40)
    eoff = np.array([0, e.nbytes], np.uint64)
    out = sst.HostClusters.alloc(e.nbytes // 2 + 1, amp_off=np.array([0, 64], np.uint64))
    out.amp_off[1] = out.amp.size + 1  # past amp_capacity
    with pytest.raises(sst.SstError) as ei:
        sst.sst_batch_host(gd.ctx, e.raw, eoff, e.fed_len, 1, w.n_feds, out, np.zeros(2, np.uint64),
                           np.zeros(4, np.uint32))
    assert ei.value.code == sst.SST_ERR_INVALID_ARG
