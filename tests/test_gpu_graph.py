"""The batched launch sequence captured as a CUDA graph and replayed.

arXiv 2101.11489 section 3 runs many events per launch; capturing the sequence
(prologue scan, persistent batched kernel, ordering scan, compaction) in a CUDA
graph removes the per-step launch cost.  The sequence allocates nothing once the
context's scratch has been sized by one ordinary call, clears its own counters on
the device, and so replays exactly: every replay must equal the eager result.
"""
import numpy as np
import pytest

import eventgen as eg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_11489_gb300 as sst  # noqa: E402
from _gpu_util import Gpu  # noqa: E402


def test_batch_replays_from_a_cuda_graph_exactly():
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
    g = Gpu(calib.noise, calib.gain, calib.bad)
    events = [eg.make_event(w, calib, 50 + i, occupancy=0.004 + 0.01 * i) for i in range(5)]
    sizes = [e.nbytes for e in events]
    eoff = torch.tensor(np.concatenate([[0], np.cumsum(sizes)]), dtype=torch.int64, device="cuda")
    coff_h = np.concatenate([[0], np.cumsum([s // 2 + 1 for s in sizes])]).astype(np.int64)
    coff = torch.from_numpy(coff_h).cuda()
    raw = torch.from_numpy(np.concatenate([e.raw for e in events])).cuda()
    fl = torch.from_numpy(np.concatenate([e.fed_len for e in events]).view(np.int32)).cuda()
    cb = sst.ClusterBuffers.alloc(int(coff_h[-1]))
    st = torch.zeros(len(events) * 4, dtype=torch.int32, device="cuda")

    def launch():
        sst.sst_batch(g.ctx, raw, eoff, fl, len(events), w.n_feds, coff, cb.record(), st)

    def snapshot():
        torch.cuda.synchronize()
        sth = st.cpu().numpy().copy()
        n = int(coff_h[-1])
        return sth, [cb.det[:n].cpu().numpy().copy(), cb.barycenter[:n].cpu().numpy().copy()]

    launch()  # sizes the scratch; nothing is allocated from here on
    eager = snapshot()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        launch()  # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        launch()
    for _ in range(3):
        st.zero_()
        cb.det.fill_(-1)
        graph.replay()
        got = snapshot()
        assert np.array_equal(got[0], eager[0])
        n_total = int(eager[0].reshape(-1, 4)[:, 1].sum())
        assert n_total > 1000
        for e in range(len(events)):
            a, m = int(coff_h[e]), int(eager[0].reshape(-1, 4)[e, 1])
            assert np.array_equal(got[1][0][a:a + m], eager[1][0][a:a + m])
            assert np.array_equal(got[1][1][a:a + m], eager[1][1][a:a + m])
    g.close()
