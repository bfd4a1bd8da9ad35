"""Local cluster positions on the GPU against the oracle (synthetic pitch per
module; arXiv 2101.11489 section 4: clusters become hits with positions).

The GPU and the oracle evaluate the same two binary32 operations, so given the
same barycenters they must agree bit for bit."""
import numpy as np
import pytest

import eventgen as eg
import oracle as orc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_11489_gb300 as sst  # noqa: E402
from _gpu_util import Gpu  # noqa: E402


def test_local_x_equals_the_oracle_bit_for_bit():
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
    g = Gpu(calib.noise, calib.gain, calib.bad)
    with pytest.raises(sst.SstError):  # no pitch yet
        sst.sst_local_x(g.ctx, torch.zeros(1, dtype=torch.int32, device="cuda"),
                        torch.zeros(1, device="cuda"), 1, torch.zeros(1, device="cuda"))
    pitch = np.random.default_rng(3).uniform(0.008, 0.0205, w.n_feds * 96).astype(np.float32)
    sst.sst_pitch_upload(g.ctx, pitch)
    e = eg.make_event(w, calib, 5)
    _, cl = g.event(e.raw, e.fed_len, w.n_feds)
    n = cl["det"].size
    assert n > 1000
    det = torch.from_numpy(cl["det"].view(np.int32)).cuda()
    bary = torch.from_numpy(cl["barycenter"]).cuda()
    x = torch.empty(n, device="cuda")
    sst.sst_local_x(g.ctx, det, bary, n, x)
    torch.cuda.synchronize()
    want = orc.local_x(cl["det"], cl["barycenter"], pitch)
    assert np.array_equal(x.cpu().numpy().view(np.uint32), want.view(np.uint32))
    # a module id outside the detector has no position
    bad_det = torch.tensor([0, w.n_feds * 96, 5], dtype=torch.int32, device="cuda")
    xb = torch.empty(3, device="cuda")
    sst.sst_local_x(g.ctx, bad_det, torch.full((3,), 130.0, device="cuda"), 3, xb)
    xb = xb.cpu().numpy()
    assert np.isnan(xb[1]) and xb[0] == np.float32(2.0) * pitch[0] and xb[2] == np.float32(2.0) * pitch[5]
    g.close()
