"""Failure detection on the GPU without a fault.

The per-event unpacker's only device wait is the look-back over the FEDs before
each FED (section 2's channel map, built on the device).  Every wait has a poll
limit; when it runs out the kernel flags the event SST_EV_TIMEOUT and finishes.
These tests shorten the limit and keep one FED from publishing its count (a flag
that nothing sets), check that the call returns with the event flagged, and that
the context then works normally again.  Nothing faults, traps or hangs.
"""
import numpy as np
import pytest

import eventgen as eg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_11489_gb300 as sst  # noqa: E402
from _gpu_util import Gpu, assert_digis_equal  # noqa: E402

N_FEDS = 24


@pytest.fixture(scope="module")
def gt():
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(N_FEDS, w.seed, w.p_bad)
    g = Gpu(calib.noise, calib.gain, calib.bad)
    yield w, calib, g
    g.close()


@pytest.mark.parametrize("withhold", [0, 5, N_FEDS - 2])
def test_a_wait_that_runs_out_flags_the_event_and_returns(gt, withhold):
    w, calib, g = gt
    e = eg.make_event(w, calib, 3, n_feds=N_FEDS)
    sst.sst_testing_set_wait(g.ctx, spin_limit=256, withhold_fed=withhold)
    try:
        dh, _ = g.event(e.raw, e.fed_len, N_FEDS)  # returns: the waits give up
    finally:
        sst.sst_testing_set_wait(g.ctx, 0, -1)
    assert dh["flags"] & sst.SST_EV_TIMEOUT
    # the context is usable again, and the same event is exact
    od, _, ost = g.oracle(e.raw, e.fed_len, N_FEDS)
    dh, _ = g.event(e.raw, e.fed_len, N_FEDS)
    assert not dh["flags"] & sst.SST_EV_TIMEOUT
    assert_digis_equal(dh, od)


def test_the_last_fed_withheld_delays_nobody(gt):
    """Only the FEDs after the withheld one wait on it: withholding the last FED
    leaves the event exact."""
    w, calib, g = gt
    e = eg.make_event(w, calib, 4, n_feds=N_FEDS)
    sst.sst_testing_set_wait(g.ctx, spin_limit=256, withhold_fed=N_FEDS - 1)
    try:
        dh, _ = g.event(e.raw, e.fed_len, N_FEDS)
    finally:
        sst.sst_testing_set_wait(g.ctx, 0, -1)
    od, _, _ = g.oracle(e.raw, e.fed_len, N_FEDS)
    assert not dh["flags"] & sst.SST_EV_TIMEOUT
    assert_digis_equal(dh, od)


def test_wait_settings_are_checked(gt):
    _, _, g = gt
    with pytest.raises(sst.SstError):
        sst.sst_testing_set_wait(g.ctx, 1 << 21, -1)
    with pytest.raises(sst.SstError):
        sst.sst_testing_set_wait(g.ctx, 0, -2)
