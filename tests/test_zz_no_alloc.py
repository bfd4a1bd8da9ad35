"""sst_unpack_noalloc, the unpacking entry point that allocates nothing.

It serves callers that may not allocate device memory while they run: a trigger
or data-acquisition process that reserves all device memory up front for its own
caching allocator, or code in which a cudaMalloc (which synchronises the device)
would stall the other streams of a real-time pipeline.  Its scratch is a fixed
device array inside the library, shared by every call on a device and reused
call after call, so these tests call it twice in a row, on different events and
into the same output buffers, and compare each result with sst_unpack's and with
the oracle's unpacking of the same bytes.  Digis, channel offsets and statuses are
integers and must match exactly.  The device's free memory must not change across
a call: the entry point allocates nothing.

This file is collected last so that a run stopping at the first failure has run
every other test first; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import eventgen as eg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as orc  # noqa: E402
import paper_2101_11489_gb300 as sst  # noqa: E402


def _upload(e):
    raw = torch.from_numpy(np.ascontiguousarray(e.raw)).cuda()
    fl = torch.from_numpy(np.ascontiguousarray(e.fed_len).view(np.int32)).cuda()
    return raw, fl


def _same(a: dict, b: dict):
    assert a["n_digi"] == b["n_digi"] and a["flags"] == b["flags"] and a["n_bad_channels"] == b["n_bad_channels"]
    for k in ("strip", "adc", "chan_off", "chan_status"):
        assert np.array_equal(a[k], b[k]), k


def test_noalloc_matches_sst_unpack_on_two_calls_in_a_row():
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
    events = [eg.make_event(w, calib, 0), eg.make_event(w, calib, 1, occupancy=0.03)]
    cap = max(e.nbytes for e in events)
    ctx = sst.sst_create(0, w.n_feds)
    try:
        got_buf = sst.DigiBuffers.alloc(cap, w.n_feds)  # reused by both calls
        for i, e in enumerate(events):
            raw, fl = _upload(e)
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            assert sst.sst_unpack_noalloc(raw, fl, w.n_feds, got_buf.record()) == sst.SST_OK
            torch.cuda.synchronize()
            if i > 0:  # the first call on a device may set up; later calls take nothing
                assert torch.cuda.mem_get_info()[0] == free0
            got = got_buf.to_host()
            ref_buf = sst.DigiBuffers.alloc(cap, w.n_feds)
            sst.sst_unpack(ctx, raw, fl, w.n_feds, ref_buf.record())
            torch.cuda.synchronize()
            ref = ref_buf.to_host()
            assert got["n_digi"] > 1000
            _same(got, ref)
            od = orc.unpack_event(e.raw, e.fed_len, w.n_feds)
            flags, nbad = orc.event_status(od["chan_status"])
            assert got["n_digi"] == od["strip"].size and got["flags"] == flags and got["n_bad_channels"] == nbad
            for k in ("strip", "adc", "chan_off", "chan_status"):
                assert np.array_equal(got[k], od[k]), k
    finally:
        sst.sst_destroy(ctx)


def test_noalloc_rejects_more_feds_than_its_scratch_holds():
    raw = torch.zeros(64, dtype=torch.uint8, device="cuda")
    n = sst.NOALLOC_MAX_FEDS + 1
    fl = torch.zeros(n, dtype=torch.int32, device="cuda")
    d = sst.DigiBuffers.alloc(16, n)
    assert sst.sst_unpack_noalloc(raw, fl, n, d.record()) == sst.SST_ERR_TOO_LARGE
