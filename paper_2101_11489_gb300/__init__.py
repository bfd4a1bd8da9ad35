"""Python binding of the GB300 silicon-strip unpacking and clustering library.

The library (``_lib/libsst.so``, built from ``csrc/`` by ``_build.py``) implements
the hot path of arXiv 2101.11489: unpacking zero-suppressed FED raw data into a
digi structure-of-arrays and three-threshold clustering (section 2), per event,
batched and served (section 3).  Its C ABI is ``include/sst.h``.

This module only marshals arguments: PyTorch tensors supply device memory (their
``data_ptr()``) and streams (``torch.cuda.current_stream().cuda_stream``); every
step of the path runs in the library's CUDA kernels.  There is no CPU fallback: if
the library is missing or fails to load, importing the functions raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsst.so")

CH_PER_FED = 96
STRIPS_PER_CH = 256
STRIPS_PER_APV = 128

SST_OK = 0
SST_ERR_INVALID_ARG = 1
SST_ERR_NO_CALIB = 2
SST_ERR_BUDGET = 3
SST_ERR_TOO_LARGE = 4
SST_ERR_BUSY = 5
SST_ERR_NOT_READY = 6
SST_ERR_TIMEOUT = 7
SST_ERR_CUDA = 8
SST_ERR_STATE = 9

SST_CH_FED_HDR = 0x01
SST_CH_FRAMING = 0x02
SST_CH_BAD_CODE = 0x04
SST_CH_RUN_RANGE = 0x08
SST_CH_RUN_ORDER = 0x10
SST_CH_TRUNC = 0x20
SST_EV_DIGI_CAPACITY = 0x100
SST_EV_CLUSTER_CAPACITY = 0x200
SST_EV_TIMEOUT = 0x400
SST_EV_SIZE = 0x800
SST_EV_AMP_CAPACITY = 0x1000
NO_AMP = 0xFFFFFFFF  # amp_first of a cluster whose amplitudes did not fit


class SstError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sst error {code}: {msg}")
        self.code = code


class sst_params(ctypes.Structure):
    _fields_ = [("t_channel", ctypes.c_float), ("t_seed", ctypes.c_float), ("t_cluster", ctypes.c_float),
                ("max_seq_holes", ctypes.c_uint8), ("max_seq_bad", ctypes.c_uint8), ("max_adj_bad", ctypes.c_uint8),
                ("reserved", ctypes.c_uint8)]


class sst_event_status(ctypes.Structure):
    _fields_ = [("n_digi", ctypes.c_uint32), ("n_clusters", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("n_bad_channels", ctypes.c_uint32)]


class sst_digis(ctypes.Structure):
    _fields_ = [("strip", ctypes.c_void_p), ("adc", ctypes.c_void_p), ("chan_off", ctypes.c_void_p),
                ("chan_status", ctypes.c_void_p), ("status", ctypes.c_void_p), ("capacity", ctypes.c_uint64)]


class sst_clusters(ctypes.Structure):
    _fields_ = [("det", ctypes.c_void_p), ("first", ctypes.c_void_p), ("width", ctypes.c_void_p),
                ("charge", ctypes.c_void_p), ("barycenter", ctypes.c_void_p), ("capacity", ctypes.c_uint64),
                ("amp", ctypes.c_void_p), ("amp_first", ctypes.c_void_p), ("amp_off", ctypes.c_void_p),
                ("amp_capacity", ctypes.c_uint64)]


class sst_tune(ctypes.Structure):
    _fields_ = [("block", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32), ("units_per_warp", ctypes.c_uint32),
                ("host_chunk_events", ctypes.c_uint32), ("tile_digis", ctypes.c_uint32),
                ("lanes_per_channel", ctypes.c_uint32)]


class sst_launch_info(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_uint32), ("block", ctypes.c_uint32), ("smem_bytes", ctypes.c_uint32),
                ("items_per_fed", ctypes.c_uint32), ("host_chunks", ctypes.c_uint32)]


class sst_server_opts(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_uint64), ("max_batch_events", ctypes.c_uint32),
                ("max_inflight", ctypes.c_uint32), ("max_requests", ctypes.c_uint32), ("n_feds", ctypes.c_uint32),
                ("zero_copy", ctypes.c_uint32)]


class sst_load_result(ctypes.Structure):
    _fields_ = [("offered_rate", ctypes.c_double), ("throughput", ctypes.c_double), ("p50_us", ctypes.c_double),
                ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double), ("max_us", ctypes.c_double),
                ("p50_admitted_us", ctypes.c_double), ("p99_admitted_us", ctypes.c_double),
                ("requests", ctypes.c_uint64), ("retries", ctypes.c_uint64)]


class sst_result_info(ctypes.Structure):
    _fields_ = [("status", sst_event_status), ("t_submit_us", ctypes.c_double), ("t_done_us", ctypes.c_double)]


_lib = None


def load_library():
    """Loads libsst.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not built; run __graft_entry__.build() or python -m {__name__}._build")
    lib = ctypes.CDLL(LIB_PATH)
    vp, u32, u64, i32, i64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64
    P = ctypes.POINTER
    sigs = {
        "sst_create": ([P(vp), ctypes.c_int, u32], i32),
        "sst_destroy": ([vp], i32),
        "sst_last_error": ([vp], ctypes.c_char_p),
        "sst_calib_upload": ([vp, vp, vp, vp, P(sst_params), vp], i32),
        "sst_unpack": ([vp, vp, u64, vp, u32, P(sst_digis), vp], i32),
        "sst_unpack_noalloc": ([vp, u64, vp, u32, P(sst_digis), vp], i32),
        "sst_cluster": ([vp, P(sst_digis), u32, P(sst_clusters), vp], i32),
        "sst_batch": ([vp, vp, vp, vp, u32, u32, vp, P(sst_clusters), vp, vp], i32),
        "sst_batch_host": ([vp, vp, vp, vp, u32, u32, P(sst_clusters), vp, vp], i32),
        "sst_batch_host_submit": ([vp, vp, vp, vp, u32, u32, P(sst_clusters), vp, vp, P(u64)], i32),
        "sst_batch_host_wait": ([vp, u64], i32),
        "sst_pitch_upload": ([vp, vp], i32),
        "sst_local_x": ([vp, vp, vp, u64, vp, vp], i32),
        "sst_set_tune": ([vp, P(sst_tune)], i32),
        "sst_get_tune": ([vp, P(sst_tune)], i32),
        "sst_autotune": ([vp, vp, vp, vp, u32, u32, vp, P(sst_clusters), vp, vp, P(sst_tune), P(ctypes.c_float)], i32),
        "sst_autotune_host": ([vp, vp, vp, vp, u32, u32, P(sst_clusters), vp, vp, P(u32), P(ctypes.c_float)], i32),
        "sst_get_launch_info": ([vp, u32, u32, P(sst_launch_info)], i32),
        "sst_profile_enable": ([vp, ctypes.c_int], i32),
        "sst_testing_set_wait": ([vp, u32, ctypes.c_int32], i32),
        "sst_profile_read": ([vp, P(u64), P(ctypes.c_double), ctypes.c_int], i32),
        "sst_server_start": ([vp, P(sst_server_opts)], i32),
        "sst_server_stop": ([vp], i32),
        "sst_submit": ([vp, vp, u64, vp, P(u64)], i32),
        "sst_poll": ([vp, u64, i64, P(sst_result_info), vp, vp, vp, vp, vp, u64], i32),
        "sst_serve_load": ([vp, vp, vp, vp, u32, u64, ctypes.c_double, u32, u32, u64, vp, P(sst_load_result)], i32),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    return ["sst_create", "sst_destroy", "sst_last_error", "sst_calib_upload", "sst_unpack", "sst_unpack_noalloc",
            "sst_cluster",
            "sst_batch", "sst_batch_host", "sst_batch_host_submit", "sst_batch_host_wait", "sst_pitch_upload", "sst_local_x", "sst_set_tune", "sst_get_tune", "sst_autotune", "sst_autotune_host", "sst_get_launch_info", "sst_profile_enable", "sst_profile_read", "sst_testing_set_wait",
            "sst_server_start", "sst_server_stop",
            "sst_submit", "sst_poll", "sst_serve_load"]


def _check(ctx, code: int, what: str):
    if code != SST_OK:
        msg = load_library().sst_last_error(ctx).decode(errors="replace") if ctx else what
        raise SstError(code, f"{what}: {msg}")


def _dp(t) -> int:
    """Device pointer of a CUDA tensor (no copy; must be contiguous)."""
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return t.data_ptr()


def _hp(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _stream(stream) -> int:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


# ---------------------------------------------------------------- C-ABI wrappers

def sst_create(device: int, n_feds: int) -> int:
    lib = load_library()
    h = ctypes.c_void_p()
    code = lib.sst_create(ctypes.byref(h), device, n_feds)
    if code != SST_OK:
        raise SstError(code, "sst_create failed")
    return h.value


def sst_destroy(ctx: int) -> None:
    _check(None, load_library().sst_destroy(ctx), "sst_destroy")


def sst_last_error(ctx: int) -> str:
    return load_library().sst_last_error(ctx).decode(errors="replace")


def sst_calib_upload(ctx: int, noise: np.ndarray, gain: np.ndarray, bad: np.ndarray, params: sst_params,
                     stream=None) -> None:
    noise = np.ascontiguousarray(noise, dtype=np.float32)
    gain = np.ascontiguousarray(gain, dtype=np.float32)
    bad = np.ascontiguousarray(bad, dtype=np.uint8)
    code = load_library().sst_calib_upload(ctx, _hp(noise), _hp(gain), _hp(bad), ctypes.byref(params),
                                           _stream(stream))
    _check(ctx, code, "sst_calib_upload")


def sst_unpack(ctx: int, raw, fed_len, n_feds: int, digis: sst_digis, stream=None) -> None:
    code = load_library().sst_unpack(ctx, _dp(raw), raw.numel(), _dp(fed_len), n_feds, ctypes.byref(digis),
                                     _stream(stream))
    _check(ctx, code, "sst_unpack")


def sst_unpack_noalloc(raw, fed_len, n_feds: int, digis: sst_digis, stream=None) -> int:
    """Unpacks like sst_unpack without a context and without allocating; returns
    the status code (SST_OK, SST_ERR_TOO_LARGE, ...) instead of raising."""
    return load_library().sst_unpack_noalloc(_dp(raw), raw.numel(), _dp(fed_len), n_feds, ctypes.byref(digis),
                                             _stream(stream))


NOALLOC_MAX_FEDS = 1024


def sst_cluster(ctx: int, digis: sst_digis, n_feds: int, clusters: sst_clusters, stream=None) -> None:
    code = load_library().sst_cluster(ctx, ctypes.byref(digis), n_feds, ctypes.byref(clusters), _stream(stream))
    _check(ctx, code, "sst_cluster")


def sst_batch(ctx: int, raw, event_off, fed_len, n_events: int, n_feds: int, clu_off, clusters: sst_clusters,
              status, stream=None) -> None:
    code = load_library().sst_batch(ctx, _dp(raw), _dp(event_off), _dp(fed_len), n_events, n_feds, _dp(clu_off),
                                    ctypes.byref(clusters), _dp(status), _stream(stream))
    _check(ctx, code, "sst_batch")


def sst_batch_host(ctx: int, raw: np.ndarray, event_off: np.ndarray, fed_len: np.ndarray, n_events: int,
                   n_feds: int, out: "HostClusters", event_first: np.ndarray, status: np.ndarray) -> None:
    """Host-memory batch: raw (uint8), event_off (uint64, n_events + 1), fed_len
    (uint32, n_events x n_feds) are read; out, event_first (uint64, n_events + 1)
    and status (uint32, n_events x 4) are written.  Synchronous."""
    for a, dt in ((raw, np.uint8), (event_off, np.uint64), (fed_len, np.uint32), (event_first, np.uint64),
                  (status, np.uint32)):
        assert a.dtype == dt and a.flags["C_CONTIGUOUS"], "sst_batch_host: wrong dtype or layout"
    assert event_off.size >= n_events + 1 and event_first.size >= n_events + 1 and status.size >= 4 * n_events
    assert fed_len.size >= n_events * n_feds and raw.size >= int(event_off[n_events])
    code = load_library().sst_batch_host(ctx, _hp(raw), _hp(event_off), _hp(fed_len), n_events, n_feds,
                                         ctypes.byref(out.record()), _hp(event_first), _hp(status))
    _check(ctx, code, "sst_batch_host")


def sst_batch_host_submit(ctx: int, raw: np.ndarray, event_off: np.ndarray, fed_len: np.ndarray, n_events: int,
                          n_feds: int, out: "HostClusters", event_first: np.ndarray, status: np.ndarray) -> int:
    """Queues a host-memory batch; returns its ticket.  The arrays belong to the
    library until sst_batch_host_wait(ticket) returns."""
    for a, dt in ((raw, np.uint8), (event_off, np.uint64), (fed_len, np.uint32), (event_first, np.uint64),
                  (status, np.uint32)):
        assert a.dtype == dt and a.flags["C_CONTIGUOUS"], "sst_batch_host_submit: wrong dtype or layout"
    assert event_off.size >= n_events + 1 and event_first.size >= n_events + 1 and status.size >= 4 * n_events
    assert fed_len.size >= n_events * n_feds and raw.size >= int(event_off[n_events])
    t = ctypes.c_uint64()
    code = load_library().sst_batch_host_submit(ctx, _hp(raw), _hp(event_off), _hp(fed_len), n_events, n_feds,
                                                ctypes.byref(out.record()), _hp(event_first), _hp(status),
                                                ctypes.byref(t))
    _check(ctx, code, "sst_batch_host_submit")
    return t.value


def sst_batch_host_wait(ctx: int, ticket: int) -> None:
    _check(ctx, load_library().sst_batch_host_wait(ctx, ticket), "sst_batch_host_wait")


def sst_pitch_upload(ctx: int, pitch: np.ndarray) -> None:
    """Strip pitch of every module (n_feds * 96 floats, host)."""
    pitch = np.ascontiguousarray(pitch, dtype=np.float32)
    _check(ctx, load_library().sst_pitch_upload(ctx, _hp(pitch)), "sst_pitch_upload")


def sst_local_x(ctx: int, det, barycenter, n: int, x, stream=None) -> None:
    """Local x of n clusters (device tensors det, barycenter -> x)."""
    _check(ctx, load_library().sst_local_x(ctx, _dp(det), _dp(barycenter), n, _dp(x), _stream(stream)),
           "sst_local_x")


TUNE_KEYS = ("block", "ctas_per_sm", "units_per_warp", "host_chunk_events", "tile_digis", "lanes_per_channel")


def _tune_dict(t: sst_tune) -> dict:
    return {k: int(getattr(t, k)) for k in TUNE_KEYS}


def sst_set_tune(ctx: int, **knobs) -> None:
    """Sets the given knobs (names as in sst_tune); the others keep their values."""
    cur = sst_get_tune(ctx)
    unknown = set(knobs) - set(TUNE_KEYS)
    if unknown:
        raise TypeError(f"unknown tune knobs {sorted(unknown)}")
    cur.update(knobs)
    t = sst_tune(*[cur[k] for k in TUNE_KEYS])
    _check(ctx, load_library().sst_set_tune(ctx, ctypes.byref(t)), "sst_set_tune")


def sst_get_tune(ctx: int) -> dict:
    t = sst_tune()
    _check(ctx, load_library().sst_get_tune(ctx, ctypes.byref(t)), "sst_get_tune")
    return _tune_dict(t)


def sst_autotune(ctx: int, raw, event_off, fed_len, n_events: int, n_feds: int, clu_off, clusters: sst_clusters,
                 status, stream=None) -> tuple[dict, float]:
    """Times the batched kernel's launch shapes on this batch; keeps and returns the fastest and its time (us)."""
    t = sst_tune()
    us = ctypes.c_float()
    code = load_library().sst_autotune(ctx, _dp(raw), _dp(event_off), _dp(fed_len), n_events, n_feds,
                                       _dp(clu_off), ctypes.byref(clusters), _dp(status), _stream(stream),
                                       ctypes.byref(t), ctypes.byref(us))
    _check(ctx, code, "sst_autotune")
    return _tune_dict(t), us.value


def sst_autotune_host(ctx: int, raw: np.ndarray, event_off: np.ndarray, fed_len: np.ndarray, n_events: int,
                      n_feds: int, clusters: "HostClusters", event_first: np.ndarray, status: np.ndarray
                      ) -> tuple[int, float]:
    """Times sst_batch_host over events per chunk on this host batch; keeps and returns the fastest chunk
    size and its wall time per call (us)."""
    best = ctypes.c_uint32()
    us = ctypes.c_float()
    code = load_library().sst_autotune_host(ctx, _hp(raw), _hp(event_off), _hp(fed_len), n_events, n_feds,
                                            ctypes.byref(clusters.record()), _hp(event_first), _hp(status),
                                            ctypes.byref(best), ctypes.byref(us))
    _check(ctx, code, "sst_autotune_host")
    return best.value, us.value


def sst_get_launch_info(ctx: int, n_events: int, n_feds: int) -> dict:
    """The batched kernel's grid, block, shared memory per CTA, work items per FED, and the host path's chunk
    count for a batch of this size under the context's knobs."""
    info = sst_launch_info()
    _check(ctx, load_library().sst_get_launch_info(ctx, n_events, n_feds, ctypes.byref(info)), "sst_get_launch_info")
    return {k: int(getattr(info, k)) for k, _ in sst_launch_info._fields_}


def save_tune(tune: dict, path: str, workload: str, extra: dict | None = None) -> None:
    """Writes a tune (as sst_get_tune returns it) for a workload to a JSON file."""
    import json
    rec = {"workload": workload, "tune": {k: int(tune[k]) for k in TUNE_KEYS}}
    if extra:
        rec.update(extra)
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)


def load_tune(path: str, workload: str) -> dict | None:
    """The tune stored for `workload` in a JSON file written by save_tune, or None."""
    import json
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("workload") != workload or set(rec.get("tune", {})) != set(TUNE_KEYS):
        return None
    return {k: int(rec["tune"][k]) for k in TUNE_KEYS}


def sst_testing_set_wait(ctx: int, spin_limit: int = 0, withhold_fed: int = -1) -> None:
    """Failure tests: polls before a look-back wait gives up (0: default) and a FED
    that never publishes its count (-1: none)."""
    _check(ctx, load_library().sst_testing_set_wait(ctx, spin_limit, withhold_fed), "sst_testing_set_wait")


def sst_profile_enable(ctx: int, enable: bool = True) -> None:
    _check(ctx, load_library().sst_profile_enable(ctx, 1 if enable else 0), "sst_profile_enable")


def sst_profile_read(ctx: int, reset: bool = True) -> tuple[int, float]:
    """(launches, summed device milliseconds) of the batched kernel since the last reset."""
    n = ctypes.c_uint64()
    ms = ctypes.c_double()
    _check(ctx, load_library().sst_profile_read(ctx, ctypes.byref(n), ctypes.byref(ms), 1 if reset else 0),
           "sst_profile_read")
    return n.value, ms.value


def sst_server_start(ctx: int, mem_budget_bytes: int, max_batch_events: int, max_inflight: int, max_requests: int,
                     n_feds: int, zero_copy=False) -> None:
    """zero_copy: False / 0 copies each event at submission; True / 1 lends the
    caller's buffer (copied to the device from there); "in_place" / 2 lends a
    pinned buffer that the kernels read directly.  A lent buffer must stay alive
    and unchanged until sst_poll returns for the ticket."""
    zc = 2 if zero_copy == "in_place" else int(zero_copy)
    o = sst_server_opts(mem_budget_bytes, max_batch_events, max_inflight, max_requests, n_feds, zc)
    _check(ctx, load_library().sst_server_start(ctx, ctypes.byref(o)), "sst_server_start")


def sst_server_stop(ctx: int) -> None:
    _check(ctx, load_library().sst_server_stop(ctx), "sst_server_stop")


def sst_submit(ctx: int, raw: np.ndarray, fed_len: np.ndarray) -> tuple[int, int]:
    """Returns (status code, ticket); the admission outcomes BUSY, BUDGET and
    TOO_LARGE are returned, not raised."""
    raw = np.ascontiguousarray(raw, dtype=np.uint8)
    fed_len = np.ascontiguousarray(fed_len, dtype=np.uint32)
    t = ctypes.c_uint64()
    code = load_library().sst_submit(ctx, _hp(raw), raw.size, _hp(fed_len), ctypes.byref(t))
    if code not in (SST_OK, SST_ERR_BUSY, SST_ERR_BUDGET, SST_ERR_TOO_LARGE):
        _check(ctx, code, "sst_submit")
    return code, t.value


def sst_serve_load(ctx: int, events, n_requests: int, rate: float, submitters: int = 8, pollers: int = 2,
                   seed: int = 1, latencies: bool = False):
    """The native Poisson client on the running server: events = [(raw u8, fed_len u32)] in host memory
    (request i is event i mod len(events)); rate in events/s, 0 = saturating.  Returns a dict of the
    sst_load_result fields (and the per-request latencies in microseconds when asked)."""
    n = len(events)
    raws = (ctypes.c_void_p * n)(*[_hp(r) for r, _ in events])
    sizes = (ctypes.c_uint64 * n)(*[int(r.size) for r, _ in events])
    fls = (ctypes.c_void_p * n)(*[_hp(np.ascontiguousarray(f)) for _, f in events])
    for _, f in events:
        assert f.dtype == np.uint32 and f.flags["C_CONTIGUOUS"], "fed_len must be contiguous uint32"
    lat = np.zeros(n_requests, np.float64) if latencies else None
    out = sst_load_result()
    code = load_library().sst_serve_load(ctx, raws, sizes, fls, n, n_requests, float(rate), submitters, pollers,
                                         seed, _hp(lat) if lat is not None else None, ctypes.byref(out))
    _check(ctx, code, "sst_serve_load")
    res = {k: getattr(out, k) for k, _ in sst_load_result._fields_}
    if lat is not None:
        res["latency_us"] = lat
    return res


def sst_poll(ctx: int, ticket: int, timeout_us: int, capacity: int = 0):
    """Returns (status code, info, clusters dict or None); NOT_READY is returned."""
    info = sst_result_info()
    arrs = {"det": np.zeros(capacity, np.uint32), "first": np.zeros(capacity, np.uint16),
            "width": np.zeros(capacity, np.uint16), "charge": np.zeros(capacity, np.uint32),
            "barycenter": np.zeros(capacity, np.float32)}
    ptrs = [(_hp(arrs[k]) if capacity else None) for k in ("det", "first", "width", "charge", "barycenter")]
    code = load_library().sst_poll(ctx, ticket, timeout_us, ctypes.byref(info), *ptrs, capacity)
    if code == SST_ERR_NOT_READY:
        return code, info, None
    _check(ctx, code, "sst_poll")
    n = min(info.status.n_clusters, capacity)
    return code, info, {k: v[:n] for k, v in arrs.items()}


# ---------------------------------------------------------------- tensor helpers

@dataclass
class DigiBuffers:
    """Device tensors behind an sst_digis record."""
    strip: object
    adc: object
    chan_off: object
    chan_status: object
    status: object

    @classmethod
    def alloc(cls, capacity: int, n_feds: int, device="cuda"):
        import torch
        return cls(torch.empty(max(capacity, 1), dtype=torch.int32, device=device),
                   torch.empty(max(capacity, 1), dtype=torch.uint8, device=device),
                   torch.empty(n_feds * CH_PER_FED + 1, dtype=torch.int32, device=device),
                   torch.empty(n_feds * CH_PER_FED, dtype=torch.uint8, device=device),
                   torch.zeros(4, dtype=torch.int32, device=device))

    def record(self) -> sst_digis:
        return sst_digis(_dp(self.strip), _dp(self.adc), _dp(self.chan_off), _dp(self.chan_status), _dp(self.status),
                         self.strip.numel())

    def to_host(self) -> dict:
        st = self.status.cpu().numpy().view(np.uint32)
        n = int(st[0])
        return {"strip": self.strip[:n].cpu().numpy().view(np.uint32).copy(),
                "adc": self.adc[:n].cpu().numpy().copy(),
                "chan_off": self.chan_off.cpu().numpy().view(np.uint32).copy(),
                "chan_status": self.chan_status.cpu().numpy().copy(),
                "n_digi": n, "n_clusters": int(st[1]), "flags": int(st[2]), "n_bad_channels": int(st[3])}


@dataclass
class ClusterBuffers:
    """Device tensors behind an sst_clusters record (int32 / int16 tensors hold the
    unsigned fields bit for bit), with optional amplitude arrays (amp u8,
    amp_first u32 per cluster; amp_off, device u64 per event + 1, for sst_batch)."""
    det: object
    first: object
    width: object
    charge: object
    barycenter: object
    amp: object = None
    amp_first: object = None
    amp_off: object = None

    @classmethod
    def alloc(cls, capacity: int, device="cuda", amp_capacity: int = 0):
        import torch
        c = max(capacity, 1)
        b = cls(torch.empty(c, dtype=torch.int32, device=device), torch.empty(c, dtype=torch.int16, device=device),
                torch.empty(c, dtype=torch.int16, device=device), torch.empty(c, dtype=torch.int32, device=device),
                torch.empty(c, dtype=torch.float32, device=device))
        if amp_capacity > 0:
            b.amp = torch.empty(amp_capacity, dtype=torch.uint8, device=device)
            b.amp_first = torch.empty(c, dtype=torch.int32, device=device)
        return b

    def record(self) -> sst_clusters:
        amp = self.amp is not None
        return sst_clusters(_dp(self.det), _dp(self.first), _dp(self.width), _dp(self.charge), _dp(self.barycenter),
                            self.det.numel(), _dp(self.amp) if amp else None, _dp(self.amp_first) if amp else None,
                            _dp(self.amp_off) if amp and self.amp_off is not None else None,
                            self.amp.numel() if amp else 0)

    def to_host(self, start: int = 0, n: int | None = None) -> dict:
        end = self.det.numel() if n is None else start + n
        h = {"det": self.det[start:end].cpu().numpy().view(np.uint32).copy(),
             "first": self.first[start:end].cpu().numpy().view(np.uint16).copy(),
             "width": self.width[start:end].cpu().numpy().view(np.uint16).copy(),
             "charge": self.charge[start:end].cpu().numpy().view(np.uint32).copy(),
             "barycenter": self.barycenter[start:end].cpu().numpy().copy()}
        if self.amp is not None:
            h["amp_first"] = self.amp_first[start:end].cpu().numpy().view(np.uint32).copy()
        return h

    def amplitudes(self) -> np.ndarray:
        return self.amp.cpu().numpy().copy()


@dataclass
class HostClusters:
    """Host arrays behind an sst_clusters record, optionally in pinned memory, with
    optional amplitude arrays (amp u8, amp_first u32 per cluster, amp_off u64 per
    event + 1: the events' slices of amp, for sst_batch_host)."""
    det: np.ndarray
    first: np.ndarray
    width: np.ndarray
    charge: np.ndarray
    barycenter: np.ndarray
    _keep: object = None  # pinned tensors that own the memory
    amp: np.ndarray = None
    amp_first: np.ndarray = None
    amp_off: np.ndarray = None

    @classmethod
    def alloc(cls, capacity: int, pinned: bool = False, amp_off=None):
        """amp_off (uint64, events + 1): also allocate amplitudes, amp_off[-1] bytes."""
        c = max(capacity, 1)
        dts = (np.uint32, np.uint16, np.uint16, np.uint32, np.float32)
        if not pinned:
            b = cls(*[np.zeros(c, d) for d in dts])
        else:
            import torch
            ts = [torch.empty(c * np.dtype(d).itemsize, dtype=torch.uint8, pin_memory=True) for d in dts]
            b = cls(*[t.numpy().view(d) for t, d in zip(ts, dts)], _keep=ts)
        if amp_off is not None:
            b.amp_off = np.ascontiguousarray(amp_off, dtype=np.uint64)
            b.amp = np.zeros(max(int(b.amp_off[-1]), 1), np.uint8)
            b.amp_first = np.zeros(c, np.uint32)
        return b

    def record(self) -> sst_clusters:
        amp = self.amp is not None
        return sst_clusters(_hp(self.det), _hp(self.first), _hp(self.width), _hp(self.charge), _hp(self.barycenter),
                            self.det.size, _hp(self.amp) if amp else None, _hp(self.amp_first) if amp else None,
                            _hp(self.amp_off) if amp else None, self.amp.size if amp else 0)

    def view(self, start: int, n: int) -> dict:
        keys = ("det", "first", "width", "charge", "barycenter") + (("amp_first",) if self.amp is not None else ())
        return {k: getattr(self, k)[start:start + n] for k in keys}


def params(t_channel=2.0, t_seed=3.0, t_cluster=5.0, max_seq_holes=0, max_seq_bad=1, max_adj_bad=0) -> sst_params:
    return sst_params(t_channel, t_seed, t_cluster, max_seq_holes, max_seq_bad, max_adj_bad, 0)
