"""Plain sequential CPU oracle for silicon-strip unpacking and clustering.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The product
library (``paper_2101_11489_gb300``) never imports it, and this package imports
nothing from the product: the two share no code, headers or constants.

The arithmetic lives in ``sst_oracle.c`` (sequential C, binary32 with one rounding
per operation, compiled with ``-ffp-contract=off``); this module only builds it and
marshals numpy arrays through ctypes.  ``bruteforce.py`` holds a third, definitional
implementation of the candidate rule for tiny modules.

Method: arXiv 2101.11489, section 2 (FED layout, zero suppression, the
three-threshold clustering).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sst_oracle.c")
_HDR = os.path.join(_HERE, "sst_oracle.h")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

CH_PER_FED = 96
STRIPS_PER_CH = 256
STRIPS_PER_APV = 128

ST_FED_HDR = 0x01
ST_FRAMING = 0x02
ST_BAD_CODE = 0x04
ST_RUN_RANGE = 0x08
ST_RUN_ORDER = 0x10
ST_TRUNC = 0x20


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no fast-math, no FMA contraction)."""
    stale = (not os.path.exists(_LIB)) or max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)) > os.path.getmtime(_LIB)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("t_channel", ctypes.c_float), ("t_seed", ctypes.c_float), ("t_cluster", ctypes.c_float),
                ("max_seq_holes", ctypes.c_int), ("max_seq_bad", ctypes.c_int), ("max_adj_bad", ctypes.c_int)]


@dataclasses.dataclass(frozen=True)
class Params:
    """The three thresholds (in units of noise) and the hole / bad-strip limits."""
    t_channel: float = 2.0
    t_seed: float = 3.0
    t_cluster: float = 5.0
    max_seq_holes: int = 0
    max_seq_bad: int = 1
    max_adj_bad: int = 0

    def _c(self) -> _Params:
        return _Params(self.t_channel, self.t_seed, self.t_cluster,
                       self.max_seq_holes, self.max_seq_bad, self.max_adj_bad)


def _P(t):
    return ctypes.POINTER(t)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p, u16p, u32p, f32p = _P(ctypes.c_uint8), _P(ctypes.c_uint16), _P(ctypes.c_uint32), _P(ctypes.c_float)
            lib.orc_pack_event.restype = ctypes.c_int64
            lib.orc_pack_event.argtypes = [u8p, u8p, ctypes.c_uint32, u8p, ctypes.c_uint64, u32p]
            lib.orc_unpack_event.restype = ctypes.c_int64
            lib.orc_unpack_event.argtypes = [u8p, u32p, ctypes.c_uint32, u32p, u8p, ctypes.c_uint64, u32p, u8p]
            lib.orc_cluster_module.restype = ctypes.c_int
            lib.orc_cluster_module.argtypes = [u8p, f32p, u8p, f32p, ctypes.c_int, _P(_Params),
                                               u16p, u16p, u32p, f32p, ctypes.c_int]
            lib.orc_cluster_event.restype = ctypes.c_int64
            lib.orc_cluster_event.argtypes = [u32p, u8p, u32p, ctypes.c_uint32, f32p, f32p, u8p, _P(_Params),
                                              u32p, u16p, u16p, u32p, f32p, ctypes.c_uint64]
            lib.orc_unpack_feds.restype = ctypes.c_int64
            lib.orc_unpack_feds.argtypes = [u8p, u32p, ctypes.c_uint32, ctypes.c_uint32, u32p, u8p, ctypes.c_uint64,
                                            u32p, u8p]
            lib.orc_cluster_feds.restype = ctypes.c_int64
            lib.orc_cluster_feds.argtypes = [u32p, u8p, u32p, ctypes.c_uint32, ctypes.c_uint32, f32p, f32p, u8p,
                                             _P(_Params), u32p, u16p, u16p, u32p, f32p, ctypes.c_uint64]
            lib.orc_cluster_amplitudes.argtypes = [u32p, u8p, u32p, f32p, f32p, u8p, _P(_Params), u32p,
                                                   u16p, u16p, ctypes.c_uint64, u32p, u8p, ctypes.c_uint64]
            lib.orc_cluster_amplitudes.restype = ctypes.c_int64
            lib.orc_local_x.argtypes = [u32p, f32p, ctypes.c_uint64, f32p, f32p]
            lib.orc_local_x.restype = None
            lib.orc_is_active.restype = ctypes.c_int
            lib.orc_is_active.argtypes = [ctypes.c_uint8, ctypes.c_float, ctypes.c_uint8, _P(_Params)]
            lib.orc_is_seed.restype = ctypes.c_int
            lib.orc_is_seed.argtypes = [ctypes.c_uint8, ctypes.c_float, ctypes.c_uint8, _P(_Params)]
            lib.orc_passes_cluster.restype = ctypes.c_int
            lib.orc_passes_cluster.argtypes = [ctypes.c_uint32, ctypes.c_float, _P(_Params)]
            lib.orc_corrected_charge.restype = ctypes.c_uint32
            lib.orc_corrected_charge.argtypes = [ctypes.c_uint8, ctypes.c_float]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, t):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(t))


# ---------------------------------------------------------------- predicates

def is_active(adc: int, noise: float, bad: int, p: Params) -> bool:
    return bool(_load().orc_is_active(adc, noise, bad, ctypes.byref(p._c())))


def is_seed(adc: int, noise: float, bad: int, p: Params) -> bool:
    return bool(_load().orc_is_seed(adc, noise, bad, ctypes.byref(p._c())))


def passes_cluster(s_raw: int, n2: float, p: Params) -> bool:
    return bool(_load().orc_passes_cluster(s_raw, n2, ctypes.byref(p._c())))


def corrected_charge(adc: int, gain: float) -> int:
    return int(_load().orc_corrected_charge(adc, gain))


# ---------------------------------------------------------------- pack / unpack

def pack_event(adc: np.ndarray, recorded: np.ndarray, n_feds: int):
    """Canonical packer: dense ADC + recorded mask -> (raw bytes, fed_len[u32])."""
    adc = np.ascontiguousarray(adc, dtype=np.uint8)
    rec = np.ascontiguousarray(recorded, dtype=np.uint8)
    assert adc.size == rec.size == n_feds * CH_PER_FED * STRIPS_PER_CH
    n_rec = int(np.count_nonzero(rec))
    cap = n_feds * (32 + 8 * 8 + 16) + n_feds * CH_PER_FED * 3 + 3 * n_rec + 64
    out = np.zeros(cap, dtype=np.uint8)
    fed_len = np.zeros(n_feds, dtype=np.uint32)
    n = _load().orc_pack_event(_ptr(adc, ctypes.c_uint8), _ptr(rec, ctypes.c_uint8), n_feds,
                               _ptr(out, ctypes.c_uint8), cap, _ptr(fed_len, ctypes.c_uint32))
    if n < 0:
        raise RuntimeError("oracle packer: capacity too small")
    return out[:n].copy(), fed_len


def unpack_event(raw: np.ndarray, fed_len: np.ndarray, n_feds: int) -> dict:
    """Raw FED records -> digis (strip, adc) in strip order, chan_off (CSR), chan_status."""
    raw = np.ascontiguousarray(raw, dtype=np.uint8)
    fed_len = np.ascontiguousarray(fed_len, dtype=np.uint32)
    assert fed_len.size == n_feds
    cap = max(int(raw.size), 1)
    strip = np.zeros(cap, dtype=np.uint32)
    adc = np.zeros(cap, dtype=np.uint8)
    chan_off = np.zeros(n_feds * CH_PER_FED + 1, dtype=np.uint32)
    chan_status = np.zeros(n_feds * CH_PER_FED, dtype=np.uint8)
    n = _load().orc_unpack_event(_ptr(raw, ctypes.c_uint8), _ptr(fed_len, ctypes.c_uint32), n_feds,
                                 _ptr(strip, ctypes.c_uint32), _ptr(adc, ctypes.c_uint8), cap,
                                 _ptr(chan_off, ctypes.c_uint32), _ptr(chan_status, ctypes.c_uint8))
    if n < 0:
        raise RuntimeError("oracle unpacker: capacity too small")
    return {"strip": strip[:n].copy(), "adc": adc[:n].copy(), "chan_off": chan_off, "chan_status": chan_status}


def event_status(chan_status: np.ndarray) -> tuple[int, int]:
    """(OR of all channel status bits, number of channels with a nonzero status)."""
    cs = np.asarray(chan_status, dtype=np.uint8)
    flags = int(np.bitwise_or.reduce(cs)) if cs.size else 0
    return flags, int(np.count_nonzero(cs))


# ---------------------------------------------------------------- clustering

def cluster_module(adc, noise, bad, gain, p: Params) -> dict:
    """One module of n <= 256 strips; gain is per strip (its APV's gain)."""
    adc = np.ascontiguousarray(adc, dtype=np.uint8)
    noise = np.ascontiguousarray(noise, dtype=np.float32)
    bad = np.ascontiguousarray(bad, dtype=np.uint8)
    gain = np.ascontiguousarray(gain, dtype=np.float32)
    n = adc.size
    assert noise.size == bad.size == gain.size == n <= STRIPS_PER_CH
    cap = STRIPS_PER_CH
    first = np.zeros(cap, np.uint16)
    width = np.zeros(cap, np.uint16)
    charge = np.zeros(cap, np.uint32)
    bary = np.zeros(cap, np.float32)
    k = _load().orc_cluster_module(_ptr(adc, ctypes.c_uint8), _ptr(noise, ctypes.c_float),
                                   _ptr(bad, ctypes.c_uint8), _ptr(gain, ctypes.c_float), n,
                                   ctypes.byref(p._c()), _ptr(first, ctypes.c_uint16),
                                   _ptr(width, ctypes.c_uint16), _ptr(charge, ctypes.c_uint32),
                                   _ptr(bary, ctypes.c_float), cap)
    if k < 0:
        raise RuntimeError("oracle module clusterizer failed")
    return {"first": first[:k].copy(), "width": width[:k].copy(), "charge": charge[:k].copy(),
            "barycenter": bary[:k].copy()}


def cluster_event(digis: dict, n_feds: int, noise, gain, bad, p: Params) -> dict:
    """Digis of one event -> cluster SoA (det, first, width, charge, barycenter)."""
    strip = np.ascontiguousarray(digis["strip"], dtype=np.uint32)
    adc = np.ascontiguousarray(digis["adc"], dtype=np.uint8)
    chan_off = np.ascontiguousarray(digis["chan_off"], dtype=np.uint32)
    noise = np.ascontiguousarray(noise, dtype=np.float32)
    gain = np.ascontiguousarray(gain, dtype=np.float32)
    bad = np.ascontiguousarray(bad, dtype=np.uint8)
    assert chan_off.size == n_feds * CH_PER_FED + 1
    n_strips = n_feds * CH_PER_FED * STRIPS_PER_CH
    assert noise.size >= n_strips and bad.size >= n_strips and gain.size >= n_strips // STRIPS_PER_APV
    cap = max(int(strip.size), 1)
    det = np.zeros(cap, np.uint32)
    first = np.zeros(cap, np.uint16)
    width = np.zeros(cap, np.uint16)
    charge = np.zeros(cap, np.uint32)
    bary = np.zeros(cap, np.float32)
    k = _load().orc_cluster_event(_ptr(strip, ctypes.c_uint32), _ptr(adc, ctypes.c_uint8),
                                  _ptr(chan_off, ctypes.c_uint32), n_feds, _ptr(noise, ctypes.c_float),
                                  _ptr(gain, ctypes.c_float), _ptr(bad, ctypes.c_uint8), ctypes.byref(p._c()),
                                  _ptr(det, ctypes.c_uint32), _ptr(first, ctypes.c_uint16),
                                  _ptr(width, ctypes.c_uint16), _ptr(charge, ctypes.c_uint32),
                                  _ptr(bary, ctypes.c_float), cap)
    if k < 0:
        raise RuntimeError("oracle event clusterizer: capacity too small")
    return {"det": det[:k].copy(), "first": first[:k].copy(), "width": width[:k].copy(),
            "charge": charge[:k].copy(), "barycenter": bary[:k].copy()}


def cluster_amplitudes(digis: dict, clusters: dict, noise, gain, bad, p: Params) -> tuple[np.ndarray, np.ndarray]:
    """Per-strip amplitudes of the clusters (gain-corrected charge of active
    strips, 0 elsewhere), back to back: returns (amp_first per cluster, amp)."""
    strip = np.ascontiguousarray(digis["strip"], dtype=np.uint32)
    adc = np.ascontiguousarray(digis["adc"], dtype=np.uint8)
    chan_off = np.ascontiguousarray(digis["chan_off"], dtype=np.uint32)
    det = np.ascontiguousarray(clusters["det"], dtype=np.uint32)
    first = np.ascontiguousarray(clusters["first"], dtype=np.uint16)
    width = np.ascontiguousarray(clusters["width"], dtype=np.uint16)
    noise = np.ascontiguousarray(noise, dtype=np.float32)
    gain = np.ascontiguousarray(gain, dtype=np.float32)
    bad = np.ascontiguousarray(bad, dtype=np.uint8)
    n = det.size
    cap = max(int(width.astype(np.int64).sum()), 1)
    amp_first = np.zeros(max(n, 1), np.uint32)
    amp = np.zeros(cap, np.uint8)
    k = _load().orc_cluster_amplitudes(_ptr(strip, ctypes.c_uint32), _ptr(adc, ctypes.c_uint8),
                                       _ptr(chan_off, ctypes.c_uint32), _ptr(noise, ctypes.c_float),
                                       _ptr(gain, ctypes.c_float), _ptr(bad, ctypes.c_uint8), ctypes.byref(p._c()),
                                       _ptr(det, ctypes.c_uint32), _ptr(first, ctypes.c_uint16),
                                       _ptr(width, ctypes.c_uint16), n, _ptr(amp_first, ctypes.c_uint32),
                                       _ptr(amp, ctypes.c_uint8), cap)
    if k < 0:
        raise RuntimeError("oracle amplitudes failed")
    return amp_first[:n].copy(), amp[:k].copy()


def process_feds(raw, fed_len, fed_base: int, n_feds: int, noise, gain, bad, p: Params) -> dict:
    """Unpack and cluster FEDs fed_base .. fed_base + n_feds - 1 of an event (their
    records back to back in raw): the clusters of that FED range, with the
    event's module ids.  Clusters never cross a FED, so an event's FED ranges can
    be processed independently (the inner level of the nested CPU scheme)."""
    raw = np.ascontiguousarray(raw, dtype=np.uint8)
    fed_len = np.ascontiguousarray(fed_len, dtype=np.uint32)
    assert fed_len.size == n_feds
    lib = _load()
    cap = max(int(raw.size), 1)
    strip = np.zeros(cap, np.uint32)
    adc = np.zeros(cap, np.uint8)
    chan_off = np.zeros(n_feds * CH_PER_FED + 1, np.uint32)
    chan_status = np.zeros(n_feds * CH_PER_FED, np.uint8)
    n = lib.orc_unpack_feds(_ptr(raw, ctypes.c_uint8), _ptr(fed_len, ctypes.c_uint32), fed_base, n_feds,
                            _ptr(strip, ctypes.c_uint32), _ptr(adc, ctypes.c_uint8), cap,
                            _ptr(chan_off, ctypes.c_uint32), _ptr(chan_status, ctypes.c_uint8))
    if n < 0:
        raise RuntimeError("oracle unpacker: capacity too small")
    noise = np.ascontiguousarray(noise, dtype=np.float32)
    gain = np.ascontiguousarray(gain, dtype=np.float32)
    bad = np.ascontiguousarray(bad, dtype=np.uint8)
    det = np.zeros(cap, np.uint32)
    first = np.zeros(cap, np.uint16)
    width = np.zeros(cap, np.uint16)
    charge = np.zeros(cap, np.uint32)
    bary = np.zeros(cap, np.float32)
    k = lib.orc_cluster_feds(_ptr(strip, ctypes.c_uint32), _ptr(adc, ctypes.c_uint8), _ptr(chan_off, ctypes.c_uint32),
                             fed_base, n_feds, _ptr(noise, ctypes.c_float), _ptr(gain, ctypes.c_float),
                             _ptr(bad, ctypes.c_uint8), ctypes.byref(p._c()), _ptr(det, ctypes.c_uint32),
                             _ptr(first, ctypes.c_uint16), _ptr(width, ctypes.c_uint16), _ptr(charge, ctypes.c_uint32),
                             _ptr(bary, ctypes.c_float), cap)
    if k < 0:
        raise RuntimeError("oracle clusterizer: capacity too small")
    return {"det": det[:k].copy(), "first": first[:k].copy(), "width": width[:k].copy(),
            "charge": charge[:k].copy(), "barycenter": bary[:k].copy(), "n_digi": int(n)}


def local_x(det: np.ndarray, barycenter: np.ndarray, pitch: np.ndarray) -> np.ndarray:
    """Local x of clusters: (barycenter - 128) * pitch[det], binary32."""
    det = np.ascontiguousarray(det, dtype=np.uint32)
    bary = np.ascontiguousarray(barycenter, dtype=np.float32)
    pitch = np.ascontiguousarray(pitch, dtype=np.float32)
    assert det.size == bary.size and (det.size == 0 or int(det.max()) < pitch.size)
    x = np.zeros(max(det.size, 1), np.float32)
    _load().orc_local_x(_ptr(det, ctypes.c_uint32), _ptr(bary, ctypes.c_float), det.size,
                        _ptr(pitch, ctypes.c_float), _ptr(x, ctypes.c_float))
    return x[:det.size].copy()


def process_event(raw, fed_len, n_feds: int, noise, gain, bad, p: Params) -> tuple[dict, dict]:
    """Unpack then cluster one event: returns (digis, clusters)."""
    d = unpack_event(raw, fed_len, n_feds)
    c = cluster_event(d, n_feds, noise, gain, bad, p)
    return d, c
