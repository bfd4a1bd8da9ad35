"""Seeded synthetic silicon-strip events and calibration.

This module stands in for the detector front end and the event builder: it draws
calibration tables (noise, gain, bad strips), deposits cluster signal, adds noise,
digitises to 8-bit ADC, applies the front end's zero suppression and writes the
result in the FED byte format.  It is the only code that both the CUDA path's tests
and the oracle's tests share, and it holds none of the method's arithmetic: no
thresholds on seeds or clusters, no unpacking, no clustering.

The paper's own sample (simulated TTBar events with pileup 70 on the 2018 CMS
geometry, arXiv 2101.11489 section 2) is not available; these synthetic events
stand in for it with the same readout geometry (96 channels x 256 strips per FED,
128-strip APVs) and occupancies of the same order.

Random numbers come from numpy's Philox counter-based generator, keyed by
(configuration seed, stream, event), so that any single event can be regenerated on
its own.
"""
from __future__ import annotations

import dataclasses
from typing import Sequence

import numpy as np

CH_PER_FED = 96
STRIPS_PER_CH = 256
STRIPS_PER_APV = 128
FE_PER_FED = 8
CH_PER_FE = 12
FED_HEADER_BYTES = 32
FED_MAGIC = 0x46545353  # bytes 'S','S','T','F'
ZS_CODE = 0x5A

_FED_HDR_DTYPE = np.dtype([("magic", "<u4"), ("fed_id", "<u2"), ("n_ch", "u1"), ("n_fe", "u1"),
                           ("fed_bytes", "<u4"), ("reserved", "<u4"), ("fe_len", "<u2", (FE_PER_FED,))])
assert _FED_HDR_DTYPE.itemsize == FED_HEADER_BYTES

# stream ids for the keyed generator
_S_NOISE, _S_GAIN, _S_BAD, _S_SIGNAL, _S_PEDNOISE, _S_OCC, _S_SAT, _S_SKEW = range(8)


def rng(seed: int, stream: int, event: int = 0) -> np.random.Generator:
    key = np.array([int(seed) & 0xFFFFFFFFFFFFFFFF, ((int(event) & 0xFFFFFFFFFFFF) << 8) | (stream & 0xFF)],
                   dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key))


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic workload: detector size, event count and signal model."""
    name: str
    n_feds: int
    n_events: int
    occupancy: tuple  # ("fixed", f) | ("uniform", lo, hi) | ("lognormal", median, sigma_ln, lo, hi)
    width: tuple  # (min, max) cluster width in strips, uniform
    p_bad: float
    seed: int
    overlap: bool = False  # allow signal clusters to overlap / touch
    sat_frac: float = 0.0  # fraction of signal strips forced to 254 / 255
    moyal_peak: float = 80.0
    moyal_scale: float = 8.0
    fed_skew: float = 1.0  # >1: per-FED occupancy multiplier drawn log-uniform in [1/skew, skew]


# The workloads of the hot path (the numbering follows the configuration list this
# project measures: plain small event, plain full event, batched, batched high
# occupancy, served stream; then the batched configuration with skewed FEDs).
WORKLOADS = {
    0: Workload("single-event-50fed", 50, 1, ("fixed", 0.01), (1, 5), 0.001, 0),
    1: Workload("single-event-440fed", 440, 1, ("fixed", 0.015), (1, 5), 0.001, 1),
    2: Workload("batch64-440fed-occ0.5-4", 440, 64, ("uniform", 0.005, 0.04), (1, 5), 0.001, 2),
    3: Workload("batch256-440fed-occ5-wide", 440, 256, ("fixed", 0.05), (1, 12), 0.02, 3,
                overlap=True, sat_frac=0.03),
    4: Workload("served-440fed-lognormal", 440, 10000, ("lognormal", 0.015, 0.6, 0.005, 0.05), (1, 5), 0.001, 4),
    # the batched configuration's stress variant: per-FED occupancy multipliers
    # log-uniform in [1/4096, 4096] (overlapping clusters allowed), so that FED
    # payloads differ about 8x within the batch despite the zero-suppression noise
    # floor (without them the batched workload's FED payloads differ about 1.6x)
    5: Workload("batch64-440fed-occ0.5-4-fedskew", 440, 64, ("uniform", 0.005, 0.04), (1, 5), 0.001, 2,
                overlap=True, fed_skew=4096.0),
}


@dataclasses.dataclass
class Calibration:
    noise: np.ndarray  # f32 [n_strips]   per-strip noise, ADC counts
    gain: np.ndarray  # f32 [n_apv]      per-APV gain
    bad: np.ndarray  # u8  [n_strips]   1 = bad strip

    @property
    def n_feds(self) -> int:
        return self.noise.size // (CH_PER_FED * STRIPS_PER_CH)


def make_calibration(n_feds: int, seed: int, p_bad: float) -> Calibration:
    n = n_feds * CH_PER_FED * STRIPS_PER_CH
    noise = rng(seed, _S_NOISE).uniform(3.0, 6.0, n).astype(np.float32)
    gain = rng(seed, _S_GAIN).uniform(0.8, 1.2, n // STRIPS_PER_APV).astype(np.float32)
    bad = (rng(seed, _S_BAD).random(n) < p_bad).astype(np.uint8)
    return Calibration(noise, gain, bad)


def event_occupancy(w: Workload, event: int) -> float:
    kind = w.occupancy[0]
    if kind == "fixed":
        return float(w.occupancy[1])
    r = rng(w.seed, _S_OCC, event)
    if kind == "uniform":
        return float(r.uniform(w.occupancy[1], w.occupancy[2]))
    if kind == "lognormal":
        _, med, sig, lo, hi = w.occupancy
        return float(np.clip(med * np.exp(sig * r.standard_normal()), lo, hi))
    raise ValueError(kind)


def make_event_strips(w: Workload, calib: Calibration, event: int, occupancy: float | None = None,
                      n_feds: int | None = None):
    """Dense per-strip ADC (u8) and the zero-suppression mask for one event.

    Signal: clusters of uniform width covering a fraction `occupancy` of the strips,
    total charge Moyal-distributed (peak `moyal_peak`, scale `moyal_scale`, drawn as
    peak + scale * (-ln Z^2) with Z standard normal), shared over the strips with
    weights uniform in [0.5, 1], scaled by the APV gain.  Noise: Gaussian with the
    strip's noise as sigma.  Digitisation: rint, negative -> 0, 254 for 254..1023,
    255 for >= 1024.  Zero suppression keeps a strip when its ADC exceeds twice its
    noise (binary32 comparison).
    """
    n_feds = calib.n_feds if n_feds is None else n_feds
    occ = event_occupancy(w, event) if occupancy is None else occupancy
    n = n_feds * CH_PER_FED * STRIPS_PER_CH
    n_mod = n_feds * CH_PER_FED
    noise = calib.noise[:n]
    r = rng(w.seed, _S_SIGNAL, event)
    wmin, wmax = w.width
    mean_w = 0.5 * (wmin + wmax)
    n_cl = int(round(occ * n / mean_w))
    signal = np.zeros(n, dtype=np.float64)
    sig_strips = np.zeros(0, dtype=np.int64)
    if n_cl > 0:
        widths = r.integers(wmin, wmax + 1, n_cl)
        if w.fed_skew > 1.0:
            fed_w = np.exp(rng(w.seed, _S_SKEW, event).uniform(-np.log(w.fed_skew), np.log(w.fed_skew), n_feds))
            p_mod = np.repeat(fed_w / fed_w.sum() / CH_PER_FED, CH_PER_FED)
            mods = r.choice(n_mod, n_cl, p=p_mod)
        else:
            mods = r.integers(0, n_mod, n_cl)
        starts = (r.random(n_cl) * (STRIPS_PER_CH - widths + 1)).astype(np.int64)
        key = mods.astype(np.int64) * STRIPS_PER_CH + starts
        if not w.overlap:
            order = np.argsort(key, kind="stable")
            key, widths = key[order], widths[order]
            ends = key + widths
            prev_end = np.concatenate([[-1], np.maximum.accumulate(ends)[:-1]])
            keep = key >= prev_end
            key, widths = key[keep], widths[keep]
        n_cl = key.size
        z = r.standard_normal(n_cl)
        q = w.moyal_peak + w.moyal_scale * (-np.log(np.maximum(z * z, 1e-300)))
        q = np.maximum(q, 0.0)
        total = int(widths.sum())
        cl_of = np.repeat(np.arange(n_cl), widths)
        offs = np.arange(total) - np.repeat(np.cumsum(widths) - widths, widths)
        sig_strips = np.repeat(key, widths) + offs
        wt = r.uniform(0.5, 1.0, total)
        wsum = np.bincount(cl_of, weights=wt, minlength=n_cl)
        share = q[cl_of] * wt / wsum[cl_of]
        np.add.at(signal, sig_strips, share * calib.gain[sig_strips // STRIPS_PER_APV].astype(np.float64))
    v = signal + noise.astype(np.float64) * rng(w.seed, _S_PEDNOISE, event).standard_normal(n)
    rv = np.rint(v)
    adc = np.where(rv < 0, 0, np.where(rv <= 253, rv, np.where(rv <= 1023, 254, 255))).astype(np.uint8)
    if w.sat_frac > 0 and sig_strips.size:
        rs = rng(w.seed, _S_SAT, event)
        uniq = np.unique(sig_strips)
        pick = uniq[rs.random(uniq.size) < w.sat_frac]
        adc[pick] = np.where(rs.random(pick.size) < 0.5, 254, 255).astype(np.uint8)
    recorded = (adc.astype(np.float32) > np.float32(2.0) * noise).astype(np.uint8)
    adc = np.where(recorded != 0, adc, 0).astype(np.uint8)
    return adc, recorded


def pack_event(adc: np.ndarray, recorded: np.ndarray, n_feds: int):
    """Front-end packer: recorded strips -> FED records (raw u8, fed_len u32[n_feds]).

    FED record: 32-byte header (u32 magic, u16 fed_id, u8 96, u8 8, u32 fed_bytes,
    u32 reserved, u16 fe_len[8]), then 8 FE units of 12 channel records, each FE unit
    padded with zeros to 8 bytes, the FED padded to 16 bytes.  Channel record: u16
    len, u8 packet code, then runs (u8 first strip, u8 width, width ADC bytes) of
    consecutive recorded strips, split at the APV boundary.
    """
    n_ch = n_feds * CH_PER_FED
    idx = np.flatnonzero(recorded[: n_ch * STRIPS_PER_CH]).astype(np.int64)
    vals = adc[idx]
    if idx.size:
        brk = np.ones(idx.size, dtype=bool)
        brk[1:] = (idx[1:] != idx[:-1] + 1) | (idx[1:] % STRIPS_PER_APV == 0)
        run_pos = np.flatnonzero(brk)
        run_g = idx[run_pos]
        run_w = np.diff(np.append(run_pos, idx.size))
        run_ch = run_g >> 8
    else:
        brk = np.zeros(0, dtype=bool)
        run_pos = run_g = run_w = run_ch = np.zeros(0, dtype=np.int64)
    nruns_ch = np.bincount(run_ch, minlength=n_ch)
    ndigi_ch = np.bincount(idx >> 8, minlength=n_ch)
    ch_len = 3 + 2 * nruns_ch + ndigi_ch
    ch_len3 = ch_len.reshape(n_feds, FE_PER_FED, CH_PER_FE)
    fe_len = ch_len3.sum(axis=2)
    fe_pad = (fe_len + 7) // 8 * 8
    fed_len = (FED_HEADER_BYTES + fe_pad.sum(axis=1) + 15) // 16 * 16
    fed_off = np.concatenate([[0], np.cumsum(fed_len)])
    fe_off = fed_off[:-1, None] + FED_HEADER_BYTES + (np.cumsum(fe_pad, axis=1) - fe_pad)
    ch_off = (fe_off[:, :, None] + (np.cumsum(ch_len3, axis=2) - ch_len3)).reshape(-1)
    buf = np.zeros(int(fed_off[-1]), dtype=np.uint8)

    hdr = np.zeros(n_feds, dtype=_FED_HDR_DTYPE)
    hdr["magic"] = FED_MAGIC
    hdr["fed_id"] = np.arange(n_feds)
    hdr["n_ch"] = CH_PER_FED
    hdr["n_fe"] = FE_PER_FED
    hdr["fed_bytes"] = fed_len
    hdr["fe_len"] = fe_len
    hb = hdr.view(np.uint8).reshape(n_feds, FED_HEADER_BYTES)
    buf[(fed_off[:-1, None] + np.arange(FED_HEADER_BYTES)).reshape(-1)] = hb.reshape(-1)

    buf[ch_off] = (ch_len & 0xFF).astype(np.uint8)
    buf[ch_off + 1] = (ch_len >> 8).astype(np.uint8)
    buf[ch_off + 2] = ZS_CODE
    if idx.size:
        run_bytes = 2 + run_w
        cs = np.cumsum(run_bytes) - run_bytes
        ch_first_run = np.searchsorted(run_ch, run_ch, side="left")
        run_off = ch_off[run_ch] + 3 + (cs - cs[ch_first_run])
        buf[run_off] = (run_g & 0xFF).astype(np.uint8)
        buf[run_off + 1] = run_w.astype(np.uint8)
        rid = np.cumsum(brk) - 1
        pos = run_off[rid] + 2 + (np.arange(idx.size) - run_pos[rid])
        buf[pos] = vals
    return buf, fed_len.astype(np.uint32)


@dataclasses.dataclass
class Event:
    raw: np.ndarray  # u8, the event's FED records back to back
    fed_len: np.ndarray  # u32 [n_feds]
    n_feds: int
    occupancy: float
    n_digi: int

    @property
    def nbytes(self) -> int:
        return int(self.raw.size)


def make_event(w: Workload, calib: Calibration, event: int, n_feds: int | None = None,
               occupancy: float | None = None) -> Event:
    n_feds = calib.n_feds if n_feds is None else n_feds
    occ = event_occupancy(w, event) if occupancy is None else occupancy
    adc, rec = make_event_strips(w, calib, event, occ, n_feds)
    raw, fed_len = pack_event(adc, rec, n_feds)
    return Event(raw, fed_len, n_feds, occ, int(np.count_nonzero(rec)))


@dataclasses.dataclass
class Batch:
    raw: np.ndarray  # u8, events back to back, each 16-byte aligned
    fed_len: np.ndarray  # u32 [n_events * n_feds]
    event_off: np.ndarray  # u64 [n_events + 1], byte offset of each event in raw
    n_events: int
    n_feds: int


def make_batch(events: Sequence[Event]) -> Batch:
    n_feds = events[0].n_feds
    assert all(e.n_feds == n_feds for e in events)
    sizes = np.array([e.nbytes for e in events], dtype=np.uint64)
    off = np.zeros(len(events) + 1, dtype=np.uint64)
    off[1:] = np.cumsum(sizes)
    raw = np.concatenate([e.raw for e in events]) if events else np.zeros(0, np.uint8)
    fed_len = np.concatenate([e.fed_len for e in events]).astype(np.uint32)
    return Batch(raw, fed_len, off, len(events), n_feds)


def make_workload(wid: int, n_events: int | None = None, first_event: int = 0):
    """Calibration and events for workload `wid` (events first_event .. first_event+n-1)."""
    w = WORKLOADS[wid]
    calib = make_calibration(w.n_feds, w.seed, w.p_bad)
    n = w.n_events if n_events is None else n_events
    events = [make_event(w, calib, first_event + i) for i in range(n)]
    return w, calib, events
