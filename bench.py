#!/usr/bin/env python3
"""Throughput of silicon-strip unpacking + three-threshold clustering on GB300.

Method: arXiv 2101.11489 (section 2: unpack zero-suppressed FED data, three-threshold
clustering; section 3: many events concurrently on one GPU).  One step = one batched
launch (sst_batch) over a batch of synthetic full-detector events already resident
in HBM: every FED of every event is unpacked and clustered.

Default workload: 64 full-detector events (440 FEDs x 96 channels x 256 strips),
per-event signal occupancy uniform in [0.5%, 4%], cluster widths 1-5, 0.1% bad
strips.  --workload batch256 selects 256 events at 5% occupancy, widths 1-12,
2% bad strips, 3% saturated strips; batch64-skew the default batch with FED
occupancies skewed so that FED payloads differ about 8x; single50 / single440 the
plain per-event configurations (one 50-FED event at 1%, one 440-FED event at 1.5%,
unpacked and clustered by sst_unpack + sst_cluster, one event per step).

Prints one JSON line (rank 0).  `value` is events/s of the batched path (device
time, CUDA events, L2 flushed between steps); `e2e` is the same through the C ABI
call for host-resident events, sst_batch_host (pinned H2D of the raw bytes, D2H of
statuses and clusters inside the timed region, overlapped over chunks of events).  `per_event` times the plain per-event launches
(sst_unpack + sst_cluster) on the same events.  --impl reference times the CPU
oracle on the host cores instead.

Under torchrun (N > 1) each rank is an independent replica on its own GPU with its
own events (the path shards by event with no exchange); timing is the maximum over
ranks and `value` the events of all ranks over that time.
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import eventgen as eg  # noqa: E402

WORKLOADS = {
    "batch64": (2, 64),
    "batch256": (3, 256),
    "batch64-skew": (5, 64),
    "single50": (0, 1),
    "single440": (1, 1),
}
PER_EVENT = {"single50", "single440"}  # the plain per-event configurations: one event per launch sequence
L2_FLUSH_BYTES = 512 << 20  # written between timed steps (L2 is 129 MB)


# ---------------------------------------------------------------- CPU side (oracle)

_W_CALIB = None


def _worker_init(wid):
    global _W_CALIB
    w = eg.WORKLOADS[wid]
    _W_CALIB = eg.make_calibration(w.n_feds, w.seed, w.p_bad)


def _gen_event(args):
    wid, ev = args
    w = eg.WORKLOADS[wid]
    e = eg.make_event(w, _W_CALIB, ev)
    return e.raw, e.fed_len, e.n_digi


def _gen_served_event(ev):
    # the served stream's occupancy mix (lognormal, median 1.5%, clipped to
    # [0.5%, 5%]) on the same detector and calibration
    e = eg.make_event(eg.WORKLOADS[4], _W_CALIB, ev)
    return e.raw, e.fed_len


_SWEEP = None  # (inner thread count, thread pool) of a CPU-sweep worker


def _sweep_init(wid, inner):
    global _SWEEP
    _worker_init(wid)
    from concurrent.futures import ThreadPoolExecutor
    _SWEEP = (inner, ThreadPoolExecutor(inner) if inner > 1 else None)


def _sweep_event(args):
    """One event through the oracle, its FEDs split into `inner` ranges of about
    equal bytes processed by threads (the inner level of the nested CPU scheme;
    the oracle's C code runs with the GIL released)."""
    raw, fl = args
    import oracle as orc
    w_calib = _W_CALIB
    inner, tp = _SWEEP
    nf = fl.size
    off = np.concatenate([[0], np.cumsum(fl.astype(np.int64))])
    cuts = sorted(set([0, nf] + [int(np.searchsorted(off, off[-1] * k / inner)) for k in range(1, inner)]))

    def part(k):
        f0, f1 = cuts[k], cuts[k + 1]
        return orc.process_feds(raw[off[f0]:off[f1]], fl[f0:f1], f0, f1 - f0, w_calib.noise, w_calib.gain,
                                w_calib.bad, orc.Params())["det"].size

    if tp is None:
        return sum(part(k) for k in range(len(cuts) - 1))
    return sum(tp.map(part, range(len(cuts) - 1)))


def cpu_sweep(args, wid, n_events):
    """Oracle throughput on the host cores for outer (events, processes) x inner
    (FED ranges of one event, threads) = cores; the nested scheme of the paper's
    CPU design beside the GPU path."""
    cores = os.cpu_count() or 1
    gen_pool = mp.get_context("spawn").Pool(cores, initializer=_worker_init, initargs=(wid,))
    events = [(r, f) for r, f, _ in gen_pool.map(_gen_event, [(wid, i) for i in range(n_events)], chunksize=1)]
    gen_pool.terminate()
    res = []
    outer = cores
    while outer >= 1:
        inner = cores // outer
        pool = mp.get_context("spawn").Pool(outer, initializer=_sweep_init, initargs=(wid, inner))
        pool.map(_sweep_event, events[:outer], chunksize=1)  # warm-up
        t0 = time.perf_counter()
        for _ in range(2):
            pool.map(_sweep_event, events, chunksize=1)
        t = (time.perf_counter() - t0) / 2
        pool.terminate()
        res.append({"outer_events": outer, "inner_fed_ranges": inner, "events_per_s": round(len(events) / t, 2),
                    "ms_per_event_latency": round(1e3 * t * outer / len(events), 2)})
        outer //= 2
    w = eg.WORKLOADS[wid]
    print(json.dumps({"metric": "events/s, CPU oracle, outer events x inner FED ranges", "unit": "events/s",
                      "cores": cores, "config": {"workload": f"{args.workload}: {w.name}", "events": n_events},
                      "cpu_sweep": res}), flush=True)


def _oracle_event(args):
    raw, fed_len = args
    import oracle as orc
    w_calib = _W_CALIB
    t0 = time.perf_counter()
    d, c = orc.process_event(raw, fed_len, fed_len.size, w_calib.noise, w_calib.gain, w_calib.bad, orc.Params())
    return time.perf_counter() - t0, int(c["det"].size)


CPU_SAMPLE_S = 12.0  # CPU seconds of oracle work in the timed CPU baseline


def time_oracle(pool, cores, events, cpu_s=CPU_SAMPLE_S):
    """Oracle (unpack + cluster, sequential C) on `cores` processes over a bounded
    sample of the events (cycled): as many as take about cpu_s seconds of CPU,
    estimated from a warm-up pass over `cores` of them.  Returns events/s, the
    sample size, its wall and CPU seconds."""
    def sample(n):
        return [(events[i % len(events)][0], events[i % len(events)][1]) for i in range(n)]
    warm = pool.map(_oracle_event, sample(cores), chunksize=1)  # warms the workers, sizes the sample
    per_event = max(sum(r[0] for r in warm) / cores, 1e-6)
    n_sample = int(min(max(cpu_s / per_event, cores), 50000))
    n_sample = -(-n_sample // cores) * cores
    t0 = time.perf_counter()
    res = pool.map(_oracle_event, sample(n_sample), chunksize=1)
    wall = time.perf_counter() - t0
    cpu = sum(r[0] for r in res)
    return n_sample / wall, n_sample, wall, cpu


# ---------------------------------------------------------------- served stream

SERVED_DISTINCT = 512  # distinct events of the served mix, cycled through the stream


def run_served(sst, ctx, events, n_feds, n_requests, batched_rate):
    """The served stream through the library's native client (sst_serve_load):
    the server's batch depth (events per launch) is picked by saturating runs, the
    saturating throughput is its capacity, then Poisson arrivals are offered at
    10% .. 120% of it and at the batched path's device rate when that is below
    the top of the sweep; p50 / p99 latency from each request's arrival to its
    completion (host clock)."""
    def point(res):
        return {"offered_rate": round(res["offered_rate"], 1) if res["offered_rate"] > 0 else "saturating",
                "events": int(res["requests"]), "throughput": round(res["throughput"], 1),
                "p50_us": round(res["p50_us"], 1), "p99_us": round(res["p99_us"], 1),
                "p99_admitted_us": round(res["p99_admitted_us"], 1), "submit_retries": int(res["retries"])}

    depth = {}
    best = None
    for mb in (16, 32, 64, 128):
        sst.sst_server_start(ctx, 8 << 30, mb, 3, 4096, n_feds, zero_copy="in_place")
        try:
            sst.sst_serve_load(ctx, events, 1000, 0.0, submitters=8, pollers=2)  # warm-up
            r = sst.sst_serve_load(ctx, events, n_requests, 0.0, submitters=8, pollers=2)
        finally:
            sst.sst_server_stop(ctx)
        depth[mb] = round(r["throughput"], 1)
        if best is None or r["throughput"] > depth[best]:
            best = mb
    sst.sst_server_start(ctx, 8 << 30, best, 3, 4096, n_feds, zero_copy="in_place")
    try:
        sst.sst_serve_load(ctx, events, 1000, 0.0, submitters=8, pollers=2)
        cap = sst.sst_serve_load(ctx, events, n_requests, 0.0, submitters=8, pollers=2)
        rates = [f * cap["throughput"] for f in (0.1, 0.3, 0.5, 0.7, 0.9, 1.0, 1.2)]
        at_batched = batched_rate if batched_rate <= 1.2 * cap["throughput"] else None
        if at_batched:
            rates.append(at_batched)
        pts = []
        for k, rate in enumerate(sorted(rates)):
            n = int(min(n_requests, max(2000, rate * 2.0)))  # at most about 2 s per point
            pts.append(point(sst.sst_serve_load(ctx, events, n, rate, submitters=8, pollers=2, seed=100 + k)))
    finally:
        sst.sst_server_stop(ctx)
    return {"capacity": point(cap), "max_batch_events": best, "batch_depth_sweep": depth, "points": pts,
            "p99_at_batched_rate_us": (next(p["p99_us"] for p in pts if p["offered_rate"] == round(at_batched, 1))
                                       if at_batched else None),
            "batched_rate": round(batched_rate, 1)}


# ---------------------------------------------------------------- clocks

class Clocks:
    """nvidia-smi samples of the GPU's clocks every 50 ms.  start() waits for the
    first sample (the tool takes a moment to come up), so that the sampling covers
    the timed region; stop() keeps the samples taken between the two calls (by
    host wall clock), or the nearest one when the region was shorter than the
    sampling interval."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.path = tempfile.mktemp(prefix="clocks", suffix=".csv")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        t_end = time.time() + 5.0
        while self.proc is not None and time.time() < t_end and not self._rows():
            time.sleep(0.02)
        self.t0 = time.time()

    def _rows(self):
        rows = []
        try:
            lines = open(self.path).read().splitlines()
        except OSError:
            return rows
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 10 and f[2].replace(".", "").isdigit():
                try:
                    t = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    continue
                rows.append([t] + f[1:])
        return rows

    def stop(self) -> dict:
        t1 = time.time()
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.06)  # one more sample after the region
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = self._rows()
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        inside = [r for r in rows if self.t0 - 0.05 <= r[0] <= t1 + 0.05]
        window = "timed region"
        if not inside:  # a region shorter than the interval: the sample nearest to it
            inside = [min(rows, key=lambda r: abs(r[0] - 0.5 * (self.t0 + t1)))]
            window = "nearest sample (timed region %.0f ms)" % ((t1 - self.t0) * 1e3)
        sm = [float(r[2]) for r in inside]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in inside for n, v in zip(names, r[6:10]) if v.lower().startswith("active")})
        pw = [float(r[4]) for r in inside if r[4].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(inside[0][3]), "samples": len(inside),
                "window": window, "power_w_max": max(pw) if pw else None, "reasons": reasons}


# ---------------------------------------------------------------- helpers

def shard(rank: int, n_events: int) -> range:
    """Event ids a rank processes: every rank is an independent replica with its own
    n_events events (rank r takes ids r * n_events ... r * n_events + n_events - 1),
    so no data moves between ranks."""
    return range(rank * n_events, (rank + 1) * n_events)


def max_over_ranks(values, world: int) -> list:
    """Element-wise maximum of per-rank timings over all ranks (identity at N = 1)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_model() -> str:
    """The host CPU as the OS describes it (model name, or the Arm part number)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def fed_spread(events) -> dict:
    """How much the FED payloads (bytes after the 32-byte header) differ: the
    largest over the smallest within each event (median and maximum over the
    events) and over all FEDs of the batch."""
    fl = np.array([e[1] for e in events], dtype=np.float64) - 32
    fl = np.maximum(fl, 1)
    within = fl.max(axis=1) / fl.min(axis=1)
    return {"within_event_median": round(float(np.median(within)), 2), "within_event_max": round(float(within.max()), 2),
            "across_batch": round(float(fl.max() / fl.min()), 2)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_traffic():
    """DRAM bytes per launch of the batched kernel from the committed ncu summary,
    or None when the kernel source has changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "k_batch_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if kernel_source_sha256() != d.get("kernel_source_sha256"):
        return None
    return d


def kernel_source_sha256():
    """SHA-256 over the sources the batched kernel is compiled from, in this order."""
    h = hashlib.sha256()
    for f in ("sst_kernels.cu", "sst_fe.cuh", "sst_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2101_11489_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def algorithmic_bytes(events, n_digi, n_clusters):
    """Bytes the path must move per launch, counted as the fused form of the method
    needs them (payload + the calibration of the recorded strips + the clusters):
    every FED payload byte read once; for every recorded strip (digi) its noise
    (4 B) and its bad-strip bit; the gains of every APV (4 B, two APVs per
    channel); fed_len and fed_off (4 + 8 B) per FED; one 16-byte cluster record
    per cluster; a 16-byte status per event."""
    payload = sum(int(e[0].size) for e in events)
    n_feds = sum(int(e[1].size) for e in events)
    return payload + 4 * n_digi + n_digi / 8 + n_feds * 96 * 2 * 4 + 12 * n_feds + 16 * n_clusters + 16 * len(events)


def kernel_bytes(events, n_digi, n_clusters):
    """Bytes the batched kernel's own dataflow touches per launch (a finer model
    than algorithmic_bytes, for comparison with the measured DRAM traffic): the
    payload; the per-strip calibration word and noise^2 of every recorded strip (4
    + 4 B); the APV multipliers (8 B per channel); the FE-unit descriptors the
    prologue wrote (8 B per unit) and the FED lengths and offsets (4 + 8 B per
    FED); the staged cluster records (16 B per cluster); the event status.  The
    bad-strip masks are read only when clusters are widened over bad strips, which
    the default parameters do not."""
    payload = sum(int(e[0].size) for e in events)
    n_feds = sum(int(e[1].size) for e in events)
    return (payload + 8 * n_digi + n_feds * 96 * 8 + n_feds * 8 * 8 + 12 * n_feds + 16 * n_clusters
            + 16 * len(events))


# ---------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="sst", choices=["sst", "reference"])
    ap.add_argument("--workload", default="batch64", choices=sorted(WORKLOADS))
    ap.add_argument("--no-autotune", action="store_true", help="default launch knobs: no stored tune, no sweep")
    ap.add_argument("--retune", action="store_true", help="run the autotuner even when a stored tune exists")
    ap.add_argument("--tune-file", default=None,
                    help="JSON file of the workload's tune (default: paper_2101_11489_gb300/tune/<workload>.json)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--served-events", type=int, default=10000, help="events per served-stream point (0: skip)")
    ap.add_argument("--cpu-sweep", action="store_true",
                    help="only time the CPU oracle over outer events x inner FED ranges on the host cores")
    args = ap.parse_args()
    rank, world, local = dist_env()
    wid, n_events = WORKLOADS[args.workload]
    w = eg.WORKLOADS[wid]
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        return run_reference(args, rank, world, wid, n_events)
    if args.cpu_sweep:
        return cpu_sweep(args, wid, n_events) if rank == 0 else None
    if args.workload in PER_EVENT:
        return run_single(args, rank, world, local, wid)

    cores = os.cpu_count() or 1
    # the process pool is started (spawn) before the first CUDA call
    pool = mp.get_context("spawn").Pool(cores, initializer=_worker_init, initargs=(wid,))
    ids = shard(rank, n_events)
    gen = pool.map(_gen_event, [(wid, i) for i in ids], chunksize=1)
    events = [(r, f) for r, f, _ in gen]
    served_pool = pool.map(_gen_served_event, range(ids.start, ids.start + SERVED_DISTINCT), chunksize=1) \
        if args.served_events > 0 and wid == 2 else []
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)

    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    import paper_2101_11489_gb300 as sst

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    ctx = sst.sst_create(local, w.n_feds)
    sst.sst_calib_upload(ctx, calib.noise, calib.gain, calib.bad, sst.params())

    sizes = np.array([e[0].size for e in events], np.int64)
    eoff = np.zeros(n_events + 1, np.int64)
    eoff[1:] = np.cumsum(sizes)
    caps = sizes // 2 + 1
    coff = np.zeros(n_events + 1, np.int64)
    coff[1:] = np.cumsum(caps)
    raw_h = np.concatenate([e[0] for e in events])
    fl_h = np.concatenate([e[1] for e in events]).astype(np.uint32)
    raw = torch.from_numpy(raw_h).to(dev)
    eoff_d = torch.from_numpy(eoff).to(dev)
    fl_d = torch.from_numpy(fl_h.view(np.int32)).to(dev)
    coff_d = torch.from_numpy(coff).to(dev)
    cb = sst.ClusterBuffers.alloc(int(coff[-1]), device=dev)
    crec = cb.record()
    st_d = torch.zeros(n_events * 4, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # launch knobs of the batched kernel: the stored tune of this workload, else the
    # autotuner's pick (then stored)
    tune = sst.sst_get_tune(ctx)
    tune_src = "default"
    tune_file = args.tune_file or os.path.join(ROOT, "paper_2101_11489_gb300", "tune", f"{args.workload}.json")
    stored = None if args.retune else sst.load_tune(tune_file, args.workload)
    if stored is not None and not args.no_autotune:
        sst.sst_set_tune(ctx, **stored)
        tune, tune_src = stored, f"stored ({os.path.relpath(tune_file, ROOT)})"
    elif not args.no_autotune:
        tune, tune_us = sst.sst_autotune(ctx, raw, eoff_d, fl_d, n_events, w.n_feds, coff_d, crec, st_d)
        tune_src = "autotuned in this run"
        try:
            os.makedirs(os.path.dirname(tune_file), exist_ok=True)
            sst.save_tune(tune, tune_file, args.workload,
                          {"us_per_launch_sequence": round(tune_us, 1),
                           "gpu": torch.cuda.get_device_name(dev)})
        except OSError:
            pass
    launch = sst.sst_get_launch_info(ctx, n_events, w.n_feds)

    def step():
        sst.sst_batch(ctx, raw, eoff_d, fl_d, n_events, w.n_feds, coff_d, crec, st_d)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---- timed region: device time of K batched steps, L2 flushed before each
    clocks = Clocks(local)
    sst.sst_profile_read(ctx, reset=True)
    sst.sst_profile_enable(ctx, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    barrier()
    t_wall = time.perf_counter() - t_wall0
    sst.sst_profile_enable(ctx, False)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    n_launch, kernel_ms = sst.sst_profile_read(ctx, reset=True)
    ms_per_step = sum(step_ms) / len(step_ms)
    ms_per_step, k_ms = max_over_ranks([ms_per_step, kernel_ms / max(n_launch, 1)], world)

    st_h = st_d.cpu().numpy().view(np.uint32).reshape(n_events, 4)
    n_digi = int(st_h[:, 0].sum())
    n_clu = int(st_h[:, 1].sum())
    flags = int(np.bitwise_or.reduce(st_h[:, 2]))

    # ---- the same step captured once as a CUDA graph and replayed (L2 flushed
    # before every replay, as above)
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        step()
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    torch.cuda.synchronize()
    g_steps = max(3, min(args.steps, 300))
    g_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(g_steps)]
    for i in range(g_steps):
        flush.fill_(i & 0xFF)
        g_ev[i][0].record(stream)
        graph.replay()
        g_ev[i][1].record(stream)
    torch.cuda.synchronize()
    g_ms = max_over_ranks([sum(a.elapsed_time(b) for a, b in g_ev) / g_steps], world)[0]
    assert np.array_equal(st_d.cpu().numpy().view(np.uint32).reshape(n_events, 4), st_h), "graph replay differs"
    del graph

    # ---- local positions of the step's clusters (synthetic strip pitch per module)
    sst.sst_pitch_upload(ctx, np.random.default_rng(11).uniform(0.008, 0.0205, w.n_feds * 96).astype(np.float32))
    n_pos = int(coff[-1])
    x_pos = torch.empty(n_pos, dtype=torch.float32, device=dev)
    sst.sst_local_x(ctx, cb.det, cb.barycenter, n_pos, x_pos)
    torch.cuda.synchronize()
    pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pa.record(stream)
    for _ in range(20):
        sst.sst_local_x(ctx, cb.det, cb.barycenter, n_clu, x_pos)
    pb.record(stream)
    torch.cuda.synchronize()
    pos_ms = pa.elapsed_time(pb) / 20
    del x_pos

    # ---- per-event launches on the same events (the paper's one-event-at-a-time form)
    pe_raw = [torch.from_numpy(e[0]).to(dev) for e in events]
    pe_fl = [torch.from_numpy(e[1].view(np.int32)).to(dev) for e in events]
    dbuf = sst.DigiBuffers.alloc(int(sizes.max()), w.n_feds, device=dev)
    drec = dbuf.record()
    pcb = sst.ClusterBuffers.alloc(int(caps.max()), device=dev)
    pcrec = pcb.record()

    def per_event_pass():
        for r, f in zip(pe_raw, pe_fl):
            sst.sst_unpack(ctx, r, f, w.n_feds, drec)
            sst.sst_cluster(ctx, drec, w.n_feds, pcrec)

    per_event_pass()
    torch.cuda.synchronize()
    pe_steps = max(3, min(args.steps // 4, 40))
    pe_ms = []
    for i in range(pe_steps):
        flush.fill_(i & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        per_event_pass()
        b.record(stream)
        torch.cuda.synchronize()
        pe_ms.append(a.elapsed_time(b))
    pe_med = max_over_ranks([statistics.median(pe_ms)], world)[0]
    pe_value = n_events / (pe_med / 1e3)

    # ---- end to end through the C ABI with host-resident events (sst_batch_host:
    # H2D of every step's events, the kernels, D2H of every cluster and status,
    # chunks of events overlapped on the library's streams)
    keep = [torch.from_numpy(a).pin_memory() for a in (raw_h, eoff.view(np.int64), fl_h.view(np.int32))]
    raw_pin, eoff_pin, fl_pin = keep[0].numpy(), keep[1].numpy().view(np.uint64), keep[2].numpy().view(np.uint32)
    # up to six sets of pinned output buffers: up to six steps are in the library's
    # pipeline, each step cut into chunks of 64 events (copies in, kernels and
    # copies out of successive chunks overlap), and step i's results are read once
    # its wait returns.  Measured on batch64 (events/s): chunks of 32 events with
    # 3, 6 or 8 steps in flight 96-99 k (five cluster copies per chunk; the copy
    # back is busy without a gap); chunks of 64 with 3 steps 98 k (the host's turn
    # between a wait and the next submission leaves the pipeline idle), with 6 or
    # 8 steps 120 k
    e2e_cap = min(int(coff[-1]), 2 * n_clu + 4096)  # cluster records per output set
    depth = max(3, min(6, (2 << 30) // (16 * e2e_cap)))  # at most about 2 GiB of pinned output sets
    e2e_chunk = min(64, n_events)
    tune_e2e = dict(tune)
    tune_e2e["host_chunk_events"] = e2e_chunk
    sst.sst_set_tune(ctx, **tune_e2e)
    outs = []
    for _ in range(depth):
        ef = torch.zeros(n_events + 1, dtype=torch.int64).pin_memory()
        sh = torch.zeros(n_events * 4, dtype=torch.int32).pin_memory()
        keep += [ef, sh]
        # room for twice the step's clusters (a step that needed more would report
        # SST_EV_CLUSTER_CAPACITY, and the status check below would fail)
        outs.append((sst.HostClusters.alloc(e2e_cap, pinned=True), ef.numpy().view(np.uint64),
                     sh.numpy().view(np.uint32).reshape(n_events, 4)))

    def e2e_run(n_steps):
        d2h, queue = 0, []

        def retire():
            t, q = queue.pop(0)
            sst.sst_batch_host_wait(ctx, t)
            return 16 * int(q[1][-1]) + q[2].nbytes + q[1].nbytes

        for i in range(n_steps):
            o = outs[i % depth]  # free: the step that used it last has been waited for
            queue.append((sst.sst_batch_host_submit(ctx, raw_pin, eoff_pin, fl_pin, n_events, w.n_feds, o[0], o[1],
                                                    o[2]), o))
            if len(queue) == depth:
                d2h += retire()
        while queue:
            d2h += retire()
        return d2h

    e2e_run(depth)
    for o in outs:
        assert np.array_equal(o[2], st_h), "sst_batch_host statuses differ from sst_batch"
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(100, min(args.steps, 200))  # enough steps to amortise the pipeline's fill and drain
    d2h_total = e2e_run(e2e_steps)
    barrier()
    sst.sst_set_tune(ctx, **tune)
    e2e_s = max_over_ranks([(time.perf_counter() - t0) / e2e_steps], world)[0]
    h2d_bytes = raw_h.nbytes + fl_h.nbytes + 2 * eoff.nbytes  # raw, FED lengths, event and cluster offsets

    # ---- served stream: continuous batching behind sst_submit / sst_poll, driven by
    # the library's native Poisson client
    served = None
    if served_pool:
        # the events live in pinned memory and are lent to the server, whose kernels
        # read them in place over the host link (zero_copy 2): no per-event copy by
        # the client, none by the copy engine
        pinned = [torch.from_numpy(r).pin_memory() for r, _ in served_pool]
        lent = [(p.numpy(), f.astype(np.uint32)) for p, (_, f) in zip(pinned, served_pool)]
        served = run_served(sst, ctx, lent, w.n_feds, args.served_events, n_events / (ms_per_step / 1e3))
        served["workload"] = ("served-440fed-lognormal: occupancy lognormal median 1.5%, clip [0.5%, 5%], "
                              f"{len(lent)} distinct events cycled, Poisson arrivals, native client "
                              "(sst_serve_load: 8 submitter and 2 poller threads), events read in place from "
                              "pinned event buffers, 8 GiB device budget, 3 batches in flight, kernels of one batch "
                              "at a time")
        del pinned, lent

    # ---- roofline of the dominant kernel (the batched kernel)
    peak, peak_kind = measured_peaks()
    b_alg = algorithmic_bytes(events, n_digi, n_clu)
    b_kern = kernel_bytes(events, n_digi, n_clu)
    achieved = b_alg / (k_ms / 1e3) / 1e9
    tr = kernel_traffic()
    traffic = None
    issue = None
    if tr is not None and tr.get("workload") == args.workload:
        traffic = tr.get("dram_bytes_per_launch")
        if tr.get("warp_instructions"):
            # the kernel is bound by instruction issue, not by HBM: one warp
            # instruction per scheduler per cycle, 4 schedulers per SM
            n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
            peak_ips = n_sm * 4 * (clk.get("sm_mhz") or 2070.0) * 1e6
            ips = tr["warp_instructions"] / (k_ms / 1e3)
            issue = {"warp_instructions_per_launch": tr["warp_instructions"], "achieved_per_s": round(ips, 1),
                     "peak_per_s": round(peak_ips, 1), "frac": round(ips / peak_ips, 4),
                     "source": "instruction count from the committed ncu capture of this kernel"}

    # ---- oracle on the host cores (rank 0 at N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, n_sample, wall, cpu_s = time_oracle(pool, cores, events)
        cpu = {"value": round(v, 2), "unit": "events/s", "cores": cores, "kind": "oracle",
               "per_core": round(v / cores, 2), "cpu_model": cpu_model(),
               "sample": f"{n_sample} events, the step's {n_events} cycled (unpack + cluster, sequential C, one "
                         f"event per process), {wall:.1f} s wall, {cpu_s:.1f} s CPU"}
    pool.terminate()

    total_events = n_events * world
    if rank == 0:
        line = {
            "metric": "events/s unpack+cluster (batched)",
            "value": round(total_events / (ms_per_step / 1e3), 1),
            "unit": "events/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(ms_per_step, 4),
            "step_ms_percentiles": {"p10": round(float(np.percentile(step_ms, 10)), 4),
                                    "median": round(float(np.median(step_ms)), 4),
                                    "p90": round(float(np.percentile(step_ms, 90)), 4)},
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {w.name}", "events_per_step": n_events, "n_feds": w.n_feds,
                       "strips_per_event": w.n_feds * 96 * 256, "l2": "flushed: 512 MiB write before every step",
                       "tune": tune, "tune_source": tune_src, "launch": launch, "digis_per_step": n_digi, "clusters_per_step": n_clu,
                       "payload_bytes_per_step": int(sizes.sum()), "status_flags": flags,
                       "fed_payload_spread": fed_spread(events),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "strips_per_s": round(total_events * w.n_feds * 96 * 256 / (ms_per_step / 1e3), 1),
            "per_event": {"value": round(pe_value * world, 1), "unit": "events/s",
                          "ms_per_event": round(pe_med / n_events, 4),
                          "what": "sst_unpack + sst_cluster, one event per launch pair, same events"},
            "batched_over_per_event": round((total_events / (ms_per_step / 1e3)) / (pe_value * world), 2),
            "graph": {"value": round(total_events / (g_ms / 1e3), 1), "unit": "events/s", "ms_per_step": round(g_ms, 4),
                      "steps": g_steps, "what": "the same step captured once as a CUDA graph and replayed"},
            "local_x": {"clusters_per_s": round(n_clu / (pos_ms / 1e3), 1), "ms": round(pos_ms, 4),
                        "what": "local x of the step's clusters from a per-module strip pitch (sst_local_x)"},
            "paper_context": {"cpu": "560 events/s, 28 Broadwell cores (real TTBar PU70 events)",
                              "gpu": "649 events/s, one Tesla P100 (real TTBar PU70 events)",
                              "note": "other hardware and real events; context, not a baseline"},
            "e2e": {"value": round(total_events / e2e_s, 1), "unit": "events/s",
                    "h2d_bytes_per_step": int(h2d_bytes), "d2h_bytes_per_step": int(d2h_total / e2e_steps),
                    "steps": e2e_steps,
                    "api": "sst_batch_host_submit / sst_batch_host_wait, pinned host buffers, up to %d steps in "
                           "flight, chunks of %d events (host_chunk_events)" % (depth, e2e_chunk)},
            "gpu_launches": 3 * args.steps,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": traffic,
                         "kernel": "k_batch", "kernels_per_step": 3, "kernel_ms": round(k_ms, 4), "algorithmic_bytes": int(b_alg),
                         "bytes_definition": "payload + 4 B noise and a bad-strip bit per recorded strip + APV "
                                             "gains + fed_len/fed_off + 16 B per cluster + 16 B status per event",
                         "traffic_model": {"bytes": int(b_kern), "achieved": round(b_kern / (k_ms / 1e3) / 1e9, 1),
                                           "frac": round(b_kern / (k_ms / 1e3) / 1e9 / peak, 4),
                                           "what": "the kernel's own dataflow: calibration word and noise^2 per "
                                                   "recorded strip, APV multipliers, FE-unit "
                                                   "descriptors, FED lengths and offsets, staged cluster records"},
                         "peak_kind": peak_kind, "issue": issue},
            "served": served,
            "cpu_baseline": cpu,
            "clocks": clk,
            "wall_s_timed_region": round(t_wall, 4),
        }
        print(json.dumps(line), flush=True)
    sst.sst_destroy(ctx)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_single(args, rank, world, local, wid):
    """The plain per-event configurations: one event per step through sst_unpack +
    sst_cluster (device buffers; the paper's per-event form), L2 flushed before
    every step; the event of the configuration, replicated per rank."""
    w = eg.WORKLOADS[wid]
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
    ev = eg.make_event(w, calib, 0)
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    import paper_2101_11489_gb300 as sst
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    ctx = sst.sst_create(local, w.n_feds)
    sst.sst_calib_upload(ctx, calib.noise, calib.gain, calib.bad, sst.params())
    raw = torch.from_numpy(ev.raw).to(dev)
    fl = torch.from_numpy(ev.fed_len.view(np.int32)).to(dev)
    cap = ev.nbytes // 2 + 1
    dbuf = sst.DigiBuffers.alloc(ev.nbytes, w.n_feds, device=dev)
    cbuf = sst.ClusterBuffers.alloc(cap, device=dev)
    drec, crec = dbuf.record(), cbuf.record()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step():
        sst.sst_unpack(ctx, raw, fl, w.n_feds, drec)
        sst.sst_cluster(ctx, drec, w.n_feds, crec)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    ev_t = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        ev_t[i][0].record(stream)
        step()
        ev_t[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = np.array([a.elapsed_time(b) for a, b in ev_t])
    mean_ms = max_over_ranks([float(ms.mean())], world)[0]
    st = dbuf.to_host()
    n_digi, n_clu = st["n_digi"], st["n_clusters"]

    # the same launch sequence captured once as a CUDA graph and replayed (L2
    # flushed before every replay): what the launch gaps of one event cost
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        step()
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    torch.cuda.synchronize()
    g_steps = max(3, min(args.steps, 300))
    g_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(g_steps)]
    for i in range(g_steps):
        flush.fill_(i & 0xFF)
        g_ev[i][0].record(stream)
        graph.replay()
        g_ev[i][1].record(stream)
    torch.cuda.synchronize()
    g_ms = max_over_ranks([float(np.median([a.elapsed_time(b) for a, b in g_ev]))], world)[0]
    assert dbuf.to_host()["n_clusters"] == n_clu, "graph replay differs"
    del graph

    # end to end through the public calls with host buffers: copy the event in
    # (pinned), unpack + cluster, read the status, then the event's clusters out
    raw_pin = torch.from_numpy(ev.raw).pin_memory()
    fl_pin = torch.from_numpy(ev.fed_len.view(np.int32)).pin_memory()
    host = sst.HostClusters.alloc(cap, pinned=True)
    st_pin = torch.zeros(4, dtype=torch.int32).pin_memory()
    dev_arrays = [cbuf.det, cbuf.first, cbuf.width, cbuf.charge, cbuf.barycenter]
    host_arrays = [torch.from_numpy(getattr(host, k).view(np.uint8)) for k in ("det", "first", "width", "charge",
                                                                             "barycenter")]

    def e2e_step():
        raw.copy_(raw_pin, non_blocking=True)
        fl.copy_(fl_pin, non_blocking=True)
        step()
        st_pin.copy_(dbuf.status.view(torch.int32), non_blocking=True)
        torch.cuda.synchronize()
        n = int(st_pin[1])
        for d, h in zip(dev_arrays, host_arrays):
            nb = n * d.element_size()
            h[:nb].copy_(d.view(torch.uint8)[:nb], non_blocking=True)
        torch.cuda.synchronize()
        return n

    for _ in range(3):
        e2e_step()
    e2e_steps = max(100, min(args.steps, 200))  # enough steps to amortise the pipeline's fill and drain
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        n_out = e2e_step()
    e2e_s = max_over_ranks([(time.perf_counter() - t0) / e2e_steps], world)[0]
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cores = os.cpu_count() or 1
        pool = mp.get_context("spawn").Pool(cores, initializer=_worker_init, initargs=(wid,))
        v, n_sample, wall, cpu_s = time_oracle(pool, cores, [(ev.raw, ev.fed_len)])
        pool.terminate()
        cpu = {"value": round(v, 2), "unit": "events/s", "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
               "sample": f"the event {n_sample} times (unpack + cluster, sequential C, one event per process), "
                         f"{wall:.1f} s wall, {cpu_s:.1f} s CPU"}
    peak, peak_kind = measured_peaks()
    b_alg = algorithmic_bytes([(ev.raw, ev.fed_len)], n_digi, n_clu)
    if rank == 0:
        print(json.dumps({
            "metric": "events/s unpack+cluster (per event)", "value": round(world * 1e3 / mean_ms, 1),
            "unit": "events/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(mean_ms, 4),
            "step_ms_percentiles": {"p10": round(float(np.percentile(ms, 10)), 4),
                                    "median": round(float(np.median(ms)), 4),
                                    "p90": round(float(np.percentile(ms, 90)), 4)},
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {w.name}", "events_per_step": 1, "n_feds": w.n_feds,
                       "strips_per_event": w.n_feds * 96 * 256, "l2": "flushed: 512 MiB write before every step",
                       "digis": int(n_digi), "clusters": int(n_clu), "payload_bytes": int(ev.nbytes),
                       "path": "sst_unpack + sst_cluster, device buffers, one event per launch sequence",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "e2e": {"value": round(world / e2e_s, 1), "unit": "events/s",
                    "h2d_bytes_per_step": int(ev.raw.nbytes + ev.fed_len.nbytes),
                    "d2h_bytes_per_step": int(16 + 16 * n_out), "steps": e2e_steps,
                    "api": "pinned copy in, sst_unpack + sst_cluster, status then the event's clusters copied out"},
            "graph": {"value": round(world * 1e3 / g_ms, 1), "unit": "events/s", "ms_per_step": round(g_ms, 4),
                      "steps": g_steps, "what": "the same launch sequence captured once as a CUDA graph and "
                                                "replayed (median step)"},
            "gpu_launches": 5 * args.steps,
            "roofline": {"bound": "hbm", "achieved": round(b_alg / (mean_ms / 1e3) / 1e9, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(b_alg / (mean_ms / 1e3) / 1e9 / peak, 4), "traffic": None,
                         "kernel": "the per-event launch sequence (k_fed_scan, k_unpack, k_cluster, k_order and a "
                                   "memset): launch- and latency-bound at one event per launch",
                         "algorithmic_bytes": int(b_alg), "peak_kind": peak_kind},
            "cpu_baseline": cpu, "clocks": clk,
        }), flush=True)
    sst.sst_destroy(ctx)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args, rank, world, wid, n_events):
    """The CPU oracle as the reference arm: each step runs the oracle over a bounded
    sample of the workload's events on all host cores."""
    if rank != 0:
        return
    w = eg.WORKLOADS[wid]
    cores = os.cpu_count() or 1
    pool = mp.get_context("spawn").Pool(cores, initializer=_worker_init, initargs=(wid,))
    # the whole step (the GPU arm's workload) while that keeps the run to about a
    # minute of oracle work per 16 cores, else a bounded sample of it
    whole = args.steps * n_events <= 20000 * max(cores, 1) // 16
    sample = n_events if whole else min(n_events, cores * 2)
    gen = pool.map(_gen_event, [(wid, i) for i in range(sample)], chunksize=1)
    events = [(r, f) for r, f, _ in gen]
    for _ in range(args.warmup):
        pool.map(_oracle_event, events[:cores], chunksize=1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        pool.map(_oracle_event, events, chunksize=1)
        times.append(time.perf_counter() - t0)
    pool.terminate()
    ms = 1e3 * sum(times) / len(times)
    v = sample / (ms / 1e3)
    print(json.dumps({
        "impl": "reference", "metric": "events/s unpack+cluster (batched)", "value": round(v, 2), "unit": "events/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {w.name}", "events_per_step": sample, "n_feds": w.n_feds},
        "cpu_baseline": {"value": round(v, 2), "unit": "events/s", "cores": cores, "kind": "oracle",
                         "sample": (f"all {n_events} events of the step" if whole else
                                    f"{sample} of the {n_events} events per step") + ", one event per process"},
        "e2e": {"value": round(v, 2), "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


if __name__ == "__main__":
    main()
