#!/usr/bin/env python3
"""Benchmark of the GB300 DFR sort.

Default workload (one "step"): the plain sort of 2^28 uint32 keys for each of
the seven seeded distributions (uniform, normal, exponential, Zipf, all-equal,
already sorted, reverse sorted) -- every stage of the hot path (root count,
per-level count, look-back scatter, classification, CTA/warp diversion sorts,
copy-back) runs inside every sort.  Inputs are restored from a pristine device
copy and L2 is flushed (256 MiB write) before every sort, outside the timed
region; each sort is timed with CUDA events on its stream.

Printed: one JSON line (rank 0).  `value` = keys sorted per second over the
whole step (Gkeys/s); `roofline` = the scatter kernel (the dominant kernel):
algorithmic bytes (read + write of every record it deals) over its measured
time, against the measured HBM copy bandwidth; `e2e` = the same metric through
the C ABI with the keys starting and ending in pinned host memory;
`cpu_baseline` = the CPU oracle on a bounded sample of the same arrays.

`--impl reference` times the CPU oracle (the only reference this method has)
on a bounded sample of the same workload.

Under torchrun every rank sorts its own replica of the workload (weak scaling,
no collective on the data path); times are the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

# ncu DRAM traffic figures (read + write bytes per key the kernel handles) of
# the u32 key-only kernels, kept in profiles/traffic.json with the sha256 of
# each kernel's own source file at the time of the capture; a figure whose
# source has changed since is not used (the roofline's traffic is then null).
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


WORKLOADS = {
    "plain_u32_2^28": dict(kind="plain", key="u32", n=1 << 28, dists=list(synth.U32_DISTRIBUTIONS)),
    "plain_u32_1M": dict(kind="plain", key="u32", n=1_000_000, dists=["uniform"]),
    "kv_u64_2^27": dict(kind="plain", key="u64kv", n=1 << 27, dists=list(synth.U64_DISTRIBUTIONS)),
    # a smaller case (still larger than L2) for full ncu captures
    "plain_u32_2^26": dict(kind="plain", key="u32", n=1 << 26, dists=["uniform"]),
    # 4096 u32 arrays, log-uniform sizes over [2^8, 2^20], uniform or Zipf per array
    "batch_u32_4096": dict(kind="batch", key="u32", count=4096, lo=1 << 8, hi=1 << 20),
    # Poisson stream of requests, log-uniform sizes over [2^10, 2^24], 70% u32 / 30% u64+u32
    "served_mixed": dict(kind="served", key="mixed", requests=100_000, lo=1 << 10, hi=1 << 24,
                         budget=16 << 30, loads=[0.25, 0.5, 0.75, 1.0]),
}
DEFAULT_WORKLOAD = "plain_u32_2^28"
SEED_OFFSET = {"plain_u32_2^28": 20, "plain_u32_1M": 1, "kv_u64_2^27": 30, "plain_u32_2^26": 20,
               "batch_u32_4096": 40, "served_mixed": 50}


def source_sha(paths) -> str:
    """sha256 (first 16 hex digits) of the files `paths` (relative to the
    repository root), concatenated in the order given."""
    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_per_key(kernel: str):
    """The ncu DRAM bytes per key of `kernel` for u32 key-only sorts, or None
    when no capture matches the kernel's current source."""
    try:
        with open(TRAFFIC_FILE) as f:
            entry = json.load(f).get(kernel)
        if entry and source_sha(entry["source"]) == entry["source_sha16"]:
            return float(entry["dram_bytes_per_key"])
    except (OSError, ValueError, KeyError, TypeError):
        pass
    return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def gen_inputs(wl: dict, seed_off: int):
    n = wl["n"]
    out = {}
    for i, dist in enumerate(wl["dists"]):
        seed = synth.BASE_SEED + seed_off + i
        if wl["key"] == "u32":
            if dist == "reverse" and "sorted" in out:
                out[dist] = out["sorted"][::-1].copy()
            else:
                out[dist] = synth.u32(dist, n, seed)
        else:
            out[dist] = synth.u64(dist, n, seed)
    return out


class ClockSampler:
    """nvidia-smi clock and throttle-reason sampling over the timed region.

    nvidia-smi polls every `interval_ms` (20 ms, so that a timed region of a
    few hundred milliseconds holds several samples; 200 ms if the short
    interval yields no sample within a few seconds; that fallback asks for
    the fields without the stamp) and stamps each sample.
    start() returns once the first sample has been written, so sampling is
    live before the warm-up; mark_start() / mark_end() bracket the timed
    region; stop() summarises the samples stamped inside it, widened by one
    interval on each side (all samples, if none falls inside or the stamps
    cannot be read).  Nothing here raises: without nvidia-smi the summary is
    None."""

    Q_PLAIN = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    Q = "timestamp," + Q_PLAIN
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
    FALLBACK_MS = 200
    FIRST_SAMPLE_S = 5.0

    def __init__(self, index: int, interval_ms: int = 20, exe: str = "nvidia-smi"):
        self.index = index
        self.interval_ms = interval_ms
        self.exe = exe
        self.proc = None
        self.f = None
        self.t0 = self.t1 = None
        self.path = os.path.join("/tmp", "dfr_clocks_%d_%d.csv" % (os.getpid(), index))

    def _launch(self, interval_ms: int, query: str) -> None:
        self.f = open(self.path, "w")
        self.interval_ms = interval_ms
        self.proc = subprocess.Popen([self.exe, "-i", str(self.index), "--query-gpu=" + query,
                                      "--format=csv,noheader,nounits", "-lms", str(interval_ms)],
                                     stdout=self.f, stderr=subprocess.DEVNULL)

    def _has_sample(self) -> bool:
        with open(self.path) as f:
            return self.summarise(f.read().splitlines(), None, None, self.interval_ms) is not None

    def _wait_first_sample(self) -> bool:
        """True once a readable sample line is in the file (an error message
        printed instead of samples does not count)."""
        end = time.monotonic() + self.FIRST_SAMPLE_S
        while time.monotonic() < end:
            if self._has_sample():
                return True
            if self.proc.poll() is not None:  # exited, e.g. refused the interval or a field
                return self._has_sample()
            time.sleep(0.01)
        return False

    def _halt(self) -> None:
        if self.proc is not None:
            try:
                self.proc.terminate()
                self.proc.wait(timeout=5)
            except Exception:
                try:
                    self.proc.kill()
                    self.proc.wait(timeout=5)
                except Exception:
                    pass
        if self.f is not None:
            self.f.close()

    def start(self) -> None:
        try:
            self._launch(self.interval_ms, self.Q)
            if not self._wait_first_sample():
                self._halt()
                self._launch(self.FALLBACK_MS, self.Q_PLAIN)
                self._wait_first_sample()
        except Exception:
            self._halt()
            self.proc = None
            try:
                os.unlink(self.path)
            except OSError:
                pass

    def mark_start(self) -> None:
        self.t0 = time.time()

    def mark_end(self) -> None:
        self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return None
        try:
            self._halt()
            with open(self.path) as f:
                lines = f.read().splitlines()
            os.unlink(self.path)
            return self.summarise(lines, self.t0, self.t1, self.interval_ms)
        except Exception:
            return None

    @classmethod
    def summarise(cls, lines, t0, t1, interval_ms):
        """Median loaded SM clock, max clock and the throttle reasons seen,
        over the samples of [t0, t1] widened by one interval (all samples
        when the window is unknown or holds none)."""
        import datetime

        rows = []
        for line in lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) == 9:  # the fallback query: no stamp
                p = [""] + p
            if len(p) < 10:
                continue
            try:
                sm, mx = float(p[2]), float(p[3])
            except ValueError:
                continue
            try:
                t = datetime.datetime.strptime(p[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                t = None
            reasons = {nm for nm, v in zip(cls.REASONS, p[6:10]) if v.lower().startswith("active")}
            rows.append((t, sm, mx, reasons))
        if not rows:
            return None
        window = "run"
        use = rows
        if t0 is not None and t1 is not None:
            pad = interval_ms * 1e-3
            inside = [r for r in rows if r[0] is not None and t0 - pad <= r[0] <= t1 + pad]
            if inside:
                use, window = inside, "timed"
        sm = [r[1] for r in use]
        loaded = [x for x in sm if x > 0.5 * max(sm)] or sm
        reasons = set().union(*(r[3] for r in use))
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r[2] for r in use),
                "reasons": sorted(reasons), "samples": len(use), "samples_total": len(rows),
                "interval_ms": interval_ms, "window": window}


def dist_setup():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(values, world, device):
    if world == 1:
        return list(values)
    import torch
    import torch.distributed as tdist

    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return t.tolist()


def job_rate(local_ms, keys_per_rank, world, device):
    """Whole-job throughput of a weak-scaling step: every rank sorts
    keys_per_rank keys; the step takes as long as the slowest rank.
    Returns (max ms over ranks, Gkeys/s of the whole job)."""
    ms = reduce_max([local_ms], world, device)[0]
    return ms, world * keys_per_rank / (ms * 1e-3) / 1e9


def barrier(world):
    if world > 1:
        import torch.distributed as tdist

        tdist.barrier()


def cpu_oracle_time(inputs, sample_n: int, key: str):
    """Single-threaded oracle on the first sample_n keys of every array."""
    import oracle

    keys = 0
    t0 = time.perf_counter()
    for dist, a in inputs.items():
        s = a[:sample_n]
        if key == "u32":
            oracle.sort_u32(s)
        else:
            oracle.sort_u64_kv(s, synth.index_payload(s.size))
        keys += s.size
    dt = time.perf_counter() - t0
    return keys, dt


def run_reference(args, wl, world, rank):
    """The reference arm: the CPU oracle, as it stands, on a bounded sample."""
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    if wl["kind"] != "plain":
        return run_reference_forms(args, wl)
    sample_n = min(wl["n"], args.cpu_sample)
    sub = dict(wl)
    sub["n"] = sample_n
    inputs = gen_inputs(sub, SEED_OFFSET.get(args.workload, 0))
    for _ in range(args.warmup):
        cpu_oracle_time(inputs, sample_n, wl["key"])
    times = []
    keys = 0
    for _ in range(args.steps):
        keys, dt = cpu_oracle_time(inputs, sample_n, wl["key"])
        times.append(dt)
    t = sum(times) / len(times)
    value = keys / t / 1e9
    line = {
        "impl": "reference", "metric": "Gkeys/s", "value": value, "unit": "Gkeys/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32" if wl["key"] == "u32" else "u64",
        "data": "synthetic", "config": config_of(args.workload, wl),
        "cpu_baseline": {"value": value, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
                         "sample": "first %d keys of each of the %d arrays per step" % (sample_n, len(inputs))},
        "e2e": {"value": value, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def profile_one(dfr, fn, stream):
    """Run fn() once with per-launch CUDA events; returns {kind: (ms, launches)}."""
    import torch

    dfr.dfr_profile_enable(True)
    dfr.dfr_profile_read()
    fn()
    torch.cuda.synchronize()
    prof = dfr.dfr_profile_read()
    dfr.dfr_profile_enable(False)
    return {k: v for k, v in prof.items() if v[1]}


def dominant_roofline(prof, stats, rec, peak, peak_kind):
    """Roofline of the kernel kind with the largest share among the two that
    move records (the scatter and the CTA sort): algorithmic bytes = a read
    and a write of every record it handles, over its measured time."""
    moved = {"scatter": 2 * rec * sum(stats["level_keys"]),
             "ctasort": 2 * rec * stats["cta_keys"],
             # the whole call as one persistent launch: every byte of the sort
             "persist": stats["model_bytes"]}
    cand = [k for k in moved if k in prof and prof[k][0] > 0]
    if not cand:
        return None
    k = max(cand, key=lambda x: prof[x][0])
    ms, launches = prof[k]
    achieved = moved[k] / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None, "kernel": "k_" + k, "peak_source": peak_kind,
            "algorithmic_bytes_per_launch": moved[k] / max(1, launches)}


def batch_inputs(wl):
    arrays, kinds = synth.batch_u32(wl["count"], synth.BASE_SEED + SEED_OFFSET["batch_u32_4096"], wl["lo"], wl["hi"])
    return arrays, kinds


def run_batch(args, wl, dfr, dev, world, rank, emit=True):
    """Many arrays: one dfr_sort_batch launch sequence against one plain
    dfr_sort_u32 call per array on one stream, uncaptured and captured in a
    CUDA graph.  Every arm sorts the same arrays, restored from a pristine copy
    and with L2 flushed before each timed repetition (untimed)."""
    import torch

    arrays, kinds = batch_inputs(wl)
    sizes = [a.size for a in arrays]
    offs, pos = [], 0
    for n in sizes:
        offs.append(pos)
        pos += (n + 63) // 64 * 64  # 256-byte aligned starts
    total_keys = int(sum(sizes))
    host = np.zeros(pos, dtype=np.uint32)
    for o, a in zip(offs, arrays):
        host[o:o + a.size] = a
    stream = torch.cuda.current_stream(dev)
    pristine = dfr.to_device(host, dev)
    work = torch.empty_like(pristine)
    kbuf = torch.empty_like(pristine)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    base, bbase = work.data_ptr(), kbuf.data_ptr()
    segs = [(dfr.DFR_U32, base + 4 * o, 0, bbase + 4 * o, 0, n) for o, n in zip(offs, sizes)]
    wsb = dfr.dfr_batch_workspace_bytes(segs)
    ws = torch.zeros(wsb, dtype=torch.uint8, device=dev)
    pwsb = dfr.dfr_workspace_bytes(dfr.DFR_U32, max(sizes))
    pws = torch.zeros(pwsb, dtype=torch.uint8, device=dev)

    def restore():
        work.copy_(pristine)
        flush.fill_(1)

    def batched():
        dfr.check(dfr.dfr_sort_batch(segs, ws, wsb, stream), "dfr_sort_batch")

    def plain():
        st = int(stream.cuda_stream)
        for o, n in zip(offs, sizes):
            rc = dfr.dfr_sort_u32(base + 4 * o, bbase + 4 * o, n, pws, pwsb, st)
            if rc:
                dfr.check(rc, "dfr_sort_u32")

    def timed(fn, steps):
        out = []
        for _ in range(steps):
            restore()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        return out

    def verify(tag):
        got = dfr.to_numpy(work, np.uint32)
        for i in range(0, len(arrays), 97):  # a sample checked against the host arrays
            o, a = offs[i], arrays[i]
            seg = got[o:o + a.size]
            if not (np.all(seg[1:] >= seg[:-1]) and np.array_equal(np.sort(a), seg)):
                raise RuntimeError("%s: array %d is not the sorted input" % (tag, i))

    # warm-up (also fills the launch-grid cache before graph capture)
    for _ in range(args.warmup):
        timed(batched, 1)
    if dfr.dfr_last_device_status(ws, stream) != dfr.DFR_OK:
        raise RuntimeError("device status after batched warm-up")
    verify("batched")
    timed(plain, 1)
    verify("plain")

    graph = torch.cuda.CUDAGraph()
    restore()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, capture_error_mode="thread_local"):
        cap_stream = torch.cuda.current_stream()
        st = int(cap_stream.cuda_stream)
        for o, n in zip(offs, sizes):
            dfr.check(dfr.dfr_sort_u32(base + 4 * o, bbase + 4 * o, n, pws, pwsb, st), "capture")
    timed(graph.replay, 1)
    verify("graph")

    clocks = ClockSampler(dev.index or 0)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    clocks.mark_start()
    l0 = dfr.dfr_launch_count()
    t_batch = timed(batched, args.steps)
    launches = dfr.dfr_launch_count() - l0
    torch.cuda.synchronize()
    clocks.mark_end()
    barrier(world)
    clk = clocks.stop()
    t_plain = timed(plain, max(1, min(args.steps, 3)))
    t_graph = timed(graph.replay, max(1, min(args.steps, 3)))
    ms, value = job_rate(statistics.mean(t_batch), total_keys, world, dev)
    ms_plain = statistics.median(t_plain)
    ms_graph = statistics.median(t_graph)

    restore()
    prof = profile_one(dfr, batched, stream)
    stats = dfr.dfr_get_stats(ws, stream)
    peak, peak_kind = measured_peaks()
    roof = dominant_roofline(prof, stats, 4, peak, peak_kind)

    e2e = None
    if not args.no_e2e:
        hin = torch.from_numpy(host.view(np.int32)).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        tt = []
        for _ in range(max(1, min(args.steps, 3))):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            work.copy_(hin, non_blocking=True)
            batched()
            hout.copy_(work, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            tt.append(e0.elapsed_time(e1))
        ems, e2e_rate = job_rate(statistics.mean(tt), total_keys, world, dev)
        e2e = {"value": e2e_rate, "unit": "Gkeys/s",
               "h2d_bytes_per_step": int(host.nbytes), "d2h_bytes_per_step": int(host.nbytes), "ms_per_step": ems}

    cpu = None
    if rank == 0 and world == 1 and args.cpu_sample > 0:
        cpu = cpu_batch_time(arrays, args.cpu_sample)
    if rank == 0:
        line = {
            "metric": "Gkeys/s", "value": value, "unit": "Gkeys/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": args.workload, "arrays": len(arrays), "total_keys": total_keys,
                       "sizes": "log-uniform [2^8, 2^20]", "keys": "uniform or Zipf(1.1) per array",
                       "uniform_arrays": kinds.count("uniform"),
                       "l2": "flushed (256 MiB write) before every repetition",
                       "inputs": "restored from a pristine device copy before every repetition (untimed)"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "batched_vs_plain": {
                "batched_gkeys_s": value / world,
                "plain_uncaptured_gkeys_s": total_keys / (ms_plain * 1e-3) / 1e9,
                "plain_graph_gkeys_s": total_keys / (ms_graph * 1e-3) / 1e9,
                "plain_uncaptured_ms": ms_plain, "plain_graph_ms": ms_graph, "batched_ms": ms / 1,
                "speedup_vs_uncaptured": ms_plain / ms, "speedup_vs_graph": ms_graph / ms},
            "sort_roofline_frac": stats["model_bytes"] / (ms * 1e-3) / 1e9 / peak,
            "kernels": {k: {"ms": v[0], "launches": v[1]} for k, v in prof.items()},
            "plan": {k: stats[k] for k in ("levels", "cta_keys", "wsort_keys", "tiny_keys", "const_keys",
                                           "cta_buckets", "wsort_buckets", "model_bytes")},
        }
        if emit:
            print(json.dumps(line), flush=True)
        return line
    return None


def cpu_batch_time(arrays, sample_keys):
    """The oracle, single-threaded, on the first arrays up to sample_keys keys."""
    import oracle

    keys, t0 = 0, time.perf_counter()
    count = 0
    for a in arrays:
        if keys >= sample_keys:
            break
        oracle.sort_u32(a)
        keys += a.size
        count += 1
    dt = time.perf_counter() - t0
    return {"value": keys / dt / 1e9, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
            "sample": "the first %d of the arrays (%d keys, %.1f s)" % (count, keys, dt)}


class _Ring:
    """First-in first-out arena for the client's request buffers: blocks are
    handed out in order and returned in the same order."""

    def __init__(self, size):
        import collections

        self.size = size
        self.live = collections.deque()  # (offset, bytes) in allocation order

    def alloc(self, nbytes):
        nbytes = (nbytes + 255) // 256 * 256
        if not self.live:
            off = 0 if nbytes <= self.size else None
        else:
            tail = self.live[0][0]
            head = self.live[-1][0] + self.live[-1][1]
            if head > tail:
                off = head if self.size - head >= nbytes else (0 if tail >= nbytes else None)
            else:  # wrapped: free space is [head, tail)
                off = head if tail - head >= nbytes else None
        if off is not None:
            self.live.append((off, nbytes))
        return off

    def free_oldest(self):
        self.live.popleft()


def served_pass(dfr, srv, gen, arena, sizes, kvs, seed, rate, ring_bytes, events):
    """One pass of the request stream.  rate = None: closed loop (submit as
    fast as buffers allow); else Poisson arrivals at `rate` requests/s.
    Each request's keys are generated on the device at its arrival (SplitMix64
    on the producer stream `gen`), then submitted with an event to wait on.
    Returns (latencies in us from the scheduled arrival, wall seconds from the
    first arrival to the last completion, keys)."""
    import collections

    R = len(sizes)
    g = np.random.Generator(np.random.PCG64(seed + 7))
    arrivals = np.cumsum(g.exponential(1.0 / rate, R)) if rate else np.zeros(R)
    ring = _Ring(ring_bytes)
    base = arena.data_ptr()
    outstanding = collections.deque()
    lats = np.zeros(R)
    t0 = time.perf_counter()
    t_last = t0
    gst = int(gen.cuda_stream)

    def retire(block):
        nonlocal t_last
        while outstanding:
            r, t, t_sched, t_call = outstanding[0]
            if block:
                rc, lat = dfr.dfr_wait(srv, t)
                done = True
            else:
                rc, done, lat = dfr.dfr_poll(srv, t)
            if not done:
                return
            if rc != dfr.DFR_OK:
                raise RuntimeError("request %d: %s" % (r, dfr.dfr_status_string(rc)))
            lats[r] = lat + (t_call - t_sched) * 1e6
            t_last = max(t_last, t_call + lat * 1e-6)
            ring.free_oldest()
            outstanding.popleft()
            block = False

    for r in range(R):
        n = int(sizes[r])
        kv = bool(kvs[r])
        kb = 8 if kv else 4
        need = n * kb + (n * 4 if kv else 0) + 256
        t_sched = t0 + arrivals[r]
        while time.perf_counter() < t_sched:
            retire(False)
        while True:
            off = ring.alloc(need)
            if off is not None:
                break
            retire(True)
        kp = base + off
        vp = base + off + ((n * kb + 255) // 256 * 256) if kv else 0
        kt = dfr.DFR_U64_KV if kv else dfr.DFR_U32
        dfr.check(dfr.dfr_fill_splitmix64(kt, kp, vp, n, synth.request_seed(seed, r), gst), "fill")
        ev = events[r % len(events)]
        ev.record(gen)
        t_call = time.perf_counter()
        rc, t = dfr.dfr_submit_after(srv, (kt, kp, vp, 0, 0, n), ev)
        if rc != dfr.DFR_OK:
            raise RuntimeError("submit: %s" % dfr.dfr_status_string(rc))
        outstanding.append((r, t, t_sched, t_call))
        retire(False)
    retire(True)
    while outstanding:
        retire(True)
    keys = int(np.sum(sizes))
    return lats, t_last - t0, keys


def run_served(args, wl, dfr, dev, world, rank):
    """Served form: a Poisson stream of sort requests through dfr_submit, at
    offered loads of 25/50/75/100% of the saturated (closed-loop) served
    throughput, against the same stream served first-in first-out with one
    plain launch sequence per request (the same server with coalescing off and
    one stream)."""
    import torch

    R = args.requests or wl["requests"]
    seed = synth.BASE_SEED + SEED_OFFSET["served_mixed"]
    sizes, kvs = synth.served_stream(R, seed, wl["lo"], wl["hi"])
    mean_n = float(np.mean(sizes))
    ring_bytes = 32 << 30
    arena = torch.empty(ring_bytes, dtype=torch.uint8, device=dev)
    gen = torch.cuda.Stream(dev)
    events = [torch.cuda.Event() for _ in range(1024)]
    torch.cuda.synchronize()

    def make_server(batched):
        srv = dfr.dfr_server_create(dev.index or 0, wl["budget"], args.serve_streams if batched else 1)
        if not batched:  # back-to-back plain launches, in arrival order, on one stream
            dfr.check(dfr.dfr_server_set_limits(srv, 1, dfr.DFR_SERVER_MAX_INFLIGHT), "limits")
        return srv

    def one(batched, rate, count=None):
        srv = make_server(batched)
        try:
            c = count or R
            lats, wall, keys = served_pass(dfr, srv, gen, arena, sizes[:c], kvs[:c], seed, rate, ring_bytes, events)
            st = dfr.dfr_server_stats(srv)
        finally:
            dfr.dfr_server_destroy(srv)
        return {"gkeys_s": keys / wall / 1e9, "p50_us": float(np.percentile(lats, 50)),
                "p99_us": float(np.percentile(lats, 99)), "mean_us": float(np.mean(lats)), "wall_s": wall,
                "requests": int(len(lats)), "batches": st["batches"]}

    # warm-up: a short closed-loop pass of each arm
    for _ in range(max(1, args.warmup)):
        one(True, None, min(R, 500))
        one(False, None, min(R, 200))

    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    clocks.mark_start()
    l0 = dfr.dfr_launch_count()
    closed = one(True, None)
    peak_keys_s = closed["gkeys_s"] * 1e9
    loads = {}
    for L in wl["loads"]:
        rate = L * peak_keys_s / mean_n
        loads["%d%%" % round(100 * L)] = {"offered_req_s": rate, "offered_gkeys_s": L * peak_keys_s / 1e9,
                                          "batched": one(True, rate),
                                          "fifo_plain": one(False, rate)}
    launches = dfr.dfr_launch_count() - l0
    clocks.mark_end()
    clk = clocks.stop()
    closed_plain = one(False, None, min(R, 20_000))

    cpu = None
    if rank == 0 and world == 1 and args.cpu_sample > 0:
        cpu = cpu_served_time(wl, args.cpu_sample, R)
    if rank == 0:
        full = loads["100%"]
        line = {
            "metric": "Gkeys/s", "value": closed["gkeys_s"], "unit": "Gkeys/s", "n_gpus": world,
            "steps": 1, "warmup": args.warmup, "ms_per_step": closed["wall_s"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32 | u64+u32", "data": "synthetic",
            "config": {"workload": args.workload, "requests": R, "sizes": "log-uniform [2^10, 2^24]",
                       "mix": "70% u32 keys only, 30% u64 keys + u32 payloads", "keys": "uniform (SplitMix64)",
                       "budget_bytes": wl["budget"], "server_streams": args.serve_streams,
                       "arrivals": "Poisson", "l2": "inputs regenerated per request (not resident in L2)"},
            "roofline": None, "cpu_baseline": cpu, "e2e": None, "gpu_launches": launches, "clocks": clk,
            "closed_loop": {"batched": closed, "fifo_plain": closed_plain},
            "loads": loads,
            "p50_us_at_100pct": full["batched"]["p50_us"], "p99_us_at_100pct": full["batched"]["p99_us"],
        }
        print(json.dumps(line), flush=True)
    return 0


def cpu_served_time(wl, sample_keys, requests=0):
    """The oracle, single-threaded, on the first requests of the served stream
    (keys regenerated on the host) up to sample_keys keys."""
    import oracle

    R = requests or wl["requests"]
    seed = synth.BASE_SEED + SEED_OFFSET["served_mixed"]
    sizes, kvs = synth.served_stream(R, seed, wl["lo"], wl["hi"])
    keys, cnt, dt = 0, 0, 0.0
    for r in range(R):
        if keys >= sample_keys:
            break
        n = int(sizes[r])
        if kvs[r]:
            k, v = synth.splitmix64(synth.request_seed(seed, r), n), synth.index_payload(n)
            t0 = time.perf_counter()
            oracle.sort_u64_kv(k, v)
        else:
            k = synth.splitmix64_u32(synth.request_seed(seed, r), n)
            t0 = time.perf_counter()
            oracle.sort_u32(k)
        dt += time.perf_counter() - t0
        keys += n
        cnt += 1
    return {"value": keys / dt / 1e9, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
            "sample": "the first %d requests of the stream (%d keys, %.1f s of sorting, keys regenerated on "
                      "the host)" % (cnt, keys, dt)}


def run_reference_forms(args, wl):
    """Reference arm of the batch and served workloads: the oracle on a
    bounded sample (the first arrays / requests), once per step."""
    if wl["kind"] == "batch":
        arrays, _ = batch_inputs(wl)
        fn = lambda: cpu_batch_time(arrays, args.cpu_sample)  # noqa: E731
    else:
        fn = lambda: cpu_served_time(wl, args.cpu_sample, args.requests)  # noqa: E731
    for _ in range(args.warmup):
        fn()
    runs = [fn() for _ in range(args.steps)]
    value = statistics.mean(r["value"] for r in runs)
    line = {
        "impl": "reference", "metric": "Gkeys/s", "value": value, "unit": "Gkeys/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32" if wl["kind"] == "batch" else "u32 | u64+u32",
        "data": "synthetic", "config": {"workload": args.workload},
        "cpu_baseline": dict(runs[-1], value=value),
        "e2e": {"value": value, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def config_of(name, wl):
    return {"workload": name, "n_per_array": wl["n"], "arrays_per_step": len(wl["dists"]),
            "distributions": wl["dists"], "key": wl["key"], "l2": "flushed (256 MiB write) before every sort",
            "inputs": "restored from a pristine device copy before every sort (untimed)"}


def run_plain(args, wl, dfr, dev, world, rank, emit=True):
    """One plain-sort workload (every array sorted alone, timed with CUDA
    events); returns rank 0's JSON line (printed when `emit`)."""
    import torch

    local = dev.index or 0
    stream = torch.cuda.current_stream(dev)
    n = wl["n"]
    kv = wl["key"] == "u64kv"
    kt = dfr.DFR_U64_KV if kv else dfr.DFR_U32
    wbytes = 8 if kv else 4
    vbytes = 4 if kv else 0
    inputs = gen_inputs(wl, SEED_OFFSET.get(args.workload, 0))

    pristine = {d: dfr.to_device(a, dev) for d, a in inputs.items()}
    work = torch.empty_like(next(iter(pristine.values())))
    vals0 = dfr.to_device(synth.index_payload(n), dev) if kv else None
    vals = torch.empty_like(vals0) if kv else None
    sorter = dfr.Sorter(kt, n, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    if args.schedule != "plan":
        c = dfr.dfr_tune_class(n)
        t = dfr.dfr_tune_get(kt, c)
        t["schedule"] = {"msd": dfr.DFR_SCHED_MSD, "lsd": dfr.DFR_SCHED_LSD, "dfr": dfr.DFR_SCHED_DFR}[args.schedule]
        dfr.check(dfr.dfr_tune_set(kt, c, t), "dfr_tune_set")

    def restore(d):
        work.copy_(pristine[d])
        if kv:
            vals.copy_(vals0)
        flush.fill_(1)

    def one_sort(d, ev0, ev1):
        restore(d)
        ev0.record(stream)
        sorter.sort_(work, vals, n, stream)
        ev1.record(stream)

    # warm-up (the clock sampler is live from here; its summary keeps the
    # samples stamped within the timed steps)
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        for d in inputs:
            one_sort(d, torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    torch.cuda.synchronize()

    # the warm-up sorts must have raised no device-side error (timeout, bounds,
    # queue capacity); parity with the oracle is the tests' job
    status = sorter.device_status(stream)
    if status != dfr.DFR_OK:
        raise RuntimeError("device status %s after warm-up" % dfr.dfr_status_string(status))

    barrier(world)
    torch.cuda.synchronize()
    clocks.mark_start()
    launches0 = dfr.dfr_launch_count()
    evs = []
    for _ in range(args.steps):
        row = []
        for d in inputs:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            one_sort(d, e0, e1)
            row.append((d, e0, e1))
        evs.append(row)
    torch.cuda.synchronize()
    clocks.mark_end()
    launches = dfr.dfr_launch_count() - launches0
    barrier(world)
    clk = clocks.stop()
    per_dist_ms = {d: [] for d in inputs}
    step_ms = []
    for row in evs:
        tot = 0.0
        for d, e0, e1 in row:
            ms = e0.elapsed_time(e1)
            per_dist_ms[d].append(ms)
            tot += ms
        step_ms.append(tot)
    ms_step_local = sum(step_ms) / len(step_ms)
    keys_per_step = n * len(inputs)
    ms_step, value = job_rate(ms_step_local, keys_per_step, world, dev)

    # Per-kernel profile of one more step (CUDA events around every launch),
    # plus the executed plan's algorithmic bytes from the device counters.
    peak, peak_kind = measured_peaks()
    dfr.dfr_profile_enable(True)
    dfr.dfr_profile_read()
    plan = {}
    prof_by_dist = {}
    prof = {}
    for d in inputs:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        one_sort(d, e0, e1)
        torch.cuda.synchronize()
        plan[d] = sorter.stats(stream)
        pd = dfr.dfr_profile_read()
        prof_by_dist[d] = {k: round(v[0], 4) for k, v in pd.items() if v[1]}
        for k, (ms_k, n_k) in pd.items():
            a, b = prof.get(k, (0.0, 0))
            prof[k] = (a + ms_k, b + n_k)
    dfr.dfr_profile_enable(False)
    rec = wbytes + vbytes
    # The dominant deal kernel: the MSD levels' scatter, or the LSD passes
    # when an LSD schedule dealt the top digits (read + write of every record
    # dealt, per launch).
    scatter_keys = sum(sum(p["level_keys"]) for p in plan.values())
    lsd_keys = sum(p["lsd_keys"] for p in plan.values())
    # The dominant record-moving kernel: the MSD levels' scatter, the LSD
    # passes (when an LSD schedule dealt the top digits) or the CTA sort --
    # algorithmic bytes = a read and a write of every record it handles.
    cta_keys = sum(p["cta_keys"] for p in plan.values())
    # A call run as one persistent launch (k_persist) moves every byte of the
    # sort in that launch: its algorithmic bytes are the plan's model bytes.
    cands = {"k_scatter": ("scatter", scatter_keys), "k_lsd_pass": ("lsd_pass", lsd_keys),
             "k_ctasort": ("ctasort", cta_keys), "k_persist": ("persist", None)}
    dom_kernel = max((k for k in cands if cands[k][0] in prof), key=lambda k: prof[cands[k][0]][0])
    dom_ms, dom_launches = prof[cands[dom_kernel][0]]
    dom_keys = cands[dom_kernel][1]
    dom_bytes = 2 * rec * dom_keys if dom_keys is not None else sum(p["model_bytes"] for p in plan.values())
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9 if dom_ms > 0 else 0.0
    traffic = None
    per_key = traffic_per_key(dom_kernel) if not kv and dom_keys is not None else None
    if per_key is not None:
        traffic = per_key * dom_keys / max(1, dom_launches)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": dom_kernel,
                "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": dom_bytes / max(1, dom_launches)}
    # Small arrays: the same sorts launched as one captured CUDA graph each
    # (dfr_graph_*), which replaces the call's kernel launches by one.
    graph_ms = {}
    if n <= (1 << 22):
        g = dfr.dfr_graph_create([(kt, work, vals if kv else 0, sorter.kbuf, sorter.vbuf if kv else 0, n)], sorter.ws,
                                 sorter.ws_bytes)
        try:
            for d in inputs:
                ts = []
                for _ in range(max(3, args.steps)):
                    restore(d)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    dfr.check(dfr.dfr_graph_launch(g, stream), "graph")
                    e1.record(stream)
                    e1.synchronize()
                    ts.append(e0.elapsed_time(e1))
                graph_ms[d] = statistics.median(ts)
        finally:
            dfr.dfr_graph_destroy(g)
    per_dist = {}
    for d in inputs:
        t = statistics.median(per_dist_ms[d])
        p = plan[d]
        per_dist[d] = {"ms": t, "gkeys_s": n / (t * 1e-3) / 1e9, "model_bytes": p["model_bytes"],
                       "sort_roofline_frac": p["model_bytes"] / (t * 1e-3) / 1e9 / peak,
                       "levels": p["levels"], "level_keys": [k for k in p["level_keys"] if k],
                       "cta_keys": p["cta_keys"], "wsort_keys": p["wsort_keys"], "tiny_keys": p["tiny_keys"],
                       "const_keys": p["const_keys"], "group_buckets": p["group_buckets"],
                       "cta_buckets": p["cta_buckets"], "wsort_buckets": p["wsort_buckets"],
                       "schedule": ("msd", "lsd", "dfr")[p["schedule"]], "lsd_keys": p["lsd_keys"],
                       "kernel_ms": prof_by_dist[d]}
        if p["est_capacity"]:
            per_dist[d]["est_overflow"] = p["est_overflow"]
            per_dist[d]["est_aborted"] = p["est_aborted"]
        if d in graph_ms:
            per_dist[d]["graph_ms"] = graph_ms[d]
            per_dist[d]["graph_gkeys_s"] = n / (graph_ms[d] * 1e-3) / 1e9
    kernel_share = {k: {"ms": v[0], "launches": v[1]} for k, v in prof.items() if v[1]}

    # End to end through the C ABI: pinned host keys -> device -> sort -> host.
    # Arrays go round-robin to `ns` streams, each with its own device buffer
    # set; a stream's next upload waits for its previous download, so with
    # three or more streams the upload engine never waits on a sort and the
    # uploads, sorts and downloads of consecutive arrays all overlap (the two
    # copy directions run on separate copy engines).  Every host<->device copy
    # of the step is inside the timed region.
    e2e = None
    if not args.no_e2e:
        ns = max(1, args.e2e_streams)
        host_in = {d: torch.from_numpy(a.view(np.int32) if a.dtype == np.uint32 else a.view(np.int64)).pin_memory()
                   for d, a in inputs.items()}
        host_out = [torch.empty_like(next(iter(host_in.values()))).pin_memory() for _ in range(ns)]
        hv_in = torch.from_numpy(synth.index_payload(n).view(np.int32)).pin_memory() if kv else None
        hv_out = [torch.empty_like(hv_in).pin_memory() for _ in range(ns)] if kv else [None] * ns
        streams = [stream] + [torch.cuda.Stream(dev) for _ in range(ns - 1)]
        works = [work] + [torch.empty_like(work) for _ in range(ns - 1)]
        valss = [vals] + [torch.empty_like(vals) for _ in range(ns - 1)] if kv else [None] * ns
        sorters = [sorter] + [dfr.Sorter(kt, n, dev) for _ in range(ns - 1)]
        e2e_ms = []
        # one untimed pass first: the extra streams' first copies and sorts
        # (first touch of their buffers) stay out of the timed steps
        for step in range(1 + max(1, min(args.steps, 3))):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(streams[0])
            for s in streams[1:]:
                s.wait_event(e0)
            for i, d in enumerate(inputs):
                j = i % ns
                with torch.cuda.stream(streams[j]):
                    works[j].copy_(host_in[d], non_blocking=True)
                    if kv:
                        valss[j].copy_(hv_in, non_blocking=True)
                    sorters[j].sort_(works[j], valss[j], n, streams[j])
                    host_out[j].copy_(works[j], non_blocking=True)
                    if kv:
                        hv_out[j].copy_(valss[j], non_blocking=True)
            for s in streams[1:]:
                joined = torch.cuda.Event()
                joined.record(s)
                streams[0].wait_event(joined)
            e1.record(streams[0])
            e1.synchronize()
            if step > 0:
                e2e_ms.append(e0.elapsed_time(e1))
        for j in range(ns):
            st = sorters[j].device_status(streams[j])
            if st != dfr.DFR_OK:
                raise RuntimeError("device status %s in the end-to-end run" % dfr.dfr_status_string(st))
        ms, e2e_rate = job_rate(sum(e2e_ms) / len(e2e_ms), keys_per_step, world, dev)
        # The host link of this machine, for context: one array's plain
        # copy each way from / to the same pinned buffers, and both at once.
        first = next(iter(inputs))
        nbytes = host_in[first].numel() * host_in[first].element_size()

        def copy_ms(pairs):
            torch.cuda.synchronize()
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(streams[0])
            for s in streams[1:]:
                s.wait_event(c0)
            for j, (dst_t, src_t) in enumerate(pairs):
                with torch.cuda.stream(streams[j % ns]):
                    dst_t.copy_(src_t, non_blocking=True)
            for s in streams[1:]:
                ev = torch.cuda.Event()
                ev.record(s)
                streams[0].wait_event(ev)
            c1.record(streams[0])
            c1.synchronize()
            return c0.elapsed_time(c1)

        h2d = nbytes / (copy_ms([(works[0], host_in[first])]) * 1e-3) / 1e9
        d2h = nbytes / (copy_ms([(host_out[0], works[0])]) * 1e-3) / 1e9
        both = 2 * nbytes / (copy_ms([(works[0], host_in[first]), (host_out[-1], works[-1])]) * 1e-3) / 1e9
        e2e = {"value": e2e_rate, "unit": "Gkeys/s",
               "h2d_bytes_per_step": keys_per_step * rec, "d2h_bytes_per_step": keys_per_step * rec,
               "ms_per_step": ms, "streams": ns,
               "overlap": "arrays round-robin over %d streams: uploads, sorts and downloads of consecutive arrays "
                          "overlap" % ns,
               "host_link_gbs": {"h2d": h2d, "d2h": d2h, "both_directions": both}}

    cpu = None
    if rank == 0 and world == 1 and args.cpu_sample > 0:
        sample_n = min(n, args.cpu_sample)
        ck, cdt = cpu_oracle_time(inputs, sample_n, wl["key"])
        cpu = {"value": ck / cdt / 1e9, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
               "sample": "first %d keys of each of the %d arrays (%d keys, %.1f s)" % (sample_n, len(inputs), ck, cdt)}

    if rank == 0:
        line = {
            "metric": "Gkeys/s", "value": value, "unit": "Gkeys/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32" if not kv else "u64+u32", "data": "synthetic",
            "config": dict(config_of(args.workload, wl), schedule=args.schedule,
                           clocks="sampled every 200 ms over the warm-up and timed steps"),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk, "per_dist": per_dist, "kernels": kernel_share,
        }
        if emit:
            print(json.dumps(line), flush=True)
        return line
    return None


def extra_summary(line):
    """The parts of another workload's line carried in the default line."""
    if line is None:
        return None
    keep = ("metric", "value", "unit", "ms_per_step", "config", "roofline", "clocks", "gpu_launches",
            "batched_vs_plain", "sort_roofline_frac")
    out = {k: line[k] for k in keep if k in line}
    if "per_dist" in line:
        out["per_dist"] = {d: {k: v[k] for k in ("ms", "gkeys_s", "sort_roofline_frac", "schedule") if k in v}
                           for d, v in line["per_dist"].items()}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dfr", choices=["dfr", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-sample", type=int, default=1 << 26)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: leave out the 2^27 key-value and 4096-array batch results")
    ap.add_argument("--e2e-streams", type=int, default=3, help="streams (device buffer sets) of the end-to-end leg")
    ap.add_argument("--dists", default="", help="comma-separated subset of the workload's distributions")
    ap.add_argument("--requests", type=int, default=0, help="served workload: requests per pass")
    ap.add_argument("--serve-streams", type=int, default=4, help="served workload: server streams")
    ap.add_argument("--schedule", default="plan", choices=["plan", "msd", "lsd", "dfr"],
                    help="plain workloads: override the launch plan's schedule of the top digits "
                         "(msd: diverting MSD; lsd: diverting LSD with one counting read; dfr: diverting "
                         "LSD with the estimated first deal, Fast Radix)")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.dists and "dists" in wl:
        wl["dists"] = [d for d in args.dists.split(",") if d in wl["dists"]]
    rank, world, local = dist_setup()

    if args.impl == "reference":
        return run_reference(args, wl, world, rank)

    import torch

    import __graft_entry__

    if world > 1:
        import torch.distributed as tdist

        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
    __graft_entry__.build()
    import paper_2207_14334_gb300 as dfr

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if wl["kind"] == "batch":
        run_batch(args, wl, dfr, dev, world, rank)
        return 0
    if wl["kind"] == "served":
        return run_served(args, wl, dfr, dev, world, rank)
    if wl["kind"] == "plain" and args.workload == DEFAULT_WORKLOAD and not args.no_extras:
        line = run_plain(args, wl, dfr, dev, world, rank, emit=False)
        extra = argparse.Namespace(**vars(args))
        extra.steps, extra.warmup, extra.no_e2e, extra.cpu_sample = 3, 3, True, 0
        extra.dists = ""
        extra.workload = "kv_u64_2^27"
        kv_line = run_plain(extra, dict(WORKLOADS[extra.workload]), dfr, dev, world, rank, emit=False)
        extra.workload = "batch_u32_4096"
        b_line = run_batch(extra, dict(WORKLOADS[extra.workload]), dfr, dev, world, rank, emit=False)
        if rank == 0:
            line["kv_u64_2^27"] = extra_summary(kv_line)
            line["batch_u32_4096"] = extra_summary(b_line)
            print(json.dumps(line), flush=True)
    else:
        run_plain(args, wl, dfr, dev, world, rank)
    if world > 1:
        import torch.distributed as tdist

        tdist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
