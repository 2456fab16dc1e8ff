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

# ncu DRAM traffic of the scatter kernel (read + write bytes per key dealt),
# taken from profiles/scatter_u32_uniform.md; valid only while the kernel
# sources hash to SCATTER_SRC_SHA (else reported as null).
SCATTER_NCU_BYTES_PER_KEY = None
SCATTER_SRC_SHA = None

WORKLOADS = {
    "plain_u32_2^28": dict(kind="plain", key="u32", n=1 << 28, dists=list(synth.U32_DISTRIBUTIONS)),
    "plain_u32_1M": dict(kind="plain", key="u32", n=1_000_000, dists=["uniform"]),
    "kv_u64_2^27": dict(kind="plain", key="u64kv", n=1 << 27, dists=list(synth.U64_DISTRIBUTIONS)),
    # a smaller case (still larger than L2) for full ncu captures
    "plain_u32_2^26": dict(kind="plain", key="u32", n=1 << 26, dists=["uniform"]),
}
DEFAULT_WORKLOAD = "plain_u32_2^28"
SEED_OFFSET = {"plain_u32_2^28": 20, "plain_u32_1M": 1, "kv_u64_2^27": 30, "plain_u32_2^26": 20}


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2207_14334_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(f.read())
    return h.hexdigest()[:16]


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
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "dfr_clocks_%d_%d.csv" % (os.getpid(), index))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        loaded = [x for x in sm if x > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


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


def config_of(name, wl):
    return {"workload": name, "n_per_array": wl["n"], "arrays_per_step": len(wl["dists"]),
            "distributions": wl["dists"], "key": wl["key"], "l2": "flushed (256 MiB write) before every sort",
            "inputs": "restored from a pristine device copy before every sort (untimed)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dfr", choices=["dfr", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-sample", type=int, default=1 << 26)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--dists", default="", help="comma-separated subset of the workload's distributions")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.dists:
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

    # warm-up
    for _ in range(args.warmup):
        for d in inputs:
            one_sort(d, torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    torch.cuda.synchronize()

    # correctness spot check of the last warm-up result (sampled: sortedness)
    status = sorter.device_status(stream)
    if status != dfr.DFR_OK:
        raise RuntimeError("device status %s after warm-up" % dfr.dfr_status_string(status))

    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
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
    ms_step = reduce_max([ms_step_local], world, dev)[0]
    keys_per_step = n * len(inputs)
    value = world * keys_per_step / (ms_step * 1e-3) / 1e9

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
    scatter_keys = sum(sum(p["level_keys"]) for p in plan.values())
    scatter_ms, scatter_launches = prof["scatter"]
    scatter_bytes = 2 * rec * scatter_keys
    achieved = scatter_bytes / (scatter_ms * 1e-3) / 1e9 if scatter_ms > 0 else 0.0
    traffic = None
    if SCATTER_NCU_BYTES_PER_KEY is not None and SCATTER_SRC_SHA == kernel_source_sha():
        traffic = SCATTER_NCU_BYTES_PER_KEY * scatter_keys / max(1, scatter_launches)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": "k_scatter",
                "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": scatter_bytes / max(1, scatter_launches)}
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
                       "kernel_ms": prof_by_dist[d]}
    kernel_share = {k: {"ms": v[0], "launches": v[1]} for k, v in prof.items() if v[1]}

    # End to end through the C ABI: pinned host keys -> device -> sort -> host.
    e2e = None
    if not args.no_e2e:
        host_in = {d: torch.from_numpy(a.view(np.int32) if a.dtype == np.uint32 else a.view(np.int64)).pin_memory()
                   for d, a in inputs.items()}
        host_out = torch.empty_like(next(iter(host_in.values()))).pin_memory()
        hv_in = torch.from_numpy(synth.index_payload(n).view(np.int32)).pin_memory() if kv else None
        hv_out = torch.empty_like(hv_in).pin_memory() if kv else None
        e2e_ms = []
        for step in range(max(1, min(args.steps, 3))):
            tot = 0.0
            for d in inputs:
                flush.fill_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                work.copy_(host_in[d], non_blocking=True)
                if kv:
                    vals.copy_(hv_in, non_blocking=True)
                sorter.sort_(work, vals, n, stream)
                host_out.copy_(work, non_blocking=True)
                if kv:
                    hv_out.copy_(vals, non_blocking=True)
                e1.record(stream)
                e1.synchronize()
                tot += e0.elapsed_time(e1)
            e2e_ms.append(tot)
        ms = reduce_max([sum(e2e_ms) / len(e2e_ms)], world, dev)[0]
        e2e = {"value": world * keys_per_step / (ms * 1e-3) / 1e9, "unit": "Gkeys/s",
               "h2d_bytes_per_step": keys_per_step * rec, "d2h_bytes_per_step": keys_per_step * rec,
               "ms_per_step": ms}

    cpu = None
    if rank == 0 and world == 1:
        sample_n = min(n, args.cpu_sample)
        ck, cdt = cpu_oracle_time(inputs, sample_n, wl["key"])
        cpu = {"value": ck / cdt / 1e9, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
               "sample": "first %d keys of each of the %d arrays (%d keys, %.1f s)" % (sample_n, len(inputs), ck, cdt)}

    if rank == 0:
        line = {
            "metric": "Gkeys/s", "value": value, "unit": "Gkeys/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32" if not kv else "u64+u32", "data": "synthetic",
            "config": config_of(args.workload, wl), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk, "per_dist": per_dist, "kernels": kernel_share,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as tdist

        tdist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
