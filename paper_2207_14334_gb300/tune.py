"""Autotuner of the launch-plan table (radix window target, radix width,
warp-sort limit, scatter / CTA-sort grid sizes) per key type and size class.

For every key type and size class it sorts uniform keys (SplitMix64, made on
the device) laid out as that class's workload -- a batch of arrays of the
class's representative length, or one array for the largest classes -- under
every candidate plan, times each with CUDA events (inputs restored and L2
flushed before every repetition, outside the timed region), and keeps the
fastest.  The plans never change a result, only the time.

For single arrays of at least dfr_lsd_min_keys keys it also tries the LSD
schedule of the top digits (Algorithm 4) on top of the best MSD plan.

The table serves both launch forms: a call of fewer than
DFR_PERSIST_AUTO_KEYS keys runs as one persistent launch, a larger one (a
big batch of the same mean length) as the level sequence.  With --both-forms
a class whose timing workload is small enough for the persistent form is
timed in both forms, and the plan kept is the one with the smallest mean of
its two times, each divided by the best time of its form (pick_plan).

Writes the table as JSON and as the C include compiled into the library
(csrc/dfr_tune_table.inc); rebuild afterwards.  Needs a GPU:

    python -m paper_2207_14334_gb300.tune --out-json tune_table.json --write-inc
"""
from __future__ import annotations

import argparse
import datetime
import itertools
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
INC = os.path.join(HERE, "csrc", "dfr_tune_table.inc")

KEY_TYPES = ("DFR_U32", "DFR_U64", "DFR_U64_KV", "DFR_U32_KV", "DFR_U64_KV64", "DFR_U32_KV64")  # row order of the C table
FIELDS = ("target_log2", "max_bits", "warp_max", "scatter_ctas_per_sm", "ctasort_ctas_per_sm", "schedule", "launch")


def class_length(c: int) -> int:
    """Representative array length of size class c (middle of its range)."""
    return 1 << (11 + 2 * c) if c < 9 else 1 << 28


def candidates(cap_log2: int):
    """The plan grid searched for one (key type, class) with the MSD schedule."""
    out = []
    for tl, mb, wm, sc, cs in itertools.product((cap_log2 - 2, cap_log2 - 1, cap_log2), (8, 7), (128, 256, 512),
                                                (0, 2), (0, 1)):
        if mb == 7 and (sc, cs) != (0, 0):
            continue  # narrower windows are tried with the default grids only
        out.append(dict(target_log2=tl, max_bits=mb, warp_max=wm, scatter_ctas_per_sm=sc, ctasort_ctas_per_sm=cs,
                        schedule=0))
    return out


def pick_plan(times):
    """The plan to keep from {plan key: {form: ms}}: the smallest mean over
    the forms it was timed in of ms / (the best ms of that form)."""
    best = {}
    for t in times.values():
        for form, ms in t.items():
            best[form] = min(ms, best.get(form, ms))
    return min(times, key=lambda k: sum(ms / best[f] for f, ms in times[k].items()) / len(times[k]))


class Case:
    """Device buffers of one workload: `count` arrays of `n` keys each."""

    def __init__(self, dfr, torch, kt: int, n: int, count: int, seed: int):
        self.dfr, self.torch, self.kt, self.n, self.count = dfr, torch, kt, n, count
        kb = dfr.KEY_BYTES[kt]
        kv = dfr.HAS_VALS[kt]
        kdt = torch.int64 if kb == 8 else torch.int32
        stride = (n + 63) // 64 * 64
        total = stride * count
        self.keys = torch.empty(total, dtype=kdt, device="cuda")
        self.src = torch.empty_like(self.keys)
        self.kbuf = torch.empty_like(self.keys)
        vb = dfr.VAL_BYTES[kt]
        self.vals = torch.empty(total, dtype=torch.int64 if vb == 8 else torch.int32, device="cuda") if kv else None
        self.vsrc = torch.empty_like(self.vals) if kv else None
        self.vbuf = torch.empty_like(self.vals) if kv else None
        for a in range(count):
            o = a * stride
            dfr.check(dfr.dfr_fill_splitmix64(kt, self.src.data_ptr() + o * kb,
                                              (self.vsrc.data_ptr() + o * vb) if kv else 0, n, seed + a), "fill")
        self.segs = [(kt, self.keys.data_ptr() + a * stride * kb,
                      (self.vals.data_ptr() + a * stride * vb) if kv else 0,
                      self.kbuf.data_ptr() + a * stride * kb, (self.vbuf.data_ptr() + a * stride * vb) if kv else 0,
                      n) for a in range(count)]
        self.wsb = dfr.dfr_batch_workspace_bytes(self.segs)
        self.ws = torch.zeros(self.wsb, dtype=torch.uint8, device="cuda")
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def time_ms(self, reps: int) -> float:
        torch, dfr = self.torch, self.dfr
        ts = []
        for _ in range(reps):
            self.keys.copy_(self.src)
            if self.vals is not None:
                self.vals.copy_(self.vsrc)
            self.flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            dfr.check(dfr.dfr_sort_batch(self.segs, self.ws, self.wsb), "sort")
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        if dfr.dfr_last_device_status(self.ws) != dfr.DFR_OK:
            raise RuntimeError("device status after tuning run")
        ts.sort()
        return ts[len(ts) // 2]


def tune(key_types, classes, reps: int, budget_keys: int, schedules=(0, 1), both_forms=False, log=print):
    import torch

    import paper_2207_14334_gb300 as dfr

    dfr.load()
    table = {}
    for ktn in key_types:
        kt = getattr(dfr, ktn)
        cap_log2 = 12  # floor(log2) of the CTA sort's capacity (6144 u32 keys, 4096 otherwise)
        for c in classes:
            n = class_length(c)
            count = max(1, min(4096, budget_keys // n))
            case = Case(dfr, torch, kt, n, count, seed=0x5EED0000 + 1000 * c + kt)
            forms = (dfr.DFR_LAUNCH_LEVELS, dfr.DFR_LAUNCH_PERSISTENT) if (
                both_forms and n * count < dfr.DFR_PERSIST_AUTO_KEYS) else (dfr.DFR_LAUNCH_AUTO,)
            plans = candidates(cap_log2)
            times = {}
            for i, plan in enumerate(plans):
                for form in forms:
                    dfr.check(dfr.dfr_tune_set(kt, c, dict(plan, launch=form)), "tune_set")
                    case.time_ms(2)
                    times.setdefault(i, {})[form] = case.time_ms(reps)
            i = pick_plan(times)
            best = (sum(times[i].values()) / len(forms), plans[i])
            # The schedule of the top digits applies to single arrays large
            # enough for the LSD phase: tried on top of the best MSD plan.
            if count == 1 and n >= dfr.dfr_lsd_min_keys(kt):
                for sched in schedules:
                    if sched == 0:
                        continue
                    plan = dict(best[1], schedule=sched)
                    dfr.check(dfr.dfr_tune_set(kt, c, plan), "tune_set")
                    case.time_ms(2)
                    ms = case.time_ms(reps)
                    if ms < best[0]:
                        best = (ms, plan)
            dfr.dfr_tune_reset()
            default_ms = case.time_ms(reps)
            table.setdefault(ktn, {})[str(c)] = dict(best[1], ms=best[0], default_ms=default_ms, n=n, arrays=count)
            log("%-10s class %d n=%-9d x%-5d best %.3f ms (default %.3f) %s" % (ktn, c, n, count, best[0],
                                                                                default_ms, best[1]))
            del case
            torch.cuda.empty_cache()
    return table


def write_inc(table, path=INC, note=""):
    default = dict(target_log2=12, max_bits=8, warp_max=512, scatter_ctas_per_sm=0, ctasort_ctas_per_sm=0, schedule=0,
                   launch=0)
    lines = ["// dfr_tune_table.inc -- the built-in launch plans, one row per key type",
             "// (" + ", ".join(KEY_TYPES) + ")",
             "// and size class (mean array",
             "// length 2^<12, [2^12, 2^14), ..., 2^28+).  Fields: target_log2, max_bits,",
             "// warp_max, scatter_ctas_per_sm, ctasort_ctas_per_sm, schedule, launch, reserved.",
             "// Written by paper_2207_14334_gb300/tune.py" + (": " + note if note else "") + "."]
    for ktn in KEY_TYPES:
        rows = []
        for c in range(10):
            e = table.get(ktn, {}).get(str(c))
            if e is None:
                e = dict(default, target_log2=12 if ktn == "DFR_U32" else 11)
            rows.append("{%d, %d, %d, %d, %d, %d, %d, 0}" % tuple(int(e.get(f, 0)) for f in FIELDS))
        body = ",\n ".join(", ".join(rows[i:i + 3]) for i in range(0, 10, 3))
        lines.append("{" + body + "},")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--key-types", default=",".join(KEY_TYPES))
    ap.add_argument("--classes", default="0,1,2,3,4,5,6,7,8,9")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--budget-keys", type=int, default=1 << 24, help="keys per batch for the small classes")
    ap.add_argument("--out-json", default="")
    ap.add_argument("--write-inc", action="store_true")
    ap.add_argument("--inc-path", default=INC)
    ap.add_argument("--both-forms", action="store_true",
                    help="time the classes that run as one persistent launch in both launch forms")
    ap.add_argument("--schedules", default="0,1",
                    help="schedules of the top digits to try on single large arrays (0 MSD, 1 LSD, 2 LSD with the "
                         "estimated deal, which falls back to MSD on skewed inputs and is left out by default)")
    args = ap.parse_args(argv)
    if os.path.dirname(HERE) not in sys.path:
        sys.path.insert(0, os.path.dirname(HERE))
    t0 = time.time()
    table = tune(args.key_types.split(","), [int(x) for x in args.classes.split(",")], args.reps, args.budget_keys,
                 schedules=tuple(int(x) for x in args.schedules.split(",")), both_forms=args.both_forms)
    import torch

    meta = {"device": torch.cuda.get_device_name(0), "date": datetime.date.today().isoformat(),
            "seconds": round(time.time() - t0, 1), "reps": args.reps, "keys": "uniform (SplitMix64)"}
    if args.out_json:
        with open(args.out_json, "w") as f:
            json.dump({"meta": meta, "table": table}, f, indent=1)
    if args.write_inc:
        write_inc(table, path=args.inc_path, note="measured on %s, %s, median of %d repetitions per plan" % (meta["device"], meta["date"],
                                                                                           args.reps))
    return 0


if __name__ == "__main__":
    sys.exit(main())
