"""The benchmark's clock sampler, against a fake nvidia-smi (CPU only): it is
live before the timed region starts, keeps the samples stamped inside that
region, falls back to a longer polling interval when the short one yields
nothing, and never raises when nvidia-smi is missing or prints unreadable
stamps."""
import datetime
import os
import stat
import sys
import time

import bench

FAKE = """#!{python}
import datetime, os, sys, time
args = sys.argv[1:]
ms = int(args[args.index("-lms") + 1])
query = [a for a in args if a.startswith("--query-gpu=")][0]
stamped = "timestamp" in query
if ms < int(os.environ.get("FAKE_MIN_MS", "0")) or (stamped and os.environ.get("FAKE_NO_STAMP_FIELD")):
    print('Field "timestamp" is not a valid field to query.')  # an error on stdout, as a tool might print it
    sys.exit(2)
mhz = os.environ.get("FAKE_MHZ", "2070")
while True:
    row = "0, %s, 2070, 812.30, 0x0000000000000004, Not Active, Not Active, Not Active, Active" % mhz
    if stamped:
        t = datetime.datetime.now().strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        row = "%s, %s" % (t if os.environ.get("FAKE_STAMP", "1") == "1" else "[N/A]", row)
    sys.stdout.write(row + "\\n")
    sys.stdout.flush()
    time.sleep(ms / 1000.0)
"""


def fake_smi(tmp_path):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE.format(python=sys.executable))
    exe.chmod(exe.stat().st_mode | stat.S_IXUSR)
    return str(exe)


def run_sampler(exe, before=0.2, timed=0.3, after=0.2):
    c = bench.ClockSampler(0, exe=exe)
    c.start()
    time.sleep(before)
    c.mark_start()
    time.sleep(timed)
    c.mark_end()
    time.sleep(after)
    return c, c.stop()


def test_samples_inside_the_timed_region(tmp_path):
    c, r = run_sampler(fake_smi(tmp_path))
    assert r["window"] == "timed" and r["interval_ms"] == 20
    assert 3 <= r["samples"] < r["samples_total"]
    assert r["sm_mhz"] == 2070 and r["sm_max_mhz"] == 2070
    assert r["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(c.path)


def test_falls_back_to_the_long_interval(tmp_path, monkeypatch):
    monkeypatch.setenv("FAKE_MIN_MS", "100")  # the fake refuses intervals under 100 ms
    _, r = run_sampler(fake_smi(tmp_path), timed=0.6, after=0.3)
    assert r["interval_ms"] == 200 and r["samples_total"] >= 1


def test_falls_back_to_the_unstamped_query(tmp_path, monkeypatch):
    monkeypatch.setenv("FAKE_NO_STAMP_FIELD", "1")  # the fake refuses the timestamp field
    _, r = run_sampler(fake_smi(tmp_path), timed=0.6, after=0.3)
    assert r["interval_ms"] == 200 and r["window"] == "run" and r["samples_total"] >= 1
    assert r["sm_mhz"] == 2070 and r["reasons"] == ["sw_power_cap"]


def test_unreadable_stamps_use_every_sample(tmp_path, monkeypatch):
    monkeypatch.setenv("FAKE_STAMP", "0")
    _, r = run_sampler(fake_smi(tmp_path))
    assert r["window"] == "run" and r["samples"] == r["samples_total"] >= 3


def test_missing_nvidia_smi(tmp_path):
    c = bench.ClockSampler(0, exe=str(tmp_path / "absent"))
    c.start()
    c.mark_start()
    c.mark_end()
    assert c.stop() is None
    assert not os.path.exists(c.path)


def test_summary_keeps_only_the_window():
    base = datetime.datetime(2026, 1, 1, 12, 0, 0)
    lines = []
    for k in range(10):
        t = (base + datetime.timedelta(milliseconds=100 * k)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        slow = k in (4, 5)
        lines.append("%s, 0, %d, 2070, 900.0, 0x0, %s, Not Active, Not Active, Not Active"
                     % (t, 1800 if slow else 2070, "Active" if slow else "Not Active"))
    lines.append("garbage line")
    t0 = (base + datetime.timedelta(milliseconds=400)).timestamp()
    t1 = (base + datetime.timedelta(milliseconds=500)).timestamp()
    r = bench.ClockSampler.summarise(lines, t0, t1, 20)
    assert r["window"] == "timed" and r["samples"] == 2 and r["samples_total"] == 10
    assert r["sm_mhz"] == 1800 and r["reasons"] == ["hw_slowdown"]
    # a window between two samples, within one interval of neither: every sample
    t0 = (base + datetime.timedelta(milliseconds=430)).timestamp()
    t1 = (base + datetime.timedelta(milliseconds=460)).timestamp()
    r = bench.ClockSampler.summarise(lines, t0, t1, 20)
    assert r["window"] == "run" and r["samples"] == 10
    assert r["sm_mhz"] == 2070 and r["reasons"] == ["hw_slowdown"]
    assert bench.ClockSampler.summarise(["x"], None, None, 20) is None
