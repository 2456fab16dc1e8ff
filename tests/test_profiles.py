"""The committed profile summaries are consistent with what bench.py reports
(CPU only): every summary gives the command that made it; the per-key DRAM
traffic bench.py scales into `roofline.traffic` is the figure the scatter
summary records, for the kernel sources hash that summary names (bench.py
reports the traffic only while the sources still hash to it)."""
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def test_every_summary_gives_its_command():
    names = sorted(n for n in os.listdir(PROFILES) if n.endswith((".md", ".txt")))
    assert names
    for n in names:
        text = open(os.path.join(PROFILES, n)).read()
        assert "Command" in text and "```" in text, n
        assert "/root/" not in text.split("```")[1], n  # commands name files of the repository only


def test_scatter_traffic_matches_its_summary():
    text = open(os.path.join(PROFILES, "k_scatter_u32_uniform_2^26.md")).read()
    assert "sha256[:16] = %s" % bench.SCATTER_SRC_SHA in text
    m = re.search(r"DRAM read \+ write per key dealt \| ([0-9.]+) B", text)
    assert m and abs(float(m.group(1)) - bench.SCATTER_NCU_BYTES_PER_KEY) < 0.01

