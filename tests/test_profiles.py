"""The committed profile summaries are consistent with what bench.py reports
(CPU only): every summary gives the command that made it, and every DRAM
traffic figure bench.py may scale into `roofline.traffic` is a well-formed
entry of profiles/traffic.json -- a per-key byte count, the kernel source
files it was captured with and their hash, and the summary it comes from.
bench.py uses a figure only while those files still hash to the recorded
value."""
import json
import os

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


def test_traffic_figures_are_well_formed():
    with open(bench.TRAFFIC_FILE) as f:
        table = json.load(f)
    assert table
    for kernel, e in table.items():
        assert kernel in ("k_scatter", "k_ctasort", "k_lsd_pass"), kernel
        assert 0.0 < float(e["dram_bytes_per_key"]) < 64.0, kernel
        assert e["source"] and all(os.path.exists(os.path.join(ROOT, p)) for p in e["source"]), kernel
        assert len(e["source_sha16"]) == 16, kernel
        assert os.path.exists(os.path.join(ROOT, e["summary"])), kernel


def test_traffic_figure_follows_the_source_hash(tmp_path, monkeypatch):
    """A figure is used only while its kernel source is unchanged."""
    src = tmp_path / "kernel.cuh"
    src.write_text("// kernel v1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    entry = {"dram_bytes_per_key": 7.5, "source": ["kernel.cuh"], "source_sha16": bench.source_sha(["kernel.cuh"]),
             "summary": "x.md"}
    table = tmp_path / "traffic.json"
    table.write_text(json.dumps({"k_scatter": entry}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(table))
    assert bench.traffic_per_key("k_scatter") == 7.5
    assert bench.traffic_per_key("k_ctasort") is None
    src.write_text("// kernel v2\n")
    assert bench.traffic_per_key("k_scatter") is None
