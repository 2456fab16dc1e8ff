"""DFR_TUNE_FILE and DFR_SPIN_LIMIT, applied by the binding when it loads the
library (CPU only: both act through host-side entry points).  Each case runs
in a fresh process, so the library's process-wide table starts built-in."""
import json
import os
import subprocess
import sys

import pytest

import paper_2207_14334_gb300 as dfr
from paper_2207_14334_gb300 import build as dfr_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROBE = """
import json, paper_2207_14334_gb300 as dfr
dfr.load()
print(json.dumps({"u32_3": dfr.dfr_tune_get(dfr.DFR_U32, 3), "u64kv_9": dfr.dfr_tune_get(dfr.DFR_U64_KV, 9)}))
"""


@pytest.fixture(scope="module", autouse=True)
def built():
    dfr_build.build()


def run(env_extra):
    env = {k: v for k, v in os.environ.items() if k not in ("DFR_TUNE_FILE", "DFR_SPIN_LIMIT")}
    env.update(env_extra)
    return subprocess.run([sys.executable, "-c", PROBE], capture_output=True, text=True, cwd=ROOT, env=env,
                          timeout=120)


def builtin():
    r = run({})
    assert r.returncode == 0, r.stderr
    return json.loads(r.stdout)


def test_tune_file_overrides_listed_entries(tmp_path):
    base = builtin()
    new = dict(base["u32_3"], target_log2=9, max_bits=6, warp_max=256, schedule=dfr.DFR_SCHED_MSD)
    p = tmp_path / "plan.json"
    p.write_text(json.dumps({"table": {"DFR_U32": {"3": new}}}))
    r = run({"DFR_TUNE_FILE": str(p)})
    assert r.returncode == 0, r.stderr
    got = json.loads(r.stdout)
    assert got["u32_3"] == new
    assert got["u64kv_9"] == base["u64kv_9"]  # entries the file does not list stay built-in


def test_checked_in_tuner_output_is_a_valid_tune_file():
    r = run({"DFR_TUNE_FILE": os.path.join(ROOT, "paper_2207_14334_gb300", "tune_table.json")})
    assert r.returncode == 0, r.stderr
    assert json.loads(r.stdout) == builtin()


@pytest.mark.parametrize("table,err", [
    ({"DFR_U32": {"3": {"target_log2": 99, "max_bits": 8, "warp_max": 256, "scatter_ctas_per_sm": 0,
                        "ctasort_ctas_per_sm": 0}}}, "invalid argument"),
    ({"DFR_U16": {"3": {}}}, "unknown key type"),
    ({"DFR_U32": {"3": {"max_bits": 8}}}, "target_log2"),
    ({"DFR_U32": {"x": {"target_log2": 11, "max_bits": 8, "warp_max": 256, "scatter_ctas_per_sm": 0,
                        "ctasort_ctas_per_sm": 0}}}, "class x"),
])
def test_refused_tune_file_fails_the_load(tmp_path, table, err):
    p = tmp_path / "bad.json"
    p.write_text(json.dumps(table))
    r = run({"DFR_TUNE_FILE": str(p)})
    assert r.returncode != 0 and err in r.stderr, r.stderr


def test_spin_limit(tmp_path):
    assert run({"DFR_SPIN_LIMIT": "100000"}).returncode == 0
    for bad in ("-1", "abc", str(1 << 32)):
        r = run({"DFR_SPIN_LIMIT": bad})
        assert r.returncode != 0 and ("DFR_SPIN_LIMIT" in r.stderr or "invalid literal" in r.stderr), r.stderr
