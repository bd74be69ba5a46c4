"""Host-side pieces of the benchmark: the workload config without
generation equals the one measured on the generated matrix, the algorithmic
byte counts follow their formulas, and the reference arm prints one JSON line
with the contract's keys (the CPU oracle on a tiny workload)."""
from __future__ import annotations

import importlib.util
import json
import os
import subprocess
import sys

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def test_spec_config_matches_generated_config():
    b = _bench()
    for n, parts in ((4096, 8), (20_000, 64)):
        sp = synth.balanced(seed=0, n=n, parts=parts)
        x = synth.generate(synth.balanced(seed=0, n=n, parts=parts))
        assert b.spec_config("balanced", sp) == b.workload_config("balanced", x)
    # random sizes are not claimed without generating
    c = b.spec_config("heterogeneous", synth.heterogeneous(seed=0))
    assert c["n_cells"] is None and c["minimal_bytes"] is None


def test_algorithmic_bytes_formulas():
    b = _bench()
    x = synth.generate(synth.balanced(seed=1, n=4096, parts=4))
    o, C, V, s, N, R = x.offset_bytes, x.n_cells, x.n_values, x.stride, x.n_cols, x.n_rows
    assert b.algorithmic_bytes("hist", x, None) == 4 * C
    assert b.algorithmic_bytes("scatter", x, None) == 4 * C + (C + 1) * o + (R + 1) * o + 12 * C
    assert b.algorithmic_bytes("scatter2", x, None) == 24 * C
    assert b.algorithmic_bytes("place", x, None) == 12 * C + 4 * C + (C + 1) * o + (N + 1) * o + 4 * C
    assert b.algorithmic_bytes("copy", x, None) == 2 * V * s  # the value-run step's bytes
    assert b.algorithmic_bytes("copy", x, None, metadata=True) == 4 * C + (C + 1) * o + 2 * V * s
    # the metric's bytes: each side read or written once
    side = 4 * C + (C + 1) * o + V * s
    assert x.minimal_bytes() == (R + 1) * o + side + (N + 1) * o + side
    assert b.l2_note(x.minimal_bytes()).startswith("fits in L2")
    assert b.l2_note(10**9).startswith("inputs larger than L2")


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--config", "1", "--steps", "2", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["config"]["workload"] == "tiny"
    ts = d["config"]["timed_sample"]  # what each timed step transposes
    assert ts["n_rows"] == 1000 and ts["n_cells"] > 0 and ts["minimal_bytes"] > 0
    assert d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]


def test_reference_arm_names_its_sample():
    """On a workload larger than the sample, the line's config is the full
    workload's and config.timed_sample describes the smaller matrix each
    timed step transposes."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "balanced", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([ln for ln in r.stdout.splitlines() if ln.strip()][0])
    assert d["config"]["n_rows"] == 4_194_304
    ts = d["config"]["timed_sample"]
    assert ts["n_rows"] == 1 << 18 and ts["n_cells"] == 32 * (1 << 18)
    assert abs(d["value"] - ts["minimal_bytes"] / (d["ms_per_step"] * 1e-3) / 1e9) < 0.01 * d["value"]
