"""The JSON line `bench.py` prints (host-only parts of the contract).

The reference arm (`--impl reference`: the oracle on every host core, a bounded sample of
the same workload) runs on the CPU, so its line is checked here in full: one JSON line
with the metric, unit and workload of our arm, a `cpu_baseline` describing the sample and
an `e2e` object with zero copies.  Our arm needs a GPU: without one it must end with an
error and print no number (no CPU fallback).
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _json_lines(text):
    out = []
    for ln in text.splitlines():
        ln = ln.strip()
        if ln.startswith("{"):
            out.append(json.loads(ln))
    return out


def test_reference_arm_prints_one_contract_line():
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = _json_lines(p.stdout)
    assert len(lines) == 1, p.stdout[-2000:]
    d = lines[0]
    assert d["impl"] == "reference"
    assert d["metric"] == "sieved coprime (p,q) pairs/s" and d["unit"] == "pairs/s"
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "c4_triangle2^20_256primes"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == "pairs/s"
    assert cb["cores"] >= 1 and "rows" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_our_arm_fails_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the arm runs (covered by the GPU runs)")
    p = subprocess.run([sys.executable, "bench.py", "--no-extras", "--steps", "3", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode != 0
    assert not any("value" in d for d in _json_lines(p.stdout))
