"""bench.py's command-line contract, checked on the CPU.

* `--impl reference` times the FP64 oracle on the host cores and prints one JSON line with the
  product arm's metric, unit and direction, `impl: reference`, a `cpu_baseline` describing the
  run and an `e2e` object with no host-device traffic.
* Under a multi-rank launch only rank 0 runs the reference arm; the other ranks exit 0 without
  output.
* The product arm has no CPU fallback: without a GPU it exits non-zero and prints no result.
"""
import json
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BENCH = os.path.join(ROOT, "bench.py")


def _run(args, **env):
    e = dict(os.environ, **env)
    return subprocess.run([sys.executable, BENCH] + args, capture_output=True, text=True,
                          env=e, cwd=ROOT, timeout=600)


def _json_lines(out):
    return [json.loads(x) for x in out.splitlines() if x.startswith("{")]


def _bench_constant(name):
    src = open(BENCH).read()
    m = re.search(rf'^{name} = "([^"]*)"', src, re.M)
    assert m, name
    return m.group(1)


def test_reference_arm_prints_one_contract_line():
    r = _run(["--impl", "reference", "--steps", "2", "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference"
    assert d["metric"] == _bench_constant("METRIC")
    assert d["unit"] == _bench_constant("UNIT")
    assert d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["vs_baseline"] is None
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == d["value"] and cb["unit"] == d["unit"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_reference_arm_other_ranks_exit_quietly():
    r = _run(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"],
             RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    assert r.returncode == 0, r.stderr[-2000:]
    assert _json_lines(r.stdout) == []


def test_product_arm_has_no_cpu_fallback():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the product arm would run")
    r = _run(["--steps", "1", "--warmup", "0"])
    assert r.returncode != 0
    assert _json_lines(r.stdout) == []
