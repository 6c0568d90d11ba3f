"""The benchmark's reference arm on the CPU (it times the oracle, no GPU):
one JSON line with the keys the benchmark contract asks for, and ranks other
than 0 exit without work."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT,
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


@pytest.mark.parametrize("workload", ["rw16", "skel20s"])
def test_reference_line(workload):
    lines = _run(["--impl", "reference", "--workload", workload, "--steps", "2", "--warmup", "1"])
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert d["config"]["workload"]
    # the same config keys as the GPU arm's line (built by the same helpers)
    extra = {"rw16": ("scenes",), "skel20s": ("joints", "step")}[workload]
    for key in ("n", "seed", "l2", "parallelism") + extra:
        assert key in d["config"], key
    assert d["config"]["parallelism"] == "single"
    cpu = d["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_other_ranks_do_no_work():
    lines = _run(["--impl", "reference", "--workload", "rw16", "--steps", "2", "--warmup", "1"],
                 {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert lines == []
