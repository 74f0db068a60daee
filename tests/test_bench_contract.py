"""bench.py on the CPU: the reference arm's JSON line (the FP64 oracle timed on a bounded
sample of the workload), the silence of non-zero ranks, the traffic record's source guard
and the algorithmic-bytes formula behind roofline.achieved."""
import hashlib
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _run(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                         capture_output=True, text=True, env=e, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return [l for l in out.stdout.splitlines() if l.startswith("{")]


def test_reference_arm_line():
    lines = _run(["--impl", "reference", "--steps", "1", "--warmup", "0",
                  "--oracle-seconds", "1"])
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["metric"] == bench.METRIC and d["impl"] == "reference"
    assert d["unit"] == "solves/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["config"]["workload"] == bench.WORKLOAD
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["unit"] == "solves/s" and "Phase II iterations" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_are_silent():
    lines = _run(["--impl", "reference", "--steps", "1", "--warmup", "0",
                  "--oracle-seconds", "1"], env={"RANK": "1", "WORLD_SIZE": "2"})
    assert lines == []


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    h = hashlib.sha256()
    for f in bench.SOLVER_SOURCES:
        with open(os.path.join(ROOT, "paper_2403_09133_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    monkeypatch.setitem(bench.SOLVER_TRAFFIC, "sources_sha256_16", h.hexdigest()[:16])
    assert bench.solver_traffic() == bench.SOLVER_TRAFFIC["bytes_per_launch"]
    monkeypatch.setitem(bench.SOLVER_TRAFFIC, "sources_sha256_16", "0" * 16)
    assert bench.solver_traffic() is None


def test_algorithmic_bytes_formula():
    # 3 n ld s per Hessian apply (P and the fixed factor read, H P written): Phase II's applies
    # at the initial rank's ld, Phase III's Newton-CG applies at the final rank's ld, both in the
    # form's element size
    n = 1000
    res = {"hessian_applies": 14, "newton_cg_iters": 5, "rank": 23, "rank0": 15}
    got = bench.algorithmic_bytes(res, n, 4)
    assert got == 14 * 3 * n * 16 * 4 + 5 * 3 * n * 24 * 4
    none = {"hessian_applies": 0, "newton_cg_iters": 0, "rank": 15, "rank0": 15}
    assert bench.algorithmic_bytes(none, n, 8) == 0
