"""The bench's JSON line on a GPU: one run of a grid whose state leaves L2
(257 x 257 x 513 FP32, the library's two-sweep passes), checked for every key
the line promises -- the metric and its value, the roofline of the dominant
kernel, the CPU oracle baseline, the end-to-end rate through host buffers, the
clock record, the launch count -- and for a passing oracle comparison."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def line():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cmd = [sys.executable, "bench.py", "--workload", "medium", "--steps", "2", "--warmup", "3",
           "--no-variants", "--cpu-seconds", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_headline_keys(line):
    assert line["metric"].startswith("19-pt Jacobi") and line["unit"] == "Gpoint-updates/s"
    assert line["value"] > 0 and line["ms_per_step"] > 0 and line["higher_is_better"] is True
    assert line["n_gpus"] == 1 and line["steps"] == 2 and line["warmup"] == 3
    assert line["dtype"] == "f32" and line["data"] == "synthetic" and line["scaling"] == "weak"
    assert "257x257x513" in line["config"]["workload"] and "L2" in line["config"]["l2"]
    assert line["gpu_launches"] > 0


def test_roofline_of_the_two_sweep_pass(line):
    r = line["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] > 0
    assert r["kernel"].startswith("k_sweep2")
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    # 56 B per interior point per pass, 50 passes for 100 sweeps
    npts = 255 * 255 * 511
    assert r["passes_per_launch"] == 50 and r["algorithmic_bytes_per_launch"] == 56 * npts * 50
    assert r["bytes_per_point_update"] == 28
    # the pass's rate against the single-sweep ceiling is the same number seen two ways
    gpts = npts * 100 / (r["launch_ms"] * 1e-3) / 1e9
    assert abs(r["single_sweep_ceiling"]["value_over_ceiling"] - gpts / (r["peak"] / 56)) < 1e-6
    assert "traffic" in r


def test_baseline_e2e_clocks_and_parity(line):
    c = line["cpu_baseline"]
    assert c["kind"] == "oracle" and c["value"] > 0 and c["cores"] >= 1 and c["sample"]
    e = line["e2e"]
    assert e["value"] > 0 and e["unit"] == line["unit"]
    assert e["h2d_bytes_per_step"] == 13 * 257 * 257 * 513 * 4 and e["d2h_bytes_per_step"] > 0
    k = line["clocks"]
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(k)
    p = line["parity"]
    assert p["pass"] is True and p["p_err"] <= p["tol"] and p["gosa_err"] <= p["tol"]
