"""The benchmark's reference arm (`bench.py --impl reference`: the FP64 CPU
oracle timed on the host cores) and its host-only oracle-timing line run
without a GPU and print one JSON line with the keys the benchmark contract
names."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, timeout=600):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       timeout=timeout, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def test_default_workload_is_the_largest_grid():
    """With no flags the benchmark times the 513 x 513 x 1025 FP32 workload
    (100 device-resident sweeps), on both arms."""
    sys.path.insert(0, ROOT)
    import bench
    args = bench.parse_args([])
    w = bench.WORKLOADS[args.workload]
    assert (w["I"], w["J"], w["K"], w["sweeps"], w["prec"]) == (513, 513, 1025, 100, "f32")
    assert args.steps >= 1 and args.warmup >= 3


def test_reference_arm_line():
    d = run_bench("--impl", "reference", "--workload", "config2", "--steps", "1", "--warmup", "0")
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["grid"] == [129, 129, 257]


@pytest.mark.slow
def test_oracle_configs_line():
    d = run_bench("--workload", "oracle-configs")
    assert d["kind"] == "oracle" and d["cores"] >= 1
    assert len(d["configs"]) == 5
    for name, c in d["configs"].items():
        assert "sample" in c, name


def test_native_arm_has_no_cpu_fallback():
    """Without a GPU the native arm fails loudly instead of printing a number,
    and the binding refuses to create a context."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "1", "--warmup", "0",
                        "--quick", "--no-variants", "--no-cpu-baseline"], capture_output=True, text=True,
                       timeout=300, cwd=ROOT)
    assert r.returncode != 0
    assert not any(ln.lstrip().startswith("{") for ln in r.stdout.splitlines())
    from paper_2002_12115_gb300 import Jacobi
    with pytest.raises(Exception):
        Jacobi(9, 9, 9, "f32")
