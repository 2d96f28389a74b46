"""bench.py's reference arm (the FP64 oracle on the host cores) prints one
JSON line with the keys of the measurement contract; run on a 16^3 instance
so that it takes seconds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "16",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["config"]["sample_n"] <= 16 and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_bench_names_the_kernel_flame_step_uses():
    """bench.py's kernel_name mirrors the library's dispatch: the row kernel
    for 16-bit storage at nx a multiple of 8 (whole 16-byte rows) from 96 to
    1024 and at 64, on half rows from 513 to 640 sites where nx is a
    multiple of 16, the one-site kernel between them and otherwise, for FP32
    and when forced."""
    sys.path.insert(0, ROOT)
    import bench
    for n in range(8, 1100, 8):
        stageable = (96 <= n <= 1024 or n == 64) and n % 8 == 0
        half = 512 < n <= 640 and n % 16 == 0
        row = stageable and (half or not 512 < n <= 640)
        for st in ("fp16", "bf16"):
            assert ("step_row_kernel" in bench.kernel_name(st, "auto", n)) == row, (st, n)
            assert ("half" in bench.kernel_name(st, "auto", n)) == half, (st, n)
            assert "step_kernel" in bench.kernel_name(st, "site", n)
        assert bench.kernel_name("fp32", "auto", n).startswith("step_kernel")
