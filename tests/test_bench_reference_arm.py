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
    """bench.py names the kernel the library chooses (flame_step_kernel),
    and that choice follows the timed rule for 16-bit storage: staged whole
    rows at most multiples of 8 from 64 to 1024, half rows at 608, 624 and
    640, the unstaged pair kernel at every other even length, the one-site
    kernel at odd lengths, for FP32 and when forced."""
    sys.path.insert(0, ROOT)
    import bench
    for n in list(range(2, 1100, 2)) + [33, 99, 257]:
        staged = n % 8 == 0 and 64 <= n <= 1024
        half = n in (608, 624, 640)
        pair = n % 2 == 0 and (not staged or 64 < n < 104 or 128 < n < 160 or 776 <= n <= 792 or
                                (512 < n <= 648 and not half))
        for st in ("fp16", "bf16"):
            name = bench.kernel_name(st, "auto", n)
            assert ("step_pair_kernel" in name) == pair, (st, n)
            assert ("half" in name) == half, (st, n)
            assert ("step_row_kernel" in name) == (n % 2 == 0 and not pair), (st, n)
            assert "step_kernel" in bench.kernel_name(st, "site", n)
        assert bench.kernel_name("fp32", "auto", n).startswith("step_kernel")


def test_reference_arm_under_torchrun_prints_one_line():
    """Launched as the multi-GPU runs are (torchrun, two ranks), rank 0 alone
    times the oracle and prints; the other rank exits 0 without work."""
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--lattice", "16", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
