"""Host logic of the host-buffer calls: the chunk plan in flame_internal.h,
compiled with the host compiler and checked exhaustively (io_plan_check.cpp);
no GPU needed."""
import os
import shutil
import subprocess
from pathlib import Path

import pytest

HERE = Path(__file__).resolve().parent
CSRC = HERE.parent / "paper_2212_11024_gb300" / "csrc"


def test_io_chunk_plan(tmp_path):
    cxx = shutil.which("g++")
    inc = Path(os.environ.get("CUDA_HOME", "/usr/local/cuda")) / "include"
    if cxx is None or not (inc / "cuda_runtime.h").exists():
        pytest.skip("needs g++ and the CUDA headers")
    exe = tmp_path / "io_plan_check"
    subprocess.run([cxx, "-O1", "-std=c++17", f"-I{inc}", f"-I{CSRC}", str(HERE / "io_plan_check.cpp"), "-o",
                    str(exe)], check=True, capture_output=True, timeout=120)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout
    assert r.stdout.strip().endswith("bad 0")
