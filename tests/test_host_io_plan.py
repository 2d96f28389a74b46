"""Host logic of the host-buffer calls: the chunk plan in flame_internal.h,
compiled with the host compiler and checked exhaustively (io_plan_check.cpp),
and the binding's check of the host arrays; no GPU needed."""
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


def test_binding_host_array_checks():
    """Flame._host (the host-buffer calls' argument check) accepts exactly
    C-contiguous FP32 host arrays of the expected shape, numpy or CPU torch,
    and passes None through; it needs no context."""
    import numpy as np
    import torch

    from paper_2212_11024_gb300.flame import Flame

    f = Flame.__new__(Flame)
    f.torch = torch
    shape = (3, 4, 5)
    a = np.zeros((3,) + shape, np.float32)
    assert f._host(a, 3, shape, "u").value == a.ctypes.data
    t = torch.zeros((3,) + shape)
    assert f._host(t, 3, shape, "u").value == t.data_ptr()
    assert f._host(t[1], 0, shape, "rho").value == t[1].data_ptr()
    assert f._host(None, 3, shape, "u") is None
    bad = [np.zeros((3,) + shape, np.float64), np.zeros((3, 3, 4, 6), np.float32),
           np.asfortranarray(a), a[:, :, :, ::2].copy()[:, :, :, :2], torch.zeros((3,) + shape, dtype=torch.float64),
           torch.zeros((3, 5, 4, 3)).transpose(1, 3)]
    for b in bad:
        with pytest.raises(ValueError):
            f._host(b, 3, shape, "u")
