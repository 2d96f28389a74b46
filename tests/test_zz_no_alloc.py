"""flame_reduce_static: the scalar diagnostics without any allocation.

Some callers cannot let the library call cudaMalloc: cudaMalloc may
synchronise the device and stall work already queued, and some hosts hand
every byte of device memory to their own caching allocator.  This entry
point keeps its scratch in a fixed device array instead.  The test calls it
through the C ABI twice in a row, with different block counts so that a
second call reading stale partial sums of the first would show, and checks
each result against flame_reduce, which computes the same sums with its own
workspace.  It also checks that block counts beyond the array's capacity are
rejected.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import turbulence

pytestmark = pytest.mark.gpu

# The two entry points run the same FP64 reduction kernel; only the order of
# the final host/device arithmetic may differ, at the level of FP64 rounding.
RTOL = 1e-12


def _compare(static, ref):
    from paper_2212_11024_gb300.flame import SCALAR_NAMES
    for i, name in enumerate(SCALAR_NAMES):
        a, b = float(static[i]), float(ref[name])
        assert abs(a - b) <= RTOL * max(abs(b), 1e-300) + 1e-300, (name, a, b)


def test_reduce_static_matches_reduce_on_two_calls():
    import torch
    from paper_2212_11024_gb300 import Flame
    from paper_2212_11024_gb300.flame import FLAME_ERR_PARAM, FLAME_OK, NSCALARS, library

    shape = (16, 20, 24)
    u, B = turbulence(shape, 41, 0.04, shells=(1, 3))
    B = B + np.array([0.0, 0.02, 0.06])[:, None, None, None]
    nz, ny, nx = shape
    sim = Flame(nx, ny, nz, 0.56, 0.6, 1.5, storage="fp32", B_ref=(0.0, 0.02, 0.06))
    sim.init(None, u, B)
    sim.step(7)
    lib = library()
    out = torch.full((NSCALARS,), float("nan"), dtype=torch.float64, device=sim.device)

    # first call (first use of the scratch array in this process, odd parity)
    rc = lib.flame_reduce_static(sim._ctx, 600, ctypes.c_void_p(out.data_ptr()))
    assert rc == FLAME_OK
    torch.cuda.synchronize()
    first = out.cpu().numpy().copy()
    _compare(first, sim.reduce())

    # second call on a changed state and with fewer blocks
    sim.step(4)
    out.fill_(float("nan"))
    rc = lib.flame_reduce_static(sim._ctx, 37, ctypes.c_void_p(out.data_ptr()))
    assert rc == FLAME_OK
    torch.cuda.synchronize()
    second = out.cpu().numpy().copy()
    _compare(second, sim.reduce())
    assert not np.allclose(first[7:11], second[7:11], rtol=1e-9)  # the state did change

    # beyond the capacity of the scratch array: a clear parameter error
    assert lib.flame_reduce_static(sim._ctx, 1025, ctypes.c_void_p(out.data_ptr())) == FLAME_ERR_PARAM
    assert lib.flame_reduce_static(sim._ctx, -1, ctypes.c_void_p(out.data_ptr())) == FLAME_ERR_PARAM
    sim.close()
