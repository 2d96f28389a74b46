"""flame_reduce_static: the scalar diagnostics without any allocation.

Some callers cannot let the library call cudaMalloc: cudaMalloc may
synchronise the device and stall work already queued, and some hosts hand
every byte of device memory to their own caching allocator.  This entry
point keeps its scratch in a fixed device array instead.  The test calls it
through the C ABI twice in a row and checks each result against
flame_reduce, which computes the same sums with its own workspace.  The
first call uses few blocks (37) and the second many (600), so the second
call reads array entries the first never wrote: if a block's partial sums
were not written before they are read, the second result would pick up the
array's initial zeros and differ.  It also checks that block counts beyond
the array's capacity are rejected.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import turbulence

pytestmark = pytest.mark.gpu

# The two entry points run the same FP64 reduction kernel with different
# block counts, so the per-site terms are summed in a different order.  Sums
# of positive terms (mass, energies, <|J|^2>, the div B estimate) then agree
# to a relative 1e-12.  Sums that cancel (momentum, <B> with a mean field
# removed, the cross-helicity after the mean-field correction) can end near
# zero, so they get an absolute bound of 1e-13 times the sum of the terms'
# magnitudes, estimated from the field scales; the maximum and the
# non-finite count do not depend on the order.
RTOL = 1e-12


def _compare(static, ref, n3, u_max, b_scale):
    from paper_2212_11024_gb300.flame import SCALAR_NAMES
    atol = {"mom_x": n3 * u_max, "mom_y": n3 * u_max, "mom_z": n3 * u_max,
            "B_x": b_scale, "B_y": b_scale, "B_z": b_scale, "H_c": u_max * b_scale}
    for i, name in enumerate(SCALAR_NAMES):
        a, b = float(static[i]), float(ref[name])
        if name in ("u_max", "nonfinite"):
            assert a == b, (name, a, b)
        elif name in atol:
            assert abs(a - b) <= 1e-13 * atol[name], (name, a, b)
        else:
            assert abs(a - b) <= RTOL * abs(b), (name, a, b)


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

    n3 = nx * ny * nz
    b_scale = float(np.abs(B).max())

    # first call (odd parity) with few blocks
    rc = lib.flame_reduce_static(sim._ctx, 37, ctypes.c_void_p(out.data_ptr()))
    assert rc == FLAME_OK
    torch.cuda.synchronize()
    first = out.cpu().numpy().copy()
    ref = sim.reduce()
    _compare(first, ref, n3, ref["u_max"], b_scale)

    # second call on a changed state, with more blocks than the first wrote
    sim.step(4)
    out.fill_(float("nan"))
    rc = lib.flame_reduce_static(sim._ctx, 600, ctypes.c_void_p(out.data_ptr()))
    assert rc == FLAME_OK
    torch.cuda.synchronize()
    second = out.cpu().numpy().copy()
    ref = sim.reduce()
    _compare(second, ref, n3, ref["u_max"], b_scale)
    assert not np.allclose(first[7:11], second[7:11], rtol=1e-9)  # the state did change

    # beyond the capacity of the scratch array: a clear parameter error
    assert lib.flame_reduce_static(sim._ctx, 1025, ctypes.c_void_p(out.data_ptr())) == FLAME_ERR_PARAM
    assert lib.flame_reduce_static(sim._ctx, -1, ctypes.c_void_p(out.data_ptr())) == FLAME_ERR_PARAM
    sim.close()
