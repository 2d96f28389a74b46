"""Degenerate cases of the method on both step kernels: the rest state and a
uniform state are fixed points of the collide-and-stream step (Sec. 3:
streaming a uniform field changes nothing and the collision leaves an
equilibrium unchanged), a zero magnetic field stays exactly zero (the Hall
and Lorentz terms vanish: pure hydrodynamics), and zero steps change
nothing."""
import numpy as np
import pytest

from gpu_helpers import turbulence

pytestmark = pytest.mark.gpu

# (storage, kernel, shape): the one-site kernel with FP32 and FP16 storage, the
# row kernel with FP16 and BF16 (64-site rows)
CASES = [("fp32", "auto", (3, 4, 10)), ("fp16", "site", (3, 4, 10)), ("fp16", "auto", (3, 4, 64)),
         ("bf16", "auto", (2, 3, 64))]


def _uniform(shape, vec):
    return np.broadcast_to(np.asarray(vec, dtype=float)[:, None, None, None], (3,) + tuple(shape)).copy()


@pytest.mark.parametrize("storage,kernel,shape", CASES)
def test_rest_state_is_an_exact_fixed_point(storage, kernel, shape):
    """u = 0 and B = B_ref everywhere: every stored deviation starts at zero.
    With 16-bit storage it stays exactly zero through both AA parities; with
    FP32 storage the collision's FP32 constants (1/3, the weights) leave
    residuals of FP32 rounding size, below the smallest FP16 subnormal."""
    from paper_2212_11024_gb300 import Flame
    nz, ny, nx = shape
    B0 = (0.03, -0.02, 0.1)
    sim = Flame(nx, ny, nz, 0.55, 0.6, 1.5, storage=storage, B_ref=B0, kernel=kernel)
    sim.init(None, _uniform(shape, (0, 0, 0)), _uniform(shape, B0))
    f0 = sim.populations().cpu().numpy()
    sim.step(7)
    f1 = sim.populations().cpu().numpy()
    m = sim.moments()
    sim.close()
    tol = 3e-8 if storage == "fp32" else 0.0
    assert np.abs(f1 - f0).max() <= tol
    assert float(m["u"].abs().max()) <= tol and float(m["J"].abs().max()) <= 10 * tol
    assert float((m["rho"] - 1.0).abs().max()) <= 27 * tol


@pytest.mark.parametrize("storage,kernel,shape", CASES)
def test_uniform_flow_in_uniform_field_is_a_fixed_point(storage, kernel, shape):
    """Uniform u and B (B_ref = B): the moments stay at their initial values --
    to FP32 rounding with FP32 storage, to the storage's rounding otherwise --
    and J stays zero."""
    from paper_2212_11024_gb300 import Flame
    nz, ny, nx = shape
    U0, B0 = (0.02, -0.01, 0.03), (0.05, 0.01, 0.1)
    sim = Flame(nx, ny, nz, 0.55, 0.6, 1.5, storage=storage, B_ref=B0, kernel=kernel)
    sim.init(None, _uniform(shape, U0), _uniform(shape, B0))
    sim.step(21)
    m = {k: v.cpu().numpy() for k, v in sim.moments().items()}
    sim.close()
    tol = {"fp32": 1e-6, "fp16": 2e-3, "bf16": 2e-2}[storage]
    for a in range(3):
        assert np.abs(m["u"][a] - U0[a]).max() < tol * np.linalg.norm(U0)
        assert np.abs(m["B"][a] - B0[a]).max() < tol * np.linalg.norm(U0)
    assert np.abs(m["J"]).max() < tol * np.linalg.norm(U0)
    # mass: the rounding of the re-encoded deviations does not conserve it exactly
    assert np.abs(m["rho"] - 1.0).max() < tol * np.linalg.norm(U0)


@pytest.mark.parametrize("storage,kernel,shape", CASES)
def test_zero_field_stays_zero(storage, kernel, shape):
    """B = 0 everywhere (and B_ref = 0): the magnetic populations stay exactly
    zero and J = 0 while the flow evolves -- the scheme reduces to the
    central-moment fluid alone, whatever d_i."""
    from paper_2212_11024_gb300 import Flame
    nz, ny, nx = shape
    u, _ = turbulence(shape, 61, 0.04)
    sim = Flame(nx, ny, nz, 0.55, 0.6, 2.5, storage=storage, kernel=kernel)
    sim.init(None, u, np.zeros((3,) + tuple(shape)))
    sim.step(9)
    f = sim.populations().cpu().numpy()
    m = sim.moments()
    sim.close()
    assert np.abs(f[27:]).max() == 0.0
    assert float(m["J"].abs().max()) == 0.0 and float(m["B"].abs().max()) == 0.0
    assert float(m["u"].abs().max()) > 0.01


@pytest.mark.parametrize("storage,kernel,shape", CASES)
def test_zero_steps_change_nothing(storage, kernel, shape):
    import torch
    from paper_2212_11024_gb300 import Flame
    nz, ny, nx = shape
    u, B = turbulence(shape, 63, 0.04)
    sim = Flame(nx, ny, nz, 0.55, 0.6, 1.5, storage=storage, kernel=kernel)
    sim.init(None, u, B)
    sim.step(3)
    a, step_a, par_a = sim.get_state()
    sim.step(0)
    b, step_b, par_b = sim.get_state()
    sim.close()
    assert torch.equal(a, b) and (step_a, par_a) == (step_b, par_b)
