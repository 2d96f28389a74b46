"""Shared helpers for the GPU parity tests (CUDA path vs FP64 oracle)."""
import numpy as np

import oracle as O
from paper_2212_11024_gb300 import inputs as I

CS2 = 1.0 / 3.0


def rest_populations(shape, rho0=1.0, Bref=(0.0, 0.0, 0.0)):
    """Reference populations of the deviation encoding, [48, nz, ny, nx]:
    the rest equilibrium of (rho0, B_ref) -- oracle equilibria at U = 0."""
    feq = O.feq_hermite(rho0, np.zeros(3)) + O.lorentz(np.array(Bref, dtype=float))
    geq = O.geq_hall(np.array(Bref, dtype=float), np.zeros(3), np.zeros(3), 0.0).reshape(21)
    v = np.concatenate([feq, geq])
    return v[:, None, None, None] * np.ones((1,) + tuple(shape))


def rel_dev_err(f_gpu, f_ref, f_rest, sl=slice(None)):
    """||f_gpu - f_ref|| / ||f_ref - f_rest|| over the slots in sl."""
    d = np.linalg.norm((f_gpu[sl] - f_ref[sl]).ravel())
    n = np.linalg.norm((f_ref[sl] - f_rest[sl]).ravel())
    return d / n


def slot_dev_errs(f_gpu, f_ref, f_rest):
    """Per population slot: ||f_gpu - f_ref|| / ||f_ref - f_rest|| ([48])."""
    d = np.sqrt(((f_gpu - f_ref) ** 2).reshape(f_ref.shape[0], -1).sum(1))
    n = np.sqrt(((f_ref - f_rest) ** 2).reshape(f_ref.shape[0], -1).sum(1))
    return d / np.maximum(n, 1e-300)


def rel_l2(x, ref):
    return float(np.linalg.norm(np.ravel(x - ref)) / np.linalg.norm(np.ravel(ref)))


def run_both(shape, tau_nu, tau_eta, d_i, u, B, steps, storage="fp32", rho=None, gradu=None, gradB=None,
             Bref=(0.0, 0.0, 0.0), literal=True, noneq=True, kernel="auto"):
    """Run the CUDA path and the oracle from the same fields; return
    (gpu populations, gpu moments, oracle populations, oracle moments), all numpy FP64."""
    from paper_2212_11024_gb300 import Flame
    nz, ny, nx = shape
    sim = Flame(nx, ny, nz, tau_nu, tau_eta, d_i, storage=storage, B_ref=Bref, init_noneq=noneq, kernel=kernel)
    sim.init(rho, u, B, gradu, gradB)
    sim.step(steps)
    sim.sync()
    fg = sim.populations().cpu().numpy()
    mg = {k: v.cpu().numpy() for k, v in sim.moments().items()}
    sim.close()
    p = O.Params(nx, ny, nz, tau_nu, tau_eta, d_i)
    pop = O.init(p, rho, u, B, gradu, gradB, noneq)
    O.step(p, pop, steps, literal=literal)
    mo = O.moments(p, pop)
    return fg, mg, pop, mo


def turbulence(shape, seed, rms, shells=(1, 2)):
    return I.turbulence(shape, seed, seed + 1, rms, rms, shells=shells)
