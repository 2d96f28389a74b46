"""The library's Fourier-space diagnostics (Sec. 4.4) against the oracle:
the wavenumber energy budget S(k), D(k) of eq. mhd_en_trans and the band
magnetic energy with its gradient (flame_energy_budget, flame_band_energy),
plus the FP32 forms of the moments and of the initialisation."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from gpu_helpers import turbulence
from oracle import spectra as S
from oracle import torch_ref as R

pytestmark = pytest.mark.gpu


def _flame(shape, tau_nu=0.55, tau_eta=0.6, d_i=1.5, storage="fp32", **kw):
    from paper_2212_11024_gb300 import Flame
    nz, ny, nx = shape
    return Flame(nx, ny, nz, tau_nu, tau_eta, d_i, storage=storage, **kw)


@pytest.mark.parametrize("shape", [(12, 10, 16), (9, 7, 11), (16, 16, 16)])
@pytest.mark.parametrize("d_i", [0.0, 1.5])
def test_budget_of_given_fields_matches_oracle(shape, d_i):
    """Same seeded FP64 fields into both: E and D to 1e-12, S to 1e-10 of
    its largest shell (FP64 throughout; cuFFT and numpy sum in another order)."""
    u, B = turbulence(shape, 31, 0.05, shells=(1, 3))
    B = B + np.array([0.0, 0.01, 0.03])[:, None, None, None]
    nu, eta = 0.05 / 3, 0.1 / 4
    sim = _flame(shape, 0.55, 0.6, d_i)
    nsh = 14
    E, Sf, D = sim.energy_budget(nsh, u, B)
    sim.close()
    E0, S0, D0 = S.energy_budget(u, B, nu, eta, nsh, d_i)
    assert np.allclose(E, E0, rtol=1e-12, atol=1e-15 * E0.max())
    assert np.allclose(D, D0, rtol=1e-12, atol=1e-15 * D0.max())
    assert np.abs(Sf - S0).max() < 1e-10 * np.abs(S0).max()
    assert np.abs(S0).max() > 1e-9


def test_budget_module_function():
    """budget.energy_budget (a context carrying nu, eta, d_i) on CUDA fields."""
    from paper_2212_11024_gb300 import budget
    shape = (12, 12, 12)
    u, B = turbulence(shape, 33, 0.04, shells=(1, 2))
    E, Sf, D = budget.energy_budget(torch.tensor(u, device="cuda"), torch.tensor(B, device="cuda"), 0.01, 0.02, 12,
                                    0.7)
    E0, S0, D0 = S.energy_budget(u, B, 0.01, 0.02, 12, 0.7)
    assert np.allclose(E, E0, rtol=1e-12) and np.allclose(D, D0, rtol=1e-12, atol=1e-15 * D0.max())
    assert np.abs(Sf - S0).max() < 1e-10 * np.abs(S0).max()


def test_budget_of_the_state_after_steps():
    """flame_energy_budget of a running FP32 lattice after 20 steps against
    the budget of the oracle's own run from the same fields: FP32-level
    agreement (E, D 1e-5 relative on the shells holding energy; S 1e-4 of
    its largest shell)."""
    shape = (16, 16, 16)
    u, B = turbulence(shape, 35, 0.04, shells=(1, 2))
    sim = _flame(shape, 0.55, 0.6, 1.2)
    sim.init(None, u, B)
    sim.step(20)
    E, Sf, D = sim.energy_budget(14)
    sim.close()
    p = O.Params(16, 16, 16, 0.55, 0.6, 1.2)
    pop = O.init(p, None, u, B)
    O.step(p, pop, 20, literal=False)
    m = O.moments(p, pop)
    E0, S0, D0 = S.energy_budget(m["u"], m["B"], 0.05 / 3, 0.1 / 4, 14, 1.2)
    big = E0 > 1e-6 * E0.max()
    assert np.allclose(E[big], E0[big], rtol=1e-5)
    assert np.allclose(D[1:], D0[1:], rtol=1e-5)
    assert np.abs(Sf - S0).max() < 1e-4 * np.abs(S0).max()


@pytest.mark.parametrize("shape", [(8, 10, 12), (7, 9, 5)])
def test_band_energy_and_gradient_match_oracle(shape):
    """L of given fields against the oracle's shell spectrum (1e-12); dL/dB
    against autograd of the FP64 reference loss (1e-12 of its largest
    entry); the adjoint seed is dL/dB on every magnetic population (as FP32)
    and zero on the fluid ones."""
    u, B = turbulence(shape, 37, 0.05, shells=(1, 3))
    B = B + np.array([0.02, 0.0, 0.04])[:, None, None, None]
    lo, hi = 2, 4
    sim = _flame(shape)
    L, g, seed = sim.band_energy(lo, hi, B, grad=True, adjoint_seed=True)
    sim.close()
    E = S.shell_spectrum(B, 10)
    assert abs(L - E[lo:hi + 1].sum()) < 1e-12 * L
    Bt = torch.tensor(B, requires_grad=True)
    (gr,) = torch.autograd.grad(R.band_energy(Bt, lo, hi), [Bt])
    gr = gr.numpy()
    assert np.abs(g.cpu().numpy() - gr).max() < 1e-12 * np.abs(gr).max()
    n3 = int(np.prod(shape))
    s = seed.cpu()
    assert torch.equal(s[:27], torch.zeros((27, n3)))
    gf = g.reshape(3, 1, n3).expand(3, 7, n3).reshape(21, n3).float().cpu()
    assert torch.equal(s[27:], gf)


def test_band_energy_of_the_state():
    """Band energy of a stepped FP32 lattice against the oracle's run (1e-5)."""
    shape = (12, 12, 16)
    u, B = turbulence(shape, 39, 0.05, shells=(1, 2))
    sim = _flame(shape, 0.56, 0.6, 1.0)
    sim.init(None, u, B)
    sim.step(15)
    L, _, _ = sim.band_energy(1, 3)
    sim.close()
    p = O.Params(16, 12, 12, 0.56, 0.6, 1.0)
    pop = O.init(p, None, u, B)
    O.step(p, pop, 15, literal=False)
    m = O.moments(p, pop)
    L0 = S.shell_spectrum(m["B"], 5)[1:4].sum()
    assert abs(L - L0) < 1e-5 * L0


@pytest.mark.parametrize("shape", [(9, 7, 11), (5, 6, 7)])
def test_spectra_on_odd_lattices(shape):
    """flame_spectra on lattices with an odd site count (fields of its FFTs
    not 16-byte multiples apart) against the oracle's run."""
    u, B = turbulence(shape, 47, 0.05, shells=(1, 2))
    nz, ny, nx = shape
    sim = _flame(shape, 0.56, 0.6, 1.0)
    sim.init(None, u, B)
    sim.step(6)
    Eu, Eb = sim.spectra(8)
    sim.close()
    p = O.Params(nx, ny, nz, 0.56, 0.6, 1.0)
    pop = O.init(p, None, u, B)
    O.step(p, pop, 6, literal=False)
    m = O.moments(p, pop)
    Eu0 = S.shell_spectrum(m["u"], 8)
    Eb0 = S.shell_spectrum(m["B"] - m["B"].reshape(3, -1).mean(1)[:, None, None, None], 8)
    assert np.allclose(Eu, Eu0, rtol=1e-5, atol=1e-6 * Eu0.max())
    assert np.allclose(Eb, Eb0, rtol=1e-5, atol=1e-6 * Eb0.max())


def test_spectral_entry_points_reject_bad_arguments():
    from paper_2212_11024_gb300.flame import FLAME_ERR_PARAM, FLAME_ERR_STATE, library
    lib = library()
    shape = (8, 8, 8)
    u, B = turbulence(shape, 41, 0.05)
    sim = _flame(shape)
    ub = torch.tensor(u, device="cuda")
    h = (ctypes.c_double * 2000)()
    L = ctypes.c_double()
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    # before flame_init the state's fields do not exist
    assert lib.flame_energy_budget(sim._ctx, 4, None, None, h, h, h) == FLAME_ERR_STATE
    assert lib.flame_band_energy(sim._ctx, 1, 2, None, ctypes.byref(L), None, None) == FLAME_ERR_STATE
    assert lib.flame_energy_budget(sim._ctx, 0, vp(ub), vp(ub), h, h, h) == FLAME_ERR_PARAM
    assert lib.flame_energy_budget(sim._ctx, 1025, vp(ub), vp(ub), h, h, h) == FLAME_ERR_PARAM
    assert lib.flame_energy_budget(sim._ctx, 4, vp(ub), None, h, h, h) == FLAME_ERR_PARAM
    assert lib.flame_band_energy(sim._ctx, 3, 2, vp(ub), ctypes.byref(L), None, None) == FLAME_ERR_PARAM
    assert lib.flame_band_energy(sim._ctx, -1, 2, vp(ub), ctypes.byref(L), None, None) == FLAME_ERR_PARAM
    assert lib.flame_band_energy(sim._ctx, 1, 2, vp(ub), None, None, None) == FLAME_ERR_PARAM
    assert sim.sync() is None
    sim.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_fp32_moments_are_the_rounded_fp64_moments(storage):
    """flame_moments_f32 equals flame_moments rounded to FP32, bit for bit
    (both take the same per-site arithmetic; only the final store differs)."""
    shape = (6, 5, 64)
    u, B = turbulence(shape, 43, 0.05)
    sim = _flame(shape, storage=storage, B_ref=(0.0, 0.0, 0.0))
    sim.init(None, u, B)
    sim.step(3)
    m64 = sim.moments()
    m32 = sim.moments(dtype=torch.float32)
    for k in m64:
        assert m32[k].dtype == torch.float32
        assert torch.equal(m32[k], m64[k].float()), k
    sim.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_fp32_initialisation_equals_fp64_of_the_same_values(storage):
    """flame_init_f32 from FP32 fields builds the same state, bit for bit, as
    flame_init from those values widened to FP64 (gradients are formed in
    FP64 from the field values either way)."""
    shape = (5, 6, 40)
    u, B = turbulence(shape, 45, 0.05)
    rho = 1.0 + 0.01 * np.sin(np.arange(np.prod(shape)).reshape(shape))
    u32, B32, r32 = u.astype(np.float32), B.astype(np.float32), rho.astype(np.float32)
    states = []
    for f in ((r32, u32, B32), (r32.astype(np.float64), u32.astype(np.float64), B32.astype(np.float64))):
        sim = _flame(shape, storage=storage)
        sim.init(*f)
        states.append(sim.get_state()[0])
        sim.close()
    assert torch.equal(states[0], states[1])
