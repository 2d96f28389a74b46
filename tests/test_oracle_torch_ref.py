"""Pins of the PyTorch FP64 restatement of the oracle (used for reference
gradients): its initial populations and steps equal the C oracle's, its band
energy equals the numpy shell spectrum, and its autograd gradients agree
with central finite differences of itself."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import spectra as S
from oracle import torch_ref as R
from paper_2212_11024_gb300 import inputs as I


def _fields(shape, seed, amp=0.05, b0=0.04):
    u, B = I.turbulence(shape, seed, seed + 1, amp, amp, shells=(1, 2))
    B[2] += b0
    return u, B


@pytest.mark.parametrize("shape,di", [((6, 5, 4), 1.5), ((4, 4, 6), 0.0)])
def test_torch_reference_equals_c_oracle(shape, di):
    u, B = _fields(shape, 3)
    nz, ny, nx = shape
    p = O.Params(nx, ny, nz, 0.56, 0.61, di)
    pop = O.init(p, None, u, B)
    t0 = R.init(torch.tensor(u), torch.tensor(B), 0.56, 0.61, torch.tensor(di, dtype=torch.float64))
    assert np.abs(t0.numpy() - pop).max() < 1e-15
    O.step(p, pop, 3)
    t3 = R.step(t0, 0.56, 0.61, torch.tensor(di, dtype=torch.float64), 3)
    assert np.abs(t3.numpy() - pop).max() < 1e-13


def test_band_energy_equals_shell_spectrum():
    u, B = _fields((8, 10, 12), 5)
    E = S.shell_spectrum(B - B.reshape(3, -1).mean(1)[:, None, None, None], 10)
    assert abs(float(R.band_energy(torch.tensor(B), 2, 4)) - E[2:5].sum()) < 1e-15


def test_reference_gradient_matches_finite_differences():
    """d/d(d_i) and a directional derivative along a random B perturbation of
    L = band energy after 4 steps, autograd vs central differences (FP64)."""
    shape = (6, 6, 6)
    u, B = _fields(shape, 9)
    rng = np.random.default_rng(0)
    dirB = rng.standard_normal(B.shape)

    def loss(Bt, di):
        pop = R.init(torch.tensor(u), Bt, 0.6, 0.6, di)
        pop = R.step(pop, 0.6, 0.6, di, 4)
        return R.band_energy(R.magnetic_field(pop), 1, 2)

    Bt = torch.tensor(B, requires_grad=True)
    di = torch.tensor(1.2, dtype=torch.float64, requires_grad=True)
    L = loss(Bt, di)
    gB, gdi = torch.autograd.grad(L, [Bt, di])
    eps = 1e-5
    with torch.no_grad():
        fd = (loss(torch.tensor(B + eps * dirB), di) - loss(torch.tensor(B - eps * dirB), di)) / (2 * eps)
        fdi = (loss(torch.tensor(B), di + eps) - loss(torch.tensor(B), di - eps)) / (2 * eps)
    assert abs(float((gB * torch.tensor(dirB)).sum()) - float(fd)) < 1e-7 * abs(float(fd))
    assert abs(float(gdi) - float(fdi)) < 1e-6 * abs(float(fdi)) + 1e-14
