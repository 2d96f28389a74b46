"""Properties of the oracle's energy budget (Sec. 4.4) that the mathematics
fixes: for spectrally solenoidal fields the nonlinear flux through a sphere
enclosing every mode vanishes (energy conservation of the ideal terms, with
or without the Hall term), and E sums to the total energy; the Orszag-Tang
fields put energy in shells 1 and 2 only, with no flux (a steady Euler
flow).  The library's implementation is compared with this one on the GPU
(tests/test_gpu_spectral.py)."""
import numpy as np

from oracle import spectra as S
from paper_2212_11024_gb300 import inputs as I


def _spectral_solenoidal(F):
    shape = F.shape[1:]
    ks = []
    for ax, n in zip((2, 1, 0), (shape[2], shape[1], shape[0])):
        k = 2 * np.pi * np.fft.fftfreq(n, 1.0 / n) / n
        if n % 2 == 0:
            k[n // 2] = 0.0
        sh = [1, 1, 1]
        sh[ax] = n
        ks.append(k.reshape(sh))
    Fh = np.stack([np.fft.fftn(F[c]) for c in range(3)])
    k = np.stack(np.broadcast_arrays(*ks))
    k2 = (k * k).sum(0)
    kd = (k * Fh).sum(0) / np.where(k2 > 0, k2, 1.0)
    Fh = Fh - k * kd
    return np.stack([np.real(np.fft.ifftn(Fh[c])) for c in range(3)])


def test_budget_flux_vanishes_for_solenoidal_fields():
    shape = (12, 10, 16)
    u, B = I.turbulence(shape, 4, 5, 0.05, 0.05, shells=(1, 3))
    u, B = _spectral_solenoidal(u), _spectral_solenoidal(B)
    nsh = 13  # every shell of this grid is < 12, so S(12) encloses all modes
    for di in (0.0, 1.5):
        E0, S0, D0 = S.energy_budget(u, B, 0.01, 0.02, nsh, di)
        assert abs(S0[-1]) < 1e-12 * np.abs(S0).max()
        assert np.abs(S0).max() > 1e-8  # the fluxes themselves are not trivial
    Etot = 0.5 * ((u * u).sum(0).mean() + (B * B).sum(0).mean())
    assert abs(E0.sum() - Etot) < 1e-15


def test_orszag_tang_budget_shell_structure():
    """Orszag-Tang fields have energy only in shells 1 and 2; their initial
    velocity is a steady Euler flow, so every flux is at round-off relative to
    E^(3/2) k."""
    u, B = I.orszag_tang((16, 16, 16), 1.0, 0.8, scale=0.01)
    E, Sf, D = S.energy_budget(u, B, 1e-3, 1e-3, 16)
    assert E[0] < 1e-30 and E[1] > 0 and E[2] > 0 and E[3:].sum() < 1e-30
    scale = E.sum() ** 1.5 * (2 * np.pi * 2 / 16)
    assert np.abs(Sf).max() < 1e-12 * scale
    assert D[-1] > 0
