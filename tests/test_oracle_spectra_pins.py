"""Pins of the spectral oracle (``oracle/spectra.py``; Sec. 4.4, the shell
spectra and the wavenumber budget of eq. mhd_en_trans) against what the
mathematics fixes, independently of the formulas the oracle writes out:

- one Fourier mode puts all its energy into the single shell round(|m|),
  with the value 1/2 <F^2> the field has in closed form (cubic, non-cubic
  and odd-sized grids; modes whose |m| rounds up and down; Nyquist modes);
- Parseval: summed over every shell the spectrum is 1/2 <|F|^2>;
- the budget of a single shear mode: no flux, and D(n) = 2 nu k^2 E for the
  spheres that enclose the mode, 0 for the others;
- the budget identity d/dt sum_{n'<n} E(n') = -S(n) - D(n) on a stepped
  oracle run, with the time derivative taken by a central difference of the
  oracle's own spectra, at a tolerance derived from the scheme's errors.
"""
import numpy as np
import pytest

import oracle as O
from oracle import spectra as S
from paper_2212_11024_gb300 import inputs as I


def _grid(shape):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x, y, z


def _mode(shape, m, amp, phase):
    """amp cos(2 pi m.x / N + phase) and its mean square in closed form."""
    nz, ny, nx = shape
    x, y, z = _grid(shape)
    arg = 2 * np.pi * (m[0] * x / nx + m[1] * y / ny + m[2] * z / nz) + phase
    f = amp * np.cos(arg)
    # a mode equal to its own conjugate (every nonzero component at the
    # Nyquist index) is real: amp^2 cos^2(phase) everywhere; otherwise the
    # mean of cos^2 over the lattice is 1/2
    self_conj = all((mi == 0) or (2 * mi == n) for mi, n in zip(m, (nx, ny, nz)))
    ms = amp * amp * np.cos(phase) ** 2 if self_conj else 0.5 * amp * amp
    return f, ms


SHAPES = [(16, 16, 16), (12, 10, 16), (9, 7, 11)]
# (m_x, m_y, m_z): |m| = 1.41 (rounds down), 1.73 (rounds up, where a floor
# would go to shell 1), 2.24, 3.61 (rounds up), 3 exactly, and axis modes
MODES = [(1, 1, 0), (1, 1, 1), (2, 1, 0), (3, 2, 0), (2, 2, 1), (0, 0, 2), (1, 0, 0), (0, 3, 1)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("m", MODES)
def test_single_mode_lands_in_one_shell(shape, m):
    nz, ny, nx = shape
    if any(2 * abs(mi) > n for mi, n in zip(m, (nx, ny, nz))):
        pytest.skip("mode beyond the grid's Nyquist index")
    rng = np.random.default_rng(sum(m) + nx)
    F = np.zeros((3,) + shape)
    ms_total = 0.0
    for c in range(3):
        F[c], ms = _mode(shape, m, rng.uniform(0.5, 2.0), rng.uniform(0, 2 * np.pi))
        ms_total += ms
    nshell = 12
    E = S.shell_spectrum(F, nshell)
    n = int(np.floor(np.sqrt(sum(mi * mi for mi in m)) + 0.5))
    expect = np.zeros(nshell)
    expect[n] = 0.5 * ms_total
    assert np.allclose(E, expect, rtol=1e-12, atol=1e-15 * ms_total)


@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 4, 10), (5, 7, 9)])
def test_nyquist_mode(shape):
    """cos(pi x) along an even axis is its own conjugate: 1/2 <F^2> = 1/2 amp^2 cos^2(phase)."""
    nz, ny, nx = shape
    m = [0, 0, 0]
    for a, n in enumerate((nx, ny, nz)):
        if n % 2 == 0:
            m[a] = n // 2
            break
    if not any(m):
        pytest.skip("no even axis")
    F = np.zeros((3,) + shape)
    F[1], ms = _mode(shape, m, 1.7, 0.4)
    n = int(np.floor(np.sqrt(sum(mi * mi for mi in m)) + 0.5))
    E = S.shell_spectrum(F, 12)
    assert abs(E[n] - 0.5 * ms) < 1e-13 and abs(E.sum() - E[n]) < 1e-15
    assert abs(0.5 * ms - 0.5 * 1.7 ** 2 * np.cos(0.4) ** 2) < 1e-15


def test_modes_in_different_shells_add():
    shape = (12, 10, 16)
    F = np.zeros((3,) + shape)
    f1, ms1 = _mode(shape, (1, 0, 0), 1.0, 0.3)
    f2, ms2 = _mode(shape, (1, 1, 1), 0.5, 1.1)
    F[0] = f1
    F[2] = f2
    E = S.shell_spectrum(F, 6)
    assert abs(E[1] - 0.5 * ms1) < 1e-14 and abs(E[2] - 0.5 * ms2) < 1e-14
    assert abs(E.sum() - E[1] - E[2]) < 1e-15


@pytest.mark.parametrize("shape", SHAPES + [(1, 1, 7), (2, 3, 1)])
def test_parseval(shape):
    """Random fields: summed over every shell the spectrum equals 1/2 <|F|^2>
    computed in real space; shells beyond nshell are dropped."""
    F = np.random.default_rng(7).standard_normal((3,) + shape)
    nz, ny, nx = shape
    nmax = int(np.ceil(np.sqrt((nx // 2) ** 2 + (ny // 2) ** 2 + (nz // 2) ** 2))) + 1
    E = S.shell_spectrum(F, nmax + 1)
    assert abs(E.sum() - 0.5 * (F * F).sum(0).mean()) < 1e-13 * (F * F).sum(0).mean()
    assert E[-1] == 0.0
    if nmax > 2:
        E2 = S.shell_spectrum(F, 2)
        assert np.allclose(E2, E[:2], rtol=1e-14, atol=0)


def test_scalar_diagnostics_closed_forms():
    """E_u, E_B (about the mean field), H_c, <|J|^2> and the enstrophy of
    single shear modes, in closed form."""
    N = 16
    shape = (N, N, N)
    x, y, z = _grid(shape)
    k = 2 * np.pi * 2 / N
    a, b, b0 = 0.03, 0.02, 0.1
    u = np.zeros((3,) + shape)
    u[0] = a * np.sin(k * z)                  # curl u = a k cos(kz) y
    B = np.zeros((3,) + shape)
    B[0] = b * np.sin(k * z)
    B[2] = b0
    J = np.zeros((3,) + shape)
    J[1] = b * k * np.cos(k * z)              # curl B
    s = S.scalars(np.ones(shape), u, B, J)
    assert abs(s["E_u"] - a * a / 4) < 1e-17
    assert abs(s["E_B"] - b * b / 4) < 1e-17
    assert abs(s["H_c"] - a * b / 2) < 1e-17
    assert abs(s["J2"] - b * b * k * k / 2) < 1e-17
    assert abs(s["enstrophy"] - a * a * k * k / 2) < 1e-15 * a * a * k * k
    assert abs(s["B_mean"][2] - b0) < 1e-16 and abs(s["mass"] - N ** 3) < 1e-9
    assert abs(s["u_max"] - a * np.abs(np.sin(k * np.arange(N))).max()) < 1e-17


@pytest.mark.parametrize("d_i", [0.0, 1.3])
def test_budget_of_a_single_shear_mode(d_i):
    """u = a sin(k z) x, B = b sin(k z) y with k = 2 pi 3/N: u.grad u = 0,
    J x B and curl(V x B) have no component on the mode, so S = 0; the mode's
    energy sits in shell 3 and D(n) = 2 nu k^2 E_u + 2 eta k^2 E_B for n > 3."""
    N = 12
    shape = (N, N, N)
    x, y, z = _grid(shape)
    k = 2 * np.pi * 3 / N
    a, b, nu, eta = 0.02, 0.015, 0.01, 0.03
    u = np.zeros((3,) + shape)
    u[0] = a * np.sin(k * z)
    B = np.zeros((3,) + shape)
    B[1] = b * np.sin(k * z)
    E, Sf, D = S.energy_budget(u, B, nu, eta, 8, d_i)
    Eu, Eb = a * a / 4, b * b / 4
    assert np.allclose(E, [0, 0, 0, Eu + Eb, 0, 0, 0, 0], rtol=1e-12, atol=1e-20)
    assert np.abs(Sf).max() < 1e-20
    expect_D = np.where(np.arange(8) > 3, 2 * nu * k * k * Eu + 2 * eta * k * k * Eb, 0.0)
    assert np.allclose(D, expect_D, rtol=1e-12, atol=1e-22)


@pytest.mark.parametrize("d_i", [0.0, 2.0])
def test_budget_identity_on_an_oracle_run(d_i):
    """Sec. 4.4: d/dt sum_{n'<n} E(n') = -S(n) - D(n).  The left side is a
    central difference over steps t - 1, t + 1 of the oracle's own shell
    spectra (pinned above); the right side is energy_budget at step t.

    Run: 32^3, solenoidal fields in shells 1..2 with u_rms = b_rms = 0.03 per
    component, tau_nu = tau_eta = 0.52 (nu = 0.02/3, eta = 0.02/4), 20 steps
    before t.  The flux S is 2-3 times D at n = 2, 3, so a sign error or a
    shell boundary taken as <= instead of < fails, and with d_i = 2 the Hall
    part of the induction flux is 20 % of S at n = 3.

    Tolerance, relative to |S(n)| + D(n): 3 Ma^2 for the weakly compressible
    scheme's O(Ma^2) departure from the incompressible budget (acoustic
    exchange, density weighting; Ma^2 = <|u|^2>/c_s^2 = 0.008 here) plus
    k_n^2/12 for the scheme's second-order lattice error at the shell's
    wavenumber k_n = 2 pi n/N.  Checked for n = 2..4 (with d_i = 0 also at
    every larger n): beyond n = 4 the Hall runs decay faster than eta k^2
    alone predicts (the scheme damps the whistler modes numerically: the
    total energy falls 11 % faster than D at d_i = 2)."""
    N, rms, tau = 32, 0.03, 0.52
    shape = (N, N, N)
    u, B = I.turbulence(shape, 11, 12, rms, rms, shells=(1, 2))
    p = O.Params(N, N, N, tau, tau, d_i)
    nu, eta = (tau - 0.5) / 3.0, (tau - 0.5) / 4.0
    pop = O.init(p, None, u, B)
    O.step(p, pop, 19, literal=False)
    ms = []
    for _ in range(3):
        m = O.moments(p, pop)
        ms.append(m)
        O.step(p, pop, 1, literal=False)
    nsh = N // 2 + 1
    cum = []
    for m in ms:
        e = S.shell_spectrum(m["u"], nsh) + S.shell_spectrum(m["B"], nsh)
        cum.append(np.concatenate([[0.0], np.cumsum(e)[:-1]]))  # sum over shells < n
    dEdt = (cum[2] - cum[0]) / 2.0
    _, Sf, D = S.energy_budget(ms[1]["u"], ms[1]["B"], nu, eta, nsh, d_i)
    ma2 = 3.0 * (ms[1]["u"] ** 2).sum(0).mean()
    top = nsh if d_i == 0 else 5
    for n in range(2, top):
        kn = 2 * np.pi * n / N
        tol = 3 * ma2 + kn * kn / 12
        err = abs(dEdt[n] + Sf[n] + D[n]) / (abs(Sf[n]) + D[n])
        assert err < tol, (n, err, tol)
