"""Host-side pins of the Table 1 validation tools (paper_2212_11024_gb300.validation):
the exact three-mode solution at the origin against the oracle's independent
construction, the maxima and error-metric definitions on synthetic signals,
and a short FP64 oracle run against the exact time series."""
import math

import numpy as np

import oracle as O
from oracle import exact_wave as X
from paper_2212_11024_gb300 import validation as V


def test_setup_matches_paper_parameters():
    s = V.lattice_setup(32, 0.01, 1e-3)
    # eps_H = 1: d_i = N, alpha_+ from d_i k = 4 pi (Sec. 4.1)
    assert s["d_i"] == 32 and abs(s["alpha_p"] - (-2 * math.pi + math.sqrt(4 * math.pi ** 2 + 1))) < 1e-15
    assert abs(s["U0"] - 0.01 / math.sqrt(3)) < 1e-18
    # Table 1's CFL: pi d_i V_A within the lattice whistler bound for N = 32, Ma = 0.01
    assert math.pi * s["d_i"] * s["U0"] < 1.0


def test_exact_origin_matches_oracle_exact_wave():
    s = V.lattice_setup(48, 0.005, 5e-4)
    t = np.linspace(0.0, 3 * s["period"], 41)
    got = V.exact_origin(t, s)
    for j, tj in enumerate(t):
        a, c = X.amplitudes(tj, s["k"], s["U0"], s["nu_lbm"], s["eta_lbm"], s["d_i"], V.B_AMP * s["U0"],
                            s["alpha_p"] * V.B_AMP * s["U0"])
        dec = math.exp(-s["nu_lbm"] * s["k"] ** 2 * tj)
        want = [a.imag + s["U0"] * V.A_AMP * dec, a.real, s["U0"] * V.C_AMP * dec]
        assert np.allclose(got[j], want, rtol=0, atol=1e-15)


def test_maxima_and_metric_definitions():
    t = np.arange(0, 2000.0, 7.0)
    w = 2 * math.pi / 250.0
    tm, vm = V.maxima(t, 1.0 + 0.5 * np.cos(w * t + 0.3))
    want = (2 * math.pi * np.arange(1, 8) - 0.3) / w
    assert np.allclose(tm[:7], want, atol=0.05) and np.allclose(vm, 1.5, atol=2e-3)
    # a numerical series running 1 % slow has eps_phi = -0.01 and eps_r from its amplitude
    s = V.lattice_setup(32, 0.01, 1e-3)
    tt = np.linspace(0, 4 * s["period"], 4001)
    ue = V.exact_origin(tt, s)
    un = V.exact_origin(tt / 1.01, s) * 1.02
    eps_phi, eps_r, _, m = V.errors(tt, un, s)
    assert m >= 2 and abs(eps_phi + 0.01) < 2e-3 and abs(eps_r - 0.02) < 2e-3
    _, _, eps_nu, _ = V.errors(tt, ue, s)
    assert abs(eps_nu) < 1e-9


def test_zmode_metrics():
    """The z-mode's amplitude at the origin: exact on the exact series (the
    A-mode removed by (A/C) u_z); a series running 1 % slow gives
    eps_phi_z = -0.01; a z-mode decaying 5 % faster gives eps_r_z = 0.05
    while the x- and y-modes decay as before."""
    s = V.lattice_setup(32, 0.01, 1e-3)
    t = np.linspace(0, 4 * s["period"], 4001)
    ue = V.exact_origin(t, s)
    a = V.zmode(ue, s)
    dec = np.exp(-s["nu_lbm"] * s["k"] ** 2 * t)
    assert np.allclose(np.abs(a), np.abs(a[0]) * dec, rtol=1e-12)
    assert np.allclose(V.zmode_errors(t, ue, s), 0.0, atol=1e-12)
    assert abs(V.zmode_errors(t, V.exact_origin(t / 1.01, s), s)[0] + 0.01) < 1e-9
    faster = ue.copy()
    extra = np.exp(-0.05 * s["nu_lbm"] * s["k"] ** 2 * t)
    faster[:, 0] = (ue[:, 0] - s["U0"] * V.A_AMP * dec) * extra + s["U0"] * V.A_AMP * dec
    faster[:, 1] = ue[:, 1] * extra
    eps_phi_z, eps_r_z = V.zmode_errors(t, faster, s)
    assert abs(eps_phi_z) < 1e-9 and abs(eps_r_z - 0.05) < 1e-9


def test_oracle_follows_exact_origin_series():
    """FP64 oracle, N = 16, one fifth of a period (Ma = 0.05, nu = 7e-3, so
    tau_nu ~ 0.51 and the modes decay by ~e^-1.4): u(0, t) within 10 % of the
    exact solution.  The scheme's error at 8 sites per wavelength is 8.4 %;
    at N = 32 it is 2.0 % (ratio 4.3, second order; too slow for this suite,
    the GPU test repeats the refinement)."""
    N, Ma, nu = 16, 0.05, 7e-3
    s = V.lattice_setup(N, Ma, nu)
    u, B = V.initial_fields(N, s["U0"], s["alpha_p"])
    p = O.Params(N, N, N, s["tau_nu"], s["tau_eta"], s["d_i"])
    pop = O.init(p, None, u, B)
    steps = int(s["period"] / 5)
    O.step(p, pop, steps, literal=False)
    m = O.moments(p, pop)
    ue = V.exact_origin([steps], s)[0]
    got = m["u"][:, 0, 0, 0]
    assert np.linalg.norm(got - ue) < 1e-1 * np.linalg.norm(ue)
