"""Validation against the exact damped Hall-MHD solution (Sec. 4.1-4.2, Table 1).

Setting (lattice units).  Box of N^3 sites, the paper's three-mode initial
condition (eqs. Xia_IC, Xia_IC2) with amplitudes A = 0.3, B = 0.2, C = 0.1,
two wavelengths per box (k = 4 pi / N), reference speed U0 = Ma / sqrt(3)
equal to the Alfven speed of the mean field B0 = U0 z, rho = 1, Hall length
d_i = eps_H N (eq. hall_param_lu2), magnetic Prandtl number 1 and
dimensionless viscosity nu (Table 1) mapped to nu_lbm = nu U0 N.

Exact solution at the origin (Pm = 1, incompressible limit): the z-mode is a
circularly polarised wave, u' = Im(a h), h = (1, i, 0) e^{ikz}, whose complex
amplitudes (a, c) obey d/dt [a, c] = [[-nu k^2, i k B0], [i k B0,
-i d_i B0 k^2 - nu k^2]] [a, c] with a(0) = B U0, c(0) = alpha_+ a(0); the x-
and y-modes are Beltrami fields perpendicular to B0 on which the Lorentz
force is a gradient and the Hall and induction terms vanish, so they only
decay as exp(-nu k^2 t).  Hence
    u(0, t) = U0 [Im a^ + A e^{-nu k^2 t}, Re a^, C e^{-nu k^2 t}],  a^ = a(t)/U0.

Metrics (Sec. 4.3): the dispersion error eps_phi = 1 - mean_i
(t_{i+1} - t_i)/(tbar_{i+1} - tbar_i) over the time maxima of |u|(0, t); the
dissipation error eps_r = rms_i (|u|(t_i) - |ubar|(tbar_i)) / |ubar|(tbar_i)
comparing the i-th maxima (phases synchronised); and the viscosity error
eps_nu = (nu~ - nu)/nu with nu~ fitted to the decay of u_z(0, t), which the
exact solution gives as U0 C exp(-nu k^2 t).  The maxima of |u| mix the
z-mode's rotation with the decay of the x- and y-modes; zmode_errors takes
the rotation alone (the z-mode's phase and amplitude, with the other modes
removed at the origin).
"""
from __future__ import annotations

import math

import numpy as np

A_AMP, B_AMP, C_AMP = 0.3, 0.2, 0.1
CS2 = 1.0 / 3.0
C2 = 0.25


def lattice_setup(N, Ma, nu, eps_H=1.0):
    """Lattice parameters of one Table 1 run (Pm = 1)."""
    U0 = Ma / math.sqrt(3.0)
    nu_l = nu * U0 * N
    k = 4.0 * math.pi / N
    d_i = eps_H * N
    alpha_p = -d_i * k / 2.0 + math.sqrt(d_i * d_i * k * k / 4.0 + 1.0)
    omega = alpha_p * k * U0  # angular frequency of the z-mode (lattice units)
    return dict(N=N, Ma=Ma, nu=nu, U0=U0, nu_lbm=nu_l, eta_lbm=nu_l, tau_nu=nu_l / CS2 + 0.5,
                tau_eta=nu_l / C2 + 0.5, k=k, d_i=d_i, alpha_p=alpha_p, period=2.0 * math.pi / omega)


def initial_fields(N, U0, alpha_p):
    """u, B [3, N, N, N] of eqs. Xia_IC / Xia_IC2."""
    z = np.arange(N, dtype=np.float64)[:, None, None]
    y = np.arange(N, dtype=np.float64)[None, :, None]
    x = np.arange(N, dtype=np.float64)[None, None, :]
    k = 4.0 * np.pi / N
    one = np.ones((N, N, N))
    u = np.zeros((3, N, N, N))
    u[0] = U0 * (B_AMP * np.sin(k * z) + A_AMP * np.cos(k * y)) * one
    u[1] = U0 * (B_AMP * np.cos(k * z) + C_AMP * np.sin(k * x)) * one
    u[2] = U0 * (C_AMP * np.cos(k * x) + A_AMP * np.sin(k * y)) * one
    B = alpha_p * u
    B[2] += U0
    return u, B


def exact_origin(t, s):
    """Exact u(0, t) [len(t), 3] for the setup dict s."""
    t = np.asarray(t, dtype=np.float64)
    k, B0, nu, d_i, U0 = s["k"], s["U0"], s["nu_lbm"], s["d_i"], s["U0"]
    M = np.array([[-nu * k * k, 1j * k * B0], [1j * k * B0, -1j * d_i * B0 * k * k - nu * k * k]])
    lam, V = np.linalg.eig(M)
    a0 = np.array([B_AMP * U0, s["alpha_p"] * B_AMP * U0], dtype=np.complex128)
    coef = np.linalg.solve(V, a0)
    a = (V[0][None, :] * coef[None, :] * np.exp(np.outer(t, lam))).sum(axis=1)
    dec = np.exp(-nu * k * k * t)
    return np.stack([np.imag(a) + U0 * A_AMP * dec, np.real(a), U0 * C_AMP * dec], axis=1)


def maxima(t, v):
    """Times and values of the interior local maxima of v(t), refined by a
    parabola through each maximum and its two neighbours."""
    t = np.asarray(t, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    i = np.where((v[1:-1] > v[:-2]) & (v[1:-1] >= v[2:]))[0] + 1
    tm, vm = [], []
    for j in i:
        y0, y1, y2 = v[j - 1], v[j], v[j + 1]
        den = y0 - 2.0 * y1 + y2
        d = 0.5 * (y0 - y2) / den if den != 0 else 0.0
        h = t[j + 1] - t[j]
        tm.append(t[j] + d * h)
        vm.append(y1 - 0.25 * (y0 - y2) * d)
    return np.array(tm), np.array(vm)


def errors(t, u_num, s):
    """(eps_phi, eps_r, eps_nu, number of periods compared) from a time series
    u_num [len(t), 3] of the velocity at the origin."""
    ue = exact_origin(t, s)
    tn, vn = maxima(t, np.linalg.norm(u_num, axis=1))
    te, ve = maxima(t, np.linalg.norm(ue, axis=1))
    m = min(len(tn), len(te))
    if m < 2:
        return float("nan"), float("nan"), float("nan"), 0
    tn, vn, te, ve = tn[:m], vn[:m], te[:m], ve[:m]
    eps_phi = 1.0 - float(np.mean(np.diff(tn) / np.diff(te)))
    eps_r = float(np.sqrt(np.mean(((vn - ve) / ve) ** 2)))
    uz = u_num[:, 2]
    good = uz > 0
    slope = np.polyfit(t[good], np.log(uz[good]), 1)[0]
    nu_t = -slope / (s["k"] ** 2)
    eps_nu = (nu_t - s["nu_lbm"]) / s["nu_lbm"]
    return eps_phi, eps_r, float(eps_nu), m - 1


def zmode(u, s):
    """The z-mode's complex amplitude at the origin, a = u_y + i (u_x - (A/C) u_z),
    from a series u [len(t), 3].  At the origin u_y is Re a alone and u_x is
    Im a plus the x-velocity of the A-mode (varying along y), while u_z is the
    C-mode's alone (varying along x); the two decay alike (they are the same
    Beltrami mode turned by 90 degrees about z, to which the lattice is
    symmetric), so (A/C) u_z removes the A-mode with the scheme's own decay."""
    u = np.asarray(u)
    return u[:, 1] + 1j * (u[:, 0] - (A_AMP / C_AMP) * u[:, 2])


def zmode_errors(t, u_num, s):
    """Dispersion and dissipation errors of the z-mode alone: eps_phi_z =
    1 - T_num / T_exact = 1 - omega_exact / omega_num (the sign convention of
    eps_phi: negative when the numerical wave is slow) with each omega the
    least-squares slope of the unwrapped phase of a(t), and eps_r_z the
    relative error of the decay rate of |a(t)| (slopes of log |a|)."""
    t = np.asarray(t, dtype=np.float64)
    an, ae = zmode(u_num, s), zmode(exact_origin(t, s), s)
    w_n = np.polyfit(t, np.unwrap(np.angle(an)), 1)[0]
    w_e = np.polyfit(t, np.unwrap(np.angle(ae)), 1)[0]
    g_n = np.polyfit(t, np.log(np.abs(an)), 1)[0]
    g_e = np.polyfit(t, np.log(np.abs(ae)), 1)[0]
    return float(1.0 - w_e / w_n), float((g_n - g_e) / g_e)


def run(N, Ma, nu, periods=10, samples_per_period=400, storage="fp32", graph_steps=64, device=None):
    """One Table 1 run on the GPU: the time series of u at the origin and the
    three error metrics."""
    import torch

    from .flame import Flame

    s = lattice_setup(N, Ma, nu)
    u, B = initial_fields(N, s["U0"], s["alpha_p"])
    nsteps = int(round(periods * s["period"]))
    every = max(1, int(s["period"] // samples_per_period))
    nsamp = nsteps // every
    sim = Flame(N, N, N, s["tau_nu"], s["tau_eta"], s["d_i"], storage=storage, B_ref=(0.0, 0.0, s["U0"]),
                device=device, graph_steps=graph_steps if every >= graph_steps else 0)
    sim.init(None, u, B)
    sites = torch.zeros(1, dtype=torch.int64, device=sim.device)
    out = torch.empty((nsamp + 1, 10), dtype=torch.float64, device=sim.device)
    sim.probe(sites, out=out[0:1])
    for j in range(1, nsamp + 1):
        sim.step(every)
        sim.probe(sites, out=out[j:j + 1])
    sim.sync()
    series = out.cpu().numpy()
    sim.close()
    t = np.arange(nsamp + 1, dtype=np.float64) * every
    eps_phi, eps_r, eps_nu, m = errors(t, series[:, 1:4], s)
    eps_phi_z, eps_r_z = zmode_errors(t, series[:, 1:4], s)
    return dict(s, steps=nsteps, sample_every=every, eps_phi=eps_phi, eps_r=eps_r, eps_nu=eps_nu,
                eps_phi_z=eps_phi_z, eps_r_z=eps_r_z, periods_compared=m,
                rho_fluct=float(np.abs(series[:, 0] - 1.0).mean()), t=t, u=series[:, 1:4])


def main(argv=None):
    """The Table 1 sweep: one JSON line per (N, Ma, nu) run (series left out).

        python -m paper_2212_11024_gb300.validation --N 32,48,64,96,128 --Ma 0.01 --nu 0.001
    """
    import argparse
    import json
    import time

    ap = argparse.ArgumentParser(description="Table 1 validation runs on the GPU")
    ap.add_argument("--N", default="32,48,64")
    ap.add_argument("--Ma", default="0.01")
    ap.add_argument("--nu", default="0.001")
    ap.add_argument("--periods", type=float, default=None,
                    help="periods per run (default: 9 at N <= 48, 7 at 64, 3 at 96, 2 beyond)")
    a = ap.parse_args(argv)
    for N in (int(v) for v in a.N.split(",")):
        for Ma in (float(v) for v in a.Ma.split(",")):
            for nu in (float(v) for v in a.nu.split(",")):
                per = a.periods or (9 if N <= 48 else 7 if N <= 64 else 3 if N <= 96 else 2)
                t0 = time.time()
                r = run(N, Ma, nu, periods=per)
                r = {k: (float(v) if isinstance(v, (np.floating, float)) else v) for k, v in r.items()
                     if k not in ("t", "u")}
                r["wall_s"] = time.time() - t0
                print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
