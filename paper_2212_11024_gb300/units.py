"""Lattice-unit parameters and the whistler CFL condition (Sec. 3.3, 3.4).

Lattice units: dx = dt = 1, c_s^2 = 1/3, C^2 = 1/4.  The relaxation times
follow from the lattice viscosity and resistivity as 1/omega = nu/c_s^2 + 1/2
(Sec. 3.1.1) and 1/omega_B = eta/C^2 + 1/2 (Sec. 3.2).  With the reference
velocity equal to the Alfven speed and rho = 1, the Hall coefficient in
lattice units is the ion inertial length in lattice spacings,
alpha_H = eps_H * N (eq. hall_param_lu2).
"""
from __future__ import annotations

import math

CS2 = 1.0 / 3.0
C2 = 0.25


def tau_from_nu(nu: float) -> float:
    return nu / CS2 + 0.5


def tau_from_eta(eta: float) -> float:
    return eta / C2 + 0.5


def nu_from_tau(tau: float) -> float:
    return CS2 * (tau - 0.5)


def eta_from_tau(tau: float) -> float:
    return C2 * (tau - 0.5)


def lattice_params(N: int, Ma: float, Re: float, Pm: float = 1.0, eps_H: float = 0.0, L0: float | None = None):
    """Lattice parameters of a run given as (N, Ma, Re, Pm, eps_H).

    U0 = Ma c_s is the reference (Alfven) velocity in lattice units, L0 the
    reference length in lattice spacings (default N), nu = U0 L0 / Re,
    eta = nu / Pm, d_i = eps_H L0 (eq. hall_param_lu2 with U0 = V_A)."""
    L = float(N if L0 is None else L0)
    U0 = Ma * math.sqrt(CS2)
    nu = U0 * L / Re
    eta = nu / Pm
    return dict(U0=U0, nu=nu, eta=eta, tau_nu=tau_from_nu(nu), tau_eta=tau_from_eta(eta), d_i=eps_H * L)


def whistler_cfl(d_i: float, speed: float) -> float:
    """pi d_i V in lattice units; the time step resolves the fastest whistler
    at k = pi when this is <= 1 (the lattice form of the Sec. 3.4 bound
    dt <= dx^2 / (pi alpha_H B_0))."""
    return math.pi * d_i * speed


def paper_mach_limit(N: int, eps_H: float) -> float:
    """The Mach-number bound printed in Sec. 3.4 (eq. CFL_LBM):
    Ma <= (sqrt(3)/pi) / (eps_H N^2).  It is N times stricter than
    whistler_cfl(eps_H N, Ma/sqrt(3)) <= 1; Table 2 satisfies it."""
    return (math.sqrt(3.0) / math.pi) / (eps_H * N * N)
