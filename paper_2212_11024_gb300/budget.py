"""Wavenumber energy budget of Sec. 4.4 (eq. mhd_en_trans) through the C ABI.

flame_energy_budget evaluates, on the GPU (cuFFT and the library's own
kernels, FP64), for fields u, B on the periodic lattice in lattice units
(F(f) = FFT(f)/N3, k = 2 pi m / N per axis, spectral derivatives with the
Nyquist wavenumber set to zero):
    S(n) = sum_{round|m| < n} Re[ F(u)* . (F(u.grad u) - F(J x B))
                                - F(B)* . F(curl(V x B)) ]
    D(n) = sum_{round|m| < n} nu k^2 |F(u)|^2 + eta k^2 |F(B)|^2
    E(n) = 1/2 sum_{shell n} (|F(u)|^2 + |F(B)|^2)
with J = curl B (spectral) and V = u - d_i J (for d_i = 0 the MHD flux as
printed).  The budget reads d/dt sum_{n' < n} E(n') = -S(n) - D(n) for the
incompressible equations; the nonlinear terms conserve energy, so S over all
shells vanishes for solenoidal fields.

``Flame.energy_budget(nshell)`` takes the fields of a running lattice; this
module's function takes given fields, with nu, eta and d_i as arguments.
"""
from __future__ import annotations

from .flame import Flame


def energy_budget(u, B, nu, eta, nshell, d_i=0.0, device=None):
    """(E, S, D) numpy FP64 [nshell] for FP64 fields u, B [3, nz, ny, nx]
    (numpy or torch, any device).  A context with tau_nu = nu/c_s^2 + 1/2,
    tau_eta = eta/C^2 + 1/2 and d_i carries the parameters (its population
    state, FP16, is never initialised)."""
    nz, ny, nx = tuple(u.shape[1:])
    dev = device if device is not None else (u.device if getattr(u, "is_cuda", False) else None)
    sim = Flame(nx, ny, nz, 3.0 * nu + 0.5, 4.0 * eta + 0.5, d_i, storage="fp16", device=dev)
    try:
        return sim.energy_budget(nshell, u, B)
    finally:
        sim.close()
