"""Exact damped circularly polarised Hall-MHD wave (Sec. 4.1, after Xia & Yang).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

Setting: uniform density rho0 = 1, mean field B0 along +z, one Fourier mode
of wavenumber k along z.  With h(z) = (1, i, 0) exp(i k z) one has
curl h = k h, and for u' = Im(a h), b' = Im(c h) every nonlinear term of the
incompressible dissipative Hall-MHD equations (Sec. 2.1, eqs. NSE and
Hall_ind) is either zero or uniform, so the complex amplitudes obey the
linear system

    da/dt = -nu k^2 a + i k B0 c
    dc/dt =  i k B0 a - (i alpha_H B0 k^2 + eta k^2) c

(the first line is the Lorentz force (curl b) x B0, the second the induction
term curl(u x B0) = B0 d_z u, the Hall term -alpha_H curl(J x B0) and
resistive diffusion).  The 2x2 matrix exponential solves it for any nu, eta.
For nu = eta it reduces to the paper's closed form: c = alpha a with
alpha_pm = -alpha_H k / 2 +- sqrt(alpha_H^2 k^2 / 4 + 1) and a(t) = a(0)
exp(i k B0 alpha t - nu k^2 t), i.e. omega_pm = -alpha_pm k (B0 = 1 units).

Everything is in lattice units: alpha_H = d_i, k = 2 pi m / N, and the
field is sampled at integer z.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def alpha_pm(k, d_i):
    """(alpha_+, alpha_-) of Sec. 4.1: -eps k/2 +- sqrt(eps^2 k^2/4 + 1)."""
    r = np.sqrt(d_i * d_i * k * k / 4.0 + 1.0)
    return -d_i * k / 2.0 + r, -d_i * k / 2.0 - r


def system_matrix(k, B0, nu, eta, d_i):
    return np.array([[-nu * k * k, 1j * k * B0],
                     [1j * k * B0, -1j * d_i * B0 * k * k - eta * k * k]], dtype=np.complex128)


def amplitudes(t, k, B0, nu, eta, d_i, a0, c0):
    """Complex (a(t), c(t)) from (a0, c0) by the matrix exponential."""
    v = scipy.linalg.expm(system_matrix(k, B0, nu, eta, d_i) * float(t)) @ np.array([a0, c0], np.complex128)
    return v[0], v[1]


def fields(t, shape, m, B0, nu, eta, d_i, a0, c0):
    """Exact u [3,nz,ny,nx] and B [3,nz,ny,nx] at time t for the mode k = 2 pi m / nz.

    The real fields are u' = Im(a h), b' = Im(c h): u'_x = Im(a e^{ikz}),
    u'_y = Re(a e^{ikz}), u'_z = 0, and B = B0 z + b'."""
    nz, ny, nx = shape
    k = 2.0 * np.pi * m / nz
    a, c = amplitudes(t, k, B0, nu, eta, d_i, a0, c0)
    z = np.arange(nz, dtype=np.float64)[:, None, None] * np.ones((1, ny, nx))
    e = np.exp(1j * k * z)
    u = np.zeros((3,) + tuple(shape))
    B = np.zeros((3,) + tuple(shape))
    u[0] = np.imag(a * e)
    u[1] = np.real(a * e)
    B[0] = np.imag(c * e)
    B[1] = np.real(c * e)
    B[2] = B0
    return u, B


def gradients(t, shape, m, B0, nu, eta, d_i, a0, c0):
    """Exact d_a u_b and d_a B_b ([9, nz, ny, nx], index 3a+b) at time t."""
    nz, ny, nx = shape
    k = 2.0 * np.pi * m / nz
    a, c = amplitudes(t, k, B0, nu, eta, d_i, a0, c0)
    z = np.arange(nz, dtype=np.float64)[:, None, None] * np.ones((1, ny, nx))
    e = np.exp(1j * k * z)
    gu = np.zeros((9,) + tuple(shape))
    gB = np.zeros((9,) + tuple(shape))
    # d_z Im(a e) = Im(i k a e), d_z Re(a e) = Re(i k a e)
    gu[3 * 2 + 0] = np.imag(1j * k * a * e)
    gu[3 * 2 + 1] = np.real(1j * k * a * e)
    gB[3 * 2 + 0] = np.imag(1j * k * c * e)
    gB[3 * 2 + 1] = np.real(1j * k * c * e)
    return gu, gB


def rel_l2(x, ref):
    return float(np.linalg.norm(np.ravel(x - ref)) / np.linalg.norm(np.ravel(ref)))
