"""Wavenumber energy budget of Sec. 4.4 (eq. mhd_en_trans), on the GPU.

For fields u, B on the periodic lattice (lattice units, F(f) = FFT(f)/N3,
k = 2 pi m / N per axis, spectral derivatives with the Nyquist wavenumber
set to zero):
    S(n) = sum_{round|m| < n} Re[ F(u)* . (F(u.grad u) - F(J x B))
                                - F(B)* . F(curl(V x B)) ]
    D(n) = sum_{round|m| < n} nu k^2 |F(u)|^2 + eta k^2 |F(B)|^2
with J = curl B (spectral) and V = u (the MHD flux as printed) or
V = u - d_i J (with the Hall term, the reading used when d_i > 0 is
requested).  The budget reads d/dt sum_{n' < n} E(n') = -S(n) - D(n) for the
incompressible equations; the nonlinear terms conserve energy, so S over all
shells vanishes.  E(n) = 1/2 sum_{shell n} (|F(u)|^2 + |F(B)|^2).

This is a post-processing tool built on torch.fft; the fields come from
Flame.moments().
"""
from __future__ import annotations

import math

import torch


def _kvec(shape, device):
    nz, ny, nx = shape

    def k1(n):
        m = torch.fft.fftfreq(n, 1.0 / n, dtype=torch.float64, device=device)
        k = 2.0 * math.pi * m / n
        if n % 2 == 0:
            k[n // 2] = 0.0  # Nyquist: no odd derivative
        return k, m

    kz, mz = k1(nz)
    ky, my = k1(ny)
    kx, mx = k1(nx)
    return (kx[None, None, :], ky[None, :, None], kz[:, None, None],
            torch.round(torch.sqrt(mx[None, None, :] ** 2 + my[None, :, None] ** 2 + mz[:, None, None] ** 2)))


def _fft(f):
    n3 = f.shape[-1] * f.shape[-2] * f.shape[-3]
    return torch.fft.fftn(f, dim=(-3, -2, -1)) / n3


def _ifft(F):
    n3 = F.shape[-1] * F.shape[-2] * F.shape[-3]
    return torch.fft.ifftn(F, dim=(-3, -2, -1)).real * n3


def _grad(Fh, kx, ky, kz):
    """Spectral gradient of a scalar field's transform -> [3, ...] real fields."""
    return torch.stack([_ifft(1j * kx * Fh), _ifft(1j * ky * Fh), _ifft(1j * kz * Fh)])


def _curl_hat(Vh, kx, ky, kz):
    return torch.stack([1j * (ky * Vh[2] - kz * Vh[1]), 1j * (kz * Vh[0] - kx * Vh[2]), 1j * (kx * Vh[1] - ky * Vh[0])])


def energy_budget(u, B, nu, eta, nshell, d_i=0.0):
    """(E, S, D) as FP64 tensors [nshell] for u, B [3, nz, ny, nx] (FP64)."""
    shape = u.shape[1:]
    kx, ky, kz, shell = _kvec(shape, u.device)
    uh = _fft(u)
    Bh = _fft(B)
    J = torch.stack([_ifft(c) for c in _curl_hat(Bh, kx, ky, kz)])
    # u . grad u
    ugu = torch.zeros_like(u)
    for b in range(3):
        g = _grad(uh[b], kx, ky, kz)
        ugu[b] = u[0] * g[0] + u[1] * g[1] + u[2] * g[2]
    JxB = torch.cross(J, B, dim=0)
    V = u - d_i * J if d_i else u
    VxB = torch.cross(V, B, dim=0)
    ind = _curl_hat(_fft(VxB), kx, ky, kz)
    Tu = (torch.conj(uh) * (_fft(ugu) - _fft(JxB))).real.sum(0)
    Tb = -(torch.conj(Bh) * ind).real.sum(0)
    k2 = kx * kx + ky * ky + kz * kz
    dis = nu * k2 * (uh.abs() ** 2).sum(0) + eta * k2 * (Bh.abs() ** 2).sum(0)
    en = 0.5 * ((uh.abs() ** 2).sum(0) + (Bh.abs() ** 2).sum(0))
    idx = shell.to(torch.int64).expand(shape).reshape(-1)
    keep = idx < nshell

    def binned(v):
        return torch.bincount(idx[keep], weights=v.expand(shape).reshape(-1)[keep], minlength=nshell)[:nshell]

    E = binned(en)
    Sc = torch.cumsum(binned(Tu + Tb), 0)
    Dc = torch.cumsum(binned(dis), 0)
    # S(n), D(n) sum over shells < n: shift by one
    zero = torch.zeros(1, dtype=torch.float64, device=u.device)
    return E, torch.cat([zero, Sc[:-1]]), torch.cat([zero, Dc[:-1]])
