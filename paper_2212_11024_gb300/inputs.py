"""Seeded synthetic initial conditions (numpy, FP64, layout [comp][z][y][x]).

This module is the only code shared by the CUDA path and the FP64 oracle;
it contains no arithmetic of the lattice-Boltzmann method itself, only the
macroscopic fields the paper starts its runs from.

- ``parallel_wave``: the circularly polarised Alfven/whistler wave along the
  mean field (Sec. 4.1, eq. Xia_IC / Xia_IC2 restricted to its z mode):
  u = amp (sin kz, cos kz, 0), B = B0 z + ratio * u, k = 2 pi m / nz.
- ``xia_three_mode``: the paper's three-mode Beltrami initial condition
  (Sec. 4.1, eqs. Xia_IC and Xia_IC2) with amplitudes A, B, C.
- ``turbulence``: random-phase solenoidal u and B with energy in the shells
  lo <= round(|m|) <= hi, equal expected energy per shell, rescaled to a
  given per-component rms.  Each Fourier mode's polarisation is projected
  orthogonal to the central-difference symbol sin(2 pi m / N), so the
  second-order central-difference divergence of the sampled field vanishes.
  Mode amplitudes are drawn over the fixed cube |m_a| <= hi in a fixed order,
  so a given seed gives the same modes on every grid size.
- ``orszag_tang``: the 3-D Orszag-Tang vortex of Sec. 4.4 on a 2 pi box.
"""
from __future__ import annotations

import numpy as np


def _coords(shape):
    nz, ny, nx = shape
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    y = np.arange(ny, dtype=np.float64)[None, :, None]
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    return x, y, z


def parallel_wave(shape, m=1, amp=1e-3, B0=0.1, ratio=1.0):
    """(u, B) of the single parallel-propagating circularly polarised mode."""
    nz = shape[0]
    k = 2.0 * np.pi * m / nz
    _, _, z = _coords(shape)
    ones = np.ones(tuple(shape))
    u = np.zeros((3,) + tuple(shape))
    u[0] = amp * np.sin(k * z) * ones
    u[1] = amp * np.cos(k * z) * ones
    B = ratio * u
    B[2] += B0
    return u, B


def parallel_wave_gradients(shape, m=1, amp=1e-3, ratio=1.0):
    """Analytic d_a u_b and d_a B_b of ``parallel_wave`` ([9, nz, ny, nx], index 3a+b)."""
    nz = shape[0]
    k = 2.0 * np.pi * m / nz
    _, _, z = _coords(shape)
    ones = np.ones(tuple(shape))
    gu = np.zeros((9,) + tuple(shape))
    gu[6] = amp * k * np.cos(k * z) * ones
    gu[7] = -amp * k * np.sin(k * z) * ones
    return gu, ratio * gu


def xia_three_mode(shape, u0, ratio, A=0.3, B=0.2, C=0.1, periods=2):
    """Sec. 4.1 initial condition: u from eq. Xia_IC, B = ratio u + u0 z (eq. Xia_IC2).

    ``periods`` wavelengths fit in the box (the paper uses 2, i.e. 4 pi / N)."""
    nz, ny, nx = shape
    x, y, z = _coords(shape)
    kx, ky, kz = 2 * np.pi * periods / nx, 2 * np.pi * periods / ny, 2 * np.pi * periods / nz
    ones = np.ones(tuple(shape))
    u = np.zeros((3,) + tuple(shape))
    u[0] = u0 * (B * np.sin(kz * z) + A * np.cos(ky * y)) * ones
    u[1] = u0 * (B * np.cos(kz * z) + C * np.sin(kx * x)) * ones
    u[2] = u0 * (C * np.cos(kx * x) + A * np.sin(ky * y)) * ones
    b = ratio * u
    b[2] += u0
    return u, b


def _band_field(shape, lo, hi, rms, seed):
    rng = np.random.default_rng(seed)
    K = 2 * hi + 1
    ms = np.arange(-hi, hi + 1)
    V = rng.standard_normal((3, K, K, K)) + 1j * rng.standard_normal((3, K, K, K))  # [c, mz, my, mx]
    mz, my, mx = np.meshgrid(ms, ms, ms, indexing="ij")
    shell = np.rint(np.sqrt(mx * mx + my * my + mz * mz)).astype(np.int64)
    sel = (shell >= lo) & (shell <= hi)
    counts = np.bincount(shell[sel], minlength=hi + 1)
    amp = np.where(sel, 1.0 / np.sqrt(np.maximum(counts[np.minimum(shell, hi)], 1)), 0.0)
    nz, ny, nx = shape
    kt = np.stack([np.sin(2 * np.pi * mx / nx), np.sin(2 * np.pi * my / ny), np.sin(2 * np.pi * mz / nz)])
    kk = (kt * kt).sum(axis=0)
    dot = (kt * V).sum(axis=0)
    V = V - kt * np.where(kk > 0, dot / np.where(kk > 0, kk, 1.0), 0.0)
    V = V * amp
    ex = np.exp(2j * np.pi * np.outer(np.arange(nx), ms) / nx)  # [x, m]
    ey = np.exp(2j * np.pi * np.outer(np.arange(ny), ms) / ny)
    ez = np.exp(2j * np.pi * np.outer(np.arange(nz), ms) / nz)
    out = np.empty((3,) + tuple(shape))
    chunk = max(1, (1 << 24) // max(1, nx * ny))
    for c in range(3):
        t1 = np.einsum("abm,xm->abx", V[c], ex)  # [mz, my, x]
        t2 = np.einsum("ym,amx->ayx", ey, t1)  # [mz, y, x]
        t2 = t2.reshape(K, ny * nx)
        for z0 in range(0, nz, chunk):
            z1 = min(nz, z0 + chunk)
            out[c, z0:z1] = np.real(ez[z0:z1] @ t2).reshape(z1 - z0, ny, nx)
    cur = np.sqrt((out * out).sum(axis=0).mean() / 3.0)
    if cur > 0:
        out *= rms / cur
    return out


def turbulence(shape, seed_u, seed_b, rms_u=0.05, rms_b=0.05, shells=(1, 4)):
    """(u, B) random-phase solenoidal fields, energy in shells lo..hi, zero mean B."""
    lo, hi = shells
    return _band_field(shape, lo, hi, rms_u, seed_u), _band_field(shape, lo, hi, rms_b, seed_b)


def orszag_tang(shape, u0=1.0, b0=0.8, scale=1.0):
    """Sec. 4.4 Orszag-Tang vortex on a 2 pi box sampled at N points per side.

    u = u0 [-2 sin y, 2 sin x, 0], B = b0 [-2 sin 2y + sin z, 2 sin x + sin z,
    sin x + sin y]; both multiplied by ``scale`` (the lattice velocity unit)."""
    nz, ny, nx = shape
    x, y, z = _coords(shape)
    X, Y, Z = 2 * np.pi * x / nx, 2 * np.pi * y / ny, 2 * np.pi * z / nz
    ones = np.ones(tuple(shape))
    u = np.zeros((3,) + tuple(shape))
    B = np.zeros((3,) + tuple(shape))
    u[0] = -2 * np.sin(Y) * ones
    u[1] = 2 * np.sin(X) * ones
    B[0] = (-2 * np.sin(2 * Y) + np.sin(Z)) * ones
    B[1] = (2 * np.sin(X) + np.sin(Z)) * ones
    B[2] = (np.sin(X) + np.sin(Y)) * ones
    return u * u0 * scale, B * b0 * scale
