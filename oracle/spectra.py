"""Shell energy spectra and scalar diagnostics, FP64 numpy (Sec. 4.4, 5).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

Pinned in ``tests/test_oracle_spectra_pins.py``: single Fourier modes land
in the one shell round(|m|) with their closed-form energy (cubic, non-cubic,
odd grids, Nyquist modes), Parseval, closed-form scalars of shear modes, the
budget of a single mode (S = 0, D = 2 nu k^2 E), and the budget identity
d/dt sum_{n'<n} E = -S(n) - D(n) on a stepped oracle run.

Conventions (the paper normalises spectra by the total energy but does not
fix the binning):
  u_hat(m) = N^-3 sum_x u(x) exp(-i k.x), k = 2 pi m / N per axis;
  shell n = round(|m|);  E(n) = 1/2 sum_{shell n} |u_hat|^2, so that the sum
  over every shell is 1/2 <|u|^2> (Parseval).
Scalars: E_u = 1/2 <|u|^2>, E_B = 1/2 <|B - <B>|^2>, H_c = <u.(B - <B>)>,
<|J|^2>, enstrophy <|curl u|^2> (spectral curl), mass, momentum, <B>.
"""
from __future__ import annotations

import numpy as np


def _wavenumbers(shape):
    nz, ny, nx = shape
    mz = np.fft.fftfreq(nz, 1.0 / nz)[:, None, None]
    my = np.fft.fftfreq(ny, 1.0 / ny)[None, :, None]
    mx = np.fft.fftfreq(nx, 1.0 / nx)[None, None, :]
    return mx, my, mz


def shell_index(shape):
    mx, my, mz = _wavenumbers(shape)
    return np.rint(np.sqrt(mx * mx + my * my + mz * mz)).astype(np.int64)


def shell_spectrum(F, nshell):
    """E(n), n < nshell, of a real vector field F [3, nz, ny, nx]."""
    shape = F.shape[1:]
    n3 = float(np.prod(shape))
    p = np.zeros(shape)
    for c in range(F.shape[0]):
        fh = np.fft.fftn(F[c]) / n3
        p += np.abs(fh) ** 2
    idx = shell_index(shape).ravel()
    keep = idx < nshell
    return 0.5 * np.bincount(idx[keep], weights=p.ravel()[keep], minlength=nshell)[:nshell]


def enstrophy(u):
    """<|curl u|^2> by the spectral curl (k = 2 pi m / N)."""
    shape = u.shape[1:]
    n3 = float(np.prod(shape))
    mx, my, mz = _wavenumbers(shape)
    kx, ky, kz = (2 * np.pi * mx / shape[2], 2 * np.pi * my / shape[1], 2 * np.pi * mz / shape[0])
    uh = [np.fft.fftn(u[c]) / n3 for c in range(3)]
    wx = 1j * (ky * uh[2] - kz * uh[1])
    wy = 1j * (kz * uh[0] - kx * uh[2])
    wz = 1j * (kx * uh[1] - ky * uh[0])
    return float(np.sum(np.abs(wx) ** 2 + np.abs(wy) ** 2 + np.abs(wz) ** 2))


def scalars(rho, u, B, J):
    """Scalar diagnostics as a dict (FP64)."""
    Bm = B.reshape(3, -1).mean(axis=1)
    b = B - Bm[:, None, None, None]
    return dict(
        mass=float(rho.sum()),
        momentum=[float((rho * u[a]).sum()) for a in range(3)],
        B_mean=[float(v) for v in Bm],
        E_u=0.5 * float((u * u).sum(axis=0).mean()),
        E_B=0.5 * float((b * b).sum(axis=0).mean()),
        H_c=float((u * b).sum(axis=0).mean()),
        J2=float((J * J).sum(axis=0).mean()),
        enstrophy=enstrophy(u),
        u_max=float(np.sqrt((u * u).sum(axis=0)).max()),
    )


def energy_budget(u, B, nu, eta, nshell, d_i=0.0):
    """(E, S, D) of Sec. 4.4 (eq. mhd_en_trans), numpy FP64, written mode by
    mode from the definitions: F = FFT/N3, k = 2 pi m/N (Nyquist k = 0 for
    derivatives), J = curl B spectrally, V = u - d_i J; S(n), D(n) sum the
    modes with round|m| < n; E(n) = 1/2 sum_{shell n} |F(u)|^2 + |F(B)|^2."""
    shape = u.shape[1:]
    n3 = float(np.prod(shape))
    ks = []
    for ax, n in zip((2, 1, 0), (shape[2], shape[1], shape[0])):
        m = np.fft.fftfreq(n, 1.0 / n)
        k = 2 * np.pi * m / n
        if n % 2 == 0:
            k[n // 2] = 0.0
        sh = [1, 1, 1]
        sh[ax] = n
        ks.append(k.reshape(sh))
    kx, ky, kz = ks
    F = lambda f: np.fft.fftn(f) / n3
    iF = lambda G: np.real(np.fft.ifftn(G)) * n3
    uh = [F(u[c]) for c in range(3)]
    Bh = [F(B[c]) for c in range(3)]
    J = np.stack([iF(1j * (ky * Bh[2] - kz * Bh[1])), iF(1j * (kz * Bh[0] - kx * Bh[2])),
                  iF(1j * (kx * Bh[1] - ky * Bh[0]))])
    ugu = np.stack([u[0] * iF(1j * kx * uh[b]) + u[1] * iF(1j * ky * uh[b]) + u[2] * iF(1j * kz * uh[b])
                    for b in range(3)])
    JxB = np.cross(J, B, axis=0)
    V = u - d_i * J
    VxB = np.cross(V, B, axis=0)
    Wh = [F(VxB[c]) for c in range(3)]
    ind = [1j * (ky * Wh[2] - kz * Wh[1]), 1j * (kz * Wh[0] - kx * Wh[2]), 1j * (kx * Wh[1] - ky * Wh[0])]
    T = sum(np.real(np.conj(uh[c]) * (F(ugu[c]) - F(JxB[c]))) - np.real(np.conj(Bh[c]) * ind[c]) for c in range(3))
    k2 = kx * kx + ky * ky + kz * kz
    dis = sum(nu * k2 * np.abs(uh[c]) ** 2 + eta * k2 * np.abs(Bh[c]) ** 2 for c in range(3))
    en = 0.5 * sum(np.abs(uh[c]) ** 2 + np.abs(Bh[c]) ** 2 for c in range(3))
    idx = shell_index(shape)
    E = np.zeros(nshell)
    S = np.zeros(nshell)
    D = np.zeros(nshell)
    for n in range(nshell):
        E[n] = en[idx == n].sum()
        S[n] = T[idx < n].sum()
        D[n] = dis[idx < n].sum()
    return E, S, D
