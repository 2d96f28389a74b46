"""Plain PyTorch FP64 (CPU) restatement of the oracle step, for reference gradients.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

Same algorithm and order as ``flame_oracle.c``, written with batched torch
operations so that ``torch.autograd`` yields exact FP64 gradients of a loss
with respect to the initial fields and the Hall length d_i:
  - f^(0): the App. A Hermite equilibrium in its tensor-product closed form
    (pinned equal to the Hermite sum in the C oracle's tests), plus the
    moment-matching Lorentz term;
  - central-moment collision literally: T(U) per site, k = T^T f,
    k* = k - S (k - k^eq), f* = solve(T^T, k*);
  - J by a batched 3x3 solve of (I + s M) J = y;
  - Hall equilibrium, BGK, and pull streaming (torch.roll);
  - initial populations from u, B with periodic central differences.
Pinned equal to the C oracle's forward in ``tests/test_oracle_torch_ref.py``.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle as _O

CS2 = 1.0 / 3.0
CC2 = 0.25
_DT = torch.float64


def _tables():
    C, W, XI, W7 = _O.lattice()
    return (torch.tensor(C, dtype=_DT), torch.tensor(W, dtype=_DT), torch.tensor(XI, dtype=_DT),
            torch.tensor(W7, dtype=_DT))


C27, W27, XI7, W7 = _tables()
I3 = torch.eye(3, dtype=_DT)
H2 = C27[:, :, None] * C27[:, None, :] - CS2 * I3  # [27, 3, 3]


def feq(rho, U):
    """rho [S], U [S,3] -> [S,27]: rho * prod_a psi(c_a, U_a)."""
    out = rho[:, None]
    for a in range(3):
        c = C27[:, a][None, :]
        u = U[:, a][:, None]
        psi = torch.where(c == 0, 2.0 / 3.0 - u * u, 0.5 * (1.0 / 3.0 + u * u + c * u))
        out = out * psi
    return out


def lorentz(B):
    """B [S,3] -> [S,27]: w_i H2_i : (|B|^2 I/2 - B B) / (2 cs^4)."""
    b2 = (B * B).sum(-1)
    M = 0.5 * b2[:, None, None] * I3 - B[:, :, None] * B[:, None, :]
    return W27[None, :] / (2 * CS2 * CS2) * torch.einsum("iab,sab->si", H2, M)


def cm_matrix(U):
    """T [S, 27 (population i), 27 (moment j)], T_j(c_i - U), corrected basis."""
    cb = C27[None, :, :] - U[:, None, :]
    x, y, z = cb[..., 0], cb[..., 1], cb[..., 2]
    x2, y2, z2 = x * x, y * y, z * z
    cols = [torch.ones_like(x), x, y, z, x * y, x * z, y * z, x2 - y2, x2 - z2, x2 + y2 + z2,
            x * y2 + x * z2, x2 * y + y * z2, x2 * z + y2 * z, x * y2 - x * z2, x2 * y - y * z2, x2 * z - y2 * z,
            x * y * z, x2 * y2 + x2 * z2 + y2 * z2, x2 * y2 + x2 * z2 - y2 * z2, x2 * y2 - x2 * z2,
            x2 * y * z, x * y2 * z, x * y * z2, x * y2 * z2, x2 * y * z2, x2 * y2 * z, x2 * y2 * z2]
    return torch.stack(cols, dim=-1)


def collide_fluid(f, fe, U, omega):
    A = cm_matrix(U).transpose(1, 2)  # [S, j, i]
    k = torch.einsum("sji,si->sj", A, f)
    ke = torch.einsum("sji,si->sj", A, fe)
    S = torch.ones(27, dtype=_DT)
    S[4:9] = omega
    ks = k - S[None, :] * (k - ke)
    return torch.linalg.solve(A, ks.unsqueeze(-1)).squeeze(-1)


def current(Lam, U, B, omegaB, dI):
    """Lam [S,3,3] (Lam[a,b]), U, B [S,3] -> J [S,3]: (I + s M) J = y."""
    A = torch.stack([Lam[:, 1, 2] - Lam[:, 2, 1], Lam[:, 2, 0] - Lam[:, 0, 2], Lam[:, 0, 1] - Lam[:, 1, 0]], -1)
    g = omegaB / CC2
    y = -g * (A - 2.0 * torch.cross(U, B, dim=-1))
    s = 2.0 * dI * g
    Bx, By, Bz = B[:, 0], B[:, 1], B[:, 2]
    zero = torch.zeros_like(Bx)
    one = torch.ones_like(Bx)
    M = torch.stack([torch.stack([one, s * Bz, -s * By], -1), torch.stack([-s * Bz, one, s * Bx], -1),
                     torch.stack([s * By, -s * Bx, one], -1)], -2)
    return torch.linalg.solve(M, y.unsqueeze(-1)).squeeze(-1)


def geq_hall(B, U, J, dI):
    """-> [S, 3 (component b), 7 (velocity i)]."""
    V = U - dI * J
    L0 = V[:, :, None] * B[:, None, :] - B[:, :, None] * V[:, None, :]  # [S, a, b]
    s = torch.einsum("ia,sab->sbi", XI7, L0)
    return W7[None, None, :] * (B[:, :, None] + s / CC2)


def site_collide(x, tau_nu, tau_eta, dI):
    """x [S, 48] -> [S, 48]."""
    omega, omegaB = 1.0 / tau_nu, 1.0 / tau_eta
    f = x[:, :27]
    g = x[:, 27:].reshape(-1, 3, 7)
    rho = f.sum(-1)
    U = (f @ C27) / rho[:, None]
    B = g.sum(-1)
    Lam = torch.einsum("ia,sbi->sab", XI7, g)
    J = current(Lam, U, B, omegaB, dI)
    fe = feq(rho, U) + lorentz(B)
    fs = collide_fluid(f, fe, U, omega)
    gs = g - omegaB * (g - geq_hall(B, U, J, dI))
    return torch.cat([fs, gs.reshape(-1, 21)], dim=-1)


def _velocities():
    return torch.cat([C27, XI7, XI7, XI7]).to(torch.int64)


def step(pop, tau_nu, tau_eta, dI, nsteps=1):
    """pop [48, nz, ny, nx] (pre-collision) -> after nsteps."""
    vel = _velocities()
    shape = pop.shape[1:]
    for _ in range(nsteps):
        x = pop.reshape(48, -1).T
        post = site_collide(x, tau_nu, tau_eta, dI).T.reshape((48,) + tuple(shape))
        pop = torch.stack([torch.roll(post[q], shifts=(int(vel[q, 2]), int(vel[q, 1]), int(vel[q, 0])),
                                      dims=(0, 1, 2)) for q in range(48)])
    return pop


def _cdiff(F, a):
    dim = 2 - a  # x is the last axis
    return 0.5 * (torch.roll(F, -1, dims=dim) - torch.roll(F, 1, dims=dim))


def init(u, B, tau_nu, tau_eta, dI, rho=None):
    """Initial populations (same reading as flame_oracle.c oracle_init) with
    central-difference gradients.  u, B [3, nz, ny, nx]."""
    shape = u.shape[1:]
    S = int(np.prod(shape))
    omega, omegaB = 1.0 / tau_nu, 1.0 / tau_eta
    r = torch.ones(S, dtype=_DT) if rho is None else rho.reshape(S)
    du = torch.stack([torch.stack([_cdiff(u[b], a) for b in range(3)]) for a in range(3)])  # [a, b, ...]
    dB = torch.stack([torch.stack([_cdiff(B[b], a) for b in range(3)]) for a in range(3)])
    du = du.reshape(3, 3, S).permute(2, 0, 1)
    dB = dB.reshape(3, 3, S).permute(2, 0, 1)
    U = u.reshape(3, S).T
    Bs = B.reshape(3, S).T
    J0 = torch.stack([dB[:, 1, 2] - dB[:, 2, 1], dB[:, 2, 0] - dB[:, 0, 2], dB[:, 0, 1] - dB[:, 1, 0]], -1)
    Pi = -(r[:, None, None] * CS2 / omega) * (du + du.transpose(1, 2))
    fne = W27[None, :] / (2 * CS2 * CS2) * torch.einsum("iab,sab->si", H2, Pi)
    f = feq(r, U) + lorentz(Bs) + fne
    gne = -(W7[None, None, :] / omegaB) * torch.einsum("ia,sab->sbi", XI7, dB)
    g = geq_hall(Bs, U, J0, dI) + gne
    x = torch.cat([f, g.reshape(S, 21)], dim=-1)
    return x.T.reshape((48,) + tuple(shape))


def magnetic_field(pop):
    return pop[27:].reshape((3, 7) + tuple(pop.shape[1:])).sum(1)


def band_energy(B, lo, hi):
    """sum_{lo <= n <= hi} E_B(n), E_B(n) = 1/2 sum_{round|m| = n} |B_hat|^2."""
    shape = B.shape[1:]
    n3 = float(np.prod(shape))
    mz = torch.fft.fftfreq(shape[0], 1.0 / shape[0], dtype=_DT)[:, None, None]
    my = torch.fft.fftfreq(shape[1], 1.0 / shape[1], dtype=_DT)[None, :, None]
    mx = torch.fft.fftfreq(shape[2], 1.0 / shape[2], dtype=_DT)[None, None, :]
    shell = torch.round(torch.sqrt(mx * mx + my * my + mz * mz))
    mask = ((shell >= lo) & (shell <= hi)).to(_DT)
    tot = 0.0
    for c in range(3):
        bh = torch.fft.fftn(B[c]) / n3
        tot = tot + 0.5 * (mask * (bh.real ** 2 + bh.imag ** 2)).sum()
    return tot
