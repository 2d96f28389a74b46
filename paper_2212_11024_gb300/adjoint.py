"""Gradients through N fused steps: torch.autograd.Function over the C ABI.

The loss is the magnetic energy in a band of spectral shells at the last
step, L = sum_{lo <= n <= hi} E_B(n) with E_B(n) = 1/2 sum_{round|m| = n}
|B_hat(m)|^2 and B_hat = FFT(B) / N3 (the spectra of Sec. 4.4).  Its
gradient with respect to the initial magnetic field, the initial velocity
and the Hall length d_i comes from the library's hand-written adjoints
(flame_step_adjoint, flame_init_adjoint), run backwards over the stored
forward states with sqrt(N) checkpointing: the forward pass keeps every k-th
state (k = ceil(sqrt(N))); the backward pass replays each segment of k steps
from its checkpoint, keeps those k states, and applies the step adjoints in
reverse.  Memory: about N/k + k state copies.
"""
from __future__ import annotations

import ctypes
import math

import torch

from .flame import Flame, _check, library


def band_energy_and_seed(B, lo, hi):
    """L and dL/dB for L = sum_{lo<=n<=hi} E_B(n) of B [3, nz, ny, nx] (FP64, any device)."""
    shape = B.shape[1:]
    n3 = float(shape[0] * shape[1] * shape[2])
    dev = B.device
    mz = torch.fft.fftfreq(shape[0], 1.0 / shape[0], dtype=torch.float64, device=dev)[:, None, None]
    my = torch.fft.fftfreq(shape[1], 1.0 / shape[1], dtype=torch.float64, device=dev)[None, :, None]
    mx = torch.fft.fftfreq(shape[2], 1.0 / shape[2], dtype=torch.float64, device=dev)[None, None, :]
    shell = torch.round(torch.sqrt(mx * mx + my * my + mz * mz))
    mask = ((shell >= lo) & (shell <= hi)).to(torch.float64)
    Bh = torch.fft.fftn(B, dim=(1, 2, 3))
    L = 0.5 * (mask * (Bh.real ** 2 + Bh.imag ** 2)).sum() / (n3 * n3)
    seed = torch.fft.ifftn(mask * Bh, dim=(1, 2, 3)).real / n3
    return L, seed


class _Run:
    """One forward run with checkpoints, and its backward sweep."""

    def __init__(self, shape, tau_nu, tau_eta, d_i, storage, B_ref, device):
        nz, ny, nx = shape
        self.sim = Flame(nx, ny, nz, tau_nu, tau_eta, d_i, storage=storage, B_ref=B_ref, device=device)
        self.shape = tuple(shape)
        self.n3 = nx * ny * nz

    def forward(self, u0, B0, nsteps, band):
        sim = self.sim
        sim.init(None, u0, B0)
        self.k = max(1, int(math.ceil(math.sqrt(max(nsteps, 1)))))
        self.ckpt = {}
        for t in range(nsteps):
            if t % self.k == 0:
                self.ckpt[t] = sim.get_state()
            sim.step(1)
        sim.sync()
        self.nsteps = nsteps
        B = sim.moments()["B"]
        L, seed = band_energy_and_seed(B, *band)
        return L, seed

    def backward(self, u0, B0, seed):
        sim = self.sim
        lib = library()
        dev = sim.device
        lam = torch.zeros((48, self.n3), dtype=torch.float32, device=dev)
        lam[27:] = seed.reshape(3, 1, self.n3).expand(3, 7, self.n3).reshape(21, self.n3).to(torch.float32)
        other = torch.empty_like(lam)
        ddi = torch.zeros(1, dtype=torch.float64, device=dev)
        ddi_total = torch.zeros(1, dtype=torch.float64, device=dev)
        starts = sorted(self.ckpt.keys())
        for s0 in reversed(starts):
            s1 = min(s0 + self.k, self.nsteps)
            blob, step, par = self.ckpt[s0]
            sim.set_state(blob, step, par)
            seg = []
            for _ in range(s0, s1):
                seg.append(sim.get_state())
                sim.step(1)
            for blob_t, _, par_t in reversed(seg):
                _check(lib.flame_step_adjoint(sim._ctx, ctypes.c_void_p(blob_t.data_ptr()), int(par_t),
                                              ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(other.data_ptr()),
                                              ctypes.c_void_p(ddi.data_ptr())), "flame_step_adjoint")
                lam, other = other, lam
                ddi_total += ddi
            del seg
        ubar = torch.empty((3,) + self.shape, dtype=torch.float64, device=dev)
        Bbar = torch.empty((3,) + self.shape, dtype=torch.float64, device=dev)
        _check(lib.flame_init_adjoint(sim._ctx, ctypes.c_void_p(u0.data_ptr()), ctypes.c_void_p(B0.data_ptr()),
                                      ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(ubar.data_ptr()),
                                      ctypes.c_void_p(Bbar.data_ptr()), ctypes.c_void_p(ddi.data_ptr())),
               "flame_init_adjoint")
        ddi_total += ddi
        sim.sync()
        return ubar, Bbar, ddi_total[0]

    def close(self):
        self.sim.close()


class FlameBandEnergy(torch.autograd.Function):
    """L = band magnetic energy after `nsteps` fused steps from (u0, B0).

    Inputs u0, B0: FP64 CUDA tensors [3, nz, ny, nx]; d_i: FP64 scalar tensor.
    Differentiable in u0, B0 and d_i (rho0 = 1, central-difference gradients
    at initialisation)."""

    @staticmethod
    def forward(ctx, u0, B0, d_i, tau_nu, tau_eta, nsteps, band, storage="fp32"):
        u0 = u0.detach().to(torch.float64).contiguous()
        B0 = B0.detach().to(torch.float64).contiguous()
        B_ref = tuple(float(v) for v in B0.reshape(3, -1).mean(dim=1))
        run = _Run(B0.shape[1:], tau_nu, tau_eta, float(d_i), storage, B_ref, B0.device)
        L, seed = run.forward(u0, B0, int(nsteps), tuple(band))
        ctx.run = run
        ctx.save_for_backward(u0, B0, seed)
        return L.detach().clone()

    @staticmethod
    def backward(ctx, gL):
        u0, B0, seed = ctx.saved_tensors
        ubar, Bbar, ddi = ctx.run.backward(u0, B0, seed)
        ctx.run.close()
        g = gL.to(torch.float64)
        return g * ubar, g * Bbar, (g * ddi).reshape(()), None, None, None, None, None


def band_energy_gradient(u0, B0, d_i, tau_nu, tau_eta, nsteps, band, storage="fp32"):
    """(L, dL/du0, dL/dB0, dL/dd_i) in one call (no autograd graph needed)."""
    u0 = torch.as_tensor(u0, dtype=torch.float64).cuda().contiguous()
    B0 = torch.as_tensor(B0, dtype=torch.float64).cuda().contiguous()
    B_ref = tuple(float(v) for v in B0.reshape(3, -1).mean(dim=1))
    run = _Run(B0.shape[1:], tau_nu, tau_eta, float(d_i), storage, B_ref, B0.device)
    try:
        L, seed = run.forward(u0, B0, int(nsteps), tuple(band))
        ubar, Bbar, ddi = run.backward(u0, B0, seed)
    finally:
        run.close()
    return float(L), ubar, Bbar, float(ddi)
