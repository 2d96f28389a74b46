"""Gradients through N fused steps: torch.autograd.Function over the C ABI.

The loss is the magnetic energy in a band of spectral shells at the last
step, L = sum_{lo <= n <= hi} E_B(n) with E_B(n) = 1/2 sum_{round|m| = n}
|B_hat(m)|^2 and B_hat = FFT(B) / N3 (the spectra of Sec. 4.4), evaluated
with its seed dL/df by the library (flame_band_energy).  Its
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
        # the loss of the last state and the adjoint seed dL/df (flame_band_energy)
        L, _, seed = sim.band_energy(band[0], band[1], adjoint_seed=True)
        return L, seed

    def backward(self, u0, B0, seed):
        sim = self.sim
        lib = library()
        dev = sim.device
        lam = seed.clone()
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
        return torch.tensor(L, dtype=torch.float64, device=B0.device)

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
