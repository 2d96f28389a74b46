"""The hand-written adjoints (flame_step_adjoint, flame_init_adjoint) and the
checkpointed gradient against FP64 references: automatic differentiation of
the PyTorch restatement of the oracle (oracle/torch_ref.py), and central
finite differences of the C oracle.

Tolerances: the adjoint runs in FP32 along the GPU's FP32 trajectory, so a
one-step VJP carries ~1e-7 relative rounding and a chain of tens of steps
~1e-6; 1e-5 (one step) and 1e-4 (chains, finite differences) leave a margin
of one to two orders of magnitude.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from gpu_helpers import turbulence
from oracle import torch_ref as R

pytestmark = pytest.mark.gpu


def _vjp_reference(pop, lam, tau_nu, tau_eta, di):
    x = torch.tensor(pop, requires_grad=True)
    d = torch.tensor(di, dtype=torch.float64, requires_grad=True)
    y = R.step(x, tau_nu, tau_eta, d, 1)
    gx, gd = torch.autograd.grad((y * torch.tensor(lam)).sum(), [x, d])
    return gx.numpy(), float(gd)


def _di_terms(pop, lam, tau_nu, tau_eta, di):
    """The per-site terms of dL/dd_i (their sum is the reference's gradient):
    the site collision of the torch restatement with one d_i per site, built
    from its own helpers, then streamed as in its step."""
    shape = pop.shape[1:]
    x = torch.tensor(pop).reshape(48, -1).T
    d = torch.full((x.shape[0],), float(di), dtype=torch.float64, requires_grad=True)
    omega, omegaB = 1.0 / tau_nu, 1.0 / tau_eta
    f, g = x[:, :27], x[:, 27:].reshape(-1, 3, 7)
    rho = f.sum(-1)
    U = (f @ R.C27) / rho[:, None]
    B = g.sum(-1)
    J = R.current(torch.einsum("ia,sbi->sab", R.XI7, g), U, B, omegaB, d)
    V = U - d[:, None] * J
    L0 = V[:, :, None] * B[:, None, :] - B[:, :, None] * V[:, None, :]
    geq = R.W7[None, None, :] * (B[:, :, None] + torch.einsum("ia,sab->sbi", R.XI7, L0) / R.CC2)
    gs = g - omegaB * (g - geq)
    fs = R.collide_fluid(f, R.feq(rho, U) + R.lorentz(B), U, omega)
    post = torch.cat([fs, gs.reshape(-1, 21)], dim=-1).T.reshape((48,) + tuple(shape))
    vel = R._velocities()
    y = torch.stack([torch.roll(post[q], shifts=(int(vel[q, 2]), int(vel[q, 1]), int(vel[q, 0])), dims=(0, 1, 2))
                     for q in range(48)])
    (a,) = torch.autograd.grad((y * torch.tensor(lam)).sum(), [d])
    return a.numpy()


@pytest.mark.parametrize("storage,nsteps,shape", [("fp32", 3, (6, 5, 7)), ("fp32", 4, (6, 5, 7)),
                                                 ("fp16", 3, (6, 5, 7)), ("fp32", 3, (5, 1, 20)),
                                                 ("fp16", 4, (8, 20, 70)), ("bf16", 3, (4, 9, 130))])
def test_step_adjoint_matches_autograd(storage, nsteps, shape):
    """One adjoint step at a state with either AA parity (3 or 4 forward steps),
    vs torch autograd of the FP64 step at the GPU's own decoded state.  The
    shapes cover blocks of one and of two warps (a one-plane y extent), rows
    longer than a block with a ragged end, and more d_i partials than the
    first summing level has blocks."""
    from paper_2212_11024_gb300 import Flame
    from paper_2212_11024_gb300.flame import library
    nz, ny, nx = shape
    u, B = turbulence(shape, 13, 0.05)
    B[2] += 0.05
    sim = Flame(nx, ny, nz, 0.57, 0.62, 1.3, storage=storage, B_ref=(0, 0, 0.05))
    sim.init(None, u, B)
    sim.step(nsteps)
    blob, _, par = sim.get_state()
    pop = sim.populations().cpu().numpy()
    rng = np.random.default_rng(nsteps)
    lam = rng.standard_normal((48,) + shape)
    lin = torch.tensor(lam.reshape(48, -1), dtype=torch.float32, device="cuda")
    lout = torch.empty_like(lin)
    ddi = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = library().flame_step_adjoint(sim._ctx, ctypes.c_void_p(blob.data_ptr()), par, ctypes.c_void_p(lin.data_ptr()),
                                      ctypes.c_void_p(lout.data_ptr()), ctypes.c_void_p(ddi.data_ptr()))
    assert rc == 0
    torch.cuda.synchronize()
    got = lout.cpu().numpy().reshape((48,) + shape)
    ref, ref_d = _vjp_reference(pop, lam, 0.57, 0.62, 1.3)
    terms = _di_terms(pop, lam, 0.57, 0.62, 1.3)
    sim.close()
    assert np.abs(got - ref).max() < 1e-5 * np.abs(ref).max()
    assert abs(terms.sum() - ref_d) < 1e-12 * np.abs(terms).sum()
    # d_i: the sites' terms cancel (a random lambda; sum |a| / |sum a| up to
    # ~5e3 here), so the bound is the FP32 rounding of each term, ~50 eps
    # per term added as independent errors, plus 1e-5 of the total.
    tol = 1e-5 * abs(ref_d) + 3e-6 * np.sqrt((terms ** 2).sum())
    assert abs(float(ddi[0]) - ref_d) < tol


@pytest.mark.parametrize("N,storage,nsteps", [(256, "fp16", 3), (256, "fp32", 4), (512, "fp16", 3)])
def test_step_adjoint_full_size_sampled_sites(N, storage, nsteps):
    """256^3 (the adjoint's benchmark lattice, d_i = 0.05 N, tau = 0.51), both
    AA parities, and 512^3 (lambda of more than 2^31 values): lambda_t at 16
    sampled sites (including the lattice's last plane, row and column)
    against autograd of the torch restatement's collision of that site
    alone, with lambda_{t+1} gathered from x + c_q.  lambda_t at a site
    depends only on its own state and on that gather, so the full-size
    launch is checked site by site."""
    import torch
    from paper_2212_11024_gb300 import Flame
    from paper_2212_11024_gb300.flame import library
    if N <= 256:
        u, B = turbulence((N, N, N), 3, 0.05, shells=(1, 4))
    else:
        # Orszag-Tang fields (Sec. 4.4), built on the device in FP32
        q = torch.arange(N, device="cuda", dtype=torch.float32) * (2 * np.pi / N)
        X, Y, Z = q.view(1, 1, N), q.view(1, N, 1), q.view(N, 1, 1)
        full = (N, N, N)
        u = torch.stack([(-2 * torch.sin(Y)).expand(full), (2 * torch.sin(X)).expand(full),
                         torch.zeros(full, device="cuda")]) * 0.02
        B = torch.stack([(-2 * torch.sin(2 * Y) + torch.sin(Z)).expand(full),
                         (2 * torch.sin(X) + torch.sin(Z)).expand(full),
                         (torch.sin(X) + torch.sin(Y)).expand(full)]) * (0.8 * 0.02)
    sim = Flame(N, N, N, 0.51, 0.51, 0.05 * N, storage=storage)
    sim.init(None, u, B)
    del u, B
    sim.step(nsteps)
    blob, _, par = sim.get_state()
    pop = sim.populations()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(nsteps)
    lin = torch.randn((48, N ** 3), dtype=torch.float32, device="cuda", generator=gen)
    lout = torch.empty_like(lin)
    ddi = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = library().flame_step_adjoint(sim._ctx, ctypes.c_void_p(blob.data_ptr()), par, ctypes.c_void_p(lin.data_ptr()),
                                      ctypes.c_void_p(lout.data_ptr()), ctypes.c_void_p(ddi.data_ptr()))
    assert rc == 0
    torch.cuda.synchronize()
    vel = R._velocities().numpy()
    rng = np.random.default_rng(nsteps)
    sites = [(N - 1, N - 1, N - 1), (0, N - 1, 0), (N - 1, 0, N - 1)] + [tuple(rng.integers(0, N, 3)) for _ in range(13)]
    worst = 0.0
    for z, y, x in sites:
        pre = torch.tensor(pop[:, z, y, x].cpu().numpy()[None, :], requires_grad=True)
        gathered = [float(lin[q, (((z + c[2]) % N) * N + (y + c[1]) % N) * N + (x + c[0]) % N]) for q, c in enumerate(vel)]
        post = R.site_collide(pre, 0.51, 0.51, torch.tensor(0.05 * N, dtype=torch.float64))
        (g,) = torch.autograd.grad((post[0] * torch.tensor(gathered, dtype=torch.float64)).sum(), [pre])
        ref = g[0].numpy()
        got = lout[:, (z * N + y) * N + x].double().cpu().numpy()
        worst = max(worst, float(np.abs(got - ref).max() / np.abs(ref).max()))
    sim.close()
    assert worst < 1e-5, worst


def test_init_adjoint_matches_autograd():
    from paper_2212_11024_gb300 import Flame
    from paper_2212_11024_gb300.flame import library
    shape = (5, 6, 4)
    nz, ny, nx = shape
    u, B = turbulence(shape, 17, 0.05)
    B[2] += 0.05
    sim = Flame(nx, ny, nz, 0.58, 0.62, 1.4)
    rng = np.random.default_rng(3)
    lam = rng.standard_normal((48,) + shape)
    ud = torch.tensor(u, device="cuda")
    Bd = torch.tensor(B, device="cuda")
    l0 = torch.tensor(lam.reshape(48, -1), dtype=torch.float32, device="cuda")
    ub = torch.empty_like(ud)
    Bb = torch.empty_like(Bd)
    ddi = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = library().flame_init_adjoint(sim._ctx, ctypes.c_void_p(ud.data_ptr()), ctypes.c_void_p(Bd.data_ptr()),
                                      ctypes.c_void_p(l0.data_ptr()), ctypes.c_void_p(ub.data_ptr()),
                                      ctypes.c_void_p(Bb.data_ptr()), ctypes.c_void_p(ddi.data_ptr()))
    assert rc == 0
    torch.cuda.synchronize()
    sim.close()
    ut = torch.tensor(u, requires_grad=True)
    Bt = torch.tensor(B, requires_grad=True)
    d = torch.tensor(1.4, dtype=torch.float64, requires_grad=True)
    pop = R.init(ut, Bt, 0.58, 0.62, d)
    gu, gB, gd = torch.autograd.grad((pop * torch.tensor(np.float32(lam).astype(np.float64))).sum(), [ut, Bt, d])
    # FP64 arithmetic, but omega, omega_B and d_i reach the kernels as FP32
    # constants (as in the forward initialisation): ~3e-8 relative.
    assert np.abs(Bb.cpu().numpy() - gB.numpy()).max() < 2e-7 * np.abs(gB.numpy()).max()
    assert np.abs(ub.cpu().numpy() - gu.numpy()).max() < 2e-7 * np.abs(gu.numpy()).max()
    assert abs(float(ddi[0]) - float(gd)) < 2e-7 * abs(float(gd))


def test_checkpointed_gradient_matches_fp64_autograd():
    """L = magnetic energy in shells 1..2 after 12 steps: gradient in u0, B0
    and d_i from the autograd Function (sqrt(N) checkpointing) vs torch
    autograd of the FP64 restatement."""
    from paper_2212_11024_gb300.adjoint import FlameBandEnergy
    shape = (8, 6, 10)
    u, B = turbulence(shape, 23, 0.04)
    B[2] += 0.03
    tau_nu, tau_eta, di, n = 0.6, 0.65, 1.5, 12
    u0 = torch.tensor(u, device="cuda", requires_grad=True)
    B0 = torch.tensor(B, device="cuda", requires_grad=True)
    d = torch.tensor(di, dtype=torch.float64, device="cuda", requires_grad=True)
    L = FlameBandEnergy.apply(u0, B0, d, tau_nu, tau_eta, n, (1, 2))
    L.backward()
    ut = torch.tensor(u, requires_grad=True)
    Bt = torch.tensor(B, requires_grad=True)
    dt = torch.tensor(di, dtype=torch.float64, requires_grad=True)
    pop = R.step(R.init(ut, Bt, tau_nu, tau_eta, dt), tau_nu, tau_eta, dt, n)
    Lr = R.band_energy(R.magnetic_field(pop), 1, 2)
    gu, gB, gd = torch.autograd.grad(Lr, [ut, Bt, dt])
    assert abs(float(L.detach()) - float(Lr.detach())) < 1e-5 * float(Lr.detach())

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    assert rel(B0.grad.cpu().numpy(), gB.numpy()) < 1e-4
    assert rel(u0.grad.cpu().numpy(), gu.numpy()) < 1e-4
    assert abs(float(d.grad) - float(gd)) < 1e-4 * abs(float(gd))


def test_config4_gradient_vs_fp64_finite_differences():
    """Config 4: 64^3, 200 steps from shell-1..4 fields (u_rms = b_rms = 0.03,
    seeds 5 and 6), loss = magnetic energy in shells 8..16 at the last step,
    tau_nu = tau_eta = 0.6, d_i = 3.2.  Directional derivatives of the GPU
    gradient along 2 seeded solenoidal directions of B0 and along d_i, vs
    central differences (eps = 1e-3) of the FP64 oracle's forward."""
    from oracle import spectra as S
    from paper_2212_11024_gb300 import inputs as I
    from paper_2212_11024_gb300.adjoint import band_energy_gradient
    N, n, band = 64, 200, (8, 16)
    tau, di = 0.6, 3.2
    u, B = I.turbulence((N, N, N), 5, 6, 0.03, 0.03, shells=(1, 4))
    L, ub, Bb, gdi = band_energy_gradient(u, B, di, tau, tau, n, band)
    Bb = Bb.cpu().numpy()

    def oracle_loss(Bf, d):
        p = O.Params(N, N, N, tau, tau, d)
        pop = O.init(p, None, u, Bf)
        O.step(p, pop, n, literal=False)
        m = O.moments(p, pop)
        Bm = m["B"] - m["B"].reshape(3, -1).mean(1)[:, None, None, None]
        return S.shell_spectrum(Bm, band[1] + 1)[band[0]:band[1] + 1].sum()

    eps = 1e-3
    for seed in (31, 32):
        _, dirB = I.turbulence((N, N, N), seed, seed + 1, 1.0, 1.0, shells=(1, 6))
        dirB /= np.linalg.norm(dirB)
        fd = (oracle_loss(B + eps * dirB, di) - oracle_loss(B - eps * dirB, di)) / (2 * eps)
        ad = float((Bb * dirB).sum())
        assert abs(ad - fd) < 1e-4 * abs(fd), (ad, fd)
    fd = (oracle_loss(B, di + eps) - oracle_loss(B, di - eps)) / (2 * eps)
    assert abs(gdi - fd) < 1e-4 * abs(fd), (gdi, fd)
