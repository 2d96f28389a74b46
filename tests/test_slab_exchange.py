"""The z-slab decomposition's exchange schedule and diagnostics reduction on
CPU ranks (gloo), without a GPU: the library's host-only flame_halo_plan and
flame_reduce_combine drive a numpy emulation of the in-place AA step.

The emulated step keeps the AA pattern's data movement exactly (even: a
site reads its own slots and writes the opposite ones; odd: it reads the
opposite slot at x - c and writes its own slot at x + c) and replaces the
collision by an integer mixing of the 48 values of a site (modulo a prime,
so every value depends on all of them and the arithmetic is exact).  A
lattice split into slabs, each rank stepping its planes and trading the
runs of flame_halo_plan after every step (exchange_distributed), must equal
the same steps on the whole periodic lattice, value for value, after every
step; a missing or misplaced run, a wrong direction or a wrong parity shows
as a mismatch.  The ghost planes start as junk, so reading one before it is
filled also shows.  The diagnostics: raw sums of synthetic fields added over
ranks (allreduce_sums) and combined by the library equal the sums of the
whole lattice."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

PRIME = 2 ** 31 - 1


def _velocities():
    c = np.zeros((48, 3), dtype=np.int64)
    opp = np.zeros(48, dtype=np.int64)
    xi7 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    opp7 = [0, 2, 1, 4, 3, 6, 5]
    for q in range(27):  # storage slot (cx+1) + 3(cy+1) + 9(cz+1)
        c[q] = (q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1)
        opp[q] = 26 - q
    for i in range(7):  # storage slot 27 + 3 i + b
        for b in range(3):
            c[27 + 3 * i + b] = xi7[i]
            opp[27 + 3 * i + b] = 27 + 3 * opp7[i] + b
    return c, opp


C, OPP = _velocities()


def _mixing():
    return np.random.default_rng(5).integers(0, 7, size=(48, 48), dtype=np.int64)


def _collide(M, pre):
    """[48, ...] -> [48, ...]: M pre modulo PRIME."""
    sh = pre.shape
    return ((M @ pre.reshape(48, -1)) % PRIME).reshape(sh)


def _shift(a, c):
    """a[.., z - cz, y - cy, x - cx] (periodic in y and x; z by slicing the caller)."""
    return np.roll(a, (int(c[1]), int(c[0])), axis=(-2, -1))


def step_global(S, parity, M):
    """One AA step of the periodic lattice S [48, nz, ny, nx], in place."""
    if parity == 0:
        post = _collide(M, S.copy())
        S[OPP] = post
    else:
        pre = np.stack([np.roll(S[OPP[q]], tuple(int(v) for v in C[q][::-1]), axis=(0, 1, 2)) for q in range(48)])
        post = _collide(M, pre)
        for q in range(48):
            S[q] = np.roll(post[q], tuple(int(v) for v in C[q][::-1]), axis=(0, 1, 2))


def step_slab(A, parity, M):
    """One AA step of the nz interior planes of a slab A [48, nz + 2, ny, nx]
    (planes 0 and nz + 1 are ghosts): z is not wrapped."""
    nz = A.shape[1] - 2
    if parity == 0:
        post = _collide(M, A[:, 1:nz + 1].copy())
        A[OPP, 1:nz + 1] = post
    else:
        pre = np.stack([_shift(A[OPP[q], 1 - C[q][2]:nz + 1 - C[q][2]], C[q]) for q in range(48)])
        post = _collide(M, pre)
        for q in range(48):
            cz = int(C[q][2])
            A[q, 1 + cz:nz + 1 + cz] = _shift(post[q], C[q])


def _worker(rank, world, port, shape, steps, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2212_11024_gb300 import flame as F
        from paper_2212_11024_gb300 import slab as SL
        nz, ny, nx = shape
        M = _mixing()
        S = np.random.default_rng(11).integers(0, PRIME, size=(48,) + shape, dtype=np.int64)
        z0s, nzs = SL.split(nz, world)
        z0, n = z0s[rank], nzs[rank]
        A = np.full((48, n + 2, ny, nx), -12345, dtype=np.int64)  # junk ghost planes
        A[:, 1:n + 1] = S[:, z0:z0 + n]
        p = F.make_params(nx, ny, n, 0.6, 0.6, 0.0, "fp32", halo_z=True)
        state = torch.from_numpy(A.reshape(-1).view(np.uint8))  # shares A's memory
        ok = True
        for t in range(steps):
            step_global(S, t % 2, M)
            step_slab(A, t % 2, M)
            SL.exchange_distributed(state, p, (t + 1) % 2, dist, rank, world, 8)
            ok = ok and np.array_equal(A[:, 1:n + 1], S[:, z0:z0 + n])
        # diagnostics: raw sums of this rank's planes of synthetic fields
        rng = np.random.default_rng(3)
        u = rng.standard_normal((3,) + shape) * 0.05
        B = rng.standard_normal((3,) + shape) * 0.05 + np.array([0.01, 0.0, 0.1])[:, None, None, None]
        rho = 1.0 + 0.01 * rng.standard_normal(shape)
        J = rng.standard_normal((3,) + shape) * 0.01

        def sums(sl):
            r, uu, bb, jj = rho[sl], u[:, sl], B[:, sl], J[:, sl]
            db = bb - np.array(p.B_ref)[:, None, None, None]
            v = np.zeros(18)
            v[0] = r.sum()
            v[1:4] = (r * uu).sum(axis=(1, 2, 3))
            v[4:7] = bb.sum(axis=(1, 2, 3))
            v[7] = (uu * uu).sum()
            v[8] = (db * db).sum()
            v[9] = (uu * db).sum()
            v[10:13] = uu.sum(axis=(1, 2, 3))
            v[13] = (jj * jj).sum()
            v[14] = np.sqrt((uu * uu).sum(0)).max()
            v[15] = 0.0
            v[16] = 0.0
            v[17] = r.size
            return v

        total = SL.allreduce_sums(sums(slice(z0, z0 + n)), dist)
        whole = sums(slice(0, nz))
        sc, sw = F.reduce_combine(p, total), F.reduce_combine(p, whole)
        red_ok = all(abs(sc[k] - sw[k]) <= 1e-12 * max(1.0, abs(sw[k])) for k in sw)
        out[rank] = (ok, red_ok)
    finally:
        dist.destroy_process_group()


def _run(world, shape, steps, port):
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_worker, args=(world, port, shape, steps, out), nprocs=world, join=True, start_method="spawn")
    return [out[r] for r in range(world)]


@pytest.mark.parametrize("world,shape,port", [(1, (5, 3, 4), 29511), (2, (5, 3, 4), 29512), (3, (7, 2, 3), 29513),
                                               (2, (2, 4, 3), 29514)])
def test_slab_exchange_matches_the_whole_lattice(world, shape, port):
    """1, 2 and 3 slabs (one plane per slab in the last case), 7 steps (both
    parities, ending odd): every slab equals its planes of the whole
    lattice after every step, and the all-reduced diagnostics equal the
    whole lattice's."""
    res = _run(world, shape, 7, port)
    assert all(ok for ok, _ in res), res
    assert all(red for _, red in res), res


def _gather_worker(rank, world, port, shape, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import spectra as S
        from paper_2212_11024_gb300 import slab as SL
        nz = shape[0]
        rng = np.random.default_rng(17)
        u = rng.standard_normal((3,) + shape)
        B = rng.standard_normal((3,) + shape) + 0.1
        z0s, nzs = SL.split(nz, world)
        z0, n = z0s[rank], nzs[rank]
        us = torch.from_numpy(u[:, z0:z0 + n].copy())
        Bs = torch.from_numpy(B[:, z0:z0 + n].copy())
        root = world - 1
        g = SL.gather_fields(us, nzs, dist, rank, world, root=root)
        gather_ok = (g is None) if rank != root else np.array_equal(g.numpy(), u)
        spec = SL.diagnostics_distributed(
            lambda uw, Bw: (S.shell_spectrum(uw.numpy(), 6), S.shell_spectrum(Bw.numpy(), 6)),
            us, Bs, nzs, dist, rank, world, root=root)
        spec_ok = np.array_equal(spec[0], S.shell_spectrum(u, 6)) and np.array_equal(spec[1], S.shell_spectrum(B, 6))
        out[rank] = (gather_ok, spec_ok)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,shape,port", [(1, (4, 3, 5), 29521), (2, (5, 4, 6), 29522), (3, (7, 3, 4), 29523)])
def test_fft_diagnostics_of_a_split_lattice(world, shape, port):
    """The slabs' fields gathered to one rank (slabs of unequal plane
    counts) equal the whole lattice's, and a diagnostic evaluated there
    reaches every rank unchanged."""
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_gather_worker, args=(world, port, shape, out), nprocs=world, join=True, start_method="spawn")
    res = [out[r] for r in range(world)]
    assert all(a and b for a, b in res), res


def test_halo_plan_runs():
    """The runs of the plan: 9 fluid + 3 magnetic slots per face, the
    populations moving across the face (c_z = -1 slots 0..8 and 45..47,
    c_z = +1 slots 18..26 and 42..44), ghosts received before an odd step and
    sent back after it; invalid arguments refused."""
    from paper_2212_11024_gb300 import flame as F
    p = F.make_params(8, 6, 5, 0.6, 0.6, 0.0, "fp16", halo_z=True)
    down, up = [(0, 9), (45, 3)], [(18, 9), (42, 3)]
    send, recv = F.halo_plan(p, 1, 0)
    assert [r[:2] for r in send] == up and all(r[2] == 1 for r in send)
    assert [r[:2] for r in recv] == down and all(r[2] == 0 for r in recv)
    send, recv = F.halo_plan(p, 1, 1)
    assert [r[:2] for r in send] == down and all(r[2] == 5 for r in send)
    assert [r[:2] for r in recv] == up and all(r[2] == 6 for r in recv)
    send, recv = F.halo_plan(p, 0, 0)
    assert [r[:2] for r in send] == down and all(r[2] == 0 for r in send)
    assert [r[:2] for r in recv] == up and all(r[2] == 1 for r in recv)
    send, recv = F.halo_plan(p, 0, 1)
    assert [r[:2] for r in send] == up and all(r[2] == 6 for r in send)
    assert [r[:2] for r in recv] == down and all(r[2] == 5 for r in recv)
    # every slot listed moves across the face it is sent through
    C27 = [(q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1) for q in range(27)]
    assert all(C27[q][2] == -1 for q in range(0, 9)) and all(C27[q][2] == 1 for q in range(18, 27))
    with pytest.raises(ValueError):
        F.halo_plan(F.make_params(8, 6, 5, 0.6, 0.6, 0.0, "fp16"), 1, 0)  # not a slab
    with pytest.raises(ValueError):
        F.halo_plan(p, 2, 0)
    with pytest.raises(ValueError):
        F.halo_plan(p, 1, 2)


def test_slab_state_bytes_and_params():
    from paper_2212_11024_gb300 import flame as F
    p = F.make_params(8, 6, 5, 0.6, 0.6, 0.0, "fp16", halo_z=True)
    assert F.state_bytes(p) == 48 * 8 * 6 * 7 * 2
    assert F.state_bytes(F.make_params(8, 6, 5, 0.6, 0.6, 0.0, "fp16", halo_z=True, variant="fd_current")) == 0
    assert F.state_bytes(F.make_params(8, 6, 5, 0.6, 0.6, 0.0, "fp16")) == 48 * 8 * 6 * 5 * 2
