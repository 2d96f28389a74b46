"""A periodic lattice split into z-slabs, the one-direction domain
decomposition of the paper's multi-GPU runs (Sec. 4: the domain is split
along a single direction and boundary nodes are exchanged every step).

Each slab is a library context with ``halo_z``: its nz planes between two
ghost planes.  Under the in-place AA pattern an even step touches only a
site's own slots, so only the odd step crosses a slab face: before it the
ghost planes receive the 9 fluid and 3 magnetic slots of the neighbour's
boundary plane that move across the face, and after it what the odd step
wrote into the ghost planes goes back to the neighbour (flame_halo_plan
lists the runs; flame_halo_exchange copies them between two contexts on one
device).  Every kernel reads and writes only its own slab's memory.

``SlabGroup`` runs all slabs of a lattice on one GPU (the copies are
cudaMemcpy2DAsync on one stream); ``exchange_distributed`` is the same
exchange between one slab per process over torch.distributed point-to-point
calls, for a slab per GPU.  The scalar diagnostics of a split lattice are the
FP64 sums of every slab (flame_reduce_sums) added -- an all-reduce across
processes -- and combined by flame_reduce_combine.  The FFT
diagnostics (spectra, the energy budget, a band energy) need the whole
lattice: the slabs' u and B are assembled (gathered to one process, for a
slab per GPU) and evaluated by a context without state over the whole
lattice (flame_create_fields, flame_spectra_fields and the field forms of
flame_energy_budget and flame_band_energy).  The gathered FP64 u and B take
48 B per site, half the FP16 state of the same lattice.
"""
from __future__ import annotations

import numpy as np

from .flame import SUM_UMAX, Flame, halo_plan, reduce_combine


def split(nz, nslabs):
    """First planes and plane counts of nslabs slabs of nz planes (each >= 1)."""
    if not 1 <= nslabs <= nz:
        raise ValueError("need 1 <= nslabs <= nz")
    counts = [nz // nslabs + (1 if s < nz % nslabs else 0) for s in range(nslabs)]
    starts = list(np.cumsum([0] + counts[:-1]))
    return [int(v) for v in starts], counts


def _with_ghosts(f, z0, nzs):
    """Planes z0 - 1 .. z0 + nzs of a periodic field [..., nz, ny, nx]."""
    import torch
    nz = f.shape[-3]
    idx = [(z0 - 1 + k) % nz for k in range(nzs + 2)]
    if isinstance(f, np.ndarray):
        return np.ascontiguousarray(np.take(f, idx, axis=-3))
    return torch.index_select(f, f.dim() - 3, torch.tensor(idx, device=f.device)).contiguous()


class SlabGroup:
    """One periodic nx x ny x nz lattice as ``nslabs`` z-slab contexts on one
    GPU, stepped together with their halo exchange; the interface of Flame
    for the calls a split lattice supports (init, step, sync, moments,
    populations, reduce, get/set of the slabs' states)."""

    def __init__(self, nx, ny, nz, nslabs, tau_nu, tau_eta, d_i, storage="fp32", device=None, **kw):
        import torch

        self.shape = (int(nz), int(ny), int(nx))
        self.z0, self.nzs = split(int(nz), int(nslabs))
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        # one stream for every slab, so steps and exchanges are ordered
        stream = torch.cuda.current_stream(dev)
        self.slabs = [Flame(nx, ny, n, tau_nu, tau_eta, d_i, storage=storage, device=dev, stream=stream,
                            halo_z=True, **kw) for n in self.nzs]
        self._whole = (int(nx), int(ny), int(nz), tau_nu, tau_eta, d_i, storage, dev, stream, kw)
        self._fields = None

    def init(self, rho, u, B):
        """Initial fields [.., nz, ny, nx] of the whole lattice: each slab gets its
        planes and one neighbouring plane on each side (periodic)."""
        for s, z0, n in zip(self.slabs, self.z0, self.nzs):
            s.init(None if rho is None else _with_ghosts(rho, z0, n), _with_ghosts(u, z0, n),
                   _with_ghosts(B, z0, n))

    def exchange(self):
        """The halo exchange through every face, after all slabs took a step."""
        k = len(self.slabs)
        for i in range(k):
            self.slabs[i].halo_exchange(self.slabs[(i + 1) % k])

    def step(self, n=1):
        for _ in range(int(n)):
            for s in self.slabs:
                s.step(1)
            self.exchange()

    def sync(self):
        for s in self.slabs:
            s.sync()

    def info(self):
        return self.slabs[0].info()

    def moments(self, dtype=None):
        import torch
        parts = [s.moments(dtype=dtype) for s in self.slabs]
        return {k: torch.cat([p[k] for p in parts], dim=-3) for k in parts[0]}

    def populations(self):
        import torch
        return torch.cat([s.populations() for s in self.slabs], dim=-3)

    def field_context(self):
        """The context without state over the whole lattice (created on first
        use) that evaluates the FFT diagnostics of the assembled fields."""
        if self._fields is None:
            nx, ny, nz, tau_nu, tau_eta, d_i, storage, dev, stream, kw = self._whole
            self._fields = Flame(nx, ny, nz, tau_nu, tau_eta, d_i, storage=storage, device=dev, stream=stream,
                                 fields_only=True, **kw)
        return self._fields

    def fields(self):
        """u and B of the whole lattice, FP64 CUDA [3, nz, ny, nx]."""
        m = self.moments()
        return m["u"], m["B"]

    def spectra(self, nshell):
        """Shell spectra (E_u, E_B) of the whole lattice (flame_spectra_fields)."""
        u, B = self.fields()
        return self.field_context().spectra(nshell, u, B)

    def energy_budget(self, nshell):
        """(E, S, D) of the whole lattice (flame_energy_budget of its fields)."""
        u, B = self.fields()
        return self.field_context().energy_budget(nshell, u, B)

    def band_energy(self, lo, hi, grad=False):
        """flame_band_energy of the whole lattice's B: (L, dL/dB or None)."""
        _, B = self.fields()
        L, g, _ = self.field_context().band_energy(lo, hi, B, grad=grad)
        return L, g

    def reduce(self):
        """FP64 scalars of the whole lattice from the slabs' raw sums."""
        sums = [s.reduce_sums() for s in self.slabs]
        total = np.sum(sums, axis=0)
        total[SUM_UMAX] = max(v[SUM_UMAX] for v in sums)
        return reduce_combine(self.slabs[0].p, total)

    def close(self):
        for s in self.slabs:
            s.close()
        if self._fields is not None:
            self._fields.close()
            self._fields = None


def _run_view(state, p, run, elem_bytes):
    """The bytes of a run (first_slot, nslots, plane) of a slab's state (a
    uint8 tensor of flame_state_bytes) as an [nslots, plane bytes] view."""
    first, nslots, plane = run
    pb = p.nx * p.ny * elem_bytes
    n3s = p.nx * p.ny * (p.nz + 2)
    return state.as_strided((nslots, pb), (n3s * elem_bytes, 1), (first * n3s + plane * p.nx * p.ny) * elem_bytes)


def exchange_distributed(state, p, parity, dist, rank, world, elem_bytes):
    """The halo exchange of one slab per process: slab `rank` of `world`
    (slab r + 1 above slab r, periodic), its state a uint8 tensor, after a
    step that left AA parity `parity`.  Through each face it sends the runs
    of flame_halo_plan to the neighbour and receives the neighbour's runs,
    with torch.distributed isend / irecv (tag: the sending face and run).
    With one process the faces trade with each other locally.  Call it on
    every rank after every step; the state must be up to date (the step
    synchronised) and is written when the call returns."""
    plans = [halo_plan(p, parity, face) for face in (0, 1)]
    if world == 1:
        for face in (0, 1):
            send, _ = plans[face]
            _, recv = plans[1 - face]
            for r in range(2):
                _run_view(state, p, recv[r], elem_bytes).copy_(_run_view(state, p, send[r], elem_bytes))
        return
    peers = ((rank - 1) % world, (rank + 1) % world)
    reqs, inbox = [], []
    for face in (0, 1):
        send, recv = plans[face]
        for r in range(2):
            buf = _run_view(state, p, send[r], elem_bytes).contiguous()
            reqs.append(dist.isend(buf, peers[face], tag=10 * face + r))
            got = state.new_empty((recv[r][1], p.nx * p.ny * elem_bytes))
            # the neighbour sends these through its opposite face
            reqs.append(dist.irecv(got, peers[face], tag=10 * (1 - face) + r))
            inbox.append((recv[r], got))
    for q in reqs:
        q.wait()
    for run, got in inbox:
        _run_view(state, p, run, elem_bytes).copy_(got)


def allreduce_sums(sums, dist):
    """Add the raw FP64 sums of every process's slab (the maximum at
    SUM_UMAX) with torch.distributed all-reduces; returns numpy FP64."""
    import torch
    t = torch.tensor(np.asarray(sums, dtype=np.float64))
    m = t[SUM_UMAX].clone().reshape(1)
    t[SUM_UMAX] = 0.0
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    t[SUM_UMAX] = m[0]
    return t.numpy()


def gather_fields(fields, nzs, dist, rank, world, root=0):
    """The whole lattice's field on `root` from every process's slab field
    [..., nzs[rank], ny, nx] (slab r + 1 above slab r): the slabs in order,
    concatenated along z, on root; None on the other ranks.  Point-to-point
    (send / recv), so slabs of different plane counts need no padding."""
    import torch
    f = fields.contiguous()
    if world == 1:
        return f
    if rank != root:
        dist.send(f, root)
        return None
    parts = []
    for r in range(world):
        if r == root:
            parts.append(f)
            continue
        buf = f.new_empty(tuple(f.shape[:-3]) + (int(nzs[r]),) + tuple(f.shape[-2:]))
        dist.recv(buf, r)
        parts.append(buf)
    return torch.cat(parts, dim=-3)


def diagnostics_distributed(compute, u, B, nzs, dist, rank, world, root=0):
    """Evaluate a whole-lattice diagnostic of a lattice split into one slab
    per process: the slabs' u and B [3, nzs[rank], ny, nx] are gathered to
    `root` (gather_fields), compute(u, B) runs there -- for instance the
    spectra of a context without state, ``lambda u, B: ctx.spectra(n, u, B)``
    -- and its result (numpy arrays or numbers) is broadcast to every rank,
    which all return it."""
    uw = gather_fields(u, nzs, dist, rank, world, root)
    Bw = gather_fields(B, nzs, dist, rank, world, root)
    out = [compute(uw, Bw) if rank == root else None]
    if world > 1:
        dist.broadcast_object_list(out, src=root)
    return out[0]
