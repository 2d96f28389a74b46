"""Step throughput of any scheme variant, storage and kernel on an n^3 lattice.

Each configuration starts from the seeded turbulence fields of the 256^3
workload recipe (random-phase solenoidal u and B, shells 1..4, rms 0.05 per
component, seeds 3 and 4), takes ``warmup`` steps, then times ``steps`` steps
with CUDA events on the library's stream (graphs of ``graph_steps``
launches).  The state (48 populations per site) is larger than L2 from 128^3
on, so the timed steps stream it from HBM.  A line reports GLUPS (10^9
lattice updates per second), the state bytes per update (192 for 16-bit
storage, 384 for FP32; the finite-difference current also moves its FP32 B
field, which is not counted) and the count of non-finite sites after the
timed steps (a run that went non-finite is still timed, but is flagged).

    python -m paper_2212_11024_gb300.throughput --n 256 --variants flame,bgk,emhd,fd_current \\
        --storage fp16,bf16,fp32 --kernels auto,site
    python -m paper_2212_11024_gb300.throughput --n 256 --adjoint --storage fp32,fp16

``--adjoint`` times flame_step_adjoint instead: one stored state, a seeded
FP32 lambda_{t+1}, 576 B per update with FP32 storage (state read, lambda
gathered and written), 480 with 16-bit storage.

``--slabs K[,K...]`` times the lattice split into K z-slabs on one GPU
(SlabGroup: every slab's step, then the AA halo exchange through every
face, one launch per slab and step), against which the one-context lines
show the decomposition's cost.

    python -m paper_2212_11024_gb300.throughput --n 256 --slabs 1,2,4 --storage fp16
"""
from __future__ import annotations

import argparse
import json

from . import inputs
from .flame import Flame

STATE_BYTES = {"fp32": 384, "fp16": 192, "bf16": 192}


def step_throughput(n, variant="flame", storage="fp16", kernel="auto", steps=200, warmup=20, d_i=None,
                    tau=0.51, graph_steps=20, fields=None, device=None):
    """Time ``steps`` steps of one configuration; returns a dict (ms per step,
    GLUPS, state bytes per update, non-finite sites).  graph_steps is 0 or
    even (flame_params)."""
    import torch

    if fields is None:
        u, B = inputs.turbulence((n, n, n), 3, 4, 0.05, 0.05, shells=(1, 4))
    else:
        u, B = fields
    d_i = 0.05 * n if d_i is None else d_i
    sim = Flame(n, n, n, tau, tau, d_i, storage=storage, variant=variant, kernel=kernel, graph_steps=graph_steps,
                device=device)
    try:
        sim.init(None, u, B)
        sim.step(warmup)
        stream = sim.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(sim.device)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        bad = int(sim.reduce()["nonfinite"])
    finally:
        sim.close()
    return dict(n=n, variant=variant, storage=storage, kernel=kernel, d_i=d_i, tau=tau, steps=steps,
                ms_per_step=ms, glups=n ** 3 / (ms * 1e-3) / 1e9, state_bytes_per_update=STATE_BYTES[storage],
                nonfinite_sites=bad)


def adjoint_throughput(n, storage="fp32", steps=30, warmup=3, d_i=None, tau=0.51, fields=None, device=None):
    """Time ``steps`` calls of flame_step_adjoint on one stored state at n^3
    (lambda_{t+1} seeded Gaussian, FP32): ms per call, GLUPS and the bytes per
    update (state read, lambda_{t+1} gathered and lambda_t written: 48 values
    each)."""
    import ctypes

    import torch

    from .flame import _check, library

    if fields is None:
        u, B = inputs.turbulence((n, n, n), 3, 4, 0.05, 0.05, shells=(1, 4))
    else:
        u, B = fields
    d_i = 0.05 * n if d_i is None else d_i
    sim = Flame(n, n, n, tau, tau, d_i, storage=storage, device=device)
    try:
        sim.init(None, u, B)
        sim.step(3)
        blob, _, par = sim.get_state()
        gen = torch.Generator(device=sim.device)
        gen.manual_seed(7)
        lam_in = torch.randn((48, n ** 3), dtype=torch.float32, device=sim.device, generator=gen)
        lam_out = torch.empty_like(lam_in)
        ddi = torch.zeros(1, dtype=torch.float64, device=sim.device)
        lib = library()
        args = (sim._ctx, ctypes.c_void_p(blob.data_ptr()), par, ctypes.c_void_p(lam_in.data_ptr()),
                ctypes.c_void_p(lam_out.data_ptr()), ctypes.c_void_p(ddi.data_ptr()))
        for _ in range(warmup):
            _check(lib.flame_step_adjoint(*args), "flame_step_adjoint")
        stream = sim.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(sim.device)
        e0.record(stream)
        for _ in range(steps):
            _check(lib.flame_step_adjoint(*args), "flame_step_adjoint")
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
    finally:
        sim.close()
    bpu = 48 * (STATE_BYTES[storage] // 96) + 2 * 48 * 4
    return dict(n=n, kernel="adjoint_step", storage=storage, steps=steps, ms_per_step=ms,
                glups=n ** 3 / (ms * 1e-3) / 1e9, bytes_per_update=bpu)


def slab_throughput(n, nslabs, storage="fp16", steps=200, warmup=20, d_i=None, tau=0.51, fields=None,
                    device=None):
    """Time ``steps`` steps of the n^3 lattice split into ``nslabs`` z-slabs
    (SlabGroup); returns a dict like step_throughput's, with the bytes the
    halo exchange moves per step."""
    import torch

    from .slab import SlabGroup

    if fields is None:
        u, B = inputs.turbulence((n, n, n), 3, 4, 0.05, 0.05, shells=(1, 4))
    else:
        u, B = fields
    d_i = 0.05 * n if d_i is None else d_i
    grp = SlabGroup(n, n, n, nslabs, tau, tau, d_i, storage=storage, device=device)
    try:
        grp.init(None, u, B)
        grp.step(warmup)
        stream = grp.slabs[0].stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        grp.step(steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        bad = int(grp.reduce()["nonfinite"])
    finally:
        grp.close()
    # per face and step: 12 slot-planes each way
    halo = 2 * 12 * n * n * (STATE_BYTES[storage] // 96) * nslabs
    return dict(n=n, slabs=nslabs, storage=storage, steps=steps, ms_per_step=ms, glups=n ** 3 / (ms * 1e-3) / 1e9,
                state_bytes_per_update=STATE_BYTES[storage], halo_bytes_per_step=halo, nonfinite_sites=bad)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--variants", default="flame,bgk,emhd,fd_current")
    ap.add_argument("--storage", default="fp16,bf16,fp32")
    ap.add_argument("--kernels", default="auto,site")
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--d-i", type=float, default=None, help="Hall length (default 0.05 n)")
    ap.add_argument("--tau", type=float, default=0.51)
    ap.add_argument("--peak-gbs", type=float, default=None,
                    help="HBM bandwidth to report the state traffic against (GB/s)")
    ap.add_argument("--adjoint", action="store_true",
                    help="time flame_step_adjoint (per storage) instead of the forward step")
    ap.add_argument("--slabs", default=None, help="slab counts to time the z-slab decomposition with (e.g. 1,2,4)")
    a = ap.parse_args(argv)
    u, B = inputs.turbulence((a.n,) * 3, 3, 4, 0.05, 0.05, shells=(1, 4))
    if a.slabs:
        for st in a.storage.split(","):
            for k in a.slabs.split(","):
                r = slab_throughput(a.n, int(k), st, a.steps, a.warmup, a.d_i, a.tau, fields=(u, B))
                if a.peak_gbs:
                    r["frac_of_peak"] = r["glups"] * r["state_bytes_per_update"] / a.peak_gbs
                print(json.dumps(r), flush=True)
        return
    if a.adjoint:
        for st in a.storage.split(","):
            r = adjoint_throughput(a.n, st, min(a.steps, 100), a.warmup, a.d_i, a.tau, fields=(u, B))
            if a.peak_gbs:
                r["frac_of_peak"] = r["glups"] * r["bytes_per_update"] / a.peak_gbs
            print(json.dumps(r), flush=True)
        return
    for v in a.variants.split(","):
        for st in a.storage.split(","):
            # FP32 storage always runs the one-site kernel
            for kern in (("site",) if st == "fp32" else a.kernels.split(",")):
                r = step_throughput(a.n, v, st, kern, a.steps, a.warmup, a.d_i, a.tau, fields=(u, B))
                if a.peak_gbs:
                    r["frac_of_peak"] = r["glups"] * r["state_bytes_per_update"] / a.peak_gbs
                print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
