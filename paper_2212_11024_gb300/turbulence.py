"""Decaying Hall-MHD turbulence runs (Sec. 5): spectra and throughput.

A run starts from seeded random-phase solenoidal u and B with their energy in
a band of shells (``inputs.turbulence``), advances the lattice in chunks of
``spectra_every`` steps and records, after every chunk, the shell spectra
E_u(n), E_B(n) (``flame_spectra``) and the FP64 scalars of ``flame_reduce``.
Throughput is the step kernel alone: CUDA events bracket each chunk of
``flame_step`` calls on the library's stream, so the diagnostics between
chunks are not counted.
"""
from __future__ import annotations

import math

import numpy as np

from . import inputs
from .flame import Flame


def decay(n, d_i, steps, spectra_every=100, storage="fp32", tau_nu=0.51, tau_eta=0.51, rms_u=0.05, rms_b=0.05,
          shells=(1, 4), seeds=(1, 2), nshell=None, graph_steps=0, device=None, fields=None):
    """One decaying-turbulence run on an n^3 periodic lattice.

    Returns a dict with ``t`` [m] (steps at each record, 0 first), ``Eu``,
    ``Eb`` [m, nshell] shell spectra, ``scalars`` (list of dicts from
    ``Flame.reduce``), ``first_nonfinite`` (end of the first chunk after
    which the state held a non-finite value, or None; the run stops there),
    ``ms_per_step`` and ``mlups`` (step kernel only, over the steps taken).
    ``fields`` = (u, B) overrides the seeded generator."""
    import torch

    if nshell is None:
        nshell = n // 2 + 1
    if fields is None:
        u, B = inputs.turbulence((n, n, n), seeds[0], seeds[1], rms_u, rms_b, shells=shells)
    else:
        u, B = fields
    sim = Flame(n, n, n, tau_nu, tau_eta, d_i, storage=storage, device=device, graph_steps=graph_steps)
    try:
        sim.init(None, u, B)
        del u, B
        t, Eu, Eb, sc = [0], [], [], []
        e, b = sim.spectra(nshell)
        Eu.append(e)
        Eb.append(b)
        sc.append(sim.reduce())
        first_bad = None
        stream = sim.stream
        ms = 0.0
        done = 0
        while done < steps:
            k = min(spectra_every, steps - done)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(k)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            done += k
            s = sim.reduce()
            if s["status"] != 0 or not math.isfinite(s["E_u"] + s["E_B"]):
                first_bad = done  # the non-finite state is sticky: the run ends here
                break
            t.append(done)
            sc.append(s)
            e, b = sim.spectra(nshell)
            Eu.append(e)
            Eb.append(b)
        n3 = float(n) ** 3
        return dict(n=n, d_i=d_i, storage=storage, tau_nu=tau_nu, tau_eta=tau_eta, steps=done,
                    t=np.array(t), Eu=np.array(Eu), Eb=np.array(Eb), scalars=sc, first_nonfinite=first_bad,
                    ms_per_step=ms / max(done, 1), mlups=n3 * done / (ms * 1e3) if ms > 0 else float("nan"))
    finally:
        sim.close()
