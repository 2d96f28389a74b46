"""What 16-bit deviation storage does to decaying Hall-MHD turbulence.

For several seeded realisations of the 256^3 workload recipe (random-phase
solenoidal u, B in shells 1..4, rms 0.05 per component, tau = 0.51,
d_i = 0.05 n) every storage configuration runs the same fields for ``steps``
steps:

  fp32 / site   the reference (FP32 storage, one-site kernel)
  fp16 / auto   FP16 deviations (row kernel)
  bf16 / auto   BF16 deviations (row kernel)
  fp16 / site   the rounding-order control: the same FP16 storage, but the
                FP32 collision evaluated in another order (one-site kernel)

Recorded: the FP64 scalars (E_u, E_B, <|J|^2>) every ``every`` steps and the
shell spectra E_u(n), E_B(n) at the end.  Reported, per configuration,
against fp32 (and the control against fp16 / auto), as the mean and the
spread over the realisations: the signed relative difference of each
shell's energy at the end, of the total energy E(t), and of the decay rate
-dE/dt (central differences of E(t)).  A difference that keeps its sign
over realisations with a spread well below its mean is a bias of the storage
format; one whose mean is within its spread is the flow's chaos amplifying
rounding differences.

    python -m paper_2212_11024_gb300.precision --n 256 --steps 500 --seeds 3
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import inputs
from .flame import Flame

CONFIGS = (("fp32", "site"), ("fp16", "auto"), ("bf16", "auto"), ("fp16", "site"))


def run(fields, n, storage, kernel, steps, every, d_i, tau, nshell, device=None):
    """One run from ``fields``; returns t, E_u(t), E_B(t), J2(t) and the final spectra."""
    u, B = fields
    g = every if every % 2 == 0 else 0
    sim = Flame(n, n, n, tau, tau, d_i, storage=storage, kernel=kernel, graph_steps=g, device=device)
    try:
        sim.init(None, u, B)
        t, eu, eb, j2 = [], [], [], []
        done = 0
        while True:
            s = sim.reduce()
            t.append(done)
            eu.append(s["E_u"])
            eb.append(s["E_B"])
            j2.append(s["J2"])
            if done >= steps or s["status"] != 0:
                break
            k = min(every, steps - done)
            sim.step(k)
            done += k
        Eu, Eb = sim.spectra(nshell)
    finally:
        sim.close()
    return dict(t=np.array(t), Eu_t=np.array(eu), Eb_t=np.array(eb), J2_t=np.array(j2), Eu=Eu, Eb=Eb,
                finished=done >= steps)


def _rel(a, b):
    return (a - b) / np.where(b != 0, np.abs(b), 1.0)


def compare(runs, ref):
    """Signed relative differences of one run against a reference run."""
    E, E0 = runs["Eu_t"] + runs["Eb_t"], ref["Eu_t"] + ref["Eb_t"]
    m = min(len(E), len(E0))
    dt = np.diff(ref["t"][:m])
    rate = -(E[2:m] - E[:m - 2]) / (dt[1:] + dt[:-1])
    rate0 = -(E0[2:m] - E0[:m - 2]) / (dt[1:] + dt[:-1])
    return dict(shell_Eu=_rel(runs["Eu"], ref["Eu"]), shell_Eb=_rel(runs["Eb"], ref["Eb"]),
                E_t=_rel(E[:m], E0[:m]), rate_t=_rel(rate, rate0))


def study(n=256, steps=500, nseeds=3, every=10, d_i=None, tau=0.51, configs=CONFIGS, device=None):
    d_i = 0.05 * n if d_i is None else d_i
    nshell = n // 2 + 1
    per = {f"{s}/{k}": [] for s, k in configs}
    t = None
    for r in range(nseeds):
        seeds = (3 + 10 * r, 4 + 10 * r)
        fields = inputs.turbulence((n, n, n), seeds[0], seeds[1], 0.05, 0.05, shells=(1, 4))
        runs = {f"{s}/{k}": run(fields, n, s, k, steps, every, d_i, tau, nshell, device) for s, k in configs}
        ref = runs["fp32/site"]
        t = ref["t"]
        for name, rr in runs.items():
            if name == "fp32/site":
                continue
            c = compare(rr, ref)
            c["vs"] = "fp32/site"
            c["finished"] = rr["finished"]
            per[name].append(c)
        if "fp16/site" in runs and "fp16/auto" in runs:
            c = compare(runs["fp16/site"], runs["fp16/auto"])
            c["vs"] = "fp16/auto"
            c["finished"] = runs["fp16/site"]["finished"]
            per.setdefault("control: fp16/site vs fp16/auto", []).append(c)
        per.setdefault("_ref_spectra", []).append(dict(Eu=ref["Eu"], Eb=ref["Eb"], E_t=ref["Eu_t"] + ref["Eb_t"]))
    shells = [s for s in (1, 2, 4, 8, 16, 32, 64, 128) if s < nshell]
    out = dict(n=n, steps=steps, seeds=nseeds, every=every, d_i=d_i, tau=tau, shells=shells, results={})
    for name, lst in per.items():
        if not lst or name == "_ref_spectra" or name == "fp32/site":
            continue
        res = dict(vs=lst[0]["vs"], finished=all(c["finished"] for c in lst))
        for key in ("shell_Eu", "shell_Eb"):
            a = np.array([c[key] for c in lst])
            res[key + "_mean"] = {str(s): float(a[:, s].mean()) for s in shells}
            res[key + "_std"] = {str(s): float(a[:, s].std(ddof=1)) if len(lst) > 1 else 0.0 for s in shells}
        for key in ("E_t", "rate_t"):
            a = np.array([c[key] for c in lst])
            idx = [i for i in range(a.shape[1]) if i % max(1, a.shape[1] // 10) == 0] + [a.shape[1] - 1]
            res[key + "_mean"] = {str(int(t[i + (1 if key == "rate_t" else 0)])): float(a[:, i].mean()) for i in idx}
            res[key + "_std"] = {str(int(t[i + (1 if key == "rate_t" else 0)])): float(a[:, i].std(ddof=1))
                                 if len(lst) > 1 else 0.0 for i in idx}
        out["results"][name] = res
    refs = per["_ref_spectra"]
    out["fp32_spectra_mean"] = {"Eu": {str(s): float(np.mean([r["Eu"][s] for r in refs])) for s in shells},
                                "Eb": {str(s): float(np.mean([r["Eb"][s] for r in refs])) for s in shells}}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--seeds", type=int, default=3)
    ap.add_argument("--every", type=int, default=10)
    ap.add_argument("--d-i", type=float, default=None)
    ap.add_argument("--tau", type=float, default=0.51)
    ap.add_argument("--configs", default=",".join(f"{s}/{k}" for s, k in CONFIGS))
    a = ap.parse_args(argv)
    configs = tuple(tuple(c.split("/")) for c in a.configs.split(","))
    print(json.dumps(study(a.n, a.steps, a.seeds, a.every, a.d_i, a.tau, configs)), flush=True)


if __name__ == "__main__":
    main()
