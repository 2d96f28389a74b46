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
    python -m paper_2212_11024_gb300.precision --experiment seeding --steps 500
    python -m paper_2212_11024_gb300.precision --experiment fork --steps 500
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


# Two experiments that separate the causes.  Both move a state between
# storage types by converting its stored values: every storage type holds the
# same quantity (a population's deviation from the rest equilibrium of
# (rho0, B_ref), divided by its lattice weight), so an FP32 state rounded to
# FP16 (round to nearest even) is exactly the FP16 state of the same
# populations, and an FP16 state widened to FP32 is exact.

def _convert(blob, src, dst):
    import torch
    dt = {"fp32": torch.float32, "fp16": torch.float16, "bf16": torch.bfloat16}
    return blob.view(dt[src]).to(dt[dst]).view(torch.uint8).contiguous()


def _spectra_after(n, storage, kernel, d_i, tau, blob, step, parity, steps, nshell, device=None):
    sim = Flame(n, n, n, tau, tau, d_i, storage=storage, kernel=kernel, device=device)
    try:
        sim.set_state(blob, step, parity)
        sim.step(steps)
        s = sim.reduce()
        Eu, Eb = sim.spectra(nshell)
    finally:
        sim.close()
    return Eu, Eb, s["E_u"] + s["E_B"]


def seeding_experiment(n=256, steps=500, nseeds=3, d_i=None, tau=0.51, device=None):
    """FP32 storage started from the FP16-rounded initial state: if it
    follows the FP16 run rather than the FP32 run, the difference is set by
    the rounding of the initial state (the seed of the small scales), not by
    the rounding of every step."""
    d_i = 0.05 * n if d_i is None else d_i
    nshell = n // 2 + 1
    shells = [s for s in (1, 2, 4, 8, 16, 32, 64, 128) if s < nshell]
    rows = {"fp32 from fp16 start vs fp32": [], "fp32 from fp16 start vs fp16": [], "fp16 vs fp32": []}
    for r in range(nseeds):
        u, B = inputs.turbulence((n, n, n), 3 + 10 * r, 4 + 10 * r, 0.05, 0.05, shells=(1, 4))
        res = {}
        for st in ("fp32", "fp16"):
            sim = Flame(n, n, n, tau, tau, d_i, storage=st, kernel="site" if st == "fp32" else "auto", device=device)
            sim.init(None, u, B)
            blob, step, par = sim.get_state()
            sim.close()
            res[st] = _spectra_after(n, st, "site" if st == "fp32" else "auto", d_i, tau, blob, step, par, steps,
                                     nshell, device)
            if st == "fp16":
                res["fp32<-fp16"] = _spectra_after(n, "fp32", "site", d_i, tau, _convert(blob, "fp16", "fp32"), step,
                                                   par, steps, nshell, device)
        for name, a, b in (("fp32 from fp16 start vs fp32", "fp32<-fp16", "fp32"),
                           ("fp32 from fp16 start vs fp16", "fp32<-fp16", "fp16"), ("fp16 vs fp32", "fp16", "fp32")):
            rows[name].append(dict(Eu=_rel(res[a][0], res[b][0]), Eb=_rel(res[a][1], res[b][1]),
                                   E=(res[a][2] - res[b][2]) / res[b][2]))
    return _summarise(rows, shells, dict(experiment="seeding", n=n, steps=steps, seeds=nseeds, d_i=d_i, tau=tau))


def fork_experiment(n=256, steps_before=500, steps_after=500, nseeds=3, d_i=None, tau=0.51, device=None):
    """Developed turbulence: an FP32 run of steps_before steps is forked into
    FP32, FP16 and BF16 (rounded state, row kernel) and an FP16 control (one-
    site kernel), which all run steps_after more steps.  Differences that
    stay within the control's are the flow's chaos; a systematic offset is a
    bias of the storage itself."""
    d_i = 0.05 * n if d_i is None else d_i
    nshell = n // 2 + 1
    shells = [s for s in (1, 2, 4, 8, 16, 32, 64, 128) if s < nshell]
    rows = {"fp16 vs fp32": [], "bf16 vs fp32": [], "control: fp16/site vs fp16/auto": []}
    for r in range(nseeds):
        u, B = inputs.turbulence((n, n, n), 3 + 10 * r, 4 + 10 * r, 0.05, 0.05, shells=(1, 4))
        sim = Flame(n, n, n, tau, tau, d_i, storage="fp32", kernel="site", device=device)
        sim.init(None, u, B)
        sim.step(steps_before)
        blob, step, par = sim.get_state()
        sim.close()
        res = {"fp32": _spectra_after(n, "fp32", "site", d_i, tau, blob, step, par, steps_after, nshell, device)}
        for st, kern in (("fp16", "auto"), ("bf16", "auto"), ("fp16", "site")):
            res[f"{st}/{kern}"] = _spectra_after(n, st, kern, d_i, tau, _convert(blob, "fp32", st), step, par,
                                                 steps_after, nshell, device)
        for name, a, b in (("fp16 vs fp32", "fp16/auto", "fp32"), ("bf16 vs fp32", "bf16/auto", "fp32"),
                           ("control: fp16/site vs fp16/auto", "fp16/site", "fp16/auto")):
            rows[name].append(dict(Eu=_rel(res[a][0], res[b][0]), Eb=_rel(res[a][1], res[b][1]),
                                   E=(res[a][2] - res[b][2]) / res[b][2]))
    return _summarise(rows, shells, dict(experiment="fork", n=n, steps_before=steps_before, steps_after=steps_after,
                                         seeds=nseeds, d_i=d_i, tau=tau))


def _summarise(rows, shells, head):
    out = dict(head, shells=shells, results={})
    for name, lst in rows.items():
        res = {}
        for key in ("Eu", "Eb"):
            a = np.array([c[key] for c in lst])
            res["shell_" + key + "_mean"] = {str(s): float(a[:, s].mean()) for s in shells}
            res["shell_" + key + "_std"] = {str(s): float(a[:, s].std(ddof=1)) if len(lst) > 1 else 0.0
                                            for s in shells}
        e = np.array([c["E"] for c in lst])
        res["E_end_mean"], res["E_end_std"] = float(e.mean()), float(e.std(ddof=1)) if len(lst) > 1 else 0.0
        out["results"][name] = res
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
    ap.add_argument("--experiment", default="study", choices=["study", "seeding", "fork"],
                    help="study: every storage from the same start; seeding: FP32 from the FP16-rounded start; "
                         "fork: storages forked from a developed FP32 state after --steps steps")
    a = ap.parse_args(argv)
    if a.experiment == "seeding":
        print(json.dumps(seeding_experiment(a.n, a.steps, a.seeds, a.d_i, a.tau)), flush=True)
        return
    if a.experiment == "fork":
        print(json.dumps(fork_experiment(a.n, a.steps, a.steps, a.seeds, a.d_i, a.tau)), flush=True)
        return
    configs = tuple(tuple(c.split("/")) for c in a.configs.split(","))
    print(json.dumps(study(a.n, a.steps, a.seeds, a.every, a.d_i, a.tau, configs)), flush=True)


if __name__ == "__main__":
    main()
