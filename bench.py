#!/usr/bin/env python3
"""Throughput of the fused FLAME Hall-MHD lattice-Boltzmann step on GB300.

Workload (default): 256^3 decaying Hall-MHD turbulence -- seeded random-phase
solenoidal u and B with energy in shells 1..4 (u_rms = b_rms = 0.05, seeds 3
and 4), rho = 1, tau_nu = tau_eta = 0.51, d_i = 0.05 * 256 = 12.8.  The
headline is FP16 deviation storage with FP32 collision; FP32 and BF16
storage are timed in the same run, FP16 / BF16 once more with the one-site
kernel forced ("fp16/site") for comparison with the row kernel, and FP16
with the unstaged pair kernel ("fp16/pair", the one other row lengths use).  A
step is one launch of the fused collide-and-stream kernel over all 256^3
sites: the row kernel (TMA-staged x rows, two sites per thread in packed
FP32 pairs) for 16-bit storage, the one-site kernel for FP32.

Metric: MLUPS (million lattice-site updates per second) and the fraction of
the measured HBM bandwidth reached by the step kernel, with the per-field
and per-shell error of the reduced-precision runs against the FP32 run.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--n 256] [--impl flame|reference]

Under torchrun (N > 1) every rank runs an independent replica of the
workload on its own GPU (weak scaling, no data-path collective); the value
is the sum of all ranks' site updates over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS and % HBM roofline at 256^3 (FP32 vs FP16-storage) at stated L2 error"
BYTES_PER_SITE = {"fp32": 48 * 4 * 2, "fp16": 48 * 2 * 2, "bf16": 48 * 2 * 2}  # AA in place: read + write 48
FALLBACK_HBM_GBS = 6800.0
# Steps per CUDA-graph replay of flame_step (flame_params.graph_steps): the
# library's fast path, one graph launch per GRAPH_STEPS kernel launches.
GRAPH_STEPS = 20
NOMINAL_HBM_GBS = 8000.0
L2_BYTES = 129 * 2 ** 20


def workload(n):
    return dict(tau_nu=0.51, tau_eta=0.51, d_i=0.05 * n, rms=0.05, shells=(1, 4), seed_u=3, seed_b=4)


def workload_name(n, storage):
    w = workload(n)
    return (f"{n}^3 decaying Hall-MHD turbulence: seeded random-phase solenoidal u, B in shells 1-4, "
            f"u_rms=b_rms={w['rms']}, rho=1, tau_nu=tau_eta={w['tau_nu']}, d_i={w['d_i']:g}; "
            f"{storage.upper()} deviation storage, FP32 collision")


# --------------------------------------------------------------------------- helpers
def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            v = float(json.load(fh)["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback (no MEASURED_PEAKS.json)"


def kernel_source_hash():
    """SHA-256 (first 16 hex digits) of the step kernels' sources with comments
    and whitespace removed, so that only a change of the code itself
    invalidates a recorded ncu traffic figure."""
    h = hashlib.sha256()
    for f in ("step.cu", "step_row.cu", "step_row.cuh", "lattice.cuh", "aa.cuh"):
        with open(os.path.join(ROOT, "paper_2212_11024_gb300", "csrc", f)) as fh:
            txt = fh.read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", "", txt)
        h.update(re.sub(r"\s+", "", txt).encode())
    return h.hexdigest()[:16]


def parse_variant(spec):
    """"fp16" -> ("fp16", "auto"); "fp16/site" -> ("fp16", "site")."""
    st, _, kern = spec.partition("/")
    return st, (kern or "auto")


def kernel_name(storage, kernel, n):
    """The step kernel flame_step launches for this storage at n^3 (the
    library's own choice, flame_step_kernel)."""
    from paper_2212_11024_gb300 import flame as F
    p = F.make_params(n, n, n, 0.51, 0.51, 0.05 * n, storage, kernel=kernel)
    return {"site": f"step_kernel<{storage}> (one site per thread)",
            "rows": f"step_row_kernel<{storage}> (staged x rows, packed FP32 pairs)",
            "half_rows": f"step_row_kernel<{storage}> (half x rows staged by bulk copies, packed FP32 pairs)",
            "pairs": f"step_pair_kernel<{storage}> (unstaged site pairs, packed FP32 pairs)"}[F.step_kernel(p)]


def recorded_traffic(storage):
    """DRAM bytes per launch of the step kernel from the committed ncu summary
    of that kernel (the row kernel for FP16/BF16, the one-site kernel for
    FP32), if it was taken on the current kernel source (else None)."""
    name = "step_row_kernel_256.md" if storage in ("fp16", "bf16") else "step_kernel_256.md"
    path = os.path.join(ROOT, "profiles", name)
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    if not m or m.group(1) != kernel_source_hash():
        return None
    m = re.search(rf"traffic_bytes_per_launch_{storage}:\s*([0-9.eE+]+)", txt)
    return float(m.group(1)) if m else None


class ClockSampler:
    """nvidia-smi clock / throttle sampling in a background thread."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.windows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), [x.strip() for x in line.split(",")]))

    def window(self, t0, t1):
        self.windows.append((t0, t1))

    def median_in(self, t0, t1):
        """Median SM clock (MHz) of the samples taken between t0 and t1."""
        sm = [float(s[1]) for t, s in self.samples if t0 <= t <= t1 and s[1].replace(".", "", 1).isdigit()]
        return statistics.median(sm) if sm else None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        inside = [s for t, s in self.samples if any(a <= t <= b for a, b in self.windows)]
        use = inside if inside else [s for _, s in self.samples]
        if not use:
            return None
        sm = [float(s[1]) for s in use if s[1].replace(".", "", 1).isdigit()]
        mx = [float(s[2]) for s in use if s[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in use for i in range(4) if len(s) > 5 + i and s[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(use), "samples_in_timed_region": len(inside)}


# --------------------------------------------------------------------------- oracle timing
def host_cores():
    """The host cores this process may run on (a launcher such as torchrun
    sets OMP_NUM_THREADS=1 per rank; the oracle legs run on rank 0 alone and
    use all of them)."""
    return len(os.sched_getaffinity(0))


def oracle_mlups(n, steps, threads=0):
    """Time `steps` oracle steps (literal 27x27 mode, FP64, OpenMP) on an n^3
    instance of the workload recipe; returns (MLUPS, seconds, cores).
    threads = 0: all host cores."""
    import numpy as np

    import oracle as O
    from paper_2212_11024_gb300 import inputs

    w = workload(n)
    cores = O.threads(threads if threads > 0 else host_cores())
    u, B = inputs.turbulence((n, n, n), w["seed_u"], w["seed_b"], w["rms"], w["rms"], shells=w["shells"])
    p = O.Params(n, n, n, w["tau_nu"], w["tau_eta"], w["d_i"])
    pop = O.init(p, None, u, B)
    del u, B
    scratch = np.empty_like(pop)
    t0 = time.perf_counter()
    O.step(p, pop, steps, literal=True, scratch=scratch)
    dt = time.perf_counter() - t0
    return n ** 3 * steps / dt / 1e6, dt, cores


# Seconds of oracle work the reference arm's warm-up and timed steps may take
# together: the workload at its full size when that is projected to fit in
# REF_FULL_S, else an n^3 instance of the same recipe sized to REF_SAMPLE_S.
REF_FULL_S, REF_SAMPLE_S = 200.0, 150.0


def run_reference(args):
    """The oracle as it stands, on the host cores, in the arm's metric, unit
    and workload.  Each timed step is one oracle step of the workload at its
    full size when the whole run is projected to take at most REF_FULL_S
    seconds (the rate taken on a 64^3 instance, which is below the full-size
    rate), else of an n^3 instance of the same recipe sized to REF_SAMPLE_S
    seconds."""
    import oracle as O

    O.build()
    rate, _, _ = oracle_mlups(min(args.n, 64), 1)  # calibration
    nsteps = max(1, args.steps + args.warmup)
    if nsteps * args.n ** 3 / (rate * 1e6) <= REF_FULL_S:
        n = args.n
    else:
        n = int((REF_SAMPLE_S / nsteps * rate * 1e6) ** (1.0 / 3.0))
        n = max(10, min(args.n, n - n % 2))
    import numpy as np

    from paper_2212_11024_gb300 import inputs

    w = workload(n)
    cores = O.threads(host_cores())
    u, B = inputs.turbulence((n, n, n), w["seed_u"], w["seed_b"], w["rms"], w["rms"], shells=w["shells"])
    p = O.Params(n, n, n, w["tau_nu"], w["tau_eta"], w["d_i"])
    pop = O.init(p, None, u, B)
    del u, B
    scratch = np.empty_like(pop)
    for _ in range(args.warmup):
        O.step(p, pop, 1, literal=True, scratch=scratch)
    t0 = time.perf_counter()
    O.step(p, pop, args.steps, literal=True, scratch=scratch)
    dt = time.perf_counter() - t0
    val = n ** 3 * args.steps / dt / 1e6
    what = (f"the {n}^3 workload itself" if n == args.n else
            f"{n}^3 periodic instance of the workload recipe (d_i = 0.05 n)")
    sample = f"{what}, one FP64 oracle step (literal 27x27 central-moment inversion) per timed step"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.n, "fp16"), "n": args.n, "shape": [args.n] * 3,
                       "sample_n": n, "compute": "fp64 (the oracle: no 16-bit storage)",
                       "parallelism": "host cores (OpenMP)"},
            "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- accuracy
ACC_STEPS = 50  # steps before the 256^3 fields are compared (chaos e-folds in ~20-25 steps)
ACC_STEPS_LONG = 500  # the 256^3 configuration's run length: fields have decorrelated, spectra compare
ORACLE_N, ORACLE_STEPS = 64, 100


def field_errors(got, ref, n, steps):
    """Relative L2 of u and B - <B> and the largest per-shell spectral error (shells 1..n/4)."""
    import numpy as np
    import torch

    gu, gb, gEu, gEb = got
    ru, rb, rEu, rEb = ref
    # shells 1..n/4 whose reference energy lies above 1e-6 of the peak: below
    # that the reduced-precision rounding noise floor dominates the shell
    shells = [k for k in range(1, n // 4 + 1)]
    res_u = [k for k in shells if rEu[k] >= 1e-6 * rEu.max()]
    res_b = [k for k in shells if rEb[k] >= 1e-6 * rEb.max()]
    sample = [k for k in (1, 2, 4, 8, 16, 32, 64) if k <= n // 4]
    rbm = rb - rb.reshape(3, -1).mean(dim=1)[:, None, None, None]
    gbm = gb - gb.reshape(3, -1).mean(dim=1)[:, None, None, None]
    return {"steps": steps, "n": n,
            "rel_l2_u": float(torch.linalg.vector_norm(gu - ru) / torch.linalg.vector_norm(ru)),
            "rel_l2_B": float(torch.linalg.vector_norm(gbm - rbm) / torch.linalg.vector_norm(rbm)),
            "max_shell_rel_err_Eu": float(np.max(np.abs(gEu[res_u] - rEu[res_u]) / rEu[res_u])),
            "max_shell_rel_err_Eb": float(np.max(np.abs(gEb[res_b] - rEb[res_b]) / rEb[res_b])),
            "resolved_shells_Eu": [min(res_u), max(res_u)], "resolved_shells_Eb": [min(res_b), max(res_b)],
            "shell_rel_err_Eu": {str(k): float(abs(gEu[k] - rEu[k]) / rEu[k]) for k in sample},
            "shell_rel_err_Eb": {str(k): float(abs(gEb[k] - rEb[k]) / rEb[k]) for k in sample}}


def oracle_restriction_errors(storages, dev):
    """The 64^3 instance of the workload recipe (same seeds, d_i = 0.05 * 64),
    100 steps: each storage variant on the GPU against the FP64 oracle."""
    import torch

    import oracle as O
    from oracle import spectra as S
    from paper_2212_11024_gb300 import Flame, inputs

    n, steps = ORACLE_N, ORACLE_STEPS
    w = workload(n)
    u, B = inputs.turbulence((n, n, n), w["seed_u"], w["seed_b"], w["rms"], w["rms"], shells=w["shells"])
    O.build()
    O.threads(host_cores())
    p = O.Params(n, n, n, w["tau_nu"], w["tau_eta"], w["d_i"])
    pop = O.init(p, None, u, B)
    O.step(p, pop, steps, literal=True)
    mo = O.moments(p, pop)
    bo = mo["B"] - mo["B"].reshape(3, -1).mean(1)[:, None, None, None]
    ref = (torch.from_numpy(mo["u"]), torch.from_numpy(mo["B"]), S.shell_spectrum(mo["u"], n // 2 + 1),
           S.shell_spectrum(bo, n // 2 + 1))
    out = {}
    for st in storages:
        sim = Flame(n, n, n, w["tau_nu"], w["tau_eta"], w["d_i"], storage=st, device=dev)
        sim.init(None, u, B)
        sim.step(steps)
        m = sim.moments()
        Eu, Eb = sim.spectra(n // 2 + 1)
        got = (m["u"].cpu(), m["B"].cpu(), Eu, Eb)
        errs = field_errors(got, ref, n, steps)
        errs["rel_l2_J"] = float(torch.linalg.vector_norm(m["J"].cpu() - torch.from_numpy(mo["J"])) /
                                 torch.linalg.vector_norm(torch.from_numpy(mo["J"])))
        errs["reference"] = "FP64 oracle (literal 27x27 collision), same 64^3 fields"
        out[st] = errs
        sim.close()
    return out


# --------------------------------------------------------------------------- replicas (N > 1)
# The decaying-turbulence runs of the paper's Sec. 5 setting that the
# benchmark records besides its headline (each from seeded random-phase
# solenoidal fields in shells 1..4, flat E(k), rho = 1, tau = 0.51):
# 128^3 FP32 storage, rms 0.05, d_i in {0, 0.05 * 128}, 1000 steps; and
# 512^3 FP16 storage, rms 0.04, d_i in {0, 0.02, 0.05, 0.1} * 512, 2000 steps.
TURBULENCE_RUNS = (
    dict(n=128, storage="fp32", rms=0.05, d_i=(0.0, 6.4), steps=1000, seeds=(1, 2)),
    dict(n=512, storage="fp16", rms=0.04, d_i=(0.0, 10.24, 25.6, 51.2), steps=2000, seeds=(1, 2)),
)


def turbulence_runs(dev, every=100):
    """Each run of TURBULENCE_RUNS: steps completed, where it went non-finite,
    step-kernel GLUPS (CUDA events around the step chunks only), the energy
    ratio E(end)/E(0) and the slope of E_B(k) over k = 8..32 at the end."""
    import numpy as np
    import torch

    from paper_2212_11024_gb300 import inputs, turbulence

    out = []
    for cfg in TURBULENCE_RUNS:
        n = cfg["n"]
        u, B = inputs.turbulence((n, n, n), *cfg["seeds"], cfg["rms"], cfg["rms"], shells=(1, 4))
        fields = (u.astype(np.float32), B.astype(np.float32))
        del u, B
        for di in cfg["d_i"]:
            r = turbulence.decay(n, di, cfg["steps"], spectra_every=every, storage=cfg["storage"], rms_u=cfg["rms"],
                                 rms_b=cfg["rms"], seeds=cfg["seeds"], graph_steps=20, device=dev, fields=fields)
            E = [s["E_u"] + s["E_B"] for s in r["scalars"]]
            k = np.arange(8, 33)
            eb = r["Eb"][-1][8:33]
            slope = float(np.polyfit(np.log(k), np.log(eb), 1)[0]) if np.all(eb > 0) else None
            out.append(dict(n=n, storage=cfg["storage"], rms=cfg["rms"], d_i=di, steps=cfg["steps"],
                            steps_done=int(r["steps"]), first_nonfinite=r["first_nonfinite"],
                            glups=r["mlups"] / 1e3, E_end_over_E0=float(E[-1] / E[0]),
                            Eb_slope_k8_32=slope, spectra_every=every))
        del fields
        torch.cuda.empty_cache()
    return out


def reduce_max(x, dist=None, device=None):
    """The largest x over the ranks of the default process group (x itself
    without one): every rank gets the slowest rank's time."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_mlups(world, sites, steps, seconds):
    """Whole-job throughput of `world` independent replicas, each updating
    `sites` sites `steps` times, over the slowest replica's time."""
    return world * sites * steps / seconds / 1e6


# --------------------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    # --lattice: the same, for launches under torchrun, whose own parser takes
    # "--n" for an ambiguous prefix of its options
    ap.add_argument("--n", "--lattice", dest="n", type=int, default=256, help="lattice edge (n^3)")
    ap.add_argument("--shape", default=None,
                    help="NX,NY,NZ: a non-cubic lattice of the same recipe (d_i = 0.05 NX), e.g. a smaller "
                         "case of the 256-site-row kernel for profiling; default n^3")
    ap.add_argument("--impl", default="flame", choices=["flame", "reference"])
    ap.add_argument("--storage", default="fp16,fp32,bf16,fp16/site,bf16/site,fp16/pair",
                    help="first entry is the headline; '/site' forces the one-site kernel, '/pair' the "
                         "unstaged pair kernel")
    ap.add_argument("--no-turbulence-runs", action="store_true",
                    help="skip the 128^3 and 512^3 decaying-turbulence runs recorded besides the headline")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the host-oracle legs (CPU baseline and the 64^3 oracle accuracy check)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    import numpy as np
    import torch

    from paper_2212_11024_gb300 import Flame, FlameError, build as B, inputs
    from paper_2212_11024_gb300 import flame as F

    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def max_over_ranks(x):
        return reduce_max(x, dist, dev)

    n = args.n
    nx, ny, nz = (int(v) for v in args.shape.split(",")) if args.shape else (n, n, n)
    n3 = nx * ny * nz
    nmin = min(nx, ny, nz)
    nshell = max(nx, ny, nz) // 2 + 1
    w = workload(nx)
    u_h, B_h = inputs.turbulence((nz, ny, nx), w["seed_u"], w["seed_b"], w["rms"], w["rms"], shells=w["shells"])
    u_d = torch.from_numpy(u_h).to(dev)
    B_d = torch.from_numpy(B_h).to(dev)
    storages = [s.strip() for s in args.storage.split(",") if s.strip()]
    head = storages[0]
    peak, peak_src = hbm_peak()
    clocks = ClockSampler(local)
    clocks.start()
    stream = torch.cuda.current_stream(dev)
    variants = {}
    for spec in storages:
        st, kern = parse_variant(spec)
        sim = Flame(nx, ny, nz, w["tau_nu"], w["tau_eta"], w["d_i"], storage=st, device=dev, kernel=kern,
                    graph_steps=GRAPH_STEPS)
        sim.init(None, u_d, B_d)
        sim.step(args.warmup)
        sim.step(GRAPH_STEPS)  # captures the graph of the timed steps' parity (untimed)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_wall0 = time.time()
        e0.record(stream)
        sim.step(args.steps)
        e1.record(stream)
        e1.synchronize()
        t_wall1 = time.time()
        barrier()
        clocks.window(t_wall0, t_wall1)
        ms = e0.elapsed_time(e1)
        ms_max = max_over_ranks(ms)
        status = "ok"
        try:
            sim.sync()
        except FlameError as ex:
            status = f"nonfinite ({ex.status})"
        sites = n3
        mlups = replica_mlups(world, sites, args.steps, ms_max * 1e-3)
        per_launch_s = ms / args.steps * 1e-3
        achieved = BYTES_PER_SITE[st] * sites / per_launch_s / 1e9
        variants[spec] = {"mlups": mlups, "ms_per_step": ms_max / args.steps, "achieved_gbs": achieved,
                          "frac_of_measured_hbm": achieved / peak, "frac_of_nominal_8tbs": achieved / NOMINAL_HBM_GBS,
                          "algorithmic_bytes_per_site": BYTES_PER_SITE[st],
                          "state_gb": 48 * sites * (4 if st == "fp32" else 2) / 1e9,
                          "kernel": kernel_name(st, kern, nx), "status": status}
        sim.close()
        del sim
        torch.cuda.empty_cache()

    # The hand-written adjoint step (flame_step_adjoint, the differentiation
    # path) on the same workload, outside the headline: 20 calls after 3.
    adjoint = {}
    if nx == ny == nz:
        from paper_2212_11024_gb300.throughput import adjoint_throughput
        for st in ("fp32", "fp16"):
            r = adjoint_throughput(nx, st, steps=20, warmup=3, d_i=w["d_i"], tau=w["tau_nu"], fields=(u_d, B_d),
                                   device=dev)
            adjoint[st] = {"glups": r["glups"], "ms_per_call": r["ms_per_step"], "bytes_per_update": r["bytes_per_update"],
                           "frac_of_measured_hbm": r["glups"] * r["bytes_per_update"] / peak}
        torch.cuda.empty_cache()

    # Accuracy at the stated step counts (outside the timed region).  The
    # 256^3 recipe is chaotic: differences e-fold every ~20-25 steps, so
    # fields are compared early, spectra by shell.
    acc_storages = [spec for spec in storages if "/" not in spec]
    accuracy = {st: {} for st in acc_storages}
    finals, longs = {}, {}
    # control for the long comparison: FP16 storage with the one-site kernel,
    # whose FP32 collision rounds in another order than the row kernel's
    control = "fp16/site" if "fp16" in acc_storages else None
    for st in acc_storages + ([control] if control else []):
        st_storage, st_kernel = parse_variant(st)
        sim = Flame(nx, ny, nz, w["tau_nu"], w["tau_eta"], w["d_i"], storage=st_storage, device=dev, kernel=st_kernel)
        sim.init(None, u_d, B_d)
        sim.step(ACC_STEPS)
        m = sim.moments(out={"u": torch.empty((3, nz, ny, nx), dtype=torch.float64, device=dev),
                             "B": torch.empty((3, nz, ny, nx), dtype=torch.float64, device=dev)})
        Eu, Eb = sim.spectra(nshell)
        finals[st] = (m["u"], m["B"], Eu, Eb)
        sim.step(ACC_STEPS_LONG - ACC_STEPS)
        try:
            sim.sync()
            m = sim.moments(out={"u": torch.empty((3, nz, ny, nx), dtype=torch.float64, device=dev),
                                 "B": torch.empty((3, nz, ny, nx), dtype=torch.float64, device=dev)})
            Eu, Eb = sim.spectra(nshell)
            longs[st] = (m["u"], m["B"], Eu, Eb)
        except FlameError:
            longs[st] = None  # non-finite by then: reported as such
        sim.close()
        del sim
    if "fp32" in finals:
        for st in acc_storages:
            if st != "fp32":
                accuracy[st]["vs_fp32_256"] = field_errors(finals[st], finals["fp32"], nmin, ACC_STEPS)
                if longs.get(st) is not None and longs.get("fp32") is not None:
                    accuracy[st]["vs_fp32_256_long"] = field_errors(longs[st], longs["fp32"], nmin, ACC_STEPS_LONG)
                else:
                    accuracy[st]["vs_fp32_256_long"] = {"steps": ACC_STEPS_LONG, "nonfinite": True}
    if control and longs.get("fp16") is not None and longs.get(control) is not None:
        accuracy["fp16"]["rounding_order_control_256_long"] = dict(
            field_errors(longs["fp16"], longs[control], nmin, ACC_STEPS_LONG),
            reference="FP16 storage, one-site kernel: the same step with the FP32 operations in another order")
    finals.clear()
    longs.clear()
    torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers: flame_init_f32_host
    # (the FP32 initial fields from page-locked host memory, copied in chunks
    # of planes overlapped with the initialisation), K steps, and
    # flame_moments_f32_host (u, B, J in FP32 to page-locked host memory,
    # copied out chunk by chunk as they are written, with flame_reduce's FP64
    # scalars computed meanwhile).  The context (its state and the CUDA graph
    # of the first steps) is set up before the timed region, and the job runs
    # once untimed before the timed run.
    del u_d, B_d
    torch.cuda.empty_cache()
    # the initial fields in one page-locked array (u, B), the results in another (u, B, J)
    in_h = torch.from_numpy(np.concatenate([u_h, B_h]).astype(np.float32)).pin_memory()
    pin_u, pin_B = in_h[0:3], in_h[3:6]
    out_h = torch.empty((9, nz, ny, nx), dtype=torch.float32).pin_memory()
    outs = {"u": out_h[0:3], "B": out_h[3:6], "J": out_h[6:9]}
    sim = Flame(nx, ny, nz, w["tau_nu"], w["tau_eta"], w["d_i"], storage=parse_variant(head)[0], device=dev,
                kernel=parse_variant(head)[1], graph_steps=GRAPH_STEPS)

    def mark():  # phase boundaries (each call below returns with its work done)
        torch.cuda.synchronize(dev)
        marks.append(time.perf_counter())

    def job():
        sim.init_host(None, pin_u, pin_B)
        mark()
        sim.step(args.steps)
        mark()
        _, r = sim.moments_host(out=outs, scalars=True)
        mark()
        return r

    # one untimed run of the whole job first (the warm-up of the end-to-end
    # path: first touches of the pinned buffers, the workspaces, the copy stream)
    marks = [time.perf_counter()]
    job()
    barrier()
    t_wall0 = time.time()
    t0 = time.perf_counter()
    marks = [t0]
    scal = job()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    clocks.window(t_wall0, time.time())
    e2e_sm = clocks.median_in(t_wall0, time.time())
    barrier()
    sim.close()
    h2d = 2 * 3 * n3 * 4
    d2h = 9 * n3 * 4 + 14 * 8
    # kernels: one initialisation and one moments launch per chunk of planes,
    # the steps, the reduction's two
    chunks = min(F.IO_CHUNKS, nz)
    e2e = {"value": replica_mlups(world, n3, args.steps, e2e_s), "unit": "MLUPS",
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
           "job": "flame_init_f32_host (FP32 u, B from one pinned host array), K x flame_step, "
                  "flame_moments_f32_host (u, B, J FP32 into one pinned host array, with the flame_reduce "
                  "scalars)", "seconds": e2e_s,
           "gpu_launches": chunks + args.steps + chunks + 2, "io_chunks": chunks,
           "final_E_u": scal["E_u"], "final_E_B": scal["E_B"],
           "phases_ms": {k: (marks[i + 1] - marks[i]) * 1e3 for i, k in
                         enumerate(("h2d overlapped with init", "steps", "moments overlapped with d2h, reduce"))},
           "sm_mhz": e2e_sm}
    clk = clocks.stop()

    turb = None
    if world == 1 and not args.no_turbulence_runs:
        turb = turbulence_runs(dev)

    # The host-oracle legs come last: their OpenMP threads keep the host cores
    # busy for a while after they finish, which would slow the host side of
    # the end-to-end job.
    if rank == 0 and not args.no_cpu_baseline:
        for st, errs in oracle_restriction_errors(acc_storages, dev).items():
            accuracy[st]["vs_oracle_64"] = errs

    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle as O

        O.build()
        # two steps (both AA parities' worth of work): ~13 s on 16 Grace cores at 256^3
        val, secs, cores = oracle_mlups(n, 2)
        cpu = {"value": val, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"two FP64 oracle steps (literal 27x27 central-moment inversion) of the {n}^3 workload, "
                         f"{secs:.1f} s on {cores} threads"}

    hv = variants[head]
    head_st, head_kern = parse_variant(head)
    traffic = recorded_traffic(head_st) if head_kern == "auto" else None
    line = {
        "metric": METRIC, "value": hv["mlups"], "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": hv["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(n, head_st) if not args.shape else
                   f"{nx}x{ny}x{nz} lattice of the same recipe (d_i = {w['d_i']:g}); {head_st.upper()} storage",
                   "n": n, "shape": [nx, ny, nz], "storage": head_st, "compute": "fp32",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "graph_steps": GRAPH_STEPS,
                   "warmup_note": f"{args.warmup} warm-up steps, then {GRAPH_STEPS} untimed steps that capture the "
                                  "CUDA graph the timed steps replay",
                   "l2": f"no flush: the {hv['state_gb']:.2f} GB state streamed each step exceeds the 129 MB L2"},
        "roofline": {"bound": "hbm", "achieved": hv["achieved_gbs"], "peak": peak, "unit": "GB/s",
                     "frac": hv["achieved_gbs"] / peak, "traffic": traffic, "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": hv["algorithmic_bytes_per_site"] * n3,
                     "kernel": kernel_name(head_st, head_kern, nx),
                     "frac_of_nominal_8tbs": hv["achieved_gbs"] / NOMINAL_HBM_GBS,
                     "kernel_source_sha256_16": kernel_source_hash()},
        "stated_l2_error": accuracy.get(head, {}).get("vs_oracle_64"),
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps, "clocks": clk,
        "variants": variants, "adjoint_step": adjoint, "accuracy": accuracy, "turbulence_runs": turb,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
