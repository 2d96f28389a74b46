"""Python binding of libflame.so (include/flame.h): argument marshalling only.

PyTorch supplies device memory and streams; every step of the method runs
in the library's CUDA kernels.  There is no CPU fallback: without the
compiled library, or without a CUDA device, the constructors raise.

    from paper_2212_11024_gb300 import Flame, inputs
    u, B = inputs.turbulence((128, 128, 128), 1, 2)
    sim = Flame(128, 128, 128, tau_nu=0.51, tau_eta=0.51, d_i=6.4, storage="fp16")
    sim.init(None, u, B)
    sim.step(100)
    m = sim.moments()          # dict of FP64 CUDA tensors rho, u, B, J
    Eu, Eb = sim.spectra(65)   # shell spectra, numpy FP64
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libflame.so")

FLAME_OK, FLAME_ERR_PARAM, FLAME_ERR_CFL, FLAME_ERR_NONFINITE, FLAME_ERR_CUDA, FLAME_ERR_STATE, FLAME_ERR_TIMEOUT = range(7)
# chunks of z planes the host-buffer calls use at most (FLAME_IO_CHUNKS)
IO_CHUNKS = 32
STORAGE = {"fp32": 1, "fp16": 2, "bf16": 3}
VARIANT = {"flame": 0, "bgk": 1, "emhd": 2, "fd_current": 3}
# flame_params.kernel: "auto" uses the row kernel (TMA-staged rows, packed
# FP32 pairs) where it applies, "site" always the one-site kernel, "row" and
# "row_half" the row kernel with whole or half rows per tile where it applies.
KERNEL = {"auto": 0, "site": 1, "row": 2, "row_half": 3, "pair": 4}
NSCALARS = 14
SCALAR_NAMES = ["mass", "mom_x", "mom_y", "mom_z", "B_x", "B_y", "B_z", "E_u", "E_B", "H_c", "J2", "u_max",
                "divB_rms", "nonfinite"]


class FlameError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {_lib().flame_status_string(status).decode()} (status {status})")


class FlameUnavailable(RuntimeError):
    pass


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("tau_nu", ctypes.c_double), ("tau_eta", ctypes.c_double), ("d_i", ctypes.c_double),
        ("storage", ctypes.c_int), ("rho0", ctypes.c_double), ("B_ref", ctypes.c_double * 3),
        ("init_noneq", ctypes.c_int), ("check_every", ctypes.c_int), ("strict_cfl", ctypes.c_int),
        ("graph_steps", ctypes.c_int), ("variant", ctypes.c_int), ("kernel", ctypes.c_int),
        ("halo_z", ctypes.c_int),
    ]


class HaloRun(ctypes.Structure):
    _fields_ = [("first_slot", ctypes.c_int), ("nslots", ctypes.c_int), ("plane", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("step", ctypes.c_longlong), ("parity", ctypes.c_int), ("nonfinite", ctypes.c_int),
                ("cfl", ctypes.c_double), ("max_speed", ctypes.c_double)]


_lock = threading.Lock()
_LIB = None


def _lib():
    global _LIB
    with _lock:
        if _LIB is not None:
            return _LIB
        if not os.path.exists(LIB_PATH):
            raise FlameUnavailable(f"{LIB_PATH} is missing: build it with paper_2212_11024_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        vp, P, i, d = ctypes.c_void_p, ctypes.POINTER, ctypes.c_int, ctypes.c_double
        sig = {
            "flame_state_bytes": (ctypes.c_size_t, [P(Params)]),
            "flame_create": (i, [P(vp), P(Params), vp, vp]),
            "flame_create_fields": (i, [P(vp), P(Params), vp]),
            "flame_step_kernel": (i, [P(Params)]),
            "flame_init": (i, [vp, vp, vp, vp, vp, vp]),
            "flame_step": (i, [vp, i]),
            "flame_sync": (i, [vp]),
            "flame_info": (i, [vp, P(Info)]),
            "flame_moments": (i, [vp, vp, vp, vp, vp]),
            "flame_populations": (i, [vp, vp]),
            "flame_reduce": (i, [vp, P(d)]),
            "flame_spectra": (i, [vp, i, P(d), P(d)]),
            "flame_spectra_fields": (i, [vp, i, vp, vp, P(d), P(d)]),
            "flame_get_state": (i, [vp, vp, P(ctypes.c_longlong), P(i)]),
            "flame_set_state": (i, [vp, vp, ctypes.c_longlong, i]),
            "flame_destroy": (None, [vp]),
            "flame_status_string": (ctypes.c_char_p, [i]),
            "flame_lattice": (i, [P(i), P(i)]),
            "flame_reduce_static": (i, [vp, i, vp]),
            "flame_probe": (i, [vp, i, vp, vp]),
            "flame_step_adjoint": (i, [vp, vp, i, vp, vp, vp]),
            "flame_init_adjoint": (i, [vp, vp, vp, vp, vp, vp, vp]),
            "flame_debug_stall_next_step": (i, [vp, ctypes.c_uint]),
            "flame_init_f32": (i, [vp, vp, vp, vp, vp, vp]),
            "flame_moments_f32": (i, [vp, vp, vp, vp, vp]),
            "flame_init_f32_host": (i, [vp, vp, vp, vp]),
            "flame_moments_f32_host": (i, [vp, vp, vp, vp, vp, P(d)]),
            "flame_band_energy": (i, [vp, i, i, vp, P(d), vp, vp]),
            "flame_energy_budget": (i, [vp, i, vp, vp, P(d), P(d), P(d)]),
            "flame_reduce_sums": (i, [vp, P(d)]),
            "flame_reduce_combine": (i, [P(Params), P(d), P(d)]),
            "flame_halo_plan": (i, [P(Params), i, i, P(HaloRun), P(HaloRun)]),
            "flame_halo_exchange": (i, [vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
        return lib


def library():
    """The loaded ctypes library (raises FlameUnavailable if not built)."""
    return _lib()


def lattice():
    """(c27 [27,3], xi7 [7,3]) velocity tables compiled into the kernels."""
    c = (ctypes.c_int * 81)()
    x = (ctypes.c_int * 21)()
    _lib().flame_lattice(c, x)
    return np.array(c[:]).reshape(27, 3), np.array(x[:]).reshape(7, 3)


def make_params(nx, ny, nz, tau_nu, tau_eta, d_i, storage="fp32", rho0=1.0, B_ref=(0.0, 0.0, 0.0),
                init_noneq=True, check_every=0, strict_cfl=False, graph_steps=0, variant="flame",
                kernel="auto", halo_z=False) -> Params:
    p = Params()
    p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
    p.tau_nu, p.tau_eta, p.d_i = float(tau_nu), float(tau_eta), float(d_i)
    p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    p.rho0 = float(rho0)
    for a in range(3):
        p.B_ref[a] = float(B_ref[a])
    p.init_noneq, p.check_every, p.strict_cfl = int(bool(init_noneq)), int(check_every), int(bool(strict_cfl))
    p.graph_steps = int(graph_steps)
    p.variant = VARIANT[variant] if isinstance(variant, str) else int(variant)
    p.kernel = KERNEL[kernel] if isinstance(kernel, str) else int(kernel)
    p.halo_z = int(bool(halo_z))
    return p


NSUMS = 18
SUM_UMAX = 14


def reduce_combine(p: Params, sums) -> dict:
    """flame_reduce_combine: the reduce() scalars from raw sums (one
    context's, or several slabs' added, with the maximum at SUM_UMAX)."""
    r = (ctypes.c_double * NSUMS)(*[float(v) for v in sums])
    h = (ctypes.c_double * NSCALARS)()
    if _lib().flame_reduce_combine(ctypes.byref(p), r, h) != 0:
        raise ValueError("flame_reduce_combine: invalid sums")
    return dict(zip(SCALAR_NAMES, list(h)))


STEP_KERNELS = {1: "site", 2: "rows", 3: "half_rows", 4: "pairs"}


def step_kernel(p: Params) -> str:
    """flame_step_kernel: which step kernel flame_step launches for these
    parameters ("site", "rows", "half_rows" or "pairs"); host only."""
    k = _lib().flame_step_kernel(ctypes.byref(p))
    if k == 0:
        raise FlameError(FLAME_ERR_PARAM, "flame_step_kernel")
    return STEP_KERNELS[k]


def halo_plan(p: Params, parity: int, face: int):
    """flame_halo_plan: ([(first_slot, nslots, plane)] * 2 sent, the same
    received) through `face` of a slab after a step leaving `parity`."""
    send, recv = (HaloRun * 2)(), (HaloRun * 2)()
    if _lib().flame_halo_plan(ctypes.byref(p), int(parity), int(face), send, recv) != 0:
        raise ValueError("flame_halo_plan: invalid arguments")
    return ([(r.first_slot, r.nslots, r.plane) for r in send], [(r.first_slot, r.nslots, r.plane) for r in recv])


def state_bytes(p: Params) -> int:
    return int(_lib().flame_state_bytes(ctypes.byref(p)))


# Checkpoints (save_checkpoint / load_checkpoint): the state blob with its
# step and AA parity, and the parameters it depends on.  The lattice, the
# storage type and the reference state of the deviation encoding (rho0,
# B_ref) define what the bytes mean and must match to resume; the relaxation
# times, d_i and the variant define the dynamics and must match too unless
# the caller asks to resume with new ones.
CHECKPOINT_LAYOUT = ("nx", "ny", "nz", "storage", "rho0", "B_ref")
CHECKPOINT_PHYSICS = ("tau_nu", "tau_eta", "d_i", "variant")


def checkpoint_meta(p: Params) -> dict:
    """The parameters a checkpoint records (plain Python values)."""
    meta = {k: getattr(p, k) for k in CHECKPOINT_LAYOUT + CHECKPOINT_PHYSICS if k != "B_ref"}
    meta["B_ref"] = [float(v) for v in p.B_ref]
    return meta


def checkpoint_mismatches(saved: dict, p: Params, same_physics: bool = True) -> list:
    """Names of the recorded parameters that differ from p (the layout ones
    always, the physics ones when same_physics)."""
    cur = checkpoint_meta(p)
    keys = CHECKPOINT_LAYOUT + (CHECKPOINT_PHYSICS if same_physics else ())
    return [k for k in keys if not np.array_equal(np.asarray(saved[k]), np.asarray(cur[k]))]


def _check(rc, what):
    if rc != FLAME_OK:
        raise FlameError(rc, what)


class Flame:
    """One periodic Hall-MHD lattice on one GPU (a flame_ctx plus its state)."""

    def __init__(self, nx, ny, nz, tau_nu, tau_eta, d_i, storage="fp32", rho0=1.0, B_ref=(0.0, 0.0, 0.0),
                 init_noneq=True, check_every=0, strict_cfl=False, device=None, stream=None, graph_steps=0,
                 variant="flame", kernel="auto", halo_z=False, fields_only=False):
        import torch

        if not torch.cuda.is_available():
            raise FlameUnavailable("no CUDA device: the FLAME step runs only on the GPU")
        lib = _lib()
        self.torch = torch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.p = make_params(nx, ny, nz, tau_nu, tau_eta, d_i, storage, rho0, B_ref, init_noneq, check_every,
                             strict_cfl, graph_steps, variant, kernel, halo_z)
        self.shape = (int(nz), int(ny), int(nx))
        # a z-slab takes its initial fields with one neighbouring plane on each side
        self.field_shape = (int(nz) + 2 * int(bool(halo_z)), int(ny), int(nx))
        self.n3 = int(nx) * int(ny) * int(nz)
        nbytes = state_bytes(self.p)
        if nbytes == 0:
            raise FlameError(FLAME_ERR_PARAM, "flame_state_bytes")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            ctx = ctypes.c_void_p()
            if fields_only:
                # no population state: the field-level diagnostics of given u, B
                self.state = None
                _check(lib.flame_create_fields(ctypes.byref(ctx), ctypes.byref(self.p),
                                               ctypes.c_void_p(self.stream.cuda_stream)), "flame_create_fields")
            else:
                self.state = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
                _check(lib.flame_create(ctypes.byref(ctx), ctypes.byref(self.p),
                                        ctypes.c_void_p(self.state.data_ptr()),
                                        ctypes.c_void_p(self.stream.cuda_stream)), "flame_create")
        self._ctx = ctx
        self._lib = lib

    # ------------------------------------------------------------------ util
    def _dev(self, a, ncomp, dtype=None):
        """Contiguous device tensor (FP64 unless dtype says otherwise) of shape
        [ncomp, nz, ny, nx] (or [nz,ny,nx])."""
        if a is None:
            return None
        t = self.torch
        dtype = t.float64 if dtype is None else dtype
        if isinstance(a, np.ndarray):
            a = t.from_numpy(np.ascontiguousarray(a))
        a = a.to(device=self.device, dtype=dtype).contiguous()
        want = (ncomp,) + self.field_shape if ncomp else self.field_shape
        if tuple(a.shape) != want:
            raise ValueError(f"expected shape {want}, got {tuple(a.shape)}")
        return a

    @staticmethod
    def _ptr(a):
        return ctypes.c_void_p(a.data_ptr()) if a is not None else None

    def _ctx_or_raise(self):
        if self._ctx is None:
            raise RuntimeError("context closed")
        return self._ctx

    # The library queues its work on self.stream, torch on its current
    # stream; when a caller passes another stream the two are ordered here.
    def _before(self):
        """Make the library's stream wait for torch's current stream, so that
        inputs torch wrote, and outputs torch allocated, are ready before the
        library touches them.  Returns the current stream."""
        cur = self.torch.cuda.current_stream(self.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)
        return cur

    def _after(self, cur, *tensors):
        """Make torch's current stream wait for the library's, so that torch
        reads the outputs only once they are written, and keep the tensors'
        memory from being reused by the caching allocator while the library's
        stream still uses it."""
        if cur != self.stream:
            cur.wait_stream(self.stream)
            for t in tensors:
                if t is not None:
                    t.record_stream(self.stream)

    # ------------------------------------------------------------------- API
    def init(self, rho, u, B, gradu=None, gradB=None):
        """flame_init from fields (numpy or torch): rho [nz,ny,nx] or None,
        u, B [3,nz,ny,nx], optional gradients [9,nz,ny,nx].  FP32 fields (u
        of dtype float32) go through flame_init_f32 as they are; anything
        else is converted to FP64 for flame_init."""
        t = self.torch
        f32 = (u.dtype == np.float32) if isinstance(u, np.ndarray) else (getattr(u, "dtype", None) is t.float32)
        dt = t.float32 if f32 else t.float64
        r, uu, bb = self._dev(rho, 0, dt), self._dev(u, 3, dt), self._dev(B, 3, dt)
        gu, gb = self._dev(gradu, 9, dt), self._dev(gradB, 9, dt)
        cur = self._before()
        # flame_init synchronises the library's stream, so the temporaries outlive their use
        fn = self._lib.flame_init_f32 if f32 else self._lib.flame_init
        rc = fn(self._ctx_or_raise(), self._ptr(r), self._ptr(uu), self._ptr(bb), self._ptr(gu), self._ptr(gb))
        self._after(cur)
        _check(rc, "flame_init_f32" if f32 else "flame_init")

    def _host(self, a, ncomp, shape, what):
        """A pointer to a C-contiguous FP32 host array (numpy or CPU torch) of
        shape [ncomp, *shape] (or shape)."""
        if a is None:
            return None
        want = ((ncomp,) + shape) if ncomp else shape
        if isinstance(a, np.ndarray):
            ok = a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
            ptr = a.ctypes.data
        else:
            ok = a.dtype is self.torch.float32 and a.device.type == "cpu" and a.is_contiguous()
            ptr = a.data_ptr()
        if not ok or tuple(a.shape) != want:
            raise ValueError(f"{what}: expected a C-contiguous FP32 host array of shape {want}")
        return ctypes.c_void_p(ptr)

    def init_host(self, rho, u, B):
        """flame_init_f32_host: the initial populations from FP32 fields in
        host memory (numpy, or CPU torch tensors; page-locked ones, e.g.
        torch's pin_memory(), let the copies overlap the initialisation):
        rho [nz,ny,nx] or None, u, B [3,nz,ny,nx] (a z-slab's with its ghost
        planes).  Returns once the host arrays are no longer in use."""
        args = (self._host(rho, 0, self.field_shape, "rho"), self._host(u, 3, self.field_shape, "u"),
                self._host(B, 3, self.field_shape, "B"))
        cur = self._before()
        rc = self._lib.flame_init_f32_host(self._ctx_or_raise(), *args)
        self._after(cur)
        _check(rc, "flame_init_f32_host")

    def moments_host(self, out=None, scalars=False):
        """flame_moments_f32_host: rho, u, B, J of the current pre-collision
        populations (FP32) written into host arrays: `out` a dict of C-contiguous
        FP32 host arrays (numpy or CPU torch; any key may be absent or None),
        or None for page-locked torch tensors of all four.  With
        scalars=True also reduce()'s scalars of the same state, computed
        while the fields are copied out.  Returns out, or (out, scalars)."""
        t = self.torch
        if out is None:
            out = dict(rho=t.empty(self.shape, dtype=t.float32).pin_memory(),
                       u=t.empty((3,) + self.shape, dtype=t.float32).pin_memory(),
                       B=t.empty((3,) + self.shape, dtype=t.float32).pin_memory(),
                       J=t.empty((3,) + self.shape, dtype=t.float32).pin_memory())
        ptrs = [self._host(out.get(k), 0 if k == "rho" else 3, self.shape, k) for k in ("rho", "u", "B", "J")]
        h = (ctypes.c_double * NSCALARS)() if scalars else None
        cur = self._before()
        rc = self._lib.flame_moments_f32_host(self._ctx_or_raise(), *ptrs, h)
        self._after(cur)
        if not scalars:
            _check(rc, "flame_moments_f32_host")
            return out
        if rc not in (FLAME_OK, FLAME_ERR_NONFINITE):
            _check(rc, "flame_moments_f32_host")
        vals = dict(zip(SCALAR_NAMES, list(h)))
        vals["status"] = rc
        return out, vals

    def step(self, n=1):
        _check(self._lib.flame_step(self._ctx_or_raise(), int(n)), "flame_step")

    def sync(self):
        _check(self._lib.flame_sync(self._ctx_or_raise()), "flame_sync")

    def info(self) -> dict:
        inf = Info()
        _check(self._lib.flame_info(self._ctx_or_raise(), ctypes.byref(inf)), "flame_info")
        return dict(step=inf.step, parity=inf.parity, nonfinite=inf.nonfinite, cfl=inf.cfl, max_speed=inf.max_speed)

    def moments(self, out=None, dtype=None) -> dict:
        """rho, u, B, J of the current pre-collision populations as CUDA
        tensors: FP64 (flame_moments) or, with dtype=torch.float32 or FP32
        tensors in `out`, FP32 (flame_moments_f32)."""
        t = self.torch
        if out is None:
            dt = t.float64 if dtype is None else dtype
            out = dict(rho=t.empty(self.shape, dtype=dt, device=self.device),
                       u=t.empty((3,) + self.shape, dtype=dt, device=self.device),
                       B=t.empty((3,) + self.shape, dtype=dt, device=self.device),
                       J=t.empty((3,) + self.shape, dtype=dt, device=self.device))
        dts = {v.dtype for v in out.values() if v is not None}
        if len(dts) != 1 or not dts <= {t.float32, t.float64}:
            raise ValueError("moments: outputs must be all FP32 or all FP64")
        f32 = dts == {t.float32}
        fn = self._lib.flame_moments_f32 if f32 else self._lib.flame_moments
        cur = self._before()
        rc = fn(self._ctx_or_raise(), self._ptr(out.get("rho")), self._ptr(out.get("u")), self._ptr(out.get("B")),
                self._ptr(out.get("J")))
        self._after(cur, *out.values())
        _check(rc, "flame_moments_f32" if f32 else "flame_moments")
        return out

    def probe(self, sites, out=None):
        """Moments at linear site indices (CUDA int64 tensor): FP64 [n, 10] =
        rho, u[3], B[3], J[3].  Asynchronous; `out` may be a preallocated slice."""
        t = self.torch
        n = int(sites.numel())
        if out is None:
            out = t.empty((n, 10), dtype=t.float64, device=self.device)
        cur = self._before()
        rc = self._lib.flame_probe(self._ctx_or_raise(), n, self._ptr(sites), self._ptr(out))
        self._after(cur, sites, out)
        _check(rc, "flame_probe")
        return out

    def populations(self):
        """Decoded pre-collision populations [48, nz, ny, nx], FP64, natural slot order."""
        t = self.torch
        f = t.empty((48,) + self.shape, dtype=t.float64, device=self.device)
        cur = self._before()
        rc = self._lib.flame_populations(self._ctx_or_raise(), self._ptr(f))
        self._after(cur, f)
        _check(rc, "flame_populations")
        return f

    def reduce(self) -> dict:
        h = (ctypes.c_double * NSCALARS)()
        rc = self._lib.flame_reduce(self._ctx_or_raise(), h)
        vals = dict(zip(SCALAR_NAMES, list(h)))
        if rc not in (FLAME_OK, FLAME_ERR_NONFINITE):
            _check(rc, "flame_reduce")
        vals["status"] = rc
        return vals

    def reduce_sums(self):
        """flame_reduce_sums: the raw FP64 sums (NSUMS values, numpy) behind
        reduce(), to be added over the slabs of a lattice and combined with
        reduce_combine."""
        h = (ctypes.c_double * NSUMS)()
        rc = self._lib.flame_reduce_sums(self._ctx_or_raise(), h)
        if rc not in (FLAME_OK, FLAME_ERR_NONFINITE):
            _check(rc, "flame_reduce_sums")
        return np.array(h[:])

    def halo_exchange(self, upper):
        """flame_halo_exchange with the slab context `upper` above this one
        (this context itself for a lattice of one slab)."""
        _check(self._lib.flame_halo_exchange(self._ctx_or_raise(), upper._ctx_or_raise()), "flame_halo_exchange")

    def reduce_static(self, nblocks=0, out=None):
        """flame_reduce_static: the reduce() scalars computed without any
        allocation in the library, into a FP64 CUDA tensor of NSCALARS
        entries (returned).  For callers that must not let the library call
        cudaMalloc; the first call on a device should precede stream capture."""
        t = self.torch
        if out is None:
            out = t.empty(NSCALARS, dtype=t.float64, device=self.device)
        cur = self._before()
        rc = self._lib.flame_reduce_static(self._ctx_or_raise(), int(nblocks), self._ptr(out))
        self._after(cur, out)
        _check(rc, "flame_reduce_static")
        return out

    def spectra(self, nshell, u=None, B=None):
        """flame_spectra: shell spectra (E_u, E_B) numpy FP64 [nshell] of the
        current state, or (flame_spectra_fields) of the given FP64 fields u, B
        [3,nz,ny,nx]."""
        Eu = (ctypes.c_double * nshell)()
        Eb = (ctypes.c_double * nshell)()
        if u is None and B is None:
            _check(self._lib.flame_spectra(self._ctx_or_raise(), int(nshell), Eu, Eb), "flame_spectra")
        else:
            uu, bb = self._dev(u, 3), self._dev(B, 3)
            cur = self._before()
            rc = self._lib.flame_spectra_fields(self._ctx_or_raise(), int(nshell), self._ptr(uu), self._ptr(bb), Eu, Eb)
            self._after(cur)
            _check(rc, "flame_spectra_fields")
        return np.array(Eu[:]), np.array(Eb[:])

    def band_energy(self, lo, hi, B=None, grad=False, adjoint_seed=False):
        """flame_band_energy: L = sum_{lo<=n<=hi} E_B(n) of the current state
        (or of the FP64 field B [3,nz,ny,nx]); with grad, also dL/dB (FP64
        CUDA [3,nz,ny,nx]); with adjoint_seed, also the FP32 [48, N3] seed of
        flame_step_adjoint.  Returns (L, dLdB or None, seed or None)."""
        t = self.torch
        bb = self._dev(B, 3)
        g = t.empty((3,) + self.shape, dtype=t.float64, device=self.device) if grad else None
        a = t.empty((48, self.n3), dtype=t.float32, device=self.device) if adjoint_seed else None
        L = ctypes.c_double()
        cur = self._before()
        rc = self._lib.flame_band_energy(self._ctx_or_raise(), int(lo), int(hi), self._ptr(bb), ctypes.byref(L),
                                         self._ptr(g), self._ptr(a))
        self._after(cur, g, a)
        _check(rc, "flame_band_energy")
        return float(L.value), g, a

    def energy_budget(self, nshell, u=None, B=None):
        """flame_energy_budget: (E, S, D) numpy FP64 [nshell] of the current
        state's u, B (or of the given FP64 fields), with this context's nu,
        eta and d_i."""
        if (u is None) != (B is None):
            raise ValueError("energy_budget: give both u and B, or neither")
        uu, bb = self._dev(u, 3), self._dev(B, 3)
        E, S, D = (ctypes.c_double * nshell)(), (ctypes.c_double * nshell)(), (ctypes.c_double * nshell)()
        cur = self._before()
        rc = self._lib.flame_energy_budget(self._ctx_or_raise(), int(nshell), self._ptr(uu), self._ptr(bb), E, S, D)
        self._after(cur)
        _check(rc, "flame_energy_budget")
        return np.array(E[:]), np.array(S[:]), np.array(D[:])

    def debug_stall_next_step(self, tries=1024):
        """Arm the wait-failure test for the next step (flame_debug_stall_next_step):
        that step's waits run out and it raises FlameError(FLAME_ERR_TIMEOUT)."""
        _check(self._lib.flame_debug_stall_next_step(self._ctx_or_raise(), int(tries)), "flame_debug_stall_next_step")

    def get_state(self):
        if self.state is None:
            raise FlameError(FLAME_ERR_STATE, "flame_get_state (a context without state)")
        dst = self.torch.empty_like(self.state)
        step = ctypes.c_longlong()
        par = ctypes.c_int()
        cur = self._before()
        rc = self._lib.flame_get_state(self._ctx_or_raise(), self._ptr(dst), ctypes.byref(step), ctypes.byref(par))
        self._after(cur, dst)
        _check(rc, "flame_get_state")
        return dst, int(step.value), int(par.value)

    def set_state(self, src, step, parity):
        if self.state is None:
            raise FlameError(FLAME_ERR_STATE, "flame_set_state (a context without state)")
        if src.numel() != self.state.numel() or src.dtype != self.state.dtype:
            raise ValueError("state blob does not match these parameters")
        src = src.contiguous()
        cur = self._before()
        rc = self._lib.flame_set_state(self._ctx_or_raise(), self._ptr(src), int(step), int(parity))
        self._after(cur, src)
        _check(rc, "flame_set_state")

    def save_checkpoint(self, path):
        """Write the state, its step and parity and checkpoint_meta() to an
        .npz file (the state goes through host memory)."""
        blob, step, parity = self.get_state()
        meta = checkpoint_meta(self.p)
        np.savez(path, state=blob.cpu().numpy(), step=np.int64(step), parity=np.int32(parity),
                 **{"meta_" + k: np.asarray(v) for k, v in meta.items()})

    def load_checkpoint(self, path, same_physics=True):
        """Resume from a save_checkpoint file.  Raises ValueError when the
        recorded lattice, storage or reference state differ from this run's
        (and its relaxation times, d_i or variant, unless same_physics is
        False)."""
        with np.load(path) as z:
            saved = {k[5:]: z[k] for k in z.files if k.startswith("meta_")}
            bad = checkpoint_mismatches(saved, self.p, same_physics)
            if bad:
                raise ValueError(f"checkpoint {path} does not match this run: {', '.join(bad)}")
            blob = self.torch.from_numpy(z["state"]).to(self.device)
            step, parity = int(z["step"]), int(z["parity"])
        self.set_state(blob, step, parity)

    def close(self):
        if getattr(self, "_ctx", None) is not None:
            self._lib.flame_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
