"""FP64 CPU oracle of the FLAME lattice-Boltzmann Hall-MHD time step.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA implementation in ``paper_2212_11024_gb300``; the two
only share the seeded input generators of ``paper_2212_11024_gb300.inputs``.

The arithmetic lives in ``flame_oracle.c`` (plain C99, FP64, OpenMP over
sites).  This module compiles it on first use with ``gcc`` and wraps it
with ctypes.  ``exact_wave`` holds the analytical damped Hall-MHD wave
(Sec. 4.1) and ``spectra`` the shell spectra and scalar diagnostics.

Parity status per function (pins live in ``tests/test_oracle_*.py``):

- equilibria, Lorentz term, CM collision, current solve, Hall equilibrium,
  streaming, initialisation: pinned (moment identities, closed forms,
  brute-force literal-vs-factored, BGK limit, exact damped wave, order of
  convergence, conservation).
- shell spectra, scalar diagnostics, energy budget (``spectra``): pinned
  (single-mode shells, Parseval, closed-form scalars, single-mode budget,
  the budget identity on a stepped run).
- turbulence beyond early times: parity unpinned (chaotic; compared per
  field only at early times and per spectral shell).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flame_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NQ = 27
NM = 7
NPOP = 48


def build(force: bool = False) -> str:
    """Compile flame_oracle.c into oracle/_build/liboracle.so (gcc, -fopenmp)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(ctypes.c_double)
        IP = ctypes.POINTER(ctypes.c_int)
        d, i = ctypes.c_double, ctypes.c_int
        sig = {
            "oracle_feq_hermite": (None, [d, P, P]),
            "oracle_feq_product": (None, [d, P, P]),
            "oracle_lorentz": (None, [P, P]),
            "oracle_lorentz_printed": (None, [P, P]),
            "oracle_cm_matrix": (None, [P, P]),
            "oracle_collide_cm_literal": (i, [P, P, P, P, P]),
            "oracle_collide_cm_factored": (None, [P, P, P, d, P]),
            "oracle_current": (i, [i, P, P, P, d, d, P]),
            "oracle_geq_hall": (None, [P, P, P, d, P]),
            "oracle_site_collide": (i, [P, d, d, d, i, P, P]),
            "oracle_step": (ctypes.c_long, [i, i, i, d, d, d, i, i, P, P]),
            "oracle_step_variant": (ctypes.c_long, [i, i, i, d, d, d, i, i, i, P, P, P]),
            "oracle_init": (i, [i, i, i, d, d, d, P, P, P, P, P, i, P]),
            "oracle_moments": (None, [i, i, i, d, d, P, P, P, P, P]),
            "oracle_lattice": (None, [IP, P, IP, P]),
            "oracle_threads": (i, [i]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle arrays are C-contiguous float64"
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def threads(n: int = 0) -> int:
    """Set (n > 0) and return the OpenMP thread count the oracle uses."""
    return _load().oracle_threads(int(n))


# ---------------------------------------------------------------- lattice
def lattice():
    """(c27 [27,3] int, w27 [27], xi7 [7,3] int, W7 [7]) as the oracle uses them."""
    lib = _load()
    c = (ctypes.c_int * 81)()
    w = np.zeros(27)
    x = (ctypes.c_int * 21)()
    W = np.zeros(7)
    lib.oracle_lattice(c, _p(w), x, _p(W))
    return (np.array(c[:], dtype=np.int64).reshape(27, 3), w,
            np.array(x[:], dtype=np.int64).reshape(7, 3), W)


# ------------------------------------------------------------- per site
def feq_hermite(rho, U):
    out = np.zeros(27)
    _load().oracle_feq_hermite(float(rho), _p(_f64(U)), _p(out))
    return out


def feq_product(rho, U):
    out = np.zeros(27)
    _load().oracle_feq_product(float(rho), _p(_f64(U)), _p(out))
    return out


def lorentz(B):
    out = np.zeros(27)
    _load().oracle_lorentz(_p(_f64(B)), _p(out))
    return out


def lorentz_printed(B):
    out = np.zeros(27)
    _load().oracle_lorentz_printed(_p(_f64(B)), _p(out))
    return out


def cm_matrix(U):
    """T(U), T[i, j] = T_j(c_i - U)."""
    out = np.zeros((27, 27))
    _load().oracle_cm_matrix(_p(_f64(U)), _p(out))
    return out


def collide_cm_literal(f, feq, U, S):
    out = np.zeros(27)
    rc = _load().oracle_collide_cm_literal(_p(_f64(f)), _p(_f64(feq)), _p(_f64(U)), _p(_f64(S)), _p(out))
    if rc != 0:
        raise ArithmeticError("singular central-moment matrix")
    return out


def collide_cm_factored(f, feq, U, omega):
    out = np.zeros(27)
    _load().oracle_collide_cm_factored(_p(_f64(f)), _p(_f64(feq)), _p(_f64(U)), float(omega), _p(out))
    return out


def current(Lam, U, B, omegaB, alphaH, literal=True):
    """J from Lambda (3x3, Lam[a,b]) per the Hall linear system."""
    J = np.zeros(3)
    rc = _load().oracle_current(int(literal), _p(_f64(np.asarray(Lam).reshape(9))), _p(_f64(U)),
                                _p(_f64(B)), float(omegaB), float(alphaH), _p(J))
    if rc != 0:
        raise ArithmeticError("singular current system")
    return J


def geq_hall(B, U, J, alphaH):
    """g^Hall(0) as [3 components, 7 velocities]."""
    out = np.zeros(21)
    _load().oracle_geq_hall(_p(_f64(B)), _p(_f64(U)), _p(_f64(J)), float(alphaH), _p(out))
    return out.reshape(3, 7)


def site_collide(pop48, tau_nu, tau_eta, d_i, literal=True):
    """Collide one site.  Returns (post[48], moments dict)."""
    out = np.zeros(48)
    mom = np.zeros(11)
    rc = _load().oracle_site_collide(_p(_f64(pop48)), float(tau_nu), float(tau_eta), float(d_i),
                                     int(literal), _p(out), _p(mom))
    if rc != 0:
        raise ArithmeticError("singular system in site collision")
    return out, dict(rho=mom[0], u=mom[1:4].copy(), B=mom[4:7].copy(), J=mom[7:10].copy(), trlam=mom[10])


# ----------------------------------------------------------------- grid
class Params:
    """Lattice-unit parameters: grid size, relaxation times, Hall length."""

    def __init__(self, nx, ny, nz, tau_nu, tau_eta, d_i):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.tau_nu, self.tau_eta, self.d_i = float(tau_nu), float(tau_eta), float(d_i)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n3(self):
        return self.nx * self.ny * self.nz


def init(p: Params, rho, u, B, gradu=None, gradB=None, noneq=True):
    """Initial populations [48, nz, ny, nx] from rho [nz,ny,nx] (or None),
    u, B [3,nz,ny,nx] and optional gradients [9,nz,ny,nx] (d_a F_b at 3a+b)."""
    pop = np.zeros((NPOP,) + p.shape)
    rc = _load().oracle_init(p.nx, p.ny, p.nz, p.tau_nu, p.tau_eta, p.d_i, _p(_f64(rho)), _p(_f64(u)),
                             _p(_f64(B)), _p(_f64(gradu)), _p(_f64(gradB)), int(bool(noneq)), _p(pop))
    assert rc == 0
    return pop


def step(p: Params, pop, nsteps=1, literal=True, scratch=None):
    """Advance pop (modified in place) by nsteps.  Returns pop."""
    assert pop.shape == (NPOP,) + p.shape and pop.dtype == np.float64 and pop.flags["C_CONTIGUOUS"]
    if scratch is None:
        scratch = np.empty_like(pop)
    bad = _load().oracle_step(p.nx, p.ny, p.nz, p.tau_nu, p.tau_eta, p.d_i, int(literal), int(nsteps),
                              _p(pop), _p(scratch))
    if bad:
        raise ArithmeticError(f"{bad} singular central-moment solves")
    return pop


VARIANTS = {"flame": 0, "bgk": 1, "emhd": 2, "fd_current": 3}


def step_variant(p: Params, pop, nsteps=1, variant="bgk", literal=True):
    """Advance pop in place with a scheme variant: "bgk" (BGK fluid collision),
    "emhd" (electron MHD magnetic equilibrium), "fd_current" (J from the
    central-difference curl of B), or "flame" (the paper's scheme)."""
    assert pop.shape == (NPOP,) + p.shape and pop.dtype == np.float64 and pop.flags["C_CONTIGUOUS"]
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    scratch = np.empty_like(pop)
    bfield = np.empty((3,) + p.shape)
    bad = _load().oracle_step_variant(p.nx, p.ny, p.nz, p.tau_nu, p.tau_eta, p.d_i, int(literal), v, int(nsteps),
                                      _p(pop), _p(scratch), _p(bfield))
    if bad:
        raise ArithmeticError(f"{bad} singular solves")
    return pop


def moments(p: Params, pop):
    """dict(rho, u, B, J, trlam) of the pre-collision populations."""
    rho = np.zeros(p.shape)
    u = np.zeros((3,) + p.shape)
    B = np.zeros((3,) + p.shape)
    J = np.zeros((3,) + p.shape)
    tr = np.zeros(p.shape)
    _load().oracle_moments(p.nx, p.ny, p.nz, p.tau_eta, p.d_i, _p(np.ascontiguousarray(pop)), _p(rho), _p(u),
                           _p(B), _p(J), _p(tr))
    return dict(rho=rho, u=u, B=B, J=J, trlam=tr)
