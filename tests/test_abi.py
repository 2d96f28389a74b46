"""Host-side checks of the C ABI (no GPU needed): the library builds, loads
and exports every entry point include/flame.h declares; host-only entry
points behave; the lattice tables compiled into the kernels are App. A's."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2212_11024_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def _declared():
    txt = open(os.path.join(ROOT, "include", "flame.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(flame_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_lattice_tables_match_app_a(lib):
    from paper_2212_11024_gb300 import flame as F
    c27, xi7 = F.lattice()
    gold = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "d3q27_velocities.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        gold[k] = [int(x) for x in v]
    assert np.array_equal(c27, np.array([gold["cx"], gold["cy"], gold["cz"]]).T)
    assert np.array_equal(xi7, [[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])


def test_params_struct_matches_header():
    """The ctypes mirror of flame_params lists the header's fields in order."""
    from paper_2212_11024_gb300 import flame as F
    txt = open(os.path.join(ROOT, "include", "flame.h")).read()
    body = txt[txt.index("typedef struct {", txt.index("flame_variant;")):txt.index("} flame_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"\b([a-zA-Z_]\w*)\s*(?:\[\d\])?\s*(?=[,;])", body)
    assert names == [f[0] for f in F.Params._fields_]


def test_state_bytes_and_param_validation(lib):
    from paper_2212_11024_gb300 import flame as F
    p = F.make_params(256, 256, 256, 0.51, 0.51, 12.8, "fp32")
    assert F.state_bytes(p) == 48 * 256 ** 3 * 4
    p = F.make_params(33, 5, 7, 0.6, 0.6, 2.0, "bf16")
    assert F.state_bytes(p) == 48 * 33 * 5 * 7 * 2
    bad = [F.make_params(0, 4, 4, 0.6, 0.6, 0.0), F.make_params(4, 4, 4, 0.5, 0.6, 0.0),
           F.make_params(4, 4, 4, 0.6, 0.4, 0.0), F.make_params(4, 4, 4, 0.6, 0.6, -1.0),
           F.make_params(4, 4, 4, 0.6, 0.6, 0.0, storage=7), F.make_params(2048, 1024, 1024, 0.6, 0.6, 0.0),
           F.make_params(4, 4, 4, 0.6, 0.6, float("nan")), F.make_params(4, 4, 4, 0.6, 0.6, 0.0, rho0=0.0),
           F.make_params(4, 4, 4, 0.6, 0.6, 0.0, kernel=5)]
    b = F.make_params(4, 4, 4, 0.6, 0.6, 0.0)
    b.halo_z = 2
    bad.append(b)
    for b in bad:
        assert F.state_bytes(b) == 0


def test_status_strings(lib):
    lib.flame_status_string.restype = ctypes.c_char_p
    texts = {lib.flame_status_string(i).decode() for i in range(7)}
    assert len(texts) == 7 and "ok" in texts


def test_flame_create_rejects_bad_arguments_without_touching_the_gpu(lib):
    """Parameter and pointer checks happen before any CUDA call."""
    from paper_2212_11024_gb300 import flame as F
    L = F.library()
    ctx = ctypes.c_void_p(1234)
    p = F.make_params(4, 4, 4, 0.6, 0.6, 0.0)
    assert L.flame_create(ctypes.byref(ctx), ctypes.byref(p), None, None) == F.FLAME_ERR_PARAM
    assert ctx.value is None
    assert L.flame_create(ctypes.byref(ctx), ctypes.byref(p), ctypes.c_void_p(0x1001), None) == F.FLAME_ERR_PARAM
    bad = F.make_params(4, 4, 4, 0.4, 0.6, 0.0)
    assert L.flame_create(ctypes.byref(ctx), ctypes.byref(bad), ctypes.c_void_p(0x1000), None) == F.FLAME_ERR_PARAM
    assert L.flame_step(None, 1) == F.FLAME_ERR_PARAM
    assert L.flame_sync(None) == F.FLAME_ERR_PARAM
    # the context without state: the same parameter checks, and no slab
    assert L.flame_create_fields(ctypes.byref(ctx), ctypes.byref(bad), None) == F.FLAME_ERR_PARAM
    assert ctx.value is None
    slab = F.make_params(4, 4, 4, 0.6, 0.6, 0.0, halo_z=True)
    assert L.flame_create_fields(ctypes.byref(ctx), ctypes.byref(slab), None) == F.FLAME_ERR_PARAM
    assert L.flame_create_fields(None, ctypes.byref(p), None) == F.FLAME_ERR_PARAM
    assert L.flame_spectra_fields(None, 4, None, None, None, None) == F.FLAME_ERR_PARAM


def test_units_match_table2_cfl():
    """Table 2 (Sec. 5): every run satisfies the printed whistler bound
    Ma <= (sqrt(3)/pi)/(eps_H N^2), and the paper's numbers for run I give
    the limit 8.4e-4 quoted beside Ma = 7e-4."""
    from paper_2212_11024_gb300 import units as U
    rows = [ln.split() for ln in open(os.path.join(ROOT, "tests", "golden", "table2_runs.txt"))
            if ln.strip() and not ln.startswith("#")]
    for run, N, Ma, eps in rows:
        lim = U.paper_mach_limit(int(N), float(eps))
        assert float(Ma) <= lim, run
        # the lattice-unit whistler number of the same run is below 1 too
        assert U.whistler_cfl(float(eps) * int(N), float(Ma) / np.sqrt(3.0)) <= 1.0
    assert abs(U.paper_mach_limit(512, 0.0025) - 8.41e-4) < 1e-6


def test_units_relaxation_times():
    from paper_2212_11024_gb300 import units as U
    assert abs(U.tau_from_nu(1.0 / 30) - 0.6) < 1e-15 and abs(U.tau_from_eta(1.0 / 40) - 0.6) < 1e-15
    lp = U.lattice_params(64, 0.05, 100.0, 1.0, 0.05)
    assert abs(lp["nu"] - 0.05 / np.sqrt(3) * 64 / 100) < 1e-15 and abs(lp["d_i"] - 3.2) < 1e-15


def test_step_kernel_choice_without_a_gpu(lib):
    """flame_step_kernel names the kernel flame_step would launch, on the
    host: the row kernel's tilings for 16-bit storage by row length, the
    one-site kernel for FP32, odd rows and when forced; 0 for bad
    parameters."""
    from paper_2212_11024_gb300 import flame as F
    L = F.library()
    bad = F.make_params(4, 4, 4, 0.4, 0.6, 0.0)
    assert L.flame_step_kernel(ctypes.byref(bad)) == 0
    want = {(256, "fp16", "auto"): "rows", (512, "bf16", "auto"): "rows", (608, "fp16", "auto"): "half_rows",
            (100, "fp16", "auto"): "pairs", (34, "bf16", "auto"): "pairs", (33, "fp16", "auto"): "site",
            (256, "fp32", "auto"): "site", (256, "fp16", "site"): "site", (256, "fp16", "pair"): "pairs",
            (100, "fp16", "row"): "site", (640, "fp16", "row"): "rows", (512, "fp16", "row_half"): "half_rows",
            (33, "fp16", "pair"): "site"}
    for (n, st, k), name in want.items():
        assert F.step_kernel(F.make_params(n, 8, 8, 0.6, 0.6, 1.0, st, kernel=k)) == name, (n, st, k)


def test_io_chunk_limit_matches_header():
    from paper_2212_11024_gb300 import flame as F
    txt = open(os.path.join(ROOT, "include", "flame.h")).read()
    m = re.search(r"FLAME_IO_CHUNKS\s*=\s*(\d+)", txt)
    assert m and int(m.group(1)) == F.IO_CHUNKS
