"""The row kernel for 16-bit storage (x rows staged in shared memory by TMA,
two sites per thread in packed FP32 pairs) against the FP64 oracle and
against the one-site kernel, for the paper's scheme and its variants (BGK
fluid, electron MHD, finite-difference current).  Row lengths 64, 128, 256
and 512 take the compile-time row length instantiations, 72, 192, 200, 328,
960, 1000 and 1024 the general one (72, 328 and 1000: blocks whose last warp
is partial; 72 and 200: runs of staged rows padded to 128 bytes)."""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import rel_dev_err, rel_l2, rest_populations, run_both, slot_dev_errs, turbulence

pytestmark = pytest.mark.gpu

# Tolerances against the FP64 oracle after 21 steps, about three times the
# largest error measured on GB300 over the lattices of each test (relative
# L2 of the fluctuations per field, of the population deviations per group
# and per slot; density absolute).  The current's relative error is larger
# on lattices a single row or plane thick ("thin"), where the fields vary
# along one or two axes only and J is small against B.
TOL = {
    # storage: u, B, J (bulk), J (thin), rho, fluid pops, magnetic pops, worst slot
    "fp16": dict(u=1e-3, B=1.2e-3, J=3e-3, J_thin=2.5e-2, rho=3e-4, fluid=1.5e-3, mag=1.5e-3, slot=7e-3),
    "bf16": dict(u=8e-3, B=1e-2, J=2.5e-2, J_thin=0.2, rho=2e-3, fluid=1.4e-2, mag=1.4e-2, slot=6e-2),
}
# the scheme's variants on the row kernel (same 21 steps)
TOL_VARIANT = {
    "fp16": dict(u=1.3e-3, B=1.2e-3, J=4.5e-3, J_thin=2.2e-2, rho=3e-4, fluid=2.3e-3, mag=1.6e-3, slot=1.1e-2),
    "bf16": dict(u=1.1e-2, B=1.1e-2, J=4e-2, J_thin=0.18, rho=2.2e-3, fluid=1.9e-2, mag=1.4e-2, slot=0.1),
}


def _thin(shape):
    return shape[0] * shape[1] < 6

# (nz, ny, nx): compile-time row lengths 64, 128, 256 and 512 and the general
# one (192, and 960 / 1024 with 480- / 512-thread blocks); single-row and
# single-plane lattices, where a row's periodic y / z neighbours are the row
# itself
SHAPES = [(6, 5, 64), (4, 3, 128), (3, 4, 192), (2, 3, 512), (1, 1, 64), (1, 2, 256), (2, 1, 960), (1, 2, 1024),
          (1, 2, 328), (2, 1, 1000), (3, 2, 72), (2, 3, 200)]
B0 = np.array([0.0, 0.02, 0.05])


def _fields(shape, seed):
    u, B = turbulence(shape, seed, 0.05, shells=(1, 2))
    return u, B + B0[:, None, None, None]


def _check_vs_oracle(shape, fg, mg, fo, mo, tol):
    b0 = B0[:, None, None, None]
    rest = rest_populations(shape, 1.0, tuple(B0))
    errs = dict(u=rel_l2(mg["u"], mo["u"]), B=rel_l2(mg["B"] - b0, mo["B"] - b0), J=rel_l2(mg["J"], mo["J"]),
                rho=float(np.abs(mg["rho"] - mo["rho"]).max()), fluid=rel_dev_err(fg, fo, rest, slice(0, 27)),
                mag=rel_dev_err(fg, fo, rest, slice(27, 48)), slot=float(slot_dev_errs(fg, fo, rest).max()))
    for k, e in errs.items():
        t = tol["J_thin"] if (k == "J" and _thin(shape)) else tol[k]
        assert e < t, (k, e, t)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_row_kernel_vs_oracle(shape, storage):
    """21 steps (ending on an odd-parity state) of Hall turbulence with a mean
    field against the FP64 oracle: per field (u, B and J fluctuations,
    density), per population group (fluid, magnetic) and for the worst single
    population slot, at the TOL bounds above."""
    u, B = _fields(shape, 41)
    fg, mg, fo, mo = run_both(shape, 0.52, 0.55, 1.5, u, B, 21, storage=storage, literal=False, Bref=tuple(B0),
                              kernel="row")
    _check_vs_oracle(shape, fg, mg, fo, mo, TOL[storage])


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("storage,ulps,steps", [("fp16", 2.0 ** -11, 51), ("bf16", 2.0 ** -8, 101)])
def test_row_kernel_agrees_with_site_kernel(shape, storage, ulps, steps):
    """Same fields, 51 (FP16) or 101 (BF16) steps, kernel "row" vs "site": both compute the collision in FP32 in a different order, so
    the stored deviations differ by a few units of the storage's last place --
    and do differ somewhere, which shows that the row kernel ran (BF16's
    8-bit significand absorbs most ordering differences: on the single-row
    lattice the two runs first differ after 51 steps).  The largest
    difference measured on GB300 is 4.2 units (FP16, 51 steps) and 3.3 (BF16,
    101 steps), so the two evaluate the same step; the bound is 12 units."""
    from paper_2212_11024_gb300 import Flame
    nz, ny, nx = shape
    u, B = _fields(shape, 43)
    pops = []
    for kernel in ("row", "site"):
        sim = Flame(nx, ny, nz, 0.52, 0.55, 1.5, storage=storage, B_ref=tuple(B0), kernel=kernel)
        sim.init(None, u, B)
        sim.step(steps)
        pops.append(sim.populations().cpu().numpy())
        sim.close()
    a, b = pops
    dev = np.abs(b - np.median(b, axis=(1, 2, 3), keepdims=True)).max()
    d = np.abs(a - b)
    assert d.max() < 12 * ulps * dev, d.max() / dev
    assert (d > 0).any()


def test_row_kernel_graph_replay_is_bit_identical():
    """graph_steps replays of the row kernel equal single launches."""
    import torch
    from paper_2212_11024_gb300 import Flame
    shape = (4, 3, 128)
    nz, ny, nx = shape
    u, B = _fields(shape, 45)
    a = Flame(nx, ny, nz, 0.52, 0.55, 1.5, storage="fp16", B_ref=tuple(B0))
    b = Flame(nx, ny, nz, 0.52, 0.55, 1.5, storage="fp16", B_ref=tuple(B0), graph_steps=8)
    for s in (a, b):
        s.init(None, u, B)
    for n in (3, 37, 20):
        a.step(n)
        b.step(n)
    assert torch.equal(a.populations(), b.populations())
    assert a.sync() is None and b.sync() is None
    a.close()
    b.close()


# one lattice per pipeline kind: 64 (two stages, refill inside the
# collision), 256 (three stages, in-place TMA stores), 512 and 960 (two
# stages, direct stores; compile-time and general row length)
@pytest.mark.parametrize("shape,storage", [((4, 3, 64), "fp16"), ((2, 3, 256), "bf16"), ((2, 3, 512), "fp16"),
                                           ((2, 1, 960), "bf16"), ((1, 2, 328), "fp16"), ((2, 2, 72), "bf16"),
                                           ((2, 2, 200), "fp16")])
def test_wait_limit_on_every_pipeline(shape, storage, variant="flame"):
    """A stalled step (barriers armed, copies never issued, 256 polls) on
    each pipeline of the row kernel reports FLAME_ERR_TIMEOUT, leaves the
    state and step count as they were, and the next step is normal."""
    import torch
    from paper_2212_11024_gb300 import Flame, FlameError
    from paper_2212_11024_gb300.flame import FLAME_ERR_TIMEOUT
    nz, ny, nx = shape
    u, B = _fields(shape, 49)
    sim = Flame(nx, ny, nz, 0.52, 0.55, 1.5, storage=storage, B_ref=tuple(B0), variant=variant, kernel="row")
    ref = Flame(nx, ny, nz, 0.52, 0.55, 1.5, storage=storage, B_ref=tuple(B0), variant=variant, kernel="row")
    for s in (sim, ref):
        s.init(None, u, B)
        s.step(2)
    sim.debug_stall_next_step(256)
    with pytest.raises(FlameError) as e:
        sim.step(1)
    assert e.value.status == FLAME_ERR_TIMEOUT
    assert sim.info()["step"] == 2
    assert torch.equal(sim.get_state()[0], ref.get_state()[0])
    sim.close()
    ref.step(1)
    assert ref.sync() is None
    ref.close()


@pytest.mark.parametrize("variant,shape", [("bgk", (2, 3, 256)), ("fd_current", (2, 3, 512)), ("emhd", (4, 3, 64))])
def test_wait_limit_for_the_variants(variant, shape):
    """The same for the scheme variants (the finite-difference current's
    stalled step reads no B field: its waits end before the collision)."""
    test_wait_limit_on_every_pipeline(shape, "fp16", variant)


def test_row_kernel_wait_limit_reports_timeout():
    """The row kernel's bounded waits: a step whose barriers are armed but
    never fed gives FLAME_ERR_TIMEOUT after the poll limit, leaves the state
    and the step count unchanged, and the GPU stays usable (a fresh context
    steps and matches a reference run bit for bit)."""
    import torch
    from paper_2212_11024_gb300 import Flame, FlameError
    from paper_2212_11024_gb300.flame import FLAME_ERR_TIMEOUT, FLAME_ERR_PARAM
    shape = (4, 3, 64)
    nz, ny, nx = shape
    u, B = _fields(shape, 47)
    sim = Flame(nx, ny, nz, 0.52, 0.55, 1.5, storage="fp16", B_ref=tuple(B0))
    sim.init(None, u, B)
    sim.step(3)
    blob0, step0, par0 = sim.get_state()
    sim.debug_stall_next_step(256)
    with pytest.raises(FlameError) as e:
        sim.step(1)
    assert e.value.status == FLAME_ERR_TIMEOUT
    blob1 = torch.empty_like(blob0)
    import ctypes
    from paper_2212_11024_gb300.flame import library
    st, pa = ctypes.c_longlong(), ctypes.c_int()
    library().flame_get_state(sim._ctx, ctypes.c_void_p(blob1.data_ptr()), ctypes.byref(st), ctypes.byref(pa))
    torch.cuda.synchronize()
    assert torch.equal(blob0, blob1) and st.value == step0 and pa.value == par0
    sim.close()
    # the site kernel has no such waits: the hook refuses
    site = Flame(nx, ny, nz, 0.52, 0.55, 1.5, storage="fp16", B_ref=tuple(B0), kernel="site")
    site.init(None, u, B)
    with pytest.raises(FlameError) as e:
        site.debug_stall_next_step(256)
    assert e.value.status == FLAME_ERR_PARAM
    site.close()
    # a fresh context on the same GPU works: 4 steps equal 3 + 1 restarted
    a = Flame(nx, ny, nz, 0.52, 0.55, 1.5, storage="fp16", B_ref=tuple(B0))
    a.init(None, u, B)
    a.step(4)
    b = Flame(nx, ny, nz, 0.52, 0.55, 1.5, storage="fp16", B_ref=tuple(B0))
    b.init(None, u, B)
    b.set_state(blob0, step0, par0)
    b.step(1)
    assert torch.equal(a.populations(), b.populations())
    a.close()
    b.close()


# the variants on compile-time (64, 256) and general (192, 960: bulk row
# copies) row lengths, including a single-row lattice
VARIANT_SHAPES = [(6, 5, 64), (3, 4, 192), (2, 3, 256), (2, 1, 960), (1, 1, 64), (2, 1, 456), (2, 2, 136)]


def _variant_run(shape, storage, kernel, variant, steps, seed):
    from paper_2212_11024_gb300 import Flame
    nz, ny, nx = shape
    u, B = _fields(shape, seed)
    sim = Flame(nx, ny, nz, 0.52, 0.55, 1.5, storage=storage, B_ref=tuple(B0), kernel=kernel, variant=variant)
    sim.init(None, u, B)
    sim.step(steps)
    f = sim.populations().cpu().numpy()
    m = {k: v.cpu().numpy() for k, v in sim.moments().items()}
    assert sim.sync() is None
    sim.close()
    return u, B, f, m


@pytest.mark.parametrize("shape", VARIANT_SHAPES)
@pytest.mark.parametrize("variant", ["bgk", "emhd", "fd_current"])
@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_row_kernel_variants_vs_oracle(shape, variant, storage):
    """21 steps of each variant with 16-bit storage on the row kernel against
    the oracle's variant, field by field, per population group and slot, at
    the TOL_VARIANT bounds above."""
    nz, ny, nx = shape
    u, B, fg, mg = _variant_run(shape, storage, "row", variant, 21, 51)
    p = O.Params(nx, ny, nz, 0.52, 0.55, 1.5)
    fo = O.init(p, None, u, B)
    O.step_variant(p, fo, 21, variant, literal=False)
    mo = O.moments(p, fo)
    _check_vs_oracle(shape, fg, mg, fo, mo, TOL_VARIANT[storage])


@pytest.mark.parametrize("shape", VARIANT_SHAPES)
@pytest.mark.parametrize("variant", ["bgk", "emhd", "fd_current"])
def test_row_kernel_variants_agree_with_site_kernel(shape, variant):
    """FP16, 51 steps of each variant, row kernel vs one-site kernel: at most
    12 half-precision units of the last place apart (4.2 measured on GB300),
    and apart somewhere (the row kernel ran)."""
    pops = [_variant_run(shape, "fp16", kernel, variant, 51, 53)[2] for kernel in ("row", "site")]
    a, b = pops
    dev = np.abs(b - np.median(b, axis=(1, 2, 3), keepdims=True)).max()
    d = np.abs(a - b)
    assert d.max() < 12 * 2.0 ** -11 * dev, d.max() / dev
    assert (d > 0).any()


@pytest.mark.parametrize("variant", ["bgk", "emhd", "fd_current"])
def test_row_kernel_variant_graph_replay_is_bit_identical(variant):
    """Graph replays of a variant's row-kernel steps (with the B pre-pass of
    the finite-difference current in the graph) equal single launches."""
    import torch
    from paper_2212_11024_gb300 import Flame
    shape = (4, 3, 128)
    nz, ny, nx = shape
    u, B = _fields(shape, 55)
    a = Flame(nx, ny, nz, 0.52, 0.55, 1.5, storage="bf16", B_ref=tuple(B0), variant=variant)
    b = Flame(nx, ny, nz, 0.52, 0.55, 1.5, storage="bf16", B_ref=tuple(B0), variant=variant, graph_steps=8)
    for s in (a, b):
        s.init(None, u, B)
    for n in (5, 19):
        a.step(n)
        b.step(n)
    assert torch.equal(a.populations(), b.populations())
    assert a.sync() is None and b.sync() is None


# Half rows per tile (kernel "row_half", rows longer than 256 sites): the
# segment's halos replace the whole row's wrap-around, the results go
# straight to HBM; the per-site arithmetic is the same, so the populations
# must equal the whole-row tiling's bit for bit.
HALF_SHAPES = [(2, 3, 320), (2, 2, 512), (1, 2, 576), (2, 1, 640), (1, 1, 960), (2, 1, 1024), (1, 2, 400),
               (2, 1, 528)]


@pytest.mark.parametrize("shape", HALF_SHAPES)
@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_half_rows_equal_whole_rows(shape, storage):
    import torch
    from paper_2212_11024_gb300 import Flame
    nz, ny, nx = shape
    u, B = _fields(shape, 57)
    sims = [Flame(nx, ny, nz, 0.52, 0.55, 1.5, storage=storage, B_ref=tuple(B0), kernel=k)
            for k in ("row", "row_half")]
    for s in sims:
        s.init(None, u, B)
    for n in (3, 4):  # an odd step count, then an even one
        for s in sims:
            s.step(n)
        assert torch.equal(sims[0].populations(), sims[1].populations())
    for s in sims:
        assert s.sync() is None
        s.close()


@pytest.mark.parametrize("variant", ["bgk", "emhd", "fd_current"])
def test_half_rows_equal_whole_rows_variants(variant):
    import torch
    from paper_2212_11024_gb300 import Flame
    shape = (2, 3, 512)
    nz, ny, nx = shape
    u, B = _fields(shape, 59)
    sims = [Flame(nx, ny, nz, 0.52, 0.55, 1.5, storage="fp16", B_ref=tuple(B0), kernel=k, variant=variant)
            for k in ("row", "row_half")]
    for s in sims:
        s.init(None, u, B)
        s.step(7)
    assert torch.equal(sims[0].populations(), sims[1].populations())
    for s in sims:
        s.close()


@pytest.mark.parametrize("shape", [(1, 2, 576), (2, 1, 640), (1, 2, 560)])
def test_half_rows_vs_oracle(shape):
    """The row lengths where whole rows leave too few warps per SM, on half
    rows, against the oracle at the row kernel's FP16 bounds."""
    u, B = _fields(shape, 41)
    fg, mg, fo, mo = run_both(shape, 0.52, 0.55, 1.5, u, B, 21, storage="fp16", literal=False, Bref=tuple(B0),
                              kernel="row_half")
    _check_vs_oracle(shape, fg, mg, fo, mo, TOL["fp16"])


@pytest.mark.parametrize("shape", [(2, 2, 512), (1, 2, 576)])
def test_wait_limit_on_half_rows(shape):
    """The bounded waits of the half-row pipeline: a stalled step reports
    FLAME_ERR_TIMEOUT and leaves the state as it was."""
    import torch
    from paper_2212_11024_gb300 import Flame, FlameError
    from paper_2212_11024_gb300.flame import FLAME_ERR_TIMEOUT
    nz, ny, nx = shape
    u, B = _fields(shape, 61)
    sim = Flame(nx, ny, nz, 0.52, 0.55, 1.5, storage="fp16", B_ref=tuple(B0), kernel="row_half")
    sim.init(None, u, B)
    sim.step(3)
    blob0 = sim.get_state()[0]
    sim.debug_stall_next_step(256)
    with pytest.raises(FlameError) as e:
        sim.step(1)
    assert e.value.status == FLAME_ERR_TIMEOUT
    import ctypes
    from paper_2212_11024_gb300.flame import library
    blob1 = torch.empty_like(blob0)
    st, pa = ctypes.c_longlong(), ctypes.c_int()
    library().flame_get_state(sim._ctx, ctypes.c_void_p(blob1.data_ptr()), ctypes.byref(st), ctypes.byref(pa))
    torch.cuda.synchronize()
    assert torch.equal(blob0, blob1) and st.value == 3
    sim.close()


@pytest.mark.parametrize("nx,expect", [(456, "row"), (544, "pair"), (608, "row_half"), (100, "pair"), (1000, "row"),
                                        (33, "site")])
def test_automatic_choice_between_the_tilings(nx, expect):
    """kernel "auto" is the tiling timed fastest at each row length (whole
    rows at most multiples of 8 in 64..1024, half rows at 608-640, the
    unstaged pair kernel at every other even length, the one-site kernel at
    odd ones).  The row kernel's tilings and the pair kernel agree bit for
    bit and differ from the one-site kernel, so auto equals the expected
    kernel bit for bit and differs from the other kind."""
    import torch
    from paper_2212_11024_gb300 import Flame
    shape = (2, 1, nx)
    nz, ny, _ = shape
    u, B = _fields(shape, 63)
    # at an odd row length no packed kernel applies: auto is the one-site kernel
    other = "site" if expect != "site" else None
    pops = {}
    for k in ("auto", expect) + ((other,) if other else ()):
        sim = Flame(nx, ny, nz, 0.52, 0.55, 1.5, storage="fp16", B_ref=tuple(B0), kernel=k)
        sim.init(None, u, B)
        sim.step(21)
        pops[k] = sim.populations()
        assert sim.sync() is None
        sim.close()
    assert torch.equal(pops["auto"], pops[expect])
    if other:
        assert not torch.equal(pops["auto"], pops[other])


# The pair kernel: the row kernel's collision on site pairs loaded and
# stored straight from HBM (any even row length).
@pytest.mark.parametrize("shape", [(2, 3, 136), (1, 2, 256), (1, 2, 552), (2, 1, 1000)])
@pytest.mark.parametrize("storage", ["fp16", "bf16"])
@pytest.mark.parametrize("variant", ["flame", "fd_current"])
def test_pair_kernel_equals_staged_rows(shape, storage, variant):
    """Where the staged row kernel also applies, the pair kernel's
    populations equal it bit for bit after an odd and an even step count."""
    import torch
    from paper_2212_11024_gb300 import Flame
    nz, ny, nx = shape
    u, B = _fields(shape, 65)
    sims = [Flame(nx, ny, nz, 0.52, 0.55, 1.5, storage=storage, B_ref=tuple(B0), kernel=k, variant=variant)
            for k in ("row", "pair")]
    for s in sims:
        s.init(None, u, B)
    for n in (3, 4):
        for s in sims:
            s.step(n)
        assert torch.equal(sims[0].populations(), sims[1].populations())
    for s in sims:
        assert s.sync() is None
        s.close()


# row lengths only the pair kernel takes: below 64, not a multiple of 8, a
# single pair per row (the wrap at both ends of a two-site row)
PAIR_SHAPES = [(3, 2, 34), (2, 3, 100), (4, 3, 2), (1, 1, 70)]


@pytest.mark.parametrize("shape", PAIR_SHAPES)
@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_pair_kernel_vs_oracle(shape, storage):
    """21 steps on the pair kernel against the FP64 oracle at the row
    kernel's TOL bounds."""
    u, B = _fields(shape, 67)
    fg, mg, fo, mo = run_both(shape, 0.52, 0.55, 1.5, u, B, 21, storage=storage, literal=False, Bref=tuple(B0),
                              kernel="pair")
    _check_vs_oracle(shape, fg, mg, fo, mo, TOL[storage])


@pytest.mark.parametrize("variant", ["bgk", "emhd", "fd_current"])
def test_pair_kernel_variants_vs_oracle(variant):
    shape = (2, 3, 34)
    nz, ny, nx = shape
    u, B, fg, mg = _variant_run(shape, "fp16", "pair", variant, 21, 69)
    p = O.Params(nx, ny, nz, 0.52, 0.55, 1.5)
    fo = O.init(p, None, u, B)
    O.step_variant(p, fo, 21, variant, literal=False)
    mo = O.moments(p, fo)
    _check_vs_oracle(shape, fg, mg, fo, mo, TOL_VARIANT["fp16"])


@pytest.mark.parametrize("shape", [(2, 3, 100), (3, 2, 34)])
def test_pair_kernel_agrees_with_site_kernel(shape):
    """FP16, 51 steps, pair kernel vs one-site kernel: at most 12 units of the
    last place apart, and apart somewhere; the pair kernel has no staged
    copies, so there is no wait to stall (FLAME_ERR_PARAM)."""
    from paper_2212_11024_gb300 import Flame, FlameError
    from paper_2212_11024_gb300.flame import FLAME_ERR_PARAM
    nz, ny, nx = shape
    u, B = _fields(shape, 71)
    pops = []
    for kernel in ("pair", "site"):
        sim = Flame(nx, ny, nz, 0.52, 0.55, 1.5, storage="fp16", B_ref=tuple(B0), kernel=kernel)
        sim.init(None, u, B)
        sim.step(51)
        pops.append(sim.populations().cpu().numpy())
        if kernel == "pair":
            with pytest.raises(FlameError) as e:
                sim.debug_stall_next_step(256)
            assert e.value.status == FLAME_ERR_PARAM
        sim.close()
    a, b = pops
    dev = np.abs(b - np.median(b, axis=(1, 2, 3), keepdims=True)).max()
    d = np.abs(a - b)
    assert d.max() < 12 * 2.0 ** -11 * dev, d.max() / dev
    assert (d > 0).any()
