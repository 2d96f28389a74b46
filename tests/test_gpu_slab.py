"""The lattice split into z-slabs on one GPU (SlabGroup: halo_z contexts,
flame_halo_exchange after every step) against the same lattice in one
context: the per-site arithmetic is the same, so the populations, moments
and the combined diagnostics must agree bit for bit (the diagnostics to
FP64 summation order), for both kernels, every storage type and the
variants a slab supports; and against the FP64 oracle at the FP32
tolerance of the single-context tests."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from gpu_helpers import rel_dev_err, rest_populations, turbulence

pytestmark = pytest.mark.gpu

B0 = np.array([0.0, 0.02, 0.05])


def _fields(shape, seed):
    u, B = turbulence(shape, seed, 0.05, shells=(1, 2))
    return u, B + B0[:, None, None, None]


def _pair(shape, nslabs, storage, variant="flame", kernel="auto"):
    from paper_2212_11024_gb300 import Flame
    from paper_2212_11024_gb300.slab import SlabGroup
    nz, ny, nx = shape
    kw = dict(storage=storage, B_ref=tuple(B0), variant=variant, kernel=kernel)
    return Flame(nx, ny, nz, 0.52, 0.55, 1.5, **kw), SlabGroup(nx, ny, nz, nslabs, 0.52, 0.55, 1.5, **kw)


@pytest.mark.parametrize("shape,nslabs", [((6, 5, 40), 1), ((6, 5, 40), 2), ((7, 4, 33), 3), ((3, 4, 24), 3)])
@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_slabs_equal_one_context_site_kernel(shape, nslabs, storage):
    """One-site kernel (FP32, and FP16 forced onto it): 1, 2 and 3 slabs,
    down to one plane per slab; equal after an odd and an even step count."""
    u, B = _fields(shape, 61)
    one, grp = _pair(shape, nslabs, storage, kernel="site")
    one.init(None, u, B)
    grp.init(None, u, B)
    for n in (7, 4):
        one.step(n)
        grp.step(n)
        assert torch.equal(one.populations(), grp.populations())
    m1, m2 = one.moments(), grp.moments()
    assert all(torch.equal(m1[k], m2[k]) for k in m1)
    grp.sync()
    one.close()
    grp.close()


@pytest.mark.parametrize("shape,nslabs", [((6, 5, 64), 2), ((5, 3, 128), 3), ((4, 2, 256), 4), ((5, 3, 40), 2),
                                          ((4, 2, 136), 3)])
@pytest.mark.parametrize("storage", ["fp16", "bf16"])
@pytest.mark.parametrize("variant", ["flame", "bgk", "emhd"])
def test_slabs_equal_one_context_row_kernel(shape, nslabs, storage, variant):
    """The row kernel on slabs (TMA-staged rows at 64, 128 and 256 sites, the
    unstaged pair kernel at 40 and 136): tiles or pairs only over the slab's
    planes, odd-step rows read from the ghost planes."""
    u, B = _fields(shape, 63)
    one, grp = _pair(shape, nslabs, storage, variant)
    one.init(None, u, B)
    grp.init(None, u, B)
    for n in (5, 6):
        one.step(n)
        grp.step(n)
        assert torch.equal(one.populations(), grp.populations())
    one.close()
    grp.close()


def test_slab_diagnostics_combine():
    """reduce() of the split lattice (the slabs' FP64 sums added and
    combined) against the single context: FP64 summation-order agreement."""
    shape = (8, 6, 64)
    u, B = _fields(shape, 65)
    one, grp = _pair(shape, 3, "fp16")
    one.init(None, u, B)
    grp.init(None, u, B)
    one.step(5)
    grp.step(5)
    a, b = one.reduce(), grp.reduce()
    for k in ("mass", "E_u", "E_B", "J2", "divB_rms"):
        assert abs(a[k] - b[k]) <= 1e-12 * abs(a[k]), k
    for k in ("mom_x", "mom_y", "mom_z"):
        assert abs(a[k] - b[k]) <= 1e-13 * a["mass"] * a["u_max"], k
    for k in ("B_x", "B_y", "B_z", "H_c"):
        assert abs(a[k] - b[k]) <= 1e-13, k
    assert a["u_max"] == b["u_max"] and a["nonfinite"] == b["nonfinite"] == 0
    one.close()
    grp.close()


def test_slabs_match_the_oracle():
    """Three slabs, FP32, 12 steps against the FP64 oracle at the
    single-context tolerance (1e-6 of the populations' dynamic part)."""
    from paper_2212_11024_gb300.slab import SlabGroup
    shape = (6, 5, 20)
    nz, ny, nx = shape
    u, B = _fields(shape, 67)
    grp = SlabGroup(nx, ny, nz, 3, 0.56, 0.61, 1.4, storage="fp32", B_ref=tuple(B0))
    grp.init(None, u, B)
    grp.step(12)
    fg = grp.populations().cpu().numpy()
    grp.close()
    p = O.Params(nx, ny, nz, 0.56, 0.61, 1.4)
    fo = O.init(p, None, u, B)
    O.step(p, fo, 12, literal=False)
    rest = rest_populations(shape, 1.0, tuple(B0))
    assert rel_dev_err(fg, fo, rest, slice(0, 27)) < 1e-6
    assert rel_dev_err(fg, fo, rest, slice(27, 48)) < 1e-6


def test_slab_fft_diagnostics_equal_one_context():
    """Spectra, the energy budget and a band energy of the split lattice (the
    slabs' u and B assembled and evaluated by a context without state)
    against the single context's own (its state's u and B): the same FP64
    fields through the same FFT code."""
    shape = (9, 6, 16)
    u, B = _fields(shape, 71)
    one, grp = _pair(shape, 3, "fp16")
    one.init(None, u, B)
    grp.init(None, u, B)
    one.step(5)
    grp.step(5)
    Eu1, Eb1 = one.spectra(9)
    Eu2, Eb2 = grp.spectra(9)
    assert np.allclose(Eu1, Eu2, rtol=1e-12, atol=0) and np.allclose(Eb1, Eb2, rtol=1e-12, atol=0)
    assert Eb1[0] == 0.0 and Eb1[1] > 0.0  # the mean field is left out
    for a, b in zip(one.energy_budget(9), grp.energy_budget(9)):
        assert np.allclose(a, b, rtol=1e-12, atol=1e-13 * np.abs(a).max())
    L1, g1, _ = one.band_energy(1, 3, grad=True)
    L2, g2 = grp.band_energy(1, 3, grad=True)
    assert abs(L1 - L2) <= 1e-12 * L1
    assert torch.allclose(g1, g2, rtol=0, atol=1e-12 * float(g1.abs().max()))
    # the field form on an ordinary context equals its state form
    m = one.moments()
    Eu3, Eb3 = one.spectra(9, m["u"], m["B"])
    assert np.allclose(Eu1, Eu3, rtol=1e-12, atol=0) and np.allclose(Eb1, Eb3, rtol=1e-12, atol=0)
    one.close()
    grp.close()


def test_context_without_state():
    """flame_create_fields: the field diagnostics work, everything that needs
    a state answers FLAME_ERR_STATE, and a slab is refused."""
    from paper_2212_11024_gb300 import Flame, FlameError
    from paper_2212_11024_gb300.flame import FLAME_ERR_PARAM, FLAME_ERR_STATE, library, make_params
    shape = (4, 6, 8)
    nz, ny, nx = shape
    u, B = _fields(shape, 73)
    f = Flame(nx, ny, nz, 0.6, 0.6, 1.0, fields_only=True)
    lib = library()
    for call in (lambda: f.init(None, u, B), lambda: f.step(1), lambda: f.moments(), lambda: f.spectra(4),
                 lambda: f.energy_budget(4), lambda: f.band_energy(1, 2), lambda: f.get_state(),
                 lambda: f.reduce()):
        with pytest.raises(FlameError) as e:
            call()
        assert e.value.status == FLAME_ERR_STATE
    blob = torch.zeros(48 * nx * ny * nz * 4, dtype=torch.uint8, device="cuda")
    assert lib.flame_set_state(f._ctx, ctypes.c_void_p(blob.data_ptr()), 0, 0) == FLAME_ERR_STATE
    ut = torch.tensor(u, device="cuda")
    Bt = torch.tensor(B, device="cuda")
    from oracle import spectra as S
    Eu, Eb = f.spectra(5, ut, Bt)
    Eu_o = S.shell_spectrum(u, 5)
    Bm = B - B.reshape(3, -1).mean(1)[:, None, None, None]
    Eb_o = S.shell_spectrum(Bm, 5)
    assert np.allclose(Eu, Eu_o, rtol=1e-12, atol=1e-18) and np.allclose(Eb, Eb_o, rtol=1e-12, atol=1e-18)
    E, _, _ = f.energy_budget(5, ut, Bt)
    # the budget's E(n) keeps B's mean mode (shell 0)
    Eb_full = S.shell_spectrum(B, 5)
    assert np.allclose(E, Eu_o + Eb_full, rtol=1e-12, atol=1e-18)
    f.close()
    ctx = ctypes.c_void_p()
    p = make_params(nx, ny, nz, 0.6, 0.6, 1.0, halo_z=True)
    assert lib.flame_create_fields(ctypes.byref(ctx), ctypes.byref(p), None) == FLAME_ERR_PARAM


def test_slab_contexts_refuse_what_they_cannot_do():
    from paper_2212_11024_gb300 import Flame, FlameError
    from paper_2212_11024_gb300.flame import FLAME_ERR_PARAM, FLAME_ERR_STATE, library
    shape = (4, 4, 16)
    u, B = _fields(shape, 69)
    nz, ny, nx = shape
    with pytest.raises(FlameError):
        Flame(nx, ny, nz, 0.6, 0.6, 1.0, halo_z=True, variant="fd_current")
    from paper_2212_11024_gb300.slab import SlabGroup
    grp = SlabGroup(nx, ny, nz, 2, 0.6, 0.6, 1.0)
    grp.init(None, u, B)
    a, b = grp.slabs
    lib = library()
    h = (ctypes.c_double * 16)()
    assert lib.flame_spectra(a._ctx, 4, h, h) == FLAME_ERR_PARAM
    L = ctypes.c_double()
    assert lib.flame_band_energy(a._ctx, 1, 2, None, ctypes.byref(L), None, None) == FLAME_ERR_PARAM
    assert lib.flame_energy_budget(a._ctx, 4, None, None, h, h, h) == FLAME_ERR_PARAM
    periodic = Flame(nx, ny, nz, 0.6, 0.6, 1.0)
    periodic.init(None, u, B)
    assert lib.flame_halo_exchange(a._ctx, periodic._ctx) == FLAME_ERR_PARAM
    a.step(1)  # a at parity 1, b at parity 0
    assert lib.flame_halo_exchange(a._ctx, b._ctx) == FLAME_ERR_STATE
    b.step(1)
    a.halo_exchange(b)
    b.halo_exchange(a)
    grp.sync()
    periodic.close()
    grp.close()
