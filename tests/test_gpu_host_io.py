"""The host-buffer calls (flame_init_f32_host, flame_moments_f32_host) move
the fields in chunks of z planes on a second stream, overlapped with the
chunks' kernels; the per-site arithmetic is that of flame_init_f32 and
flame_moments_f32, so the state and the fields must equal theirs bit for bit
on the same FP32 fields: for fewer z planes than chunks, a plane count the
chunks do not divide, and more planes than chunks; from page-locked and from
pageable host memory; for a z-slab context (fields with ghost planes); and
the scalars must equal flame_reduce's."""
import ctypes

import numpy as np
import pytest
import torch

from gpu_helpers import turbulence

pytestmark = pytest.mark.gpu

B0 = np.array([0.0, 0.03, 0.06])
SHAPES = [(5, 8, 16), (37, 12, 40), (70, 6, 64)]  # (nz, ny, nx): nz below, between and above the chunk limit


def _fields32(shape, seed):
    u, B = turbulence(shape, seed, 0.05, shells=(1, 2))
    return u.astype(np.float32), (B + B0[:, None, None, None]).astype(np.float32)


def _flame(shape, storage, **kw):
    from paper_2212_11024_gb300 import Flame
    nz, ny, nx = shape
    return Flame(nx, ny, nz, 0.53, 0.56, 1.2, storage=storage, B_ref=tuple(B0), **kw)


def _host(a, pinned):
    return torch.from_numpy(a).pin_memory() if pinned else np.ascontiguousarray(a)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("pinned", [True, False])
def test_init_host_equals_device_init(shape, storage, pinned):
    u, B = _fields32(shape, 71)
    rho = (1.0 + 0.01 * np.cos(np.arange(np.prod(shape)) * 0.37).reshape(shape)).astype(np.float32)
    a, b = _flame(shape, storage), _flame(shape, storage)
    try:
        a.init(torch.from_numpy(rho), torch.from_numpy(u), torch.from_numpy(B))  # FP32 fields: flame_init_f32
        b.init_host(_host(rho, pinned), _host(u, pinned), _host(B, pinned))
        sa, sb = a.get_state()[0], b.get_state()[0]
        assert torch.equal(sa, sb)
        assert a.info()["max_speed"] == b.info()["max_speed"]
        # rho omitted: rho = 1 on both paths
        a.init(None, torch.from_numpy(u), torch.from_numpy(B))
        b.init_host(None, _host(u, pinned), _host(B, pinned))
        assert torch.equal(a.get_state()[0], b.get_state()[0])
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("steps", [3, 4])
def test_moments_host_equals_device_moments(shape, storage, steps):
    u, B = _fields32(shape, 72)
    sim = _flame(shape, storage)
    try:
        sim.init_host(None, _host(u, True), _host(B, True))
        sim.step(steps)
        dev = sim.moments(dtype=torch.float32)
        ref = sim.reduce()
        out, scal = sim.moments_host(scalars=True)
        for k in ("rho", "u", "B", "J"):
            assert torch.equal(out[k], dev[k].cpu()), k
        assert scal["status"] == ref["status"] == 0
        for k, v in ref.items():
            assert scal[k] == v, k
        # some fields only, into pageable numpy arrays
        part = {"u": np.full((3,) + shape, np.nan, np.float32), "J": np.full((3,) + shape, np.nan, np.float32)}
        assert sim.moments_host(out=part) is part
        assert np.array_equal(part["u"], dev["u"].cpu().numpy())
        assert np.array_equal(part["J"], dev["J"].cpu().numpy())
    finally:
        sim.close()


@pytest.mark.parametrize("pinned", [True, False])
def test_host_io_with_fields_in_one_array(pinned):
    """Fields the caller keeps in one host array (adjacent in memory) move in
    one copy per chunk: the same results as separate arrays."""
    shape = (37, 12, 40)
    u, B = _fields32(shape, 75)
    rho = (1.0 + 0.02 * np.sin(np.arange(np.prod(shape)) * 0.11).reshape(shape)).astype(np.float32)
    a, b = _flame(shape, "fp16"), _flame(shape, "fp16")
    try:
        inp = np.concatenate([u, B, rho[None]])  # u, B, rho: the workspace's order
        inp = torch.from_numpy(inp).pin_memory() if pinned else inp
        a.init_host(_host(rho, True), _host(u, True), _host(B, True))
        b.init_host(inp[6], inp[0:3], inp[3:6])
        assert torch.equal(a.get_state()[0], b.get_state()[0])
        a.step(3)
        ref = a.moments_host()
        buf = torch.full((10,) + shape, float("nan"), dtype=torch.float32)
        buf = buf.pin_memory() if pinned else buf.numpy()
        out = a.moments_host(out={"rho": buf[0], "u": buf[1:4], "B": buf[4:7], "J": buf[7:10]})
        for k in ("rho", "u", "B", "J"):
            assert np.array_equal(np.asarray(out[k]), ref[k].numpy()), k
        # B left out: u and J are then adjacent in the workspace as in buf
        buf2 = np.full((6,) + shape, np.nan, np.float32)
        out2 = a.moments_host(out={"u": buf2[0:3], "J": buf2[3:6]})
        assert np.array_equal(out2["u"], ref["u"].numpy()) and np.array_equal(out2["J"], ref["J"].numpy())
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_host_io_of_a_slab(storage):
    """A z-slab (planes 9..20 of a 33-plane lattice, ghost planes 8 and 21):
    its initial fields with the ghost planes, its moments of the 12 updated
    planes."""
    nz, ny, nx = 33, 6, 24
    u, B = _fields32((nz, ny, nx), 73)
    z = np.arange(8, 22)
    us, Bs = np.ascontiguousarray(u[:, z]), np.ascontiguousarray(B[:, z])
    a = _flame((12, ny, nx), storage, halo_z=True)
    b = _flame((12, ny, nx), storage, halo_z=True)
    try:
        a.init(None, torch.from_numpy(us), torch.from_numpy(Bs))
        b.init_host(None, _host(us, True), _host(Bs, False))
        # the updated planes 1..12 of the 14 held (the ghost planes are
        # written by the halo exchange, not by the initialisation)
        es = 4 if storage == "fp32" else 2
        sa = a.get_state()[0].view(48, 14, ny, nx * es)[:, 1:13]
        sb = b.get_state()[0].view(48, 14, ny, nx * es)[:, 1:13]
        assert torch.equal(sa, sb)
        dev = a.moments(dtype=torch.float32)
        out = b.moments_host()
        for k in ("rho", "u", "B", "J"):
            assert tuple(out[k].shape)[-3:] == (12, ny, nx)
            assert torch.equal(out[k], dev[k].cpu()), k
    finally:
        a.close()
        b.close()


def test_host_io_errors():
    from paper_2212_11024_gb300 import Flame
    from paper_2212_11024_gb300 import flame as F
    lib = F.library()
    shape = (6, 4, 8)
    u, B = _fields32(shape, 74)
    sim = _flame(shape, "fp32")
    fields = Flame(8, 4, 6, 0.53, 0.56, 1.2, fields_only=True)
    try:
        # moments before any initial state
        assert lib.flame_moments_f32_host(sim._ctx, None, None, None, None, None) == F.FLAME_ERR_STATE
        hu, hB = np.ascontiguousarray(u), np.ascontiguousarray(B)
        assert lib.flame_init_f32_host(sim._ctx, None, None, ctypes.c_void_p(hB.ctypes.data)) == F.FLAME_ERR_PARAM
        assert lib.flame_init_f32_host(sim._ctx, None, ctypes.c_void_p(hu.ctypes.data), None) == F.FLAME_ERR_PARAM
        assert lib.flame_init_f32_host(None, None, ctypes.c_void_p(hu.ctypes.data),
                                       ctypes.c_void_p(hB.ctypes.data)) == F.FLAME_ERR_PARAM
        # a context without a population state
        assert lib.flame_init_f32_host(fields._ctx, None, ctypes.c_void_p(hu.ctypes.data),
                                       ctypes.c_void_p(hB.ctypes.data)) == F.FLAME_ERR_STATE
        # the binding checks type, layout and shape before the call
        with pytest.raises(ValueError):
            sim.init_host(None, u.astype(np.float64), B)
        with pytest.raises(ValueError):
            sim.init_host(None, u[:, :, :, :4], B)
        with pytest.raises(ValueError):
            sim.init_host(None, np.asfortranarray(u), B)
        sim.init_host(None, hu, hB)
        with pytest.raises(ValueError):
            sim.moments_host(out={"u": np.empty((3, 6, 4, 7), np.float32)})
        # all outputs NULL: nothing to copy, still a valid call
        assert lib.flame_moments_f32_host(sim._ctx, None, None, None, None, None) == F.FLAME_OK
    finally:
        sim.close()
        fields.close()
