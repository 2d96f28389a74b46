"""Checkpoint and resume through a file: the resumed run continues bit for
bit, and a checkpoint of another lattice is refused."""
import numpy as np
import pytest

from gpu_helpers import turbulence

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage,shape", [("fp16", (4, 3, 128)), ("fp32", (3, 4, 10))])
def test_resume_from_file_is_bit_identical(storage, shape, tmp_path):
    import torch
    from paper_2212_11024_gb300 import Flame
    nz, ny, nx = shape
    u, B = turbulence(shape, 71, 0.04)
    path = tmp_path / "ck.npz"
    a = Flame(nx, ny, nz, 0.55, 0.6, 1.5, storage=storage)
    a.init(None, u, B)
    a.step(5)  # odd parity: the checkpoint records it
    a.save_checkpoint(path)
    a.step(7)
    b = Flame(nx, ny, nz, 0.55, 0.6, 1.5, storage=storage)
    b.load_checkpoint(path)
    assert b.info()["step"] == 5 and b.info()["parity"] == 1
    b.step(7)
    assert torch.equal(a.populations(), b.populations())
    a.close()
    b.close()
    c = Flame(nx, ny, nz, 0.55, 0.6, 3.0, storage=storage)
    with pytest.raises(ValueError, match="d_i"):
        c.load_checkpoint(path)
    c.load_checkpoint(path, same_physics=False)  # new d_i on the same state
    c.close()
    d = Flame(nx, ny + 1, nz, 0.55, 0.6, 1.5, storage=storage)
    with pytest.raises(ValueError, match="ny"):
        d.load_checkpoint(path)
    d.close()


def test_checkpoint_round_trip_on_non_default_streams(tmp_path):
    """A context created on its own stream orders its work against torch's
    current stream: the checkpoint saved while steps are still queued holds
    the state after those steps, and a context on a third stream resumes from
    it bit for bit (a 256^3-sized step keeps the library's stream busy while
    torch copies the blob to the host)."""
    import torch
    from paper_2212_11024_gb300 import Flame
    shape = (64, 64, 256)
    nz, ny, nx = shape
    u, B = turbulence(shape, 73, 0.04)
    path = tmp_path / "ck.npz"
    ref = Flame(nx, ny, nz, 0.55, 0.6, 1.5, storage="fp16")
    ref.init(None, u, B)
    ref.step(9)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    a = Flame(nx, ny, nz, 0.55, 0.6, 1.5, storage="fp16", stream=s1)
    a.init(None, u, B)
    a.step(9)               # queued on s1, not synchronised
    a.save_checkpoint(path)
    b = Flame(nx, ny, nz, 0.55, 0.6, 1.5, storage="fp16", stream=s2)
    b.load_checkpoint(path)
    assert torch.equal(b.populations(), ref.populations())
    for s in (ref, b):
        s.step(4)
    assert torch.equal(b.populations(), ref.populations())
    m_ref, m_b = ref.moments(), b.moments()
    assert all(torch.equal(m_ref[k], m_b[k]) for k in m_ref)
    for s in (ref, a, b):
        assert s.sync() is None
        s.close()
