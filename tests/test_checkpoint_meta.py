"""Checkpoint metadata (host logic, no GPU): what a checkpoint records and
which differences refuse a resume."""
import numpy as np

from paper_2212_11024_gb300.flame import checkpoint_meta, checkpoint_mismatches, make_params


def _roundtrip(meta, tmp_path):
    path = tmp_path / "meta.npz"
    np.savez(path, **{"meta_" + k: np.asarray(v) for k, v in meta.items()})
    with np.load(path) as z:
        return {k[5:]: z[k] for k in z.files if k.startswith("meta_")}


def test_identical_parameters_resume(tmp_path):
    p = make_params(64, 32, 16, 0.55, 0.6, 3.2, storage="fp16", B_ref=(0.0, 0.02, 0.1), variant="bgk")
    saved = _roundtrip(checkpoint_meta(p), tmp_path)
    assert checkpoint_mismatches(saved, p) == []


def test_layout_differences_always_refuse(tmp_path):
    p = make_params(64, 32, 16, 0.55, 0.6, 3.2, storage="fp16", B_ref=(0.0, 0.02, 0.1))
    saved = _roundtrip(checkpoint_meta(p), tmp_path)
    for other, name in ((make_params(32, 64, 16, 0.55, 0.6, 3.2, storage="fp16", B_ref=(0.0, 0.02, 0.1)), "nx"),
                        (make_params(64, 32, 16, 0.55, 0.6, 3.2, storage="bf16", B_ref=(0.0, 0.02, 0.1)), "storage"),
                        (make_params(64, 32, 16, 0.55, 0.6, 3.2, storage="fp16", B_ref=(0.0, 0.0, 0.1)), "B_ref"),
                        (make_params(64, 32, 16, 0.55, 0.6, 3.2, storage="fp16", rho0=1.1, B_ref=(0.0, 0.02, 0.1)),
                         "rho0")):
        assert name in checkpoint_mismatches(saved, other)
        assert name in checkpoint_mismatches(saved, other, same_physics=False)


def test_physics_differences_refuse_unless_allowed(tmp_path):
    p = make_params(64, 32, 16, 0.55, 0.6, 3.2, storage="fp16")
    saved = _roundtrip(checkpoint_meta(p), tmp_path)
    q = make_params(64, 32, 16, 0.55, 0.6, 6.4, storage="fp16", variant="emhd")
    assert checkpoint_mismatches(saved, q) == ["d_i", "variant"]
    assert checkpoint_mismatches(saved, q, same_physics=False) == []
