"""Decaying-turbulence driver (Sec. 5) on the GPU against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from oracle import spectra as S

pytestmark = pytest.mark.gpu


def test_decay_records_match_oracle_and_conserve():
    """turbulence.decay at 24^3: records at 0, 40, 80, 120; the spectra at
    step 40 equal the oracle's after the same 40 steps; Parseval holds; mass
    is conserved; the total energy of the d_i = 0 run never grows."""
    from paper_2212_11024_gb300 import inputs, turbulence
    n = 24
    nshell = int(np.ceil(np.sqrt(3.0) * n / 2)) + 1
    u, B = inputs.turbulence((n, n, n), 31, 32, 0.02, 0.02, shells=(1, 3))
    r = turbulence.decay(n, 0.0, 120, spectra_every=40, storage="fp32", tau_nu=0.6, tau_eta=0.6, nshell=nshell,
                         fields=(u, B))
    assert r["first_nonfinite"] is None
    assert list(r["t"]) == [0, 40, 80, 120]
    assert r["Eu"].shape == (4, nshell) and r["Eb"].shape == (4, nshell)
    assert r["mlups"] > 0
    for j, sc in enumerate(r["scalars"]):
        assert abs(r["Eu"][j].sum() - sc["E_u"]) < 1e-6 * sc["E_u"]
        assert abs(r["Eb"][j].sum() - sc["E_B"]) < 1e-6 * sc["E_B"]
        assert abs(sc["mass"] - n ** 3) < 1e-9 * n ** 3
    tot = np.array([sc["E_u"] + sc["E_B"] for sc in r["scalars"]])
    assert np.all(np.diff(tot) < 0)
    p = O.Params(n, n, n, 0.6, 0.6, 0.0)
    pop = O.init(p, None, u, B)
    O.step(p, pop, 40, literal=False)
    m = O.moments(p, pop)
    Eu_ref = S.shell_spectrum(m["u"], nshell)
    Eb_ref = S.shell_spectrum(m["B"] - m["B"].reshape(3, -1).mean(axis=1)[:, None, None, None], nshell)
    for got, ref in ((r["Eu"][1], Eu_ref), (r["Eb"][1], Eb_ref)):
        big = ref > 1e-6 * ref.max()
        assert np.allclose(got[big], ref[big], rtol=2e-5)


def test_decay_hall_fp16_tracks_fp32():
    """A Hall run in FP16 storage records every chunk; its spectra stay close
    to the FP32 run of the same fields over the first 40 steps (resolved
    shells, relative 1e-2)."""
    from paper_2212_11024_gb300 import inputs, turbulence
    n = 32
    u, B = inputs.turbulence((n, n, n), 33, 34, 0.03, 0.03, shells=(1, 4))
    a = turbulence.decay(n, 0.05 * n, 80, spectra_every=40, storage="fp32", fields=(u, B))
    b = turbulence.decay(n, 0.05 * n, 80, spectra_every=40, storage="fp16", fields=(u, B))
    assert a["first_nonfinite"] is None and b["first_nonfinite"] is None
    for key in ("Eu", "Eb"):
        ref = a[key][1]
        big = ref > 1e-4 * ref.max()
        assert np.allclose(b[key][1][big], ref[big], rtol=1e-2), key


def test_step_throughput_reports_every_configuration():
    """The throughput helper times a variant on either kernel and reports a
    finite state."""
    from paper_2212_11024_gb300.throughput import step_throughput
    for variant, storage, kernel in (("bgk", "fp16", "auto"), ("fd_current", "bf16", "site"), ("emhd", "fp32", "site")):
        r = step_throughput(64, variant, storage, kernel, steps=6, warmup=3, d_i=1.0, tau=0.6, graph_steps=2)
        assert r["glups"] > 0 and r["nonfinite_sites"] == 0
        assert r["state_bytes_per_update"] == (384 if storage == "fp32" else 192)


def test_adjoint_throughput_reports_a_time():
    from paper_2212_11024_gb300.throughput import adjoint_throughput
    for storage in ("fp32", "bf16"):
        r = adjoint_throughput(32, storage, steps=3, warmup=1)
        assert r["glups"] > 0 and r["bytes_per_update"] == (576 if storage == "fp32" else 480)
