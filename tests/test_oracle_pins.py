"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check compares the oracle with something other than itself: values
printed in the paper (tests/golden), moment identities the paper states,
closed forms, special cases that reduce to a textbook operator, and brute
force (the literal 27x27 inversion against the factored form).
"""
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")
CS2 = 1.0 / 3.0
C2 = 0.25


def _golden_velocities():
    rows = {}
    with open(os.path.join(GOLD, "d3q27_velocities.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, *vals = line.split()
            rows[name] = [int(v) for v in vals]
    return np.array([rows["cx"], rows["cy"], rows["cz"]]).T


def _rand_state(rng, scale=0.05):
    """A random pre-collision site state near a moving, magnetised equilibrium."""
    rho = 1.0 + 0.1 * rng.uniform(-1, 1)
    U = scale * rng.uniform(-1, 1, 3)
    B = 0.1 * rng.uniform(-1, 1, 3)
    f = O.feq_product(rho, U) + O.lorentz(B)
    f = f * (1.0 + 0.05 * rng.uniform(-1, 1, 27))
    return f


C, W, XI, W7 = O.lattice()


# ------------------------------------------------------------------ lattice
def test_d3q27_velocities_match_app_a():
    assert np.array_equal(C, _golden_velocities())


def test_d3q27_opposites_and_weights():
    # App. A ordering: velocity i and i+13 are opposite for i = 1..13.
    for i in range(1, 14):
        assert np.array_equal(C[i], -C[i + 13])
    # Sec. 3.1.1 weights (golden file), isotropy up to fourth order.
    with open(os.path.join(GOLD, "weights.txt")) as fh:
        line = [ln for ln in fh if ln.startswith("d3q27")][0].split()[1:]
    vals = [eval(v) for v in line]  # fractions like 8/27
    n2 = (C * C).sum(axis=1)
    for n in range(4):
        assert np.allclose(W[n2 == n], vals[n], rtol=0, atol=1e-17)
    assert abs(W.sum() - 1) < 1e-15
    assert np.allclose(W @ C, 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", W, C, C), CS2 * np.eye(3), atol=1e-16)
    assert abs((W * C[:, 0] ** 4).sum() - 3 * CS2 ** 2) < 1e-16
    assert abs((W * C[:, 0] ** 2 * C[:, 1] ** 2).sum() - CS2 ** 2) < 1e-16


def test_d3q7_weights_give_C2():
    assert abs(W7.sum() - 1) < 1e-16
    assert np.allclose(W7 @ XI, 0)
    # Sec. 3.2: sum W xi xi = C^2 I with 2C = sqrt(3) cs, i.e. C^2 = 1/4.
    assert np.allclose(np.einsum("i,ia,ib->ab", W7, XI, XI), C2 * np.eye(3))
    assert abs(4 * C2 - 3 * CS2) < 1e-16


# --------------------------------------------------------------- equilibria
@pytest.mark.parametrize("seed", range(5))
def test_hermite_sum_equals_product_form(seed):
    rng = np.random.default_rng(seed)
    rho, U = 0.8 + 0.4 * rng.random(), 0.4 * rng.uniform(-1, 1, 3)
    assert np.allclose(O.feq_hermite(rho, U), O.feq_product(rho, U), rtol=0, atol=2e-16)


def test_hermite_equilibrium_truncations():
    # Only the 1st and 2nd order terms for a velocity along x: the x-only
    # 1-D Maxwellian moments must hold exactly (mass, momentum, cs^2 + u^2).
    U = np.array([0.3, 0.0, 0.0])
    f = O.feq_hermite(1.0, U)
    assert abs(f.sum() - 1) < 1e-15
    assert abs(f @ C[:, 0] - 0.3) < 1e-15
    assert abs(f @ C[:, 0] ** 2 - (CS2 + 0.09)) < 1e-15
    # at U = 0 the equilibrium is rho * w
    assert np.allclose(O.feq_hermite(1.3, np.zeros(3)), 1.3 * W, atol=1e-16)


@pytest.mark.parametrize("seed", range(5))
def test_fmhd_moments_match_paper(seed):
    """Sec. 3.1.1: sum f = rho, sum f c = rho U, sum f c c = rho UU + p I + |B|^2 I/2 - BB."""
    rng = np.random.default_rng(100 + seed)
    rho, U, B = 0.9 + 0.2 * rng.random(), 0.1 * rng.uniform(-1, 1, 3), 0.2 * rng.uniform(-1, 1, 3)
    f = O.feq_hermite(rho, U) + O.lorentz(B)
    assert abs(f.sum() - rho) < 1e-15
    assert np.allclose(f @ C, rho * U, atol=1e-16)
    Pi = np.einsum("i,ia,ib->ab", f, C, C)
    want = rho * np.outer(U, U) + rho * CS2 * np.eye(3) + 0.5 * (B @ B) * np.eye(3) - np.outer(B, B)
    assert np.allclose(Pi, want, atol=1e-15)
    # third-order moments of the product form: per-axis Maxwellian moments
    assert abs(f @ (C[:, 0] * C[:, 1] * C[:, 2]) - rho * U[0] * U[1] * U[2]) < 1e-16


def test_printed_lorentz_term_adds_mass():
    """The Lorentz term as printed in Sec. 3.1.1 / App. A has mass 3|B|^2 and
    second moment 2|B|^2 I - BB; the moment-matching form used instead has
    neither defect (reading of the paper, see the oracle header)."""
    B = np.array([0.1, -0.2, 0.05])
    lp = O.lorentz_printed(B)
    assert abs(lp.sum() - 3 * (B @ B)) < 1e-15
    assert np.allclose(np.einsum("i,ia,ib->ab", lp, C, C), 2 * (B @ B) * np.eye(3) - np.outer(B, B), atol=1e-15)
    lm = O.lorentz(B)
    assert abs(lm.sum()) < 1e-16 and np.allclose(lm @ C, 0, atol=1e-17)


# ---------------------------------------------------- central-moment basis
def _printed_basis(cb):
    x, y, z = cb
    return [1, x, y, z, x * y, x * z, y * z, x * x - y * y, x * x - z * z, x * x + y * y + z * z,
            x * y * y + x * z * z, x * y * y + y * z * z, x * x * y + y * y * z,
            x * y * y - x * z * z, x * y * y - y * z * z, x * x * y - y * y * z, x * y * z,
            x * x * y * y + x * x * z * z + y * y * z * z, x * x * y * y + x * x * z * z - y * y * z * z,
            x * x * y * y - x * x * z * z, x * x * y * z, x * y * y * z, x * y * z * z,
            x * y * y * z * z, x * x * y * z * z, x * x * y * y * z, x * x * y * y * z * z]


def test_printed_basis_is_singular_corrected_is_not():
    """Sec. 3.1.2 prints T11, T12, T14, T15 such that the 27 columns are
    linearly dependent; the oracle's corrected basis is well conditioned."""
    Tp = np.array([_printed_basis(c.astype(float)) for c in C])
    assert np.linalg.matrix_rank(Tp) < 27
    T = O.cm_matrix(np.zeros(3))
    assert np.linalg.matrix_rank(T) == 27
    assert np.linalg.cond(T) < 100


@pytest.mark.parametrize("seed", range(4))
def test_equilibrium_central_moments(seed):
    """k^eq = T^T f^(0) equals rho times products of 1-D Gaussian central
    moments (mu_0 = 1, mu_1 = 0, mu_2 = cs^2), column by column."""
    rng = np.random.default_rng(200 + seed)
    rho, U = 1.0 + 0.1 * rng.random(), 0.1 * rng.uniform(-1, 1, 3)
    k = O.cm_matrix(U).T @ O.feq_hermite(rho, U)
    c2, c4, c6 = CS2, CS2 ** 2, CS2 ** 3
    want = np.zeros(27)
    want[0] = rho
    want[9] = 3 * c2 * rho
    want[17] = 3 * c4 * rho
    want[18] = c4 * rho
    want[26] = c6 * rho
    assert np.allclose(k, want, atol=1e-15)


# ---------------------------------------------------------------- collision
def _cm(f, U, cols):
    T = O.cm_matrix(U)
    return T[:, cols].T @ f


@pytest.mark.parametrize("seed", range(6))
def test_cm_collision_literal_equals_factored(seed):
    rng = np.random.default_rng(300 + seed)
    f = _rand_state(rng)
    rho = f.sum()
    U = (f @ C) / rho
    B = 0.1 * rng.uniform(-1, 1, 3)
    feq = O.feq_hermite(rho, U) + O.lorentz(B)
    om = 1.0 / (0.5 + rng.random())
    S = np.ones(27)
    S[4:9] = om
    a = O.collide_cm_literal(f, feq, U, S)
    b = O.collide_cm_factored(f, feq, U, om)
    assert np.allclose(a, b, rtol=0, atol=1e-14)


@pytest.mark.parametrize("seed", range(4))
def test_cm_collision_conserves_and_relaxes(seed):
    rng = np.random.default_rng(400 + seed)
    f = _rand_state(rng)
    rho = f.sum()
    U = (f @ C) / rho
    feq = O.feq_hermite(rho, U) + O.lorentz(0.1 * rng.uniform(-1, 1, 3))
    om = 1.6
    S = np.ones(27)
    S[4:9] = om
    fs = O.collide_cm_literal(f, feq, U, S)
    assert abs(fs.sum() - rho) < 1e-15
    assert np.allclose(fs @ C, f @ C, atol=1e-16)
    # central moments from their definition sum f cbar^a cbar^b, computed here
    cb = C - U
    def cmom(g, a, b):
        return float(g @ (cb[:, a] * cb[:, b]))
    for a, b in [(0, 1), (0, 2), (1, 2)]:
        assert abs(cmom(fs, a, b) - ((1 - om) * cmom(f, a, b) + om * cmom(feq, a, b))) < 1e-15
    for a, b in [(0, 1), (0, 2)]:
        d = lambda g: cmom(g, a, a) - cmom(g, b, b)
        assert abs(d(fs) - ((1 - om) * d(f) + om * d(feq))) < 1e-15
    tr = lambda g: sum(cmom(g, a, a) for a in range(3))
    assert abs(tr(fs) - tr(feq)) < 1e-15
    # every third- and higher-order central moment is at equilibrium
    T = O.cm_matrix(U)
    assert np.allclose(T[:, 10:].T @ fs, T[:, 10:].T @ feq, atol=1e-15)


def test_cm_collision_bgk_limit():
    """Sec. 3.1.2: S = omega I recovers BGK, f* = f - omega (f - f^eq)."""
    rng = np.random.default_rng(5)
    f = _rand_state(rng)
    rho = f.sum()
    U = (f @ C) / rho
    feq = O.feq_hermite(rho, U)
    om = 1.3
    fs = O.collide_cm_literal(f, feq, U, om * np.ones(27))
    assert np.allclose(fs, f - om * (f - feq), atol=1e-15)
    fs1 = O.collide_cm_literal(f, feq, U, np.ones(27))
    assert np.allclose(fs1, feq, atol=1e-15)


# ------------------------------------------------------------------ current
@pytest.mark.parametrize("seed", range(5))
def test_current_solve_residual_and_closed_form(seed):
    rng = np.random.default_rng(500 + seed)
    Lam = 0.01 * rng.standard_normal((3, 3))
    U, B = 0.05 * rng.standard_normal(3), 0.2 * rng.standard_normal(3)
    omB, aH = 1.0 / 0.6, 3.0 * rng.random()
    J = O.current(Lam, U, B, omB, aH, literal=True)
    Jc = O.current(Lam, U, B, omB, aH, literal=False)
    assert np.allclose(J, Jc, rtol=1e-13, atol=1e-17)
    # eq. soe_current_density: (I + s M) J = -(omega_B/C^2) J_0 with the
    # paper's J_0 vector and M J = J x B.
    J0 = np.array([Lam[1, 2] - Lam[2, 1] - 2 * (U[1] * B[2] - U[2] * B[1]),
                   Lam[2, 0] - Lam[0, 2] - 2 * (U[2] * B[0] - U[0] * B[2]),
                   Lam[0, 1] - Lam[1, 0] - 2 * (U[0] * B[1] - U[1] * B[0])])
    M = np.array([[0, B[2], -B[1]], [-B[2], 0, B[0]], [B[1], -B[0], 0]])
    s = 2 * aH * omB / C2
    assert np.allclose((np.eye(3) + s * M) @ J, -(omB / C2) * J0, atol=1e-15)
    assert np.allclose(M @ J, np.cross(J, B), atol=1e-16)
    # App. B: det = 1 + s^2 |B|^2 > 0 (the paper's D = C^6 + 4 C^2 a^2 w^2 |B|^2, scaled by C^6)
    assert abs(np.linalg.det(np.eye(3) + s * M) - (1 + s * s * (B @ B))) < 1e-12


def test_current_ideal_limit_is_dellar():
    """alpha_H = 0: J = -(omega_B/C^2) (A - 2 U x B) (Dellar 2002)."""
    rng = np.random.default_rng(9)
    Lam = 0.01 * rng.standard_normal((3, 3))
    U, B = 0.05 * rng.standard_normal(3), 0.2 * rng.standard_normal(3)
    A = np.array([Lam[1, 2] - Lam[2, 1], Lam[2, 0] - Lam[0, 2], Lam[0, 1] - Lam[1, 0]])
    J = O.current(Lam, U, B, 1.7, 0.0)
    assert np.allclose(J, -(1.7 / C2) * (A - 2 * np.cross(U, B)), atol=1e-16)


def test_hall_equilibrium_moments():
    """eq. gHall_eq: sum_i g = B; sum_i xi_a g_b = V_a B_b - B_a V_b, V = U - a_H J (traceless)."""
    rng = np.random.default_rng(11)
    B, U, J = rng.standard_normal(3) * 0.1, rng.standard_normal(3) * 0.05, rng.standard_normal(3) * 0.01
    aH = 2.5
    g = O.geq_hall(B, U, J, aH)  # [b, i]
    assert np.allclose(g.sum(axis=1), B, atol=1e-16)
    Lam0 = np.einsum("ia,bi->ab", XI, g)
    V = U - aH * J
    assert np.allclose(Lam0, np.outer(V, B) - np.outer(B, V), atol=1e-16)
    assert abs(np.trace(Lam0)) < 1e-17


# -------------------------------------------------------------- grid level
def _smooth_random(shape, seed, amp):
    from paper_2212_11024_gb300 import inputs as I
    u, B = I.turbulence(shape, seed, seed + 1, amp, amp, shells=(1, 2))
    return u, B


def test_init_moments_and_current_from_exact_gradients():
    """Initial populations return rho, u, B exactly, and the current of the
    step's linear system equals curl B of the supplied gradient (eq.
    LB_density_current read as J = curl B)."""
    from paper_2212_11024_gb300 import inputs as I
    shape = (16, 4, 4)
    k = 2 * np.pi / 16
    u, B = I.parallel_wave(shape, 1, 1e-3, 0.1, 0.8)
    gu, gB = I.parallel_wave_gradients(shape, 1, 1e-3, 0.8)
    p = O.Params(4, 4, 16, 0.6, 0.7, 2.0)
    pop = O.init(p, None, u, B, gu, gB)
    m = O.moments(p, pop)
    assert np.allclose(m["rho"], 1.0, atol=1e-15)
    assert np.allclose(m["u"], u, atol=1e-16)
    assert np.allclose(m["B"], B, atol=1e-16)
    curl = np.stack([gB[3 * 1 + 2] - gB[3 * 2 + 1], gB[3 * 2 + 0] - gB[3 * 0 + 2], gB[3 * 0 + 1] - gB[3 * 1 + 0]])
    assert np.allclose(m["J"], curl, atol=1e-15)
    # for this wave curl b = k b
    assert np.allclose(m["J"][:2], k * (B[:2]), atol=1e-15)


def test_conservation():
    """Global mass, momentum and mean B are invariants of the periodic step
    (Sec. 3.1.2: S conserves mass and momentum; the magnetic BGK conserves
    sum g).  Tr(Lambda) (eq. LB_B_div) is zero at t = 0 for a field whose
    central-difference divergence is zero."""
    shape = (8, 8, 8)
    u, B = _smooth_random(shape, 7, 0.05)
    B[2] += 0.05
    p = O.Params(8, 8, 8, 0.55, 0.6, 1.5)
    pop = O.init(p, None, u, B)
    m0 = O.moments(p, pop)
    O.step(p, pop, 10)
    m1 = O.moments(p, pop)
    assert abs(m1["rho"].sum() - m0["rho"].sum()) < 1e-12
    for a in range(3):
        assert abs((m1["rho"] * m1["u"][a]).sum() - (m0["rho"] * m0["u"][a]).sum()) < 1e-13
        assert abs(m1["B"][a].sum() - m0["B"][a].sum()) < 1e-13
    assert np.abs(m0["trlam"]).max() < 1e-15


def test_divB_estimate_converges_second_order():
    """eq. LB_B_div: -(omega_B/C^2) Tr(Lambda) estimates div B.  The paper
    reports it stays at round-off; for a general 3-D field it is a
    discretisation error instead, which must fall at least like N^-2 under
    diffusive refinement (fixed tau, steps ~ N^2, amplitudes ~ 1/N,
    d_i ~ N), relative to |grad B|."""
    from paper_2212_11024_gb300 import inputs as I
    ratios = []
    for N in (8, 16, 32):
        s = N / 8
        u, B = I.turbulence((N, N, N), 7, 8, 0.05 / s, 0.05 / s, shells=(1, 2))
        B[2] += 0.05 / s
        p = O.Params(N, N, N, 0.55, 0.6, 1.5 * s)
        pop = O.init(p, None, u, B)
        O.step(p, pop, int(10 * s * s), literal=False)
        m = O.moments(p, pop)
        Bf = m["B"]
        grad = np.sqrt(sum(((np.roll(Bf[a], -1, axis=2 - b) - np.roll(Bf[a], 1, axis=2 - b)) / 2) ** 2
                           for a in range(3) for b in range(3)).mean())
        div = np.sqrt((((1 / 0.6) / C2 * m["trlam"]) ** 2).mean())
        ratios.append(div / grad)
    r = np.array(ratios)
    assert np.all(r[:-1] / r[1:] > 4.0), r


def test_translation_equivariance():
    """Shifting the initial fields by one lattice cell along each axis shifts
    the result by the same cell: catches streaming-direction errors."""
    shape = (6, 5, 4)
    u, B = _smooth_random(shape, 21, 0.05)
    p = O.Params(4, 5, 6, 0.6, 0.6, 1.0)
    pop = O.init(p, None, u, B)
    O.step(p, pop, 3)
    for ax in (1, 2, 3):
        pop_s = O.init(p, None, np.roll(u, 1, axis=ax), np.roll(B, 1, axis=ax))
        O.step(p, pop_s, 3)
        assert np.allclose(pop_s, np.roll(pop, 1, axis=ax), atol=1e-15)


def test_grid_literal_equals_factored():
    shape = (6, 6, 6)
    u, B = _smooth_random(shape, 31, 0.06)
    p = O.Params(6, 6, 6, 0.53, 0.58, 2.0)
    a = O.init(p, None, u, B)
    b = a.copy()
    O.step(p, a, 4, literal=True)
    O.step(p, b, 4, literal=False)
    assert np.allclose(a, b, rtol=0, atol=1e-14)


def test_streaming_moves_populations_along_their_velocity():
    """eq. stream: with omega = omega_B = 1 and a uniform state plus one
    perturbed population at one site, after the collision the perturbation's
    post-collision value sits at x + c_i.  Checked via linearity: the
    difference between perturbed and unperturbed runs is zero everywhere
    except at the 27 + 7 neighbour sites."""
    p = O.Params(5, 5, 5, 1.0, 1.0, 0.0)
    u = np.zeros((3, 5, 5, 5))
    B = np.zeros((3, 5, 5, 5))
    B[2] = 0.1
    base = O.init(p, None, u, B)
    pert = base.copy()
    pert[:, 2, 2, 2] += 1e-6 * np.linspace(1, 2, 48)
    O.step(p, base, 1)
    O.step(p, pert, 1)
    d = np.abs(pert - base).max(axis=0)  # [z, y, x]
    hit = {(2 + c[2], 2 + c[1], 2 + c[0]) for c in C}
    for z in range(5):
        for y in range(5):
            for x in range(5):
                if (z, y, x) not in hit:
                    assert d[z, y, x] == 0.0
    assert d[2, 2, 2] > 0


# -------------------------------------------------------- exact damped wave
def _wave_error(N, nxy, steps, di, B0, amp, tau_nu=0.6, tau_eta=0.6, literal=False):
    from oracle import exact_wave as X
    from paper_2212_11024_gb300 import inputs as I
    shape = (N, nxy, nxy)
    k = 2 * np.pi / N
    ap, _ = X.alpha_pm(k, di)
    u, B = I.parallel_wave(shape, 1, amp, B0, ap)
    gu, gB = I.parallel_wave_gradients(shape, 1, amp, ap)
    p = O.Params(nxy, nxy, N, tau_nu, tau_eta, di)
    pop = O.init(p, None, u, B, gu, gB)
    O.step(p, pop, steps, literal=literal)
    m = O.moments(p, pop)
    nu, eta = (tau_nu - 0.5) * CS2, (tau_eta - 0.5) * C2
    ue, Be = X.fields(steps, shape, 1, B0, nu, eta, di, amp, ap * amp)
    bz = np.array([0, 0, B0])[:, None, None, None]
    return X.rel_l2(m["u"], ue), X.rel_l2(m["B"] - bz, Be - bz), m


def test_exact_wave_function_matches_paper_closed_form():
    """For nu = eta the 2x2 solution is the paper's: b' = alpha_+ u',
    phase exp(i k B0 alpha t), decay exp(-nu k^2 t) (Sec. 4.1)."""
    from oracle import exact_wave as X
    k, B0, nu, di = 2 * np.pi / 32, 0.1, 0.02, 2.0
    ap, am = X.alpha_pm(k, di)
    assert abs(ap * am + 1) < 1e-15 and abs(ap + am + di * k) < 1e-15
    for alpha in (ap, am):
        a, c = X.amplitudes(137.0, k, B0, nu, nu, di, 1.0, alpha)
        want = np.exp(1j * k * B0 * alpha * 137.0 - nu * k * k * 137.0)
        assert abs(a - want) < 1e-12 and abs(c - alpha * want) < 1e-12
    # d_i = 0: Alfven waves, alpha = +-1
    assert X.alpha_pm(k, 0.0) == (1.0, -1.0)
    # config-1 numbers: alpha_+ = 0.82274, omega_+ = -alpha_+ k B0 = -0.016155
    ap1, _ = X.alpha_pm(2 * np.pi / 32, 2.0)
    assert abs(ap1 - 0.82274) < 5e-6
    assert abs(-ap1 * (2 * np.pi / 32) * 0.1 + 0.016155) < 1e-6


def test_exact_wave_config1_reduced_grid():
    """Config 1 (N = 32, B0 = 0.1 z, d_i = 2, tau = 0.6, amplitude 1e-3, 200
    steps).  The fields are uniform in x and y, so a 4 x 4 x 32 periodic grid
    gives the same result as 32^3.  The remaining error is the scheme's
    second-order dispersion error: about 0.027 rad of phase after 3.05 rad
    of propagation; its N^-2 scaling is pinned by the next test."""
    eu, eb, m = _wave_error(32, 4, 200, 2.0, 0.1, 1e-3, literal=True)
    assert eu < 3.5e-2 and eb < 5e-2
    assert np.abs(m["rho"] - 1).max() < 1e-12


@pytest.mark.parametrize("di", [2.0, 0.0])
def test_exact_wave_second_order_convergence(di):
    """Diffusive scaling (fixed tau, steps ~ N^2, B0 and amplitude ~ 1/N,
    d_i ~ N): the error against the exact solution falls as N^-2
    (Sec. 4.2-4.3 report second order).  d_i = 0 is the ideal-MHD Alfven
    limit."""
    errs = []
    for N in (16, 32, 64):
        s = N / 32
        eu, eb, _ = _wave_error(N, 2, int(round(200 * s * s)), di * s, 0.1 / s, 1e-3 / s)
        errs.append((eu, eb))
    errs = np.array(errs)
    for j in range(2):
        slopes = np.log2(errs[:-1, j] / errs[1:, j])
        assert np.all(slopes > 1.7) and np.all(slopes < 2.4), (errs, slopes)


def test_exact_wave_unequal_viscosity_resistivity():
    """tau_nu != tau_eta (nu != eta): the 2x2 exact solution still applies."""
    eu, eb, _ = _wave_error(32, 2, 200, 2.0, 0.1, 1e-3, tau_nu=0.7, tau_eta=0.55)
    assert eu < 4e-2 and eb < 5e-2


# ----------------------------------------------------------- scheme variants
def test_variant_bgk_equals_literal_bgk_limit():
    """Variant "bgk" is the central-moment operator with S = omega I
    (Sec. 3.1.2): the grid step equals per-site BGK collisions plus streaming,
    in both the literal and the factored oracle modes."""
    shape = (5, 4, 6)
    u, B = _smooth_random(shape, 41, 0.05)
    p = O.Params(6, 4, 5, 0.57, 0.6, 1.1)
    a = O.init(p, None, u, B)
    b = a.copy()
    O.step_variant(p, a, 3, "bgk", literal=True)
    O.step_variant(p, b, 3, "bgk", literal=False)
    assert np.allclose(a, b, rtol=0, atol=1e-14)
    # per-site check of one collision against f - omega (f - f^eq)
    pop = O.init(p, None, u, B)
    x = pop[:, 0, 0, 0]
    f = x[:27]
    rho = f.sum()
    U = (f @ C) / rho
    g = x[27:].reshape(3, 7)
    Bv = g.sum(1)
    feq = O.feq_hermite(rho, U) + O.lorentz(Bv)
    S = np.full(27, 1 / 0.57)
    assert np.allclose(O.collide_cm_literal(f, feq, U, S), f - (1 / 0.57) * (f - feq), atol=1e-15)


def test_variant_emhd_exact_whistler():
    """Electron MHD (end of Sec. 5): with U dropped from the magnetic
    equilibrium the field obeys db/dt = -d_i curl(J x B0) + eta lap b, so the
    parallel circularly polarised mode evolves as c(t) = c0 exp(-(i d_i B0
    k^2 + eta k^2) t) whatever the flow does.  Checked after 200 steps at
    N = 32 and 64 (diffusive scaling): second-order convergence."""
    from paper_2212_11024_gb300 import inputs as I
    errs = []
    for N in (32, 64):
        s = N / 32
        di, B0, amp, steps = 2.0 * s, 0.1 / s, 1e-3 / s, int(200 * s * s)
        shape = (N, 2, 2)
        k = 2 * np.pi / N
        u, B = I.parallel_wave(shape, 1, amp, B0, 0.5)
        gu, gB = I.parallel_wave_gradients(shape, 1, amp, 0.5)
        p = O.Params(2, 2, N, 0.6, 0.6, di)
        pop = O.init(p, None, u, B, gu, gB)
        O.step_variant(p, pop, steps, "emhd", literal=False)
        m = O.moments(p, pop)
        eta = 0.1 * 0.25
        c = 0.5 * amp * np.exp(-(1j * di * B0 * k * k + eta * k * k) * steps)
        z = np.arange(N)
        want = np.stack([np.imag(c * np.exp(1j * k * z)), np.real(c * np.exp(1j * k * z))])
        got = m["B"][:2, :, 0, 0]
        errs.append(np.linalg.norm(got - want) / np.linalg.norm(want))
    assert errs[0] < 8e-2 and 3.0 < errs[0] / errs[1] < 5.5, errs


def test_variant_fd_current_converges_to_exact_wave():
    """Current from the central-difference curl of B: the parallel
    Hall-MHD wave still converges to the exact solution at second order."""
    from oracle import exact_wave as X
    from paper_2212_11024_gb300 import inputs as I
    errs = []
    for N in (16, 32, 64):
        s = N / 32
        di, B0, amp, steps = 2.0 * s, 0.1 / s, 1e-3 / s, int(round(200 * s * s))
        shape = (N, 2, 2)
        k = 2 * np.pi / N
        ap, _ = X.alpha_pm(k, di)
        u, B = I.parallel_wave(shape, 1, amp, B0, ap)
        gu, gB = I.parallel_wave_gradients(shape, 1, amp, ap)
        p = O.Params(2, 2, N, 0.6, 0.6, di)
        pop = O.init(p, None, u, B, gu, gB)
        O.step_variant(p, pop, steps, "fd_current", literal=False)
        m = O.moments(p, pop)
        ue, _ = X.fields(steps, shape, 1, B0, 0.1 / 3, 0.1 / 4, di, amp, ap * amp)
        errs.append(X.rel_l2(m["u"], ue))
    r = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(r > 3.0) and np.all(r < 5.5), (errs, r)
