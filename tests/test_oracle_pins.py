"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks an oracle routine against something other than the oracle itself: closed
forms worked by hand (tests/golden), invariants, special cases that reduce to textbook
results, an independent two-body propagator, scipy's high-order ODE integrator, networkx's
connected components, and brute force on tiny inputs. A plausible slip in the oracle (a
dropped term, a wrong sign, a transposed index) fails at least one of them.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1404_2324_gb300 import ics
from tests import twobody_ref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
G = ics.G_GAUSS


def _load_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ------------------------------------------------------------------ changeover K (Sect. 2.1)
def test_changeover_golden_table():
    rc = 0.37
    for row in _load_golden("changeover_K.txt"):
        y, K, dKdy = (float(s) for s in row)
        r = rc * (0.1 + 0.9 * y)
        assert O.changeover(r, rc) == pytest.approx(K, rel=1e-14, abs=1e-15)
        assert O.changeover_dr(r, rc) * 0.9 * rc == pytest.approx(dKdy, rel=1e-13, abs=1e-15)


def test_changeover_limits_symmetry_monotone():
    rc = 0.05
    assert O.changeover(0.1 * rc, rc) == 0.0
    assert O.changeover(0.05 * rc, rc) == 0.0
    assert O.changeover(rc, rc) == 1.0
    assert O.changeover(2 * rc, rc) == 1.0
    ys = np.linspace(0.0, 1.0, 401)
    Ks = [O.changeover(rc * (0.1 + 0.9 * y), rc) for y in ys]
    assert all(b >= a for a, b in zip(Ks, Ks[1:]))
    for y in ys:  # K(y) + K(1-y) = 1 (the rational form is point-symmetric about y = 1/2)
        k1 = O.changeover(rc * (0.1 + 0.9 * y), rc)
        k2 = O.changeover(rc * (0.1 + 0.9 * (1 - y)), rc)
        assert k1 + k2 == pytest.approx(1.0, abs=2e-15)


def test_changeover_derivative_matches_finite_difference():
    rc = 0.2
    for y in [0.05, 0.3, 0.5, 0.77, 0.95]:
        r = rc * (0.1 + 0.9 * y)
        h = 1e-6 * rc
        fd = (O.changeover(r + h, rc) - O.changeover(r - h, rc)) / (2 * h)
        assert O.changeover_dr(r, rc) == pytest.approx(fd, rel=1e-8)


def test_weight_gradient_mode_is_minus_gradient_of_HB():
    """kmode 1 is -d/dr of the pair potential -G m m K/r (Eq. Hb): weight/r^2 = -(d/dr)(K/r)*... ."""
    rc = 0.1
    for y in [0.1, 0.4, 0.6, 0.9]:
        r = rc * (0.1 + 0.9 * y)
        h = 1e-7 * r
        dphi = ((O.changeover(r + h, rc) / (r + h)) - (O.changeover(r - h, rc) / (r - h))) / (2 * h)
        # force on i towards j per G m_i m_j: -d/dr(-K/r) directed inward = -dphi ... in units 1/r^2
        assert O.weight_B(r * r, rc, 1) / (r * r) == pytest.approx(-dphi, rel=1e-7)
        assert O.weight_B(r * r, rc, 0) == pytest.approx(O.changeover(r, rc), rel=1e-15)
    assert O.weight_B(4 * rc * rc, rc, 1) == 1.0


# ------------------------------------------------------------------ critical radius (Eq. rcrit)
def test_rcrit_closed_form_circular_and_unbound():
    p = O.params(G=G, m0=1.0, dt=6.0)
    m = np.array([3e-5, 1e-9, 1e-7])
    r = np.array([1.0, 2.0, 0.7])
    vc = np.sqrt(G / r)
    x = np.zeros((3, 3)); x[:, 0] = r
    v = np.zeros((3, 3)); v[:, 1] = vc
    v[2, 1] = 3.0 * vc[2]  # unbound: Hill radius from |x|
    rc = O.rcrit(p, 6.0, m, np.ones(3, np.int32), x, v)
    for k in range(3):
        a = r[k]  # circular: a = r; unbound: reading uses |x|
        rh = a * (m[k] / 3.0) ** (1.0 / 3.0)
        spd = np.linalg.norm(v[k])
        assert rc[k] == pytest.approx(max(3.0 * rh, 0.4 * 6.0 * spd), rel=1e-14)
    assert rc[0] == pytest.approx(3.0 * (3e-5 / 3) ** (1 / 3), rel=1e-14)  # Hill branch wins
    assert rc[1] == pytest.approx(0.4 * 6.0 * vc[1], rel=1e-14)            # velocity branch wins


# ------------------------------------------------------------------ kick (Eq. Hb)
def _random_cluster(n, seed, spread=0.05):
    rng = np.random.default_rng(seed)
    x = np.array([1.0, 0.0, 0.0]) + spread * rng.standard_normal((n, 3))
    m = np.exp(rng.uniform(np.log(1e-9), np.log(1e-6), n))
    return m, x


def test_kick_far_field_is_textbook_direct_sum():
    """With every pair outside rc (K = 1) the kick is plain Newtonian direct summation."""
    p = O.params(G=G)
    m, x = _random_cluster(12, 1)
    rc = np.full(12, 1e-6)
    a = O.accel_B(p, m, np.ones(12, np.int32), x, rc)
    d = x[None, :, :] - x[:, None, :]            # d[i, j] = x_j - x_i
    r = np.linalg.norm(d, axis=-1) + np.eye(12)
    ref = G * np.einsum("j,ijk->ik", m, d / r[..., None] ** 3 * (1 - np.eye(12))[..., None])
    np.testing.assert_allclose(a, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_kick_is_minus_gradient_of_HB_in_gradient_mode():
    """kmode 1: m_i a_i = -dH_B/dx_i with H_B = -sum G m_i m_j K(r_ij)/r_ij (numerical gradient)."""
    p = O.params(G=G, kmode=1)
    m, x = _random_cluster(6, 2, spread=0.02)
    rc = np.full(6, 0.03)  # several pairs inside the transition zone
    a = O.accel_B(p, m, np.ones(6, np.int32), x, rc)

    def HB(xx):
        e = 0.0
        for i in range(6):
            for j in range(i + 1, 6):
                r = np.linalg.norm(xx[j] - xx[i])
                e -= G * m[i] * m[j] * O.changeover(r, 0.03) / r
        return e

    h = 1e-7
    for i in range(6):
        for c in range(3):
            xp = x.copy(); xp[i, c] += h
            xm = x.copy(); xm[i, c] -= h
            g = (HB(xp) - HB(xm)) / (2 * h)
            assert -g / m[i] == pytest.approx(a[i, c], rel=2e-6, abs=1e-6 * np.abs(a).max())


def test_kick_two_bodies_in_transition_zone_closed_form():
    """Two bodies at y = 1/4 (K = 1/10, golden table): a_1 = G m_2 K / r^2 along the line."""
    p = O.params(G=G, kmode=0)
    rc = 0.04
    r = rc * (0.1 + 0.9 * 0.25)
    x = np.array([[1.0, 0.0, 0.0], [1.0, r, 0.0]])
    m = np.array([2e-7, 5e-7])
    a = O.accel_B(p, m, np.ones(2, np.int32), x, np.array([rc, 0.5 * rc]))
    assert a[0, 1] == pytest.approx(G * m[1] * 0.1 / r ** 2, rel=1e-13)
    assert a[1, 1] == pytest.approx(-G * m[0] * 0.1 / r ** 2, rel=1e-13)
    assert a[0, 0] == 0.0 and a[0, 2] == 0.0


def test_kick_newton_third_law_and_ghosts():
    p = O.params(G=G)
    m, x = _random_cluster(20, 3, spread=0.03)
    rc = np.random.default_rng(4).uniform(0.005, 0.03, 20)
    alive = np.ones(20, np.int32); alive[5] = 0
    a = O.accel_B(p, m, alive, x, rc)
    mom = (m[:, None] * a * alive[:, None]).sum(0)
    assert np.abs(mom).max() <= 1e-14 * np.abs(m[:, None] * a).max() * 20
    assert np.all(a[5] == 0.0)
    m2 = m.copy(); m2[5] = 123.0  # a ghost's mass must not matter
    np.testing.assert_array_equal(O.accel_B(p, m2, alive, x, rc), a)


def test_precheck_brute_force():
    p = O.params(G=G)
    m, x = _random_cluster(40, 5, spread=0.1)
    rc = np.random.default_rng(6).uniform(0.005, 0.04, 40)
    alive = np.ones(40, np.int32); alive[7] = 0
    got = O.precheck(p, alive, x, rc)
    want = [(i, j) for i in range(40) for j in range(i + 1, 40)
            if alive[i] and alive[j] and np.linalg.norm(x[j] - x[i]) < 3 * max(rc[i], rc[j]) * (1 - 1e-12)]
    border = [(i, j) for i in range(40) for j in range(i + 1, 40)
              if abs(np.linalg.norm(x[j] - x[i]) / (3 * max(rc[i], rc[j])) - 1) < 1e-12]
    assert not border
    assert [tuple(r) for r in got] == want
    assert len(want) > 5


# ------------------------------------------------------------------ Sun drift (Eq. Hc)
def test_sun_drift_closed_form():
    p = O.params(G=G, m0=1.3)
    rng = np.random.default_rng(7)
    m = rng.uniform(1e-7, 1e-5, 5)
    v = rng.standard_normal((5, 3)) * 0.01
    x = rng.standard_normal((5, 3))
    alive = np.ones(5, np.int32)
    P = O.momentum(m, alive, v)
    np.testing.assert_allclose(P, (m[:, None] * v).sum(0), rtol=1e-14)
    xs = O.sun_drift(p, alive, x, P, 3.0)
    np.testing.assert_allclose(xs, x + 3.0 * P / 1.3, rtol=1e-14, atol=1e-16)


# ------------------------------------------------------------------ Kepler drift (Eq. fg)
def test_stumpff_against_trig_closed_forms():
    for z in [1e-8, 0.05, 0.3, 2.0, 9.0, 40.0, 150.0, -0.05, -2.0, -30.0]:
        c = O.stumpff(z)
        if z > 0:
            s = np.sqrt(z)
            ref = [np.cos(s), np.sin(s) / s, (1 - np.cos(s)) / z, (s - np.sin(s)) / s ** 3]
        else:
            s = np.sqrt(-z)
            ref = [np.cosh(s), np.sinh(s) / s, (np.cosh(s) - 1) / -z, (np.sinh(s) - s) / s ** 3]
        tol = 1e-12 if abs(z) > 1e-3 else 1e-7  # the closed forms cancel badly near z = 0
        np.testing.assert_allclose(c, ref, rtol=tol * max(1.0, abs(z) / 10))
    np.testing.assert_allclose(O.stumpff(0.0), [1.0, 1.0, 0.5, 1.0 / 6.0], rtol=1e-16)


@pytest.mark.parametrize("e", [0.0001, 0.05, 0.3, 0.7, 0.95])
def test_kepler_drift_matches_classical_solution(e):
    mu = G * 1.0
    rng = np.random.default_rng(int(e * 1e4))
    for _ in range(10):
        a = rng.uniform(0.3, 5.0)
        x, v = ics.elements_to_cartesian(mu, a, e, rng.uniform(0, 1), rng.uniform(0, 6.28),
                                         rng.uniform(0, 6.28), rng.uniform(0, 6.28))
        dt = rng.uniform(-40.0, 40.0)
        x1, v1, st, it = O.kepler_drift(mu, x, v, dt)
        assert st == 0
        if e < 0.01:
            continue  # the classical route is ill-conditioned near e = 0; covered by invariants
        xr, vr = twobody_ref.propagate(mu, x, v, dt)
        assert np.linalg.norm(x1 - xr) <= 2e-13 * np.linalg.norm(xr)
        assert np.linalg.norm(v1 - vr) <= 2e-13 * np.linalg.norm(vr)


def test_kepler_drift_hyperbolic_matches_classical_solution():
    mu = G
    x = np.array([1.0, 0.1, -0.05])
    v = np.array([0.005, 0.03, 0.002])  # v^2 > 2 mu / r
    for dt in [1.0, 25.0, -60.0, 300.0]:
        x1, v1, st, _ = O.kepler_drift(mu, x, v, dt)
        assert st == 0
        xr, vr = twobody_ref.propagate(mu, x, v, dt)
        assert np.linalg.norm(x1 - xr) <= 1e-12 * np.linalg.norm(xr)
        assert np.linalg.norm(v1 - vr) <= 1e-12 * np.linalg.norm(vr)


def test_kepler_drift_invariants_and_reversibility():
    mu = G
    rng = np.random.default_rng(11)
    for _ in range(50):
        x, v = ics.elements_to_cartesian(mu, rng.uniform(0.3, 3), rng.uniform(0, 0.6),
                                         rng.uniform(0, 1), *rng.uniform(0, 6.28, 3))
        dt = rng.uniform(1, 30)
        x1, v1, st, it = O.kepler_drift(mu, x, v, dt)
        assert st == 0 and it <= 8
        E0 = 0.5 * v @ v - mu / np.linalg.norm(x)
        E1 = 0.5 * v1 @ v1 - mu / np.linalg.norm(x1)
        assert abs(E1 - E0) <= 1e-14 * abs(E0)
        L0, L1 = np.cross(x, v), np.cross(x1, v1)
        assert np.linalg.norm(L1 - L0) <= 1e-14 * np.linalg.norm(L0)
        x2, v2, st, _ = O.kepler_drift(mu, x1, v1, -dt)
        assert np.linalg.norm(x2 - x) <= 1e-13 * np.linalg.norm(x)
        assert np.linalg.norm(v2 - v) <= 1e-13 * np.linalg.norm(v)


def test_kepler_drift_zero_step_and_iteration_cap():
    x = np.array([1.0, 0.0, 0.0]); v = np.array([0.0, 0.017, 0.0])
    x1, v1, st, _ = O.kepler_drift(G, x, v, 0.0)
    assert st == 0 and np.array_equal(x1, x) and np.array_equal(v1, v)
    x1, v1, st, _ = O.kepler_drift(G, x, v, 10.0, maxit=1)
    assert st == 1 and np.array_equal(x1, x)  # not converged: state untouched, flagged


# ------------------------------------------------------------------ Hermite encounter test (Eqs. teqn, polydelta)
def test_hermite_exact_for_straight_line_motion():
    """For uniform relative motion |dx(t)|^2 is quadratic, the cubic Hermite interpolant is exact,
    and the minimum is the closed-form closest approach. A wrong sign in a, b or c fails this."""
    rng = np.random.default_rng(12)
    for _ in range(200):
        d0 = rng.standard_normal(3) * 0.01
        w = rng.standard_normal(3) * 0.003
        tau = rng.choice([6.0, -4.0, 10.2])
        d1 = d0 + w * tau
        got = O.hermite_min(d0, w, d1, w, tau)
        tstar = -(d0 @ w) / (w @ w) / tau  # in units of the step
        ts = min(max(tstar, 0.0), 1.0)
        want = np.sum((d0 + w * tau * ts) ** 2)
        assert got == pytest.approx(want, rel=1e-9, abs=1e-12 * (d0 @ d0))


def test_hermite_minimum_brute_force_grid():
    rng = np.random.default_rng(13)
    for _ in range(200):
        dx0, dv0, dx1, dv1 = (rng.standard_normal(3) * s for s in (0.01, 0.002, 0.01, 0.002))
        tau = 5.0
        P0, P1 = dx0 @ dx0, dx1 @ dx1
        Pd0, Pd1 = 2 * dx0 @ dv0, 2 * dx1 @ dv1
        t = np.linspace(0, 1, 200001)
        # cubic Hermite basis of Sect. 2.2 on a fine grid
        P = (P0 * (1 + 2 * t) * (1 - t) ** 2 + P1 * t ** 2 * (3 - 2 * t)
             + Pd0 * t * (1 - t) ** 2 * tau + Pd1 * t ** 2 * (t - 1) * tau)
        got = O.hermite_min(dx0, dv0, dx1, dv1, tau)
        assert got <= P.min() + 1e-12 * max(P0, P1)
        assert got >= P.min() - 1e-9 * max(P0, P1)


def test_encounter_list_brute_force():
    rng = np.random.default_rng(14)
    n = 30
    x0 = rng.uniform(-0.1, 0.1, (n, 3)) + [1, 0, 0]
    v0 = rng.standard_normal((n, 3)) * 0.002
    tau = 6.0
    x1 = x0 + v0 * tau
    v1 = v0.copy()
    rc = rng.uniform(0.01, 0.06, n)
    alive = np.ones(n, np.int32)
    cand = np.array([(i, j) for i in range(n) for j in range(i + 1, n)], np.int32)
    got = O.encounters(alive, x0, v0, x1, v1, rc, cand, tau)
    want = []
    for i, j in cand:
        d0, w = x0[j] - x0[i], v0[j] - v0[i]
        ts = min(max(-(d0 @ w) / (w @ w) / tau, 0.0), 1.0)
        if np.sum((d0 + w * tau * ts) ** 2) < max(rc[i], rc[j]) ** 2:
            want.append((i, j))
    assert [tuple(r) for r in got] == want and len(want) > 3


# ------------------------------------------------------------------ grouping (Appendix)
def test_groups_are_connected_components():
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(15)
    n = 300
    pairs = set()
    for _ in range(150):
        i, j = sorted(rng.choice(n, 2, replace=False))
        pairs.add((int(i), int(j)))
    pairs = sorted(pairs)
    single = np.zeros(n, np.int32); single[[3, 77]] = 1
    got = O.groups(n, pairs, single)
    Gr = nx.Graph(); Gr.add_edges_from(pairs); Gr.add_nodes_from([3, 77])
    want = sorted(sorted(c) for c in nx.connected_components(Gr))
    assert [list(g) for g in got] == want
    assert all(list(g) == sorted(g) for g in got)
    assert [g[0] for g in got] == sorted(g[0] for g in got)


# ------------------------------------------------------------------ Bulirsch-Stoer (Sect. 3.2)
def test_bs_single_body_is_kepler_orbit():
    p = O.params(G=G, m0=1.0)
    x, v = ics.elements_to_cartesian(G, 1.2, 0.4, 0.1, 0.3, 0.5, 0.7)
    out = O.bs_group(p, [0], 6.0, [1e-9], [0.0], [1], x.reshape(1, 3), v.reshape(1, 3), [0.01])
    xr, vr = twobody_ref.propagate(G, x, v, 6.0)
    assert out["status"] == 0
    assert np.linalg.norm(out["x"] - xr) <= 1e-11 * np.linalg.norm(xr)
    assert np.linalg.norm(out["v"] - vr) <= 1e-11 * np.linalg.norm(vr)


def test_bs_isolated_pair_is_two_body_orbit():
    """m0 = 0 and K = 0 (huge rc): the group is an isolated two-body problem."""
    p = O.params(G=G, m0=0.0, collisions=0)
    m = np.array([3e-4, 1e-4])
    mu = G * m.sum()
    xr_rel, vr_rel = ics.elements_to_cartesian(mu, 0.01, 0.6, 0.2, 0.1, 0.4, 2.0)
    com_x, com_v = np.array([1.0, 0.2, 0.0]), np.array([0.001, 0.017, 0.0])
    x = np.array([com_x - m[1] / m.sum() * xr_rel, com_x + m[0] / m.sum() * xr_rel])
    v = np.array([com_v - m[1] / m.sum() * vr_rel, com_v + m[0] / m.sum() * vr_rel])
    tau = 6.0  # a third of the relative orbit's period
    out = O.bs_group(p, [0, 1], tau, m, [0, 0], [1, 1], x, v, [1e6, 1e6])
    rel_x, rel_v = twobody_ref.propagate(mu, xr_rel, vr_rel, tau)
    assert out["status"] == 0
    np.testing.assert_allclose(out["x"][1] - out["x"][0], rel_x, rtol=0, atol=1e-11 * np.linalg.norm(rel_x))
    np.testing.assert_allclose(out["v"][1] - out["v"][0], rel_v, rtol=0, atol=1e-11 * np.linalg.norm(rel_v))
    cm = (m[:, None] * out["x"]).sum(0) / m.sum()
    np.testing.assert_allclose(cm, com_x + com_v * tau, rtol=1e-13, atol=1e-15)


def test_bs_matches_scipy_dop853_for_four_bodies():
    from scipy.integrate import solve_ivp
    p = O.params(G=G, m0=1.0, collisions=0)
    rng = np.random.default_rng(16)
    m = np.array([2e-6, 5e-6, 1e-6, 3e-6])
    x = np.array([1.0, 0.0, 0.0]) + rng.standard_normal((4, 3)) * 0.01
    v = np.array([0.0, 0.0172, 0.0]) + rng.standard_normal((4, 3)) * 0.0004
    tau = 6.0

    def rhs(t, y):
        X = y[:12].reshape(4, 3); V = y[12:].reshape(4, 3)
        A = -G * X / np.linalg.norm(X, axis=1)[:, None] ** 3
        for i in range(4):
            for j in range(4):
                if i != j:
                    d = X[j] - X[i]
                    A[i] += G * m[j] * d / np.linalg.norm(d) ** 3
        return np.concatenate([V.ravel(), A.ravel()])

    sol = solve_ivp(rhs, (0, tau), np.concatenate([x.ravel(), v.ravel()]), method="DOP853",
                    rtol=1e-13, atol=1e-16)
    out = O.bs_group(p, [0, 1, 2, 3], tau, m, np.zeros(4), np.ones(4, np.int32), x, v, np.full(4, 1e6))
    np.testing.assert_allclose(out["x"].ravel(), sol.y[:12, -1], rtol=1e-10)
    np.testing.assert_allclose(out["v"].ravel(), sol.y[12:, -1], rtol=1e-9)


def test_bs_collision_merges_conserving_mass_momentum_and_energy():
    """Isolated pair (m0 = 0, K = 0) on a head-on course: the merger conserves mass and linear
    momentum exactly, and E + U (U booked per Sect. 3.2) equals the energy before contact."""
    p = O.params(G=G, m0=0.0)
    m = np.array([4e-7, 1e-7])
    R = np.array([2e-5, 1e-5])
    x = np.array([[1.0, 0.0, 0.0], [1.0, 0.002, 0.0]])
    v = np.array([[0.0, 0.0172, 0.0], [0.0, 0.0172 - 0.001, 0.0]])  # closing in ~2 days
    P0 = (m[:, None] * v).sum(0)
    E0 = 0.5 * (m * (v * v).sum(1)).sum() - G * m[0] * m[1] / 0.002
    out = O.bs_group(p, [0, 1], 6.0, m, R, [1, 1], x, v, [1e6, 1e6])
    assert out["status"] == 0
    assert [tuple(c) for c in out["collisions"]] == [(0, 1)]
    assert list(out["alive"]) == [1, 0]  # heavier body survives
    assert out["m"][0] == pytest.approx(5e-7, rel=1e-15) and out["m"][1] == 0.0
    assert out["R"][0] == pytest.approx((2e-5 ** 3 + 1e-5 ** 3) ** (1 / 3), rel=1e-14)
    Pm = out["m"][0] * out["v"][0]
    np.testing.assert_allclose(Pm, P0, rtol=1e-13, atol=1e-13 * np.linalg.norm(P0))
    E1 = 0.5 * out["m"][0] * out["v"][0] @ out["v"][0]
    assert E1 + out["U"] == pytest.approx(E0, rel=1e-9)
    assert out["U"] > 0.0 or out["U"] < 0.0


def test_merge_rule_equal_masses_keeps_smaller_index():
    p = O.params(G=G, m0=1.0)
    m = np.array([1e-7, 1e-7])
    out = O.bs_group(p, [0, 1], 6.0, m, [1e-5, 1e-5], [1, 1],
                     np.array([[1.0, 0.0, 0.0], [1.0, 0.001, 0.0]]),
                     np.array([[0.0, 0.0172, 0.0], [0.0, 0.0172 - 0.001, 0.0]]), [0.05, 0.05])
    assert list(out["alive"]) == [1, 0]


# ------------------------------------------------------------------ whole step (Eq. z1, Sect. 2.3)
def _sim(d, **kw):
    p = O.params(G=d["G"], m0=d["m0"], dt=d["dt"], order=d.get("order", 2), **kw)
    return O.Sim(p, d["m"], d["R"], d["x"], d["v"])


def test_yoshida_weights_golden():
    """The oracle's substep weights (Sect. 2.3) equal Yoshida's (1990) published values, which in
    turn satisfy the order conditions of a symmetric composition of a symmetric 2nd-order step:
    sum w = 1, sum w^3 = 0 (order 4) and sum w^5 = 0 (order 6). A weight mistyped in its 8th digit
    misses the golden row at 1e-14 and leaves sum w^3 ~ 1e-8."""
    rows = {r[0]: [float(s) for s in r[1:]] for r in _load_golden("yoshida.txt")}
    c = 2 ** (1 / 3)
    assert rows["order4"] == pytest.approx([1 / (2 - c), -c / (2 - c), 1 / (2 - c)], rel=1e-15)
    for order in (4, 6):
        w = np.array(rows[f"order{order}"])
        assert abs(w.sum() - 1.0) < 1e-14
        assert abs((w ** 3).sum()) < 1e-13
        if order == 6:
            assert abs((w ** 5).sum()) < 1e-13
        assert list(w) == list(w[::-1])  # symmetric sequence
        np.testing.assert_allclose(O.substep_weights(order), w, rtol=1e-14, atol=0)
    assert list(O.substep_weights(2)) == [1.0]


def _composed_leapfrog_error(w, h_list, mp):
    """Global error at t = 1 of the pendulum q'' = -sin q (q, p = 1, 0.3) integrated by the
    composition of leapfrog steps with weights w, in 40-digit arithmetic, against mpmath's Taylor
    integrator. Leapfrog is symmetric and of order 2, so the composition has the order of w."""
    mp.mp.dps = 40
    f = mp.odefun(lambda t, y: [y[1], -mp.sin(y[0])], 0, [mp.mpf(1), mp.mpf("0.3")])
    qr, pr = f(1)
    errs = []
    for h in h_list:
        n = int(round(1.0 / h))
        hh = mp.mpf(1) / n
        q, p = mp.mpf(1), mp.mpf("0.3")
        for _ in range(n):
            for wk in w:
                s = wk * hh
                p -= s / 2 * mp.sin(q)
                q += s * p
                p -= s / 2 * mp.sin(q)
        errs.append(abs(q - qr) + abs(p - pr))
    return [float(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]


def test_sixth_order_weights_give_sixth_order_convergence():
    """The oracle's 6th-order weights, used in a composition of a symmetric 2nd-order step, give a
    global error that falls by 2^6 = 64 per halving of the step down to h = 1/40 (40 digits, so
    rounding plays no part). A weight off by 1e-8 leaves an O(h^2) error of ~1e-8 h^2, which takes
    over at these steps (the planted-mistake test below)."""
    mp = pytest.importorskip("mpmath")
    w = [mp.mpf(float(x)) for x in O.substep_weights(6)]
    ratios = _composed_leapfrog_error(w, (0.2, 0.1, 0.05, 0.025), mp)
    assert all(58.0 < r < 70.0 for r in ratios), ratios


def test_sixth_order_convergence_check_detects_an_eighth_digit_error():
    mp = pytest.importorskip("mpmath")
    w = [mp.mpf(float(x)) for x in O.substep_weights(6)]
    w[2] = w[4] = w[2] * (1 + mp.mpf("1e-8"))  # plant the mistake in a copy of the weights
    w[3] = 1 - 2 * (w[0] + w[1] + w[2])
    ratios = _composed_leapfrog_error(w, (0.05, 0.025), mp)
    assert not (58.0 < ratios[0] < 70.0), ratios


def test_single_massless_body_step_is_exact_kepler_orbit():
    """m_1 = 0: P = 0, no kick, and a step is exactly the Kepler drift (any order)."""
    x, v = ics.elements_to_cartesian(G, 1.0, 0.2, 0.05, 1.0, 2.0, 3.0)
    for order in (2, 4, 6):
        d = dict(G=G, m0=1.0, dt=6.0, order=order, m=np.zeros(1), R=np.zeros(1),
                 x=x.reshape(1, 3), v=v.reshape(1, 3))
        s = _sim(d)
        s.step(20)
        st = s.state()
        xr, vr = twobody_ref.propagate(G, x, v, 120.0)
        assert np.linalg.norm(st["x"][0] - xr) <= 1e-13 * np.linalg.norm(xr) * 20
        assert np.linalg.norm(st["v"][0] - vr) <= 1e-13 * np.linalg.norm(vr) * 20


def _far_planets(n=3, seed=17):
    rng = np.random.default_rng(seed)
    a = np.array([0.7, 1.3, 2.4, 3.9, 5.5])[:n]
    m = np.array([3e-6, 1e-5, 5e-6, 2e-6, 4e-6])[:n]
    x, v = ics.elements_to_cartesian(G * (1 + m), a, rng.uniform(0.01, 0.05, n), rng.uniform(0, 0.02, n),
                                     *rng.uniform(0, 6.28, (3, n)))
    return dict(G=G, m0=1.0, dt=4.0, m=m, R=ics.radius_from_mass(m), x=x, v=v)


def test_time_reversal_encounter_free():
    d = _far_planets()
    for order in (2, 4):
        d["order"] = order
        s = _sim(d)
        s.step(25)
        st = s.state()
        back = dict(d, x=st["x"], v=st["v"], dt=-d["dt"])
        s2 = _sim(back)
        s2.step(25)
        st2 = s2.state()
        assert s.stats()["encounters"] == 0
        np.testing.assert_allclose(st2["x"], d["x"], rtol=0, atol=1e-12 * np.abs(d["x"]).max())
        np.testing.assert_allclose(st2["v"], d["v"], rtol=0, atol=1e-12 * np.abs(d["v"]).max())


def _angmom(state, m0=1.0):
    x, v, m = state["x"], state["v"], state["m"]
    # democratic variables: L = sum m_i x_i x v_i(barycentric) = inertial angular momentum
    P = (m[:, None] * v).sum(0)
    vb = v - P / (m0 + m.sum())
    return (m[:, None] * np.cross(x, vb)).sum(0)


def test_angular_momentum_conserved_with_encounters():
    d = ics.disk32(1)
    s = _sim(d)
    L0 = _angmom(s.state())
    s.step(200)
    assert s.stats()["encounters"] > 5  # BS groups took part
    L1 = _angmom(s.state())
    assert np.linalg.norm(L1 - L0) <= 1e-12 * np.linalg.norm(L0)


def test_energy_error_scaling_with_order():
    """Encounter-free system: halving tau divides the energy error by ~4 (2nd), ~16 (4th) and ~64
    (6th order: at tau = 8 and 4 days, and 16 and 8 days, the errors stay above rounding)."""
    base = _far_planets(3, seed=18)
    for order, expect, dts in ((2, 4.0, (8.0, 4.0)), (4, 16.0, (8.0, 4.0)), (6, 64.0, (8.0, 4.0)),
                               (6, 64.0, (16.0, 8.0))):
        errs = []
        for dt in dts:
            d = dict(base, dt=dt, order=order)
            s = _sim(d)
            E0, _ = s.energy()
            emax = 0.0
            nsteps = int(round(400.0 / dt))
            for _ in range(nsteps):
                s.step(1)
                E, U = s.energy()
                emax = max(emax, abs((E + U - E0) / E0))
            errs.append(emax)
        ratio = errs[0] / errs[1]
        assert expect / 1.6 < ratio < expect * 1.6, (order, errs)


def test_whole_step_matches_direct_integration_at_splitting_order():
    from scipy.integrate import solve_ivp
    base = _far_planets(3, seed=19)
    m = base["m"]

    def rhs(t, y):  # full Newtonian problem in heliocentric coordinates
        X = y[:9].reshape(3, 3); V = y[9:].reshape(3, 3)
        A = -G * (1 + m)[:, None] * X / np.linalg.norm(X, axis=1)[:, None] ** 3
        for i in range(3):
            for j in range(3):
                if i != j:
                    d = X[j] - X[i]
                    A[i] += G * m[j] * (d / np.linalg.norm(d) ** 3 - X[j] / np.linalg.norm(X[j]) ** 3)
        return np.concatenate([V.ravel(), A.ravel()])

    T = 200.0
    sol = solve_ivp(rhs, (0, T), np.concatenate([base["x"].ravel(), base["v"].ravel()]),
                    method="DOP853", rtol=1e-13, atol=1e-15)
    xr = sol.y[:9, -1].reshape(3, 3)
    errs = []
    for dt in (4.0, 2.0):
        s = _sim(dict(base, dt=dt, order=2))
        s.step(int(T / dt))
        errs.append(np.abs(s.state()["x"] - xr).max())
    assert errs[0] < 1e-6
    assert 2.5 < errs[0] / errs[1] < 6.0  # O(tau^2)


def test_energy_closed_form_single_body():
    """One body: E (democratic) equals the barycentric two-body energy."""
    p = O.params(G=G, m0=1.0)
    m = np.array([1e-3])
    xh = np.array([[1.1, 0.2, 0.0]]); vh = np.array([[0.001, 0.016, 0.001]])
    M = 1.0 + m[0]
    V0 = -m[0] * vh[0] / M          # central body's barycentric velocity
    V1 = vh[0] + V0
    Eref = 0.5 * 1.0 * V0 @ V0 + 0.5 * m[0] * V1 @ V1 - G * m[0] / np.linalg.norm(xh[0])
    s = O.Sim(p, m, np.zeros(1), xh, vh)
    E, U = s.energy()
    assert E == pytest.approx(Eref, rel=1e-14) and U == 0.0


def test_disk32_energy_bounded_and_no_reuse_violations():
    d = ics.disk32(1)
    s = _sim(d)
    E0, _ = s.energy()
    errs = []
    for _ in range(10):
        s.step(100)
        E, U = s.energy()
        errs.append(abs((E + U - E0) / E0))
    st = s.stats()
    assert max(errs) < 1e-7
    assert st["reuse_violations"] == 0 and st["kepler_fallbacks"] == 0
    assert st["candidates"] >= st["encounters"] > 0  # prechecker never misses (candidates contain all)
