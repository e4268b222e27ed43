"""The lower bound that lets the encounter and contact tests skip the root search (Sect. 2.2, Eqs.
teqn and polydelta).

Over s in [0, 1] the cubic Hermite interpolant of the squared separation is
h00 P0 + h01 P1 + tau (h10 Pd0 + h11 Pd1), with h00 + h01 = 1, h00, h01 >= 0 and
0 <= s (1 - s)^2, s^2 (1 - s) <= 4/27. Hence it never falls below
min(P0, P1) - (4/27) |tau| (|Pd0| + |Pd1|). The kernels decide "minimum < threshold" without the
roots when this bound clears the threshold by a relative margin of 1e-12; these tests check the
inequality itself, by brute force over a fine grid, on random and on extreme data.
"""
import numpy as np


def cubic(s, tau, P0, P1, Pd0, Pd1):
    h00 = 2 * s**3 - 3 * s**2 + 1
    h01 = -2 * s**3 + 3 * s**2
    h10 = s**3 - 2 * s**2 + s
    h11 = s**3 - s**2
    return h00 * P0 + h01 * P1 + tau * (h10 * Pd0 + h11 * Pd1)


def bound(tau, P0, P1, Pd0, Pd1):
    return np.minimum(P0, P1) - (4.0 / 27.0) * abs(tau) * (abs(Pd0) + abs(Pd1))


def test_bound_holds_on_random_cubics():
    rng = np.random.default_rng(7)
    s = np.linspace(0.0, 1.0, 4001)[:, None]
    n = 20000
    P0 = rng.uniform(0, 1, n) * 10.0 ** rng.uniform(-8, 2, n)
    P1 = rng.uniform(0, 1, n) * 10.0 ** rng.uniform(-8, 2, n)
    Pd0 = rng.normal(size=n) * 10.0 ** rng.uniform(-6, 2, n)
    Pd1 = rng.normal(size=n) * 10.0 ** rng.uniform(-6, 2, n)
    tau = rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-3, 1, n)
    vals = cubic(s, tau, P0, P1, Pd0, Pd1).min(axis=0)
    lb = bound(tau, P0, P1, Pd0, Pd1)
    scale = P0 + P1 + abs(tau) * (abs(Pd0) + abs(Pd1))
    assert np.all(vals >= lb - 1e-14 * scale)


def test_bound_is_attained_by_the_extreme_slopes():
    """The constant 4/27 cannot be lowered: P0 = P1 = 0 with Pd1 = 0 reaches -(4/27) tau |Pd0| at
    s = 1/3 (and with Pd0 = 0, -(4/27) tau |Pd1| at s = 2/3)."""
    s = np.array([1.0 / 3.0, 2.0 / 3.0])
    a = cubic(s[0], 1.0, 0.0, 0.0, -1.0, 0.0)
    b = cubic(s[1], 1.0, 0.0, 0.0, 0.0, 1.0)
    assert np.isclose(a, -4.0 / 27.0, rtol=1e-15) and np.isclose(b, -4.0 / 27.0, rtol=1e-15)
    assert np.isclose(bound(1.0, 0.0, 0.0, -1.0, 0.0), -4.0 / 27.0)


def test_bound_never_skips_a_pair_that_meets():
    """Pairs built to pass inside the threshold at an interior time: the bound never clears it."""
    rng = np.random.default_rng(11)
    for _ in range(2000):
        tau = rng.uniform(0.1, 10.0)
        d0 = rng.normal(size=3)
        v = rng.normal(size=3)
        tmin = rng.uniform(0.05, 0.95) * tau
        # straight line through a closest point at tmin, distance dc
        dc = rng.uniform(0.0, 0.1)
        perp = np.cross(v, d0)
        perp = dc * perp / np.linalg.norm(perp)
        x0 = perp - v * tmin
        x1 = perp + v * (tau - tmin)
        P0, P1 = x0 @ x0, x1 @ x1
        Pd0, Pd1 = 2 * x0 @ v, 2 * x1 @ v
        thr = (1.01 * dc) ** 2
        lb = bound(tau, P0, P1, Pd0, Pd1)
        assert not (lb - 1e-12 * (P0 + P1 + (4 / 27) * tau * (abs(Pd0) + abs(Pd1))) > thr)
