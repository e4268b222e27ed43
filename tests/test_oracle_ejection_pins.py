"""Pins of the oracle's ejections (Sect. 3.2, Ejections): a body farther than Rcut from the central
mass, or closer than RcutSun, is removed at the end of the step and its state recorded; the energy
it takes away is booked into U.

The removal step and the recorded state are checked against an independent two-body propagator
(orbital elements and Kepler's equation, `twobody_ref.propagate`) for a body too light to perturb
anything; the energy bookkeeping is checked by the invariant E + U across an ejection, where the
removed body's own energy is orders of magnitude larger than the integrator's step-to-step error.
"""
import numpy as np
import pytest

import oracle as O
from paper_1404_2324_gb300 import ics
from tests.twobody_ref import propagate

G = ics.G_GAUSS


def _light_body_radii(x, v, dt, steps):
    """|x| at the end of steps 1..steps on the exact Kepler orbit about m0 = 1."""
    return np.array([np.linalg.norm(propagate(G, x, v, k * dt)[0]) for k in range(1, steps + 1)])


def _pick_threshold(r, above, floor=1.2):
    """A threshold between two consecutive step radii, far from both (the first crossing step);
    outward crossings start beyond floor."""
    for k in range(1, len(r)):
        lo, hi = sorted((r[k - 1], r[k]))
        if (above and r[k] > r[k - 1] and r[k - 1] > floor) or (not above and r[k] < r[k - 1] and r[k] < 0.6):
            if hi - lo > 1e-3 and all(abs(rr - 0.5 * (lo + hi)) > 1e-4 for rr in r[: k + 1]):
                return 0.5 * (lo + hi), k + 1
    raise AssertionError("no usable crossing")


def _single(x, v, dt, **kw):
    m = np.array([1e-13])
    p = O.params(G=G, m0=1.0, dt=dt, order=2, **kw)
    return O.Sim(p, m, np.array([1e-9]), np.array([x]), np.array([v]))


def test_escape_beyond_rcut_at_the_kepler_step():
    x, v = np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.3 * np.sqrt(2 * G), 0.01])
    dt = 6.0
    r = _light_body_radii(x, v, dt, 60)
    rcut, kstar = _pick_threshold(r, above=True)
    s = _single(x, v, dt, rcut=rcut)
    for k in range(1, kstar + 1):
        s.step(1)
        alive = s.state()["alive"][0]
        assert alive == (1 if k < kstar else 0), (k, kstar)
    ej = s.ejections()
    assert ej.shape == (1, 8) and ej[0, 0] == 0 and ej[0, 1] == kstar
    xk, vk = propagate(G, x, v, kstar * dt)
    np.testing.assert_allclose(ej[0, 2:5], xk, rtol=1e-9)
    np.testing.assert_allclose(ej[0, 5:8], vk, rtol=1e-9)
    assert s.stats()["ejections"] == 1
    s.close()


def test_plunge_inside_rcut_sun_at_the_kepler_step():
    # e = 0.9, a = 1: periapsis 0.1 AU; start at apoapsis
    a, e = 1.0, 0.9
    x = np.array([-a * (1 + e), 0.0, 0.0])
    v = np.array([0.0, -np.sqrt(G / a * (1 - e) / (1 + e)), 0.0])
    dt = 1.0
    r = _light_body_radii(x, v, dt, 400)
    rsun, kstar = _pick_threshold(r, above=False)
    s = _single(x, v, dt, rcut_sun=rsun)
    s.step(kstar - 1)
    assert s.state()["alive"][0] == 1
    s.step(1)
    assert s.state()["alive"][0] == 0
    ej = s.ejections()
    assert ej.shape == (1, 8) and ej[0, 1] == kstar
    np.testing.assert_allclose(ej[0, 2:5], propagate(G, x, v, kstar * dt)[0], rtol=1e-8)
    s.close()


def test_off_by_default():
    x, v = np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.3 * np.sqrt(2 * G), 0.0])
    s = _single(x, v, 6.0)
    s.step(200)  # far beyond any sensible Rcut
    assert s.state()["alive"][0] == 1 and s.ejections().shape == (0, 8) and s.stats()["ejections"] == 0
    s.close()


def _three_body(rcut):
    """A Jupiter-mass planet at 5.2 AU, an Earth at 1 AU and an Earth-mass body escaping from 0.8
    AU at 1.35 times the escape speed (it passes 8 AU after ~170 steps of 2 days)."""
    m = np.array([1e-3, 3e-6, 3e-6])
    x = np.array([[5.2, 0.0, 0.0], [0.0, 1.0, 0.0], [-0.8, 0.0, 0.05]])
    v = np.array([[0.0, np.sqrt(G / 5.2), 0.0], [-np.sqrt(G), 0.0, 0.0], [0.0, -1.35 * np.sqrt(2 * G / 0.8), 0.0]])
    p = O.params(G=G, m0=1.0, dt=2.0, order=4, rcut=rcut)
    return O.Sim(p, m, ics.radius_from_mass(m), x, v)


def test_energy_booked_into_U_keeps_E_plus_U():
    s = _three_body(rcut=8.0)
    tot = []
    E, U = s.energy()
    tot.append(E + U)
    ejected_at = None
    for k in range(1, 400):
        s.step(1)
        E, U = s.energy()
        tot.append(E + U)
        if ejected_at is None and s.state()["alive"][2] == 0:
            ejected_at = k
            removed = U  # U before this step was 0 (no mergers here)
    assert ejected_at is not None and s.ejections()[0, 0] == 2
    steps = np.abs(np.diff(tot))
    quiet = np.delete(steps, ejected_at - 1)
    # the jump at the ejection step is no larger than an ordinary step's change of E + U, while the
    # energy the body took away is many orders of magnitude larger
    assert steps[ejected_at - 1] <= 3 * quiet.max() + 1e-18
    assert abs(removed) > 1e4 * quiet.max()
    # and E + U drifts no more than the same system's E without the ejection test
    s2 = _three_body(rcut=0.0)
    E0, _ = s2.energy()
    e2 = [E0]
    for k in range(1, 400):
        s2.step(1)
        e2.append(s2.energy()[0])
    assert abs(tot[-1] - tot[0]) <= 10 * max(abs(np.array(e2) - E0).max(), 1e-18)
    s.close()
    s2.close()


def test_test_particle_escape_at_the_kepler_step():
    xp = np.array([[0.4, 0.0, 0.0]])
    vp = np.array([[0.0, np.sqrt(G / 0.4), 0.0]])
    mp = np.array([1e-6])
    xt = np.array([[1.0, 0.0, 0.0], [0.0, 1.5, 0.0]])
    vt = np.array([[0.0, 1.25 * np.sqrt(2 * G), 0.0], [-np.sqrt(G / 1.5), 0.0, 0.0]])
    dt = 6.0
    r = _light_body_radii(xt[0], vt[0], dt, 80)
    rcut, kstar = _pick_threshold(r, above=True, floor=2.0)
    p = O.params(G=G, m0=1.0, dt=dt, order=2, rcut=rcut)
    t = O.TPSim(p, mp, ics.radius_from_mass(mp), xp, vp, xt, vt)
    t.step(kstar - 1)
    assert list(t.state()["tp_alive"]) == [1, 1]
    t.step(1)
    assert list(t.state()["tp_alive"]) == [0, 1]
    assert t.stats()["tp_ejected"] == 1 and t.ejections().shape == (0, 8)
    t.close()


@pytest.mark.parametrize("order", [2, 4])
def test_ejected_body_no_longer_acts(order):
    """After the removal the remaining bodies move as if the body had never been there from that
    step on: a run started from the post-ejection state without it agrees."""
    m = np.array([1e-3, 3e-6, 3e-6])
    x = np.array([[5.2, 0.0, 0.0], [0.0, 1.0, 0.0], [-0.8, 0.0, 0.05]])
    v = np.array([[0.0, np.sqrt(G / 5.2), 0.0], [-np.sqrt(G), 0.0, 0.0], [0.0, -1.35 * np.sqrt(2 * G / 0.8), 0.0]])
    p = O.params(G=G, m0=1.0, dt=2.0, order=order, rcut=8.0)
    a = O.Sim(p, m, ics.radius_from_mass(m), x, v)
    k = 0
    while a.state()["alive"][2] == 1:
        a.step(1)
        k += 1
        assert k < 600
    st = a.state()
    b = O.Sim(O.params(G=G, m0=1.0, dt=2.0, order=order), m[:2], ics.radius_from_mass(m[:2]), st["x"][:2], st["v"][:2])
    a.step(20)
    b.step(20)
    sa, sb = a.state(), b.state()
    np.testing.assert_allclose(sa["x"][:2], sb["x"], rtol=1e-12)
    np.testing.assert_allclose(sa["v"][:2], sb["v"], rtol=1e-10)
    a.close()
    b.close()
