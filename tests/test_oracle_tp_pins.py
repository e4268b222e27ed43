"""Pins of the oracle's test-particle mode (Sect. 3.3) against the pinned main mode and closed forms.

A test particle (TP) must move exactly like a massless body of the main mode: both feel the same
K-weighted kick, Sun drift and Kepler drift. In an encounter the main mode integrates the planet
and the massless body together by BS, while the TP mode keeps the planet on its Kepler path. A
planet whose only group partners are massless feels no pair force, so its BS path is its Kepler
orbit to the BS tolerance, and the two modes agree to ~1e-10.
"""
import numpy as np
import pytest

import oracle as O
from paper_1404_2324_gb300 import ics
from tests import twobody_ref

G = ics.G_GAUSS


def _planets_and_tps(seed=1, ntp=6, near=True):
    rng = np.random.default_rng(seed)
    mp = np.array([3e-6, 1e-5, 5e-6])
    xp, vp = ics.elements_to_cartesian(G * (1 + mp), np.array([0.8, 1.5, 2.6]), np.array([0.02, 0.03, 0.01]),
                                       np.array([0.01, 0.02, 0.0]), *rng.uniform(0, 6.28, (3, 3)))
    if near:  # TPs close to planet 1 so that encounters and BS happen
        xt = xp[1] + rng.normal(0, 0.03, (ntp, 3)) * [1, 1, 0.1]
        vt = vp[1] + rng.normal(0, 0.0008, (ntp, 3)) * [1, 1, 0.1]
    else:
        xt, vt = ics.elements_to_cartesian(G, rng.uniform(1.9, 2.2, ntp), rng.uniform(0, 0.05, ntp),
                                           rng.uniform(0, 0.02, ntp), *rng.uniform(0, 6.28, (3, ntp)))
    return mp, xp, vp, xt, vt


@pytest.mark.parametrize("order", [2, 4])
def test_tp_equals_massless_body_of_main_mode(order):
    mp, xp, vp, xt, vt = _planets_and_tps(near=True)
    p = O.params(G=G, m0=1.0, dt=6.0, order=order, collisions=0, bs_eps=1e-13)
    tp = O.TPSim(p, mp, np.zeros(3), xp, vp, xt, vt)
    m_all = np.concatenate([mp, np.zeros(len(xt))])
    main = O.Sim(p, m_all, np.zeros(len(m_all)), np.vstack([xp, xt]), np.vstack([vp, vt]))
    # the two modes differ only through BS step-size control (one group vs one TP at a time), so
    # the gap follows the BS tolerance: ~1e-14 after a step, a few 1e-12 after 15 close passes
    for steps, bound, vbound in ((1, 1e-13, 1e-10), (14, 2e-11, 2e-9)):
        tp.step(steps)
        main.step(steps)
        a, b = tp.state(), main.state()
        assert np.abs(a["xt"] - b["x"][3:]).max() <= bound * np.abs(b["x"][3:]).max()
        assert np.abs(a["vt"] - b["v"][3:]).max() <= vbound * np.abs(b["v"][3:]).max()
        np.testing.assert_allclose(a["x"], b["x"][:3], rtol=1e-12)
    assert tp.stats()["tp_encounters"] > 0 and tp.stats()["tp_bs_steps"] > 0


def test_tp_without_encounters_matches_main_mode_exactly():
    mp, xp, vp, xt, vt = _planets_and_tps(near=False, seed=2)
    p = O.params(G=G, m0=1.0, dt=6.0, order=2)
    tp = O.TPSim(p, mp, np.zeros(3), xp, vp, xt, vt)
    m_all = np.concatenate([mp, np.zeros(len(xt))])
    main = O.Sim(p, m_all, np.zeros(len(m_all)), np.vstack([xp, xt]), np.vstack([vp, vt]))
    tp.step(20)
    main.step(20)
    assert tp.stats()["tp_encounters"] == 0
    a, b = tp.state(), main.state()
    np.testing.assert_array_equal(a["xt"], b["x"][3:])  # same operations in the same order
    np.testing.assert_array_equal(a["vt"], b["v"][3:])


def test_tp_with_massless_planets_is_kepler_orbit():
    rng = np.random.default_rng(3)
    xt, vt = ics.elements_to_cartesian(G, rng.uniform(0.5, 3, 4), rng.uniform(0, 0.3, 4), rng.uniform(0, 0.2, 4),
                                       *rng.uniform(0, 6.28, (3, 4)))
    mp = np.zeros(2)
    xp, vp = ics.elements_to_cartesian(G, np.array([1.0, 2.0]), np.zeros(2), np.zeros(2), np.zeros(2), np.zeros(2),
                                       np.array([0.0, 3.0]))
    p = O.params(G=G, m0=1.0, dt=5.0, order=4)
    tp = O.TPSim(p, mp, np.zeros(2), xp, vp, xt, vt)
    tp.step(12)
    st = tp.state()
    for i in range(4):
        xr, vr = twobody_ref.propagate(G, xt[i], vt[i], 60.0)
        assert np.linalg.norm(st["xt"][i] - xr) <= 1e-12 * np.linalg.norm(xr)


def test_tp_hitting_a_planet_is_removed_and_planet_untouched():
    mp = np.array([1e-6])
    xp = np.array([[1.0, 0.0, 0.0]]); vp = np.array([[0.0, 0.0172, 0.0]])
    xt = np.array([[1.0, 0.003, 0.0], [1.5, 0.0, 0.0]])
    vt = np.array([[0.0, 0.0172 - 0.0015, 0.0], [0.0, 0.014, 0.0]])
    Rp = np.array([1e-4])
    p = O.params(G=G, m0=1.0, dt=6.0)
    tp = O.TPSim(p, mp, Rp, xp, vp, xt, vt, Rt=np.array([1e-5, 1e-5]))
    ref = O.Sim(p, mp, Rp, xp, vp)
    tp.step(2)
    ref.step(2)
    st = tp.state()
    assert list(st["tp_alive"]) == [0, 1]
    assert tp.stats()["tp_removed"] == 1
    np.testing.assert_array_equal(st["x"], ref.state()["x"])  # the planet never feels a TP
