"""Ejections (Sect. 3.2) and the batched stop below Nmin (Sect. 3.4) on the GPU against the oracle:
which bodies leave at the end of which step, their recorded heliocentric state, the energy booked
into U, and the motion of the bodies that stay."""
import numpy as np
import pytest

import oracle as O
from paper_1404_2324_gb300 import genga, ics

pytestmark = pytest.mark.gpu

G = ics.G_GAUSS


def _escape_system():
    """A Jupiter-mass planet at 5.2 AU, an Earth at 1 AU, two Earth-mass bodies escaping from
    +-0.8 AU at 1.35 and 1.3 times the escape speed, and a body on an e = 0.9 orbit (periapsis
    0.1 AU) that passes inside RcutSun = 0.3 AU."""
    m = np.array([1e-3, 3e-6, 3e-6, 2e-6, 1e-7])
    ve = np.sqrt(2 * G / 0.8)
    x = np.array([[5.2, 0.0, 0.0], [0.0, 1.0, 0.0], [-0.8, 0.0, 0.05], [0.8, 0.0, -0.03], [-1.9, 0.0, 0.0]])
    v = np.array([[0.0, np.sqrt(G / 5.2), 0.0], [-np.sqrt(G), 0.0, 0.0], [0.0, -1.35 * ve, 0.0], [0.0, 1.3 * ve, 0.0],
                  [0.0, -np.sqrt(G * 0.1 / 1.9), 0.0]])
    return m, ics.radius_from_mass(m), x, v


def _gpu_params(**kw):
    p = genga.genga_default_params()
    for k, val in kw.items():
        setattr(p, k, val)
    return p


def _with_central(m, R, x, v, m0=1.0):
    return (np.concatenate([[m0], m]), np.concatenate([[0.0], R]), np.vstack([np.zeros(3), x]),
            np.vstack([np.zeros(3), v]))


@pytest.mark.parametrize("order", [2, 4])
def test_escapes_and_plunge_follow_the_oracle(order):
    m, R, x, v = _escape_system()
    dt, steps, rcut, rsun = 2.0, 260, 8.0, 0.3
    o = O.Sim(O.params(G=G, m0=1.0, dt=dt, order=order, rcut=rcut, rcut_sun=rsun), m, R, x, v)
    g = genga.Genga(*_with_central(m, R, x, v), G, dt, order, params=_gpu_params(rcut=rcut, rcut_sun=rsun))
    try:
        for k in range(steps):
            o.step(1)
            g.step(1)
            if k % 20 == 19 or k == steps - 1:
                st, os_ = g.state(), o.state()
                assert np.array_equal(st["alive"][1:], os_["alive"]), k
        oe = o.ejections()
        ge = genga.genga_ejections(g.ctx)
        assert len(oe) == 3  # both escapers and the plunging body
        assert np.array_equal(ge[:, 0], oe[:, 0] + 1) and np.array_equal(ge[:, 1], oe[:, 1])
        np.testing.assert_allclose(ge[:, 2:], oe[:, 2:], rtol=1e-9, atol=1e-13)
        E, U = g.energy()
        Eo, Uo = o.energy()
        np.testing.assert_allclose(U, Uo, rtol=1e-9)
        np.testing.assert_allclose(E + U, Eo + Uo, rtol=1e-9)  # U is ~3 % of E here
        st, os_ = g.state(), o.state()
        live = os_["alive"] == 1
        np.testing.assert_allclose(st["x"][1:][live], os_["x"][live], rtol=1e-9)
        np.testing.assert_allclose(st["v"][1:][live], os_["v"][live], rtol=1e-8)
        code, _ = genga.genga_status(g.ctx)
        assert code & genga.ST_BS_FAILED == 0
    finally:
        g.close()
        o.close()


def test_many_ejections_in_one_step():
    """The 2048-body disk with Rcut inside its outer edge: every body beyond 3.5 AU leaves at the
    end of the first step, at once; the rest then move as in the oracle."""
    d = ics.disk2048(2)
    rcut = 3.5
    p = O.params(G=d["G"], m0=d["m0"], dt=d["dt"], order=4, rcut=rcut)
    o = O.Sim(p, d["m"], d["R"], d["x"], d["v"])
    g = genga.Genga(*_with_central(d["m"], d["R"], d["x"], d["v"], d["m0"]), d["G"], d["dt"], 4,
                    params=_gpu_params(rcut=rcut))
    try:
        o.step(1)
        g.step(1)
        oe, ge = o.ejections(), genga.genga_ejections(g.ctx)
        assert 100 < len(oe) < 1024
        assert np.array_equal(ge[:, 0], oe[:, 0] + 1) and np.all(ge[:, 1] == 1)
        np.testing.assert_allclose(ge[:, 2:5], oe[:, 2:5], rtol=1e-12)
        np.testing.assert_allclose(ge[:, 5:], oe[:, 5:], rtol=1e-10)
        np.testing.assert_allclose(g.energy()[1], o.energy()[1], rtol=1e-10)
        o.step(4)
        g.step(4)
        st, os_ = g.state(), o.state()
        assert np.array_equal(st["alive"][1:], os_["alive"])
        live = os_["alive"] == 1
        ex = np.linalg.norm(st["x"][1:][live] - os_["x"][live], axis=1) / np.linalg.norm(os_["x"][live], axis=1)
        assert ex.max() <= 1e-10
    finally:
        g.close()
        o.close()


def test_test_particles_and_planets_leave():
    """Planets and particles beyond Rcut (or inside RcutSun) leave at the same step as in the oracle."""
    d = ics.tp_disk(3, n_tp=2048)
    rcut, rsun = 4.0, 0.35
    p = O.params(G=d["G"], m0=d["m0"], dt=d["dt"], order=2, rcut=rcut, rcut_sun=rsun)
    o = O.TPSim(p, d["m"], d["R"], d["x"], d["v"], d["x_tp"], d["v_tp"], d["R_tp"])
    m = np.concatenate([[d["m0"]], d["m"]])
    R = np.concatenate([[0.0], d["R"]])
    h = genga.genga_init_tp(m, R, np.vstack([np.zeros(3), d["x"]]), np.vstack([np.zeros(3), d["v"]]), d["G"], d["dt"],
                            2, d["x_tp"], d["v_tp"], d["R_tp"])
    try:
        genga.genga_set_params(h, _gpu_params(rcut=rcut, rcut_sun=rsun))
        for _ in range(3):
            o.step(1)
            genga.genga_step(h, 1)
            g = genga.genga_get_state_tp(h, len(d["x_tp"]))
            assert np.array_equal(g["tp_alive"], o.state()["tp_alive"])
        gp = genga.genga_get_state(h, len(d["m"]) + 1)
        assert np.array_equal(gp["alive"][1:], o.state()["alive"])
        assert genga.genga_tp_status(h)["tp_ejected"] == o.stats()["tp_ejected"] > 0
        oe, ge = o.ejections(), genga.genga_ejections(h)
        assert len(oe) > 0 and np.array_equal(ge[:, 0], oe[:, 0] + 1) and np.array_equal(ge[:, 1], oe[:, 1])
        np.testing.assert_allclose(ge[:, 2:], oe[:, 2:], rtol=1e-10)
    finally:
        genga.genga_free(h)
        o.close()


def test_batched_ejections_and_nmin_stop():
    """Three systems: the escape system, a two-planet system whose outer planet escapes (then fewer
    than Nmin = 2 bodies: stopped, everything removed) and a quiet one."""
    m1, R1, x1, v1 = _escape_system()
    m2 = np.array([3e-6, 1e-6])
    x2 = np.array([[1.0, 0.0, 0.0], [0.0, -0.9, 0.0]])
    v2 = np.array([[0.0, np.sqrt(G), 0.0], [1.3 * np.sqrt(2 * G / 0.9), 0.0, 0.0]])
    R2 = ics.radius_from_mass(m2)
    m3 = np.array([2e-6, 4e-6, 1e-6])
    x3 = np.array([[0.7, 0.0, 0.0], [0.0, 1.3, 0.01], [-2.0, 0.0, 0.0]])
    v3 = np.array([[0.0, np.sqrt(G / 0.7), 0.0], [-np.sqrt(G / 1.3), 0.0, 0.0], [0.0, -np.sqrt(G / 2.0), 0.0]])
    R3 = ics.radius_from_mass(m3)
    systems = [(m1, R1, x1, v1), (m2, R2, x2, v2), (m3, R3, x3, v3)]
    off = np.cumsum([0] + [len(s[0]) for s in systems])
    cat = [np.concatenate([s[k] for s in systems]) for k in range(4)]
    dt, steps, rcut, rsun = 2.0, 260, 8.0, 0.3
    h = genga.genga_init_batch(off, np.ones(3), cat[0], cat[1], cat[2], cat[3], G, dt, 2, 1)
    orc = [O.Sim(O.params(G=G, m0=1.0, dt=dt, order=2, rcut=rcut, rcut_sun=rsun), *s) for s in systems]
    try:
        genga.genga_set_params(h, _gpu_params(rcut=rcut, rcut_sun=rsun, nmin=2))
        stop_step, E_at_stop = None, None
        for k in range(1, steps + 1):
            genga.genga_step(h, 1)
            for o in orc:
                o.step(1)
            if stop_step is None and orc[1].state()["alive"].sum() < 2:
                stop_step = k
                E_at_stop = sum(orc[1].energy())  # E + U of system 2 just before its removals
        g = genga.genga_get_state_batch(h, off[-1])
        assert stop_step is not None
        assert np.array_equal(g["alive"][off[0]:off[1]], orc[0].state()["alive"])
        assert not g["alive"][off[1]:off[2]].any()  # stopped: every body removed
        assert np.array_equal(g["alive"][off[2]:off[3]], orc[2].state()["alive"]) and g["alive"][off[2]:off[3]].all()
        for s, o in ((0, orc[0]), (2, orc[2])):
            live = o.state()["alive"] == 1
            np.testing.assert_allclose(g["x"][off[s]:off[s + 1]][live], o.state()["x"][live], rtol=1e-9)
        ge = genga.genga_ejections(h)
        ge = ge[np.lexsort((ge[:, 0], ge[:, 1]))]
        oe = np.vstack([orc[0].ejections() + [off[0], 0, 0, 0, 0, 0, 0, 0],
                        orc[1].ejections() + [off[1], 0, 0, 0, 0, 0, 0, 0]])
        oe = oe[np.lexsort((oe[:, 0], oe[:, 1]))]
        assert np.array_equal(ge[:, :2], oe[:, :2])
        np.testing.assert_allclose(ge[:, 2:], oe[:, 2:], rtol=1e-9, atol=1e-13)
        _, U = genga.genga_energy_batch(h, 3)
        np.testing.assert_allclose(U, orc[0].energy()[1] + E_at_stop, rtol=1e-9)
    finally:
        genga.genga_free(h)
        for o in orc:
            o.close()


def test_off_by_default_changes_nothing():
    m, R, x, v = _escape_system()
    g = genga.Genga(*_with_central(m, R, x, v), G, 2.0, 2)
    try:
        g.step(300)
        assert g.state()["alive"].all() and len(genga.genga_ejections(g.ctx)) == 0
        assert genga.genga_launch_count(g.ctx) == 4 + 7  # no ejection kernel in the step graph
    finally:
        g.close()
