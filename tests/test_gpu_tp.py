"""Test-particle mode (Sect. 3.3) on the GPU against the oracle's test-particle mode.

Both sides take the same inputs: planets of the test-particle recipe plus test particles, some of
them placed within 0.02 AU of the inner planets so that encounters, Bulirsch-Stoer and removals all
happen. Planets must agree as in the main mode. A particle without an encounter agrees to 1e-13
after one step. A particle passing deep inside a planet's Hill sphere is chaotic: the oracle itself,
started 1e-15 away, moves its velocity by up to ~1e-9 within one step there. Such a particle may
deviate by a small multiple of that self-sensitivity; everything else meets 1e-12 (one step) or
1e-10 (twenty steps) outright.
"""
import numpy as np
import pytest

import oracle as O
from paper_1404_2324_gb300 import genga, ics

pytestmark = pytest.mark.gpu


def _inputs(n_tp=1000, n_near=64, seed=3):
    d = ics.tp_disk(seed, n_tp=n_tp)
    rng = np.random.default_rng(seed)
    # put some particles next to the inner planets (a few planet radii to a few Hill radii away)
    for k in range(n_near):
        j = k % 3
        d["x_tp"][k] = d["x"][j] + rng.normal(0, 0.01, 3) * [1, 1, 0.2]
        d["v_tp"][k] = d["v"][j] + rng.normal(0, 3e-4, 3) * [1, 1, 0.2]
    d["R_tp"] = np.full(n_tp, 1e-6)
    return d


def _gpu(d, order):
    m = np.concatenate([[d["m0"]], d["m"]])
    R = np.concatenate([[0.0], d["R"]])
    x = np.vstack([np.zeros(3), d["x"]])
    v = np.vstack([np.zeros(3), d["v"]])
    return genga.genga_init_tp(m, R, x, v, d["G"], d["dt"], order, d["x_tp"], d["v_tp"], d["R_tp"])


def _oracle(d, order):
    p = O.params(G=d["G"], m0=d["m0"], dt=d["dt"], order=order)
    return O.TPSim(p, d["m"], d["R"], d["x"], d["v"], d["x_tp"], d["v_tp"], d["R_tp"])


def _tp_err(g, o):
    live = o["tp_alive"] == 1
    ex = np.linalg.norm(g["xt"][live] - o["xt"][live], axis=1) / np.linalg.norm(o["xt"][live], axis=1)
    ev = np.linalg.norm(g["vt"][live] - o["vt"][live], axis=1) / np.linalg.norm(o["vt"][live], axis=1)
    return np.maximum(ex, ev), live


def _sensitivity(d, order, steps):
    """Per particle, the largest relative move of the oracle when its start is perturbed by 1e-15
    (positions or velocities of the test particles, two draws each)."""
    base = _oracle(d, order)
    base.step(steps)
    ref = base.state()
    base.close()
    worst = np.zeros(len(d["x_tp"]))
    for seed in range(4):
        rng = np.random.default_rng(100 + seed)
        dp = dict(d)
        key = ("x_tp", "v_tp")[seed % 2]
        dp[key] = d[key] * (1 + 1e-15 * rng.standard_normal(d[key].shape))
        o = _oracle(dp, order)
        o.step(steps)
        st = o.state()
        o.close()
        both = (st["tp_alive"] == 1) & (ref["tp_alive"] == 1)
        e, live = _tp_err(st, {**ref, "tp_alive": both.astype(ref["tp_alive"].dtype)})
        worst[np.where(both)[0]] = np.maximum(worst[np.where(both)[0]], e)
    return worst


def _check(g, os_, sens, tol, mult):
    assert np.array_equal(g["tp_alive"], os_["tp_alive"])
    e, live = _tp_err(g, os_)
    s = sens[live]
    bad = (e > tol) & (e > mult * s)
    over = e > tol
    print(f"{int(over.sum())} of {len(e)} particles above {tol:g}"
          + (f"; largest {e[over].max():.2e}, largest error/sensitivity {(e[over] / np.maximum(s[over], 1e-300)).max():.1f}"
             if over.any() else ""))
    assert not bad.any(), list(zip(np.where(live)[0][bad], e[bad], s[bad]))
    return e, live


@pytest.mark.parametrize("order", [2, 4, 6])
def test_tp_mode_matches_oracle(order):
    d = _inputs()
    n_tp = len(d["x_tp"])
    h = _gpu(d, order)
    o = _oracle(d, order)
    try:
        genga.genga_step(h, 1)
        o.step(1)
        g = genga.genga_get_state_tp(h, n_tp)
        os_ = o.state()
        e, live = _check(g, os_, _sensitivity(d, order, 1), 1e-12, 10.0)
        met = np.zeros(n_tp, bool)
        met[[int(t) for t, _ in o.encounters(-1)]] = True
        assert e[~met[live]].max() <= 1e-13
        gp = genga.genga_get_state(h, len(d["m"]) + 1)
        np.testing.assert_allclose(gp["x"][1:], os_["x"], rtol=1e-13)
        genga.genga_step(h, 19)
        o.step(19)
        g = genga.genga_get_state_tp(h, n_tp)
        os_ = o.state()
        e, live = _check(g, os_, _sensitivity(d, order, 20), 1e-10, 30.0)
        assert np.mean(e <= 1e-10) >= 0.95, np.sort(e)[-10:]
        st = genga.genga_tp_status(h)
        ost = o.stats()
        assert st["tp_encounters"] > 0 and st["tp_bs_steps"] > 0 and st["tp_removed"] > 0
        for k in ("tp_candidates", "tp_encounters", "tp_removed"):
            assert abs(st[k] - ost[k]) <= 0.01 * ost[k] + 2, (k, st[k], ost[k])
    finally:
        genga.genga_free(h)
        o.close()


def test_tp_hitting_a_planet_is_removed():
    mp = np.array([1.0, 1e-6])
    R = np.array([0.0, 1e-4])
    x = np.array([[0, 0, 0], [1.0, 0.0, 0.0]])
    v = np.array([[0, 0, 0], [0.0, 0.0172, 0.0]])
    xt = np.array([[1.0, 0.003, 0.0], [1.5, 0.0, 0.0]])
    vt = np.array([[0.0, 0.0172 - 0.0015, 0.0], [0.0, 0.014, 0.0]])
    h = genga.genga_init_tp(mp, R, x, v, ics.G_GAUSS, 6.0, 2, xt, vt, np.array([1e-5, 1e-5]))
    genga.genga_step(h, 2)
    g = genga.genga_get_state_tp(h, 2)
    assert list(g["tp_alive"]) == [0, 1]
    assert genga.genga_tp_status(h)["tp_removed"] == 1
    genga.genga_free(h)


def test_planets_evolve_as_in_the_main_mode():
    """Test particles are massless: the planets of a test-particle run are bit-identical to a main-mode
    run of the planets alone."""
    d = _inputs(n_tp=77)
    h = _gpu(d, 4)
    m = np.concatenate([[d["m0"]], d["m"]])
    s = genga.Genga(m, np.concatenate([[0.0], d["R"]]), np.vstack([np.zeros(3), d["x"]]),
                    np.vstack([np.zeros(3), d["v"]]), d["G"], d["dt"], 4)
    try:
        genga.genga_step(h, 10)
        s.step(10)
        a = genga.genga_get_state(h, len(m))
        b = s.state()
        assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["v"], b["v"])
    finally:
        genga.genga_free(h)
        s.close()


@pytest.mark.parametrize("n_planets,n_tp", [(33, 4), (2, 0)])
def test_tp_sizes_out_of_range_are_rejected(n_planets, n_tp):
    m = np.concatenate([[1.0], np.full(n_planets, 1e-6)])
    x = np.vstack([np.zeros(3), np.stack([np.arange(1, n_planets + 1), np.zeros(n_planets), np.zeros(n_planets)], 1)])
    v = np.vstack([np.zeros(3), np.zeros((n_planets, 3))])
    v[1:, 1] = 0.0172 / np.sqrt(x[1:, 0])
    xt = np.tile([[1.5, 0.0, 0.0]], (n_tp, 1))
    vt = np.tile([[0.0, 0.014, 0.0]], (n_tp, 1))
    with pytest.raises(genga.GengaError):
        genga.genga_init_tp(m, np.zeros(n_planets + 1), x, v, ics.G_GAUSS, 6.0, 2, xt, vt, np.zeros(n_tp))


@pytest.mark.parametrize("order", [2, 4])
def test_first_step_particle_planet_encounter_pairs_match(order):
    """From identical inputs, the (particle, planet) encounter pairs of the last substep of the first
    step match the oracle's (the Hermite test runs in the same arithmetic; the states it sees differ
    by rounding): any pair in which the lists differ must flip in the oracle itself under a 1e-15
    change of the particles' start."""
    d = _inputs()
    h = _gpu(d, order)
    o = _oracle(d, order)
    try:
        genga.genga_step(h, 1)
        o.step(1)
        gp = {tuple(p) for p in genga.genga_tp_encounters(h)}
        op = {(i, j + 1) for i, j in o.encounters(-1)}  # planets numbered with the central mass at 0
    finally:
        genga.genga_free(h)
        o.close()
    assert len(op) > 10
    diff = gp ^ op
    flip = set()
    rng = np.random.default_rng(0)
    for _ in range(8 if diff else 0):
        dp = dict(d, x_tp=d["x_tp"] * (1 + 1e-15 * rng.standard_normal(d["x_tp"].shape)))
        q = _oracle(dp, order)
        q.step(1)
        flip |= op ^ {(i, j + 1) for i, j in q.encounters(-1)}
        q.close()
    print(f"order {order}: {len(op)} pairs, {len(diff)} differ, {len(diff & flip)} of them at the threshold")
    assert diff <= flip, sorted(diff - flip)


def test_particles_meeting_a_planet_in_a_group_match_oracle():
    """Particles deep in the Hill sphere of a planet that is itself in a close encounter with a second
    planet (the paper's reading: the particle's Bulirsch-Stoer sees the planet on its Kepler path, see
    tests/test_oracle_tp_reading.py for the size of that approximation): the GPU follows the oracle."""
    from tests.test_oracle_tp_reading import config
    m, R, x, v, xt, vt = config(True)
    d = dict(G=ics.G_GAUSS, m0=1.0, dt=6.0, m=m, R=R, x=x, v=v, x_tp=xt, v_tp=vt, R_tp=np.zeros(len(xt)))
    h = _gpu(d, 4)
    o = _oracle(d, 4)
    try:
        genga.genga_step(h, 1)
        o.step(1)
        assert (1, 2) in {tuple(p) for p in genga.genga_encounters(h)}  # the planets' group (central mass at 0)
        met = {int(i) for i, j in genga.genga_tp_encounters(h) if j == 1}
        assert len(met) >= 8
        g = genga.genga_get_state_tp(h, len(xt))
        _check(g, o.state(), _sensitivity(d, 4, 1), 1e-12, 10.0)
        genga.genga_step(h, 4)
        o.step(4)
        g = genga.genga_get_state_tp(h, len(xt))
        _check(g, o.state(), _sensitivity(d, 4, 5), 1e-10, 30.0)
    finally:
        genga.genga_free(h)
        o.close()
