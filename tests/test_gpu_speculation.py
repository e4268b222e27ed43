"""Bulirsch-Stoer groups that need many substeps (Sect. 3.2): tight planet binaries in the batched
mode and particles bound to a planet in the test-particle mode.

The step control halves H on a failed attempt and doubles it after an accepted one, so such groups
alternate failed attempts at 2H with accepted ones at H. The GPU kernels attempt H and H/2 side by
side and keep the H/2 result only where the serial control would have attempted H/2 next; these
inputs drive that path hard. The number of accepted substeps must be the oracle's (the oracle runs
the serial control). A binary integrated over 8 to 32 substeps amplifies rounding: the oracle
itself, started 1e-15 away, moves by up to ~4e-11 in one step (a bound particle by up to ~1e-9),
while the binaries' substep counts do not change. A system (a particle) must therefore agree to
1e-12, or to within ten times the oracle's own sensitivity.
"""
import numpy as np
import pytest

import oracle as O
from paper_1404_2324_gb300 import genga, ics

pytestmark = pytest.mark.gpu

G = ics.G_GAUSS


def _circ(mu, r, phi, incl=0.0):
    """Position and velocity of a circular orbit of radius r at phase phi about mass parameter mu."""
    c, s = np.cos(phi), np.sin(phi)
    x = r * np.array([c, s * np.cos(incl), s * np.sin(incl)])
    v = np.sqrt(mu / r) * np.array([-s, c * np.cos(incl), c * np.sin(incl)])
    return x, v


def binaries(n_sys=48, seed=31):
    """Per system: a binary of two planets (masses log-U[3e-5, 1e-4], separation 1.5e-3..3e-3 AU,
    mutual period of one to three days) on a circular orbit at 0.1..0.3 AU, in every third system a
    third planet loosely bound to the pair, and two distant planets."""
    rng = np.random.default_rng(seed)
    m, x, v, off = [], [], [], [0]
    for s in range(n_sys):
        mA, mB = np.exp(rng.uniform(np.log(3e-5), np.log(1e-4), 2))
        xA, vA = _circ(G * (1.0 + mA), rng.uniform(0.1, 0.3), rng.uniform(0, 2 * np.pi))
        sep, psi = rng.uniform(1.5e-3, 3e-3), rng.uniform(0, 2 * np.pi)
        dx, dv = _circ(G * (mA + mB), sep, psi, rng.uniform(0.0, 0.3))
        body_m = [mA, mB]
        body_x = [xA - mB / (mA + mB) * dx, xA + mA / (mA + mB) * dx]
        body_v = [vA - mB / (mA + mB) * dv, vA + mA / (mA + mB) * dv]
        if s % 3 == 0:  # a third member inside the pair's critical radius
            mC = np.exp(rng.uniform(np.log(1e-6), np.log(1e-5)))
            ex, ev = _circ(G * (mA + mB), 4.0 * sep, rng.uniform(0, 2 * np.pi), 0.2)
            body_m.append(mC)
            body_x.append(xA + ex)
            body_v.append(vA + 0.8 * ev)
        for _ in range(2):
            xf, vf = _circ(G, rng.uniform(1.0, 4.0), rng.uniform(0, 2 * np.pi), rng.uniform(0, 0.02))
            body_m.append(1e-6)
            body_x.append(xf)
            body_v.append(vf)
        m += body_m
        x += body_x
        v += body_v
        off.append(len(m))
    m = np.array(m)
    return dict(m0=np.ones(n_sys), G=G, m=m, R=ics.radius_from_mass(m), x=np.array(x), v=np.array(v),
                offsets=np.array(off), dt=6.0)


def _rel(a, b, live):
    ex = np.linalg.norm(a["x"][live] - b["x"][live], axis=1) / np.linalg.norm(b["x"][live], axis=1)
    ev = np.linalg.norm(a["v"][live] - b["v"][live], axis=1) / np.linalg.norm(b["v"][live], axis=1)
    return np.maximum(ex, ev)


def _oracle_system(b, sl, x, v):
    o = O.Sim(O.params(G=G, m0=1.0, dt=b["dt"], order=2), b["m"][sl], b["R"][sl], x, v)
    o.step(1)
    st, n, gmax = o.state(), o.stats()["bs_steps"], max(len(k) for k in o.groups(0))
    o.close()
    return st, n, gmax


def test_tight_binaries_follow_the_oracle_in_the_batched_mode():
    b = binaries()
    off, n = b["offsets"], b["offsets"][-1]
    h = genga.genga_init_batch(off, b["m0"], b["m"], b["R"], b["x"], b["v"], b["G"], b["dt"], 2, 1)
    try:
        genga.genga_step(h, 1)
        g = genga.genga_get_state_batch(h, n)
        code, cnt = genga.genga_status(h)
    finally:
        genga.genga_free(h)
    bs_steps = []
    for s in range(len(off) - 1):
        sl = slice(off[s], off[s + 1])
        st, nbs, gmax = _oracle_system(b, sl, b["x"][sl], b["v"][sl])
        bs_steps.append(nbs)
        assert gmax >= 2
        assert np.array_equal(g["alive"][sl], st["alive"])
        live = st["alive"] == 1
        err = _rel({k: g[k][sl] for k in ("x", "v")}, st, live).max()
        if err > 1e-12:  # the oracle's own sensitivity to a 1e-15 change of the start
            sens = 0.0
            for seed in range(4):
                rng = np.random.default_rng(200 + seed)
                key = ("x", "v")[seed % 2]
                pert = {k: b[k][sl].copy() for k in ("x", "v")}
                pert[key] *= 1 + 1e-15 * rng.standard_normal(pert[key].shape)
                sp, _, _ = _oracle_system(b, sl, pert["x"], pert["v"])
                both = live & (sp["alive"] == 1)
                sens = max(sens, _rel(sp, st, both).max())
            assert err <= 10.0 * sens, (s, err, sens)
    assert min(bs_steps) >= 4 and max(bs_steps) >= 8, (min(bs_steps), max(bs_steps))  # many substeps
    assert code & (genga.ST_BS_FAILED | genga.ST_GROUP_TOO_LARGE) == 0
    assert cnt["bs_steps"] == sum(bs_steps)


def bound_particles(n_bound=96, n_free=32, seed=32):
    """A Jupiter-mass planet at 1 AU and two small planets, with particles on circular orbits about
    the big planet at 0.002..0.01 AU (periods of one to eleven days) and others far from all
    planets."""
    rng = np.random.default_rng(seed)
    mp = np.array([1e-3, 1e-6, 3e-6])
    xs, vs = zip(*[_circ(G * (1 + mp[0]), 1.0, 0.3), _circ(G, 1.6, 2.0), _circ(G, 2.5, 4.0)])
    xp, vp = np.array(xs), np.array(vs)
    xt, vt = [], []
    for k in range(n_bound):
        dx, dv = _circ(G * mp[0], rng.uniform(0.002, 0.01), rng.uniform(0, 2 * np.pi), rng.uniform(0, 0.5))
        xt.append(xp[0] + dx)
        vt.append(vp[0] + dv)
    for k in range(n_free):
        x1, v1 = _circ(G, rng.uniform(3.0, 4.0), rng.uniform(0, 2 * np.pi), rng.uniform(0, 0.1))
        xt.append(x1)
        vt.append(v1)
    return dict(m0=1.0, m=mp, R=ics.radius_from_mass(mp), x=xp, v=vp, x_tp=np.array(xt), v_tp=np.array(vt),
                R_tp=np.full(n_bound + n_free, 1e-7), dt=6.0)


def test_bound_particles_follow_the_oracle_in_the_test_particle_mode():
    d = bound_particles()
    n_tp = len(d["x_tp"])
    m = np.concatenate([[1.0], d["m"]])
    R = np.concatenate([[0.0], d["R"]])
    h = genga.genga_init_tp(m, R, np.vstack([np.zeros(3), d["x"]]), np.vstack([np.zeros(3), d["v"]]), G, d["dt"], 2,
                            d["x_tp"], d["v_tp"], d["R_tp"])
    o = O.TPSim(O.params(G=G, m0=1.0, dt=d["dt"], order=2), d["m"], d["R"], d["x"], d["v"], d["x_tp"], d["v_tp"],
                d["R_tp"])
    try:
        genga.genga_step(h, 1)
        o.step(1)
        g = genga.genga_get_state_tp(h, n_tp)
        st = genga.genga_tp_status(h)
        os_, ost = o.state(), o.stats()
    finally:
        genga.genga_free(h)
        o.close()
    assert np.array_equal(g["tp_alive"], os_["tp_alive"])
    live = os_["tp_alive"] == 1
    err = _rel({"x": g["xt"], "v": g["vt"]}, {"x": os_["xt"], "v": os_["vt"]}, live)
    if err.max() > 1e-12:  # per particle, the oracle's own sensitivity to a 1e-15 change of the start
        sens = np.zeros(n_tp)
        for seed in range(4):
            rng = np.random.default_rng(300 + seed)
            key = ("x_tp", "v_tp")[seed % 2]
            dp = dict(d)
            dp[key] = d[key] * (1 + 1e-15 * rng.standard_normal(d[key].shape))
            op = O.TPSim(O.params(G=G, m0=1.0, dt=d["dt"], order=2), d["m"], d["R"], d["x"], d["v"], dp["x_tp"],
                         dp["v_tp"], d["R_tp"])
            op.step(1)
            sp = op.state()
            op.close()
            both = live & (sp["tp_alive"] == 1)
            e = _rel({"x": sp["xt"], "v": sp["vt"]}, {"x": os_["xt"], "v": os_["vt"]}, both)
            sens[both] = np.maximum(sens[both], e)
        bad = (err > 1e-12) & (err > 10.0 * sens[live])
        assert not bad.any(), list(zip(np.where(live)[0][bad], err[bad], sens[live][bad]))
    assert ost["tp_bs_steps"] >= 4 * 96  # the bound particles need several substeps each
    # a particle circling the planet at a few planet-Hill-radius hundredths is chaotic even in its
    # step decisions: the oracle's own substep count moves by up to 2 (of ~1510) when the start
    # changes by 1e-15, so twice that is allowed
    assert abs(st["tp_bs_steps"] - ost["tp_bs_steps"]) <= 4, (st["tp_bs_steps"], ost["tp_bs_steps"])
    assert st["tp_encounters"] == ost["tp_encounters"]
