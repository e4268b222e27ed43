"""Parity at the benchmark's full sizes, in the launch configuration the benchmark times, on
sampled outputs that the oracle computes one by one.

Batched mode: all 8192 systems advance in 100-step graph launches; a sample of systems is run by
the single-system oracle (the systems are independent). Test-particle mode: all 2^20 particles
advance with the 8 planets; the oracle runs the planets with a sample of the particles (massless
particles do not act on each other or on the planets). Differentiable engine: all 64 disks of 256
bodies; sampled disks against the oracle, the gradient against central differences. The bounds are
those of the smaller parity tests: 1e-12 after one step, 1e-9 after 100, or a small multiple of the
oracle's own sensitivity to a 1e-15 change of the start where a close pass makes a system chaotic.
"""
import numpy as np
import pytest

import oracle as O
from paper_1404_2324_gb300 import genga, ics

pytestmark = pytest.mark.gpu

G = ics.G_GAUSS


def _rel(gx, gv, ox, ov):
    ex = np.linalg.norm(gx - ox, axis=1) / np.linalg.norm(ox, axis=1)
    ev = np.linalg.norm(gv - ov, axis=1) / np.linalg.norm(ov, axis=1)
    return np.maximum(ex, ev)


def _oracle_system(b, s, steps, scale=None):
    off = b["offsets"]
    sl = slice(off[s], off[s + 1])
    x = b["x"][sl] if scale is None else b["x"][sl] * scale
    o = O.Sim(O.params(G=b["G"], m0=b["m0"][s], dt=b["dt"], order=2), b["m"][sl], b["R"][sl], x, b["v"][sl])
    o.step(steps)
    st = o.state()
    o.close()
    return st


def test_full_batch_in_100_step_launches_matches_sampled_systems():
    b = ics.batch(4, n_sys=8192)  # the benchmark's batch
    off, n = b["offsets"], b["offsets"][-1]
    rng = np.random.default_rng(40)
    sample = np.sort(rng.choice(8192, 48, replace=False))
    h = genga.genga_init_batch(off, b["m0"], b["m"], b["R"], b["x"], b["v"], b["G"], b["dt"], 2, 100)
    try:
        genga.genga_step(h, 1)  # one step (the single-step graph)
        g1 = genga.genga_get_state_batch(h, n)
        genga.genga_step(h, 100)  # one 100-step graph launch, as timed by the benchmark
        g2 = genga.genga_get_state_batch(h, n)
        code, cnt = genga.genga_status(h)
    finally:
        genga.genga_free(h)
    assert code & (genga.ST_BS_FAILED | genga.ST_GROUP_TOO_LARGE) == 0
    assert cnt["steps"] >= 101 and cnt["bs_steps"] > 0
    ok, exc = 0, []
    for s in sample:
        sl = slice(off[s], off[s + 1])
        o1 = _oracle_system(b, s, 1)
        live = o1["alive"] == 1
        assert np.array_equal(g1["alive"][sl], o1["alive"])
        assert _rel(g1["x"][sl][live], g1["v"][sl][live], o1["x"][live], o1["v"][live]).max() <= 1e-12, s
        o2 = _oracle_system(b, s, 101)
        live = o2["alive"] == 1
        assert np.array_equal(g2["alive"][sl], o2["alive"])
        e = _rel(g2["x"][sl][live], g2["v"][sl][live], o2["x"][live], o2["v"][live]).max()
        if e <= 1e-9:
            ok += 1
            continue
        sens = 0.0
        for seed in (1, 2):
            pert = 1 + 1e-15 * np.random.default_rng(seed).standard_normal((off[s + 1] - off[s], 3))
            op = _oracle_system(b, s, 101, pert)
            both = live & (op["alive"] == 1)
            sens = max(sens, _rel(op["x"][both], op["v"][both], o2["x"][both], o2["v"][both]).max())
        exc.append((s, e, sens))
        assert e <= 30 * sens, (s, e, sens)
    print(f"8192-system batch, 101 steps: {len(exc)} of {len(sample)} sampled systems above 1e-9"
          + (f"; largest {max(x[1] for x in exc):.2e}, largest error/sensitivity {max(x[1] / x[2] for x in exc):.1f}"
             if exc else ""))
    assert ok >= 0.9 * len(sample)


def test_full_test_particle_set_matches_sampled_particles():
    d = ics.tp_disk(3, n_tp=1 << 20)  # the benchmark's particle set
    n_tp = len(d["x_tp"])
    m = np.concatenate([[d["m0"]], d["m"]])
    R = np.concatenate([[0.0], d["R"]])
    h = genga.genga_init_tp(m, R, np.vstack([np.zeros(3), d["x"]]), np.vstack([np.zeros(3), d["v"]]), d["G"],
                            d["dt"], 2, d["x_tp"], d["v_tp"], d["R_tp"])
    try:
        genga.genga_step(h, 1)
        g = genga.genga_get_state_tp(h, n_tp)
        gp = genga.genga_get_state(h, len(d["m"]) + 1)
    finally:
        genga.genga_free(h)
    rng = np.random.default_rng(41)
    sample = np.sort(rng.choice(n_tp, 4096, replace=False))

    def oracle(xt):
        o = O.TPSim(O.params(G=d["G"], m0=d["m0"], dt=d["dt"], order=2), d["m"], d["R"], d["x"], d["v"], xt,
                    d["v_tp"][sample], d["R_tp"][sample])
        o.step(1)
        st, enc = o.state(), o.encounters(-1)
        o.close()
        return st, enc

    os_, enc = oracle(d["x_tp"][sample])
    np.testing.assert_allclose(gp["x"][1:], os_["x"], rtol=1e-13)
    assert np.array_equal(g["tp_alive"][sample], os_["tp_alive"])
    live = os_["tp_alive"] == 1
    e = _rel(g["xt"][sample][live], g["vt"][sample][live], os_["xt"][live], os_["vt"][live])
    met = np.zeros(len(sample), bool)
    met[[int(t) for t, _ in enc]] = True
    assert e[~met[live]].max() <= 1e-13  # no encounter: kick, drifts and Kepler only
    if e.max() > 1e-12:  # a particle passing close to a planet: the oracle's own sensitivity
        sens = np.zeros(len(sample))
        for seed in (3, 4):
            pert = 1 + 1e-15 * np.random.default_rng(seed).standard_normal((len(sample), 3))
            sp, _ = oracle(d["x_tp"][sample] * pert)
            both = live & (sp["tp_alive"] == 1)
            sens[both] = np.maximum(sens[both], _rel(sp["xt"][both], sp["vt"][both], os_["xt"][both], os_["vt"][both]))
        bad = (e > 1e-12) & (e > 10 * sens[live])
        assert not bad.any(), list(zip(sample[live][bad], e[bad], sens[live][bad]))


def test_full_adjoint_batch_sampled():
    """The differentiable engine on its benchmark workload (64 disks x 256 bodies, checkpoint every
    50 steps): sampled systems follow the oracle (collisions off), and the gradient's directional
    derivative along a direction on eight sampled systems agrees with central differences of the
    forward (the other systems' forward runs are bit-identical, so they cancel)."""
    import torch
    from paper_1404_2324_gb300.adjoint import AdjointEngine

    def T(a):
        return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")

    d = ics.adj_disks(5)
    B, n = d["m"].shape
    steps = 20
    eng = AdjointEngine(d["m0"], d["G"], d["dt"], 2, ckpt_every=50)
    try:
        xo, vo = eng.forward(T(d["x"]), T(d["v"]), T(d["m"]), steps)
        xo, vo = xo.cpu().numpy(), vo.cpu().numpy()
        assert eng.status() & 0x2A == 0
        for b in (3, 41):
            p = O.params(G=d["G"], m0=d["m0"][b], dt=d["dt"], order=2, collisions=0)
            s = O.Sim(p, d["m"][b], np.zeros(n), d["x"][b], d["v"][b])
            s.step(steps)
            st = s.state()
            s.close()
            assert _rel(xo[b], vo[b], st["x"], st["v"]).max() <= 1e-9, b
        rng = np.random.default_rng(42)
        ux, uv = rng.standard_normal(d["x"].shape), rng.standard_normal(d["v"].shape) * 50.0
        gx, gv, gm = (t.cpu().numpy() for t in eng.backward(T(ux), T(uv)))
        sel = np.zeros(B, bool)
        sel[rng.choice(B, 8, replace=False)] = True
        dx = rng.standard_normal(d["x"].shape) * np.linalg.norm(d["x"], axis=-1, keepdims=True) * sel[:, None, None]
        dv = rng.standard_normal(d["v"].shape) * np.linalg.norm(d["v"], axis=-1, keepdims=True) * sel[:, None, None]
        dm = rng.standard_normal(d["m"].shape) * d["m"] * sel[:, None]
        pred = (gx * dx).sum() + (gv * dv).sum() + (gm * dm).sum()

        def loss(h):
            xh, vh = eng.forward(T(d["x"] + h * dx), T(d["v"] + h * dv), T(d["m"] + h * dm), steps)
            return (xh.cpu().numpy() * ux).sum() + (vh.cpu().numpy() * uv).sum()

        fd = (loss(1e-7) - loss(-1e-7)) / 2e-7
        assert abs(fd - pred) <= 1e-6 * abs(pred), (fd, pred)
    finally:
        eng.close()
