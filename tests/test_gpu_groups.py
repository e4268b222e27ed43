"""Large encounter groups on the GPU: groups of 5 or more members are integrated by the cluster BS
kernel (one thread-block cluster per group, one CTA per extrapolation level), smaller ones by the
one-CTA kernel, groups of 33 to 64 members by the wide one-CTA kernel (512 threads). A compact
swarm puts one large group through these kernels; its result must follow the oracle like any
other group (Sect. 3.2, Bulirsch-Stoer). A group above 64 members is reported, not integrated.
"""
import numpy as np
import pytest

import oracle as O
from paper_1404_2324_gb300 import genga, ics
from tests.gpu_util import rel_state_error, with_central

pytestmark = pytest.mark.gpu


def swarm(n_swarm, n_far=8, seed=21, spread=0.004):
    """n_swarm bodies within a few 1e-3 AU of each other at 1 AU (one encounter group), plus n_far
    bodies on ordinary orbits elsewhere."""
    rng = np.random.default_rng(seed)
    G = ics.G_GAUSS
    xs = np.array([1.0, 0.0, 0.0]) + rng.normal(0.0, spread, (n_swarm, 3)) * [1.0, 1.0, 0.2]
    vc = np.sqrt(G / 1.0)
    vs = np.array([0.0, vc, 0.0]) + rng.normal(0.0, 2e-5, (n_swarm, 3))
    ms = np.exp(rng.uniform(np.log(1e-10), np.log(1e-9), n_swarm))
    far = ics._disk(rng, n_far, 1e-8, 1e-7, 1.5, 3.0, 0.01, 0.005)
    d = dict(m0=1.0, G=G, m=np.concatenate([ms, far["m"]]), x=np.vstack([xs, far["x"]]),
             v=np.vstack([vs, far["v"]]), dt=6.0)
    d["R"] = ics.radius_from_mass(d["m"]) * 1e-3  # small radii: no contact inside the swarm
    return d


def _pair(d, order):
    m, R, x, v = with_central(d)
    g = genga.Genga(m, R, x, v, d["G"], d["dt"], order)
    p = O.params(G=d["G"], m0=d["m0"], dt=d["dt"], order=order)
    o = O.Sim(p, d["m"], d["R"], d["x"], d["v"])
    return g, o


@pytest.mark.parametrize("order", [2, 4])
def test_large_group_follows_the_oracle(order):
    d = swarm(12)
    g, o = _pair(d, order)
    try:
        g.step(1)
        o.step(1)
        sizes = [len(k) for k in o.groups(0)]
        assert max(sizes) >= 5  # the cluster kernel took part
        err, same = rel_state_error(g, o)
        assert same and err <= 1e-12, err
        g.step(9)
        o.step(9)
        err, same = rel_state_error(g, o)
        assert same and err <= 1e-9, err
        code, cnt = g.status()
        assert code & (genga.ST_BS_FAILED | genga.ST_GROUP_TOO_LARGE) == 0
        assert cnt["bs_steps"] == o.stats()["bs_steps"]
    finally:
        g.close()
        o.close()


def test_group_of_thirty_two_members():
    d = swarm(32, n_far=4, seed=22, spread=0.003)
    g, o = _pair(d, 2)
    try:
        g.step(1)
        o.step(1)
        assert max(len(k) for k in o.groups(0)) == 32
        err, same = rel_state_error(g, o)
        assert same and err <= 1e-12, err
        assert g.status()[0] & genga.ST_GROUP_TOO_LARGE == 0
    finally:
        g.close()
        o.close()


@pytest.mark.parametrize("n_swarm", [40, 64])
def test_groups_above_thirty_two_members(n_swarm):
    d = swarm(n_swarm, n_far=4, seed=24 + n_swarm, spread=0.003)
    g, o = _pair(d, 2)
    try:
        g.step(1)
        o.step(1)
        assert max(len(k) for k in o.groups(0)) == n_swarm
        err, same = rel_state_error(g, o)
        assert same and err <= 1e-12, err
        code, cnt = g.status()
        assert code & (genga.ST_BS_FAILED | genga.ST_GROUP_TOO_LARGE) == 0
        assert cnt["bs_steps"] == o.stats()["bs_steps"]
    finally:
        g.close()
        o.close()


def test_large_group_in_a_batched_system():
    """A batched system of 48 bodies, 40 of them in one swarm (queue 3, the wide kernel), next to
    two ordinary systems."""
    ds = [swarm(40, n_far=8, seed=30, spread=0.003), swarm(3, n_far=5, seed=31), swarm(2, n_far=10, seed=32)]
    off = np.cumsum([0] + [len(d["m"]) for d in ds])
    cat = {k: np.concatenate([d[k] for d in ds]) for k in ("m", "R", "x", "v")}
    h = genga.genga_init_batch(off, np.ones(3), cat["m"], cat["R"], cat["x"], cat["v"], ds[0]["G"], ds[0]["dt"], 2, 1)
    try:
        genga.genga_step(h, 1)
        gs = genga.genga_get_state_batch(h, off[-1])
        code, _ = genga.genga_status(h)
        assert code & (genga.ST_BS_FAILED | genga.ST_GROUP_TOO_LARGE) == 0
        for s, d in enumerate(ds):
            o = O.Sim(O.params(G=d["G"], m0=d["m0"], dt=d["dt"], order=2), d["m"], d["R"], d["x"], d["v"])
            o.step(1)
            if s == 0:
                assert max(len(k) for k in o.groups(0)) == 40
            st = o.state()
            sl = slice(off[s], off[s + 1])
            assert np.array_equal(gs["alive"][sl], st["alive"])
            live = st["alive"] == 1
            e = np.linalg.norm(gs["x"][sl][live] - st["x"][live], axis=1) / np.linalg.norm(st["x"][live], axis=1)
            assert e.max() <= 1e-12, (s, e.max())
            o.close()
    finally:
        genga.genga_free(h)


def test_group_above_the_cap_is_reported():
    d = swarm(80, n_far=4, seed=23, spread=0.003)
    m, R, x, v = with_central(d)
    g = genga.Genga(m, R, x, v, d["G"], d["dt"], 2)
    try:
        g.step(1)
        assert g.status()[0] & genga.ST_GROUP_TOO_LARGE
    finally:
        g.close()
