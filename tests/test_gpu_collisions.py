"""Collision reports and spins on the GPU (Sect. 3.2, Collisions) against the oracle: every merger
leaves a report of both bodies' positions, velocities and spins at the start of the BS substep in
which the contact was found, and the survivor's spin takes the pair's orbital angular momentum.
Reports are compared field by field: step, substep, time, pair and survivor exactly, states within
the parity tolerance."""
import numpy as np
import pytest

import oracle as O
from paper_1404_2324_gb300 import genga, ics
from tests.gpu_util import with_central
from tests.test_gpu_groups import swarm

pytestmark = pytest.mark.gpu


def _key(rec):
    """The library's report order: step, substep, time, i, j."""
    return np.lexsort((rec[:, 4], rec[:, 3], rec[:, 2], rec[:, 1], rec[:, 0]))


def _compare_reports(gr, orr, offset=0, tol=1e-9):
    """gr: the library's reports (caller indices, central mass at 0 in the main mode); orr: the
    oracle's (body indices from 0), shifted by `offset` to the library's numbering."""
    orr = orr[_key(orr)].copy()
    for f in (3, 4, 23):
        orr[:, f] += offset
    assert len(gr) == len(orr), (len(gr), len(orr))
    np.testing.assert_array_equal(gr[:, [0, 1, 3, 4, 23]], orr[:, [0, 1, 3, 4, 23]])
    np.testing.assert_allclose(gr[:, 2], orr[:, 2], rtol=0, atol=1e-12 * np.abs(orr[:, 2]).max(initial=1.0))
    for sl in (slice(5, 8), slice(14, 17)):  # positions
        np.testing.assert_allclose(gr[:, sl], orr[:, sl], rtol=0, atol=tol * np.abs(orr[:, sl]).max())
    for sl in (slice(8, 11), slice(17, 20)):  # velocities
        np.testing.assert_allclose(gr[:, sl], orr[:, sl], rtol=0, atol=tol * np.abs(orr[:, sl]).max())
    sp = np.abs(orr[:, 11:14]).max(initial=0.0) + np.abs(orr[:, 20:23]).max(initial=0.0)
    np.testing.assert_allclose(gr[:, 11:14], orr[:, 11:14], rtol=0, atol=tol * sp + 1e-300)
    np.testing.assert_allclose(gr[:, 20:23], orr[:, 20:23], rtol=0, atol=tol * sp + 1e-300)


def _run_pair(d, order, steps, spin0=None):
    m, R, x, v = with_central(d)
    g = genga.Genga(m, R, x, v, d["G"], d["dt"], order)
    o = O.Sim(O.params(G=d["G"], m0=d["m0"], dt=d["dt"], order=order), d["m"], d["R"], d["x"], d["v"])
    if spin0 is not None:
        g.set_spin(np.vstack([np.zeros(3), spin0]))
        o.set_spin(spin0)
    g.step(steps)
    o.step(steps)
    return g, o


@pytest.mark.parametrize("seed,order,steps", [(3, 2, 100), (7, 2, 100), (3, 4, 30)])
def test_collision_reports_match_oracle(seed, order, steps):
    """disk32 with radii enlarged 1000x: mergers from the first step on."""
    d = ics.disk32(seed)
    d["R"] = d["R"] * 1000.0
    rng = np.random.default_rng(seed)
    spin0 = rng.standard_normal((len(d["m"]), 3)) * 1e-14
    g, o = _run_pair(d, order, steps, spin0)
    try:
        gr, orr = g.collisions(), o.collision_records()
        assert len(orr) >= 1
        _compare_reports(gr, orr, offset=1)
        gs, os_ = g.state(), o.state()
        np.testing.assert_array_equal(gs["alive"][1:], os_["alive"])
        np.testing.assert_array_equal(gs["m"][1:], os_["m"])  # merged masses: the same sums
        gsp, osp = g.spin()[1:], o.spin()
        np.testing.assert_allclose(gsp, osp, rtol=0, atol=1e-9 * np.abs(osp).max())
        code, cnt = g.status()
        assert cnt["mergers"] == len(orr) and code & genga.ST_COLL_OVERFLOW == 0
    finally:
        g.close()
        o.close()


def test_angular_momentum_with_spin_is_conserved_on_the_gpu():
    d = ics.disk32(9)
    d["R"] = d["R"] * 1000.0
    m, R, x, v = with_central(d)
    g = genga.Genga(m, R, x, v, d["G"], d["dt"], 2)

    def Ltot():
        st = g.state()
        mm, xx, vv = st["m"][1:], st["x"][1:], st["v"][1:]
        live = st["alive"][1:] == 1
        vb = vv - (mm[:, None] * vv).sum(0) / (d["m0"] + mm.sum())
        return (mm[live, None] * np.cross(xx[live], vb[live])).sum(0) + g.spin()[1:][live].sum(0)

    try:
        L0 = Ltot()
        g.step(160)
        assert g.status()[1]["mergers"] >= 3
        L1 = Ltot()
        assert np.linalg.norm(L1 - L0) <= 1e-11 * np.linalg.norm(L0)
    finally:
        g.close()


def test_mergers_in_a_large_group_are_reported():
    """A 150-member swarm with radii of 1e-4 AU: three mergers on the grid-wide BS kernel."""
    d = swarm(150, n_far=4, seed=40, spread=0.003)
    d["R"][:150] = 1e-4
    g, o = _run_pair(d, 2, 1)
    try:
        orr = o.collision_records()
        assert len(orr) >= 2
        _compare_reports(g.collisions(), orr, offset=1, tol=1e-11)
    finally:
        g.close()
        o.close()


def test_batched_collision_reports_match_oracle():
    """Three 32-body systems (radii enlarged 1000x in two) in the batched mode: each system's reports
    equal the oracle's for that system, with the flat body indices."""
    ds = [ics.disk32(3), ics.disk32(5), ics.disk32(7)]
    ds[0]["R"] = ds[0]["R"] * 1000.0
    ds[2]["R"] = ds[2]["R"] * 1000.0
    off = np.cumsum([0] + [len(d["m"]) for d in ds])
    cat = {k: np.concatenate([d[k] for d in ds]) for k in ("m", "R", "x", "v")}
    h = genga.genga_init_batch(off, np.ones(3), cat["m"], cat["R"], cat["x"], cat["v"], ds[0]["G"], ds[0]["dt"], 2, 1)
    try:
        genga.genga_step(h, 90)
        gr = genga.genga_collisions(h)
        refs = []
        for s, d in enumerate(ds):
            o = O.Sim(O.params(G=d["G"], m0=d["m0"], dt=d["dt"], order=2), d["m"], d["R"], d["x"], d["v"])
            o.step(90)
            r = o.collision_records()
            for f in (3, 4, 23):
                r[:, f] += off[s]
            refs.append(r)
            o.close()
        orr = np.vstack(refs)
        assert len(orr) >= 3
        _compare_reports(gr, orr, offset=0)
        spin = genga.genga_get_spin(h, off[-1])
        assert np.abs(spin).max() > 0.0  # survivors carry the pairs' orbital angular momentum
    finally:
        genga.genga_free(h)
