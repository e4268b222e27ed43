"""Pins of the oracle's collision bookkeeping (Sect. 3.2, Collisions): the spin of a merged body
follows from angular-momentum conservation, and every merger leaves a report of both bodies'
positions, velocities and spins at the last time before the contact. CPU only."""
import numpy as np
import pytest

import oracle as O
from paper_1404_2324_gb300 import ics

G = ics.G_GAUSS


def _total_L(m, x, v, spin, alive):
    """Orbital angular momentum in democratic variables (heliocentric x, barycentric v: the inertial
    total) plus the bodies' spins."""
    live = np.asarray(alive) == 1
    return (m[live, None] * np.cross(x[live], v[live])).sum(0) + spin[live].sum(0)


def _grazing_pair():
    """Two bodies at 1 AU closing at 1e-3 AU/day with an impact parameter of half their radii sum."""
    m = np.array([4e-7, 1e-7])
    R = np.array([2e-5, 1e-5])
    vc = np.sqrt(G)
    x = np.array([[1.0, 0.0, 0.0], [1.0 + 1.5e-5, 0.002, 0.0]])
    v = np.array([[0.0, vc, 0.0], [0.0, vc - 0.001, 0.0]])
    return m, R, x, v


def test_merger_conserves_angular_momentum_with_spin():
    m, R, x, v = _grazing_pair()
    spin0 = np.array([[1e-15, -2e-15, 3e-14], [0.0, 4e-15, -1e-14]])
    p = O.params(G=G, m0=1.0)
    L0 = _total_L(m, x, v, spin0, [1, 1])
    out = O.bs_group(p, [0, 1], 6.0, m, R, [1, 1], x, v, [0.05, 0.05], spin=spin0)
    assert [tuple(c) for c in out["collisions"]] == [(0, 1)]
    L1 = _total_L(out["m"], out["x"], out["v"], out["spin"], out["alive"])
    # the pair's orbital angular momentum about its centre of mass (~1e-15 here against |L| ~ 1e-8)
    # must move into the spin: without it the total would change by ~1e-7 of itself
    assert np.linalg.norm(L1 - L0) <= 1e-12 * np.linalg.norm(L0)
    assert np.all(out["spin"][1] == 0.0)  # the ghost carries nothing
    # a merger without any orbital term would leave the summed spins, which is measurably off
    assert np.linalg.norm(out["spin"][0] - spin0.sum(0)) > 1e-3 * np.linalg.norm(out["spin"][0])


def test_collision_report_is_the_state_before_contact():
    m, R, x, v = _grazing_pair()
    p = O.params(G=G, m0=1.0)
    out = O.bs_group(p, [0, 1], 6.0, m, R, [1, 1], x, v, [0.05, 0.05])
    assert len(out["records"]) == 1
    r = out["records"][0]
    assert (r[3], r[4], r[23]) == (0, 1, 0)  # pair ascending; the heavier body survives
    assert 0.0 <= r[2] < 6.0
    xi, xj = r[5:8], r[14:17]
    assert np.linalg.norm(xj - xi) > R.sum()  # not yet touching at the reported time
    # the reported time and state lie on the pair's path: the first body's state at the report,
    # integrated on its own BS from t = 0, is the reported one (the substeps before the contact)
    if r[2] > 0.0:
        early = O.bs_group(p, [0, 1], r[2], m, R, [1, 1], x, v, [0.05, 0.05])
        np.testing.assert_allclose(early["x"][0], xi, rtol=1e-10)
    else:
        np.testing.assert_array_equal(xi, x[0])


def test_whole_run_conserves_angular_momentum_through_mergers():
    """disk32 with radii enlarged 1000x: five mergers in 300 steps; orbital angular momentum plus
    spins is conserved by the whole step (Sect. 2.1 splitting: every part is rotation invariant) and
    by the mergers (spin bookkeeping), to round-off and the BS tolerance."""
    d = ics.disk32(3)
    R = d["R"] * 1000.0
    p = O.params(G=d["G"], m0=d["m0"], dt=d["dt"], order=2)
    s = O.Sim(p, d["m"], R, d["x"], d["v"])
    st = s.state()

    def Ltot(state, spin):
        P = (state["m"][:, None] * state["v"]).sum(0)
        vb = state["v"] - P / (d["m0"] + state["m"].sum())  # heliocentric -> barycentric
        return _total_L(state["m"], state["x"], vb, spin, state["alive"])

    L0 = Ltot(st, s.spin())
    s.step(300)
    recs = s.collision_records()
    assert s.stats()["collisions"] == len(recs) >= 2
    st1 = s.state()
    L1 = Ltot(st1, s.spin())
    assert np.linalg.norm(L1 - L0) <= 1e-11 * np.linalg.norm(L0)
    Lnospin = Ltot(st1, np.zeros_like(s.spin()))
    assert np.linalg.norm(Lnospin - L0) > 10 * np.linalg.norm(L1 - L0)
    # reports: steps ascending, pairs ascending, survivor is the heavier body of the pair at merge time
    assert np.all(np.diff(recs[:, 0]) >= 0)
    assert np.all(recs[:, 3] < recs[:, 4])
    assert np.all((recs[:, 23] == recs[:, 3]) | (recs[:, 23] == recs[:, 4]))
