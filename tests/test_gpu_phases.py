"""GPU parity of each step of the method, fed the oracle's inputs (phase entry points of the C ABI).

Tolerances: FP64 kernels that differ from the oracle only in summation order and in ~1-ulp
reciprocal/square-root estimates agree to a few 1e-16 per operation; the bounds below (1e-13 on
accelerations relative to the largest, 1e-13 on Kepler drifts, 1e-11 on Bulirsch-Stoer groups,
whose step-size decisions use the same rule on values that differ by ulps) leave two to three
orders of margin. Decisions taken on integers or exact comparisons (precheck, encounter lists,
groups) must match bit for bit.
"""
import numpy as np
import pytest

import oracle as O
from paper_1404_2324_gb300 import genga, ics
from tests.gpu_util import aos, dev, soa, torch

pytestmark = pytest.mark.gpu


def _ulp_err(got, ref_ld):
    ref = ref_ld.astype(np.float64)
    return np.max(np.abs((got.astype(np.longdouble) - ref_ld) / np.spacing(np.abs(ref)).astype(np.longdouble)))


def test_refined_reciprocal_and_roots_within_two_ulp():
    rng = np.random.default_rng(1)
    x = np.exp(rng.uniform(np.log(1e-30), np.log(1e30), 200000))
    xin = dev(x)
    out = torch().empty_like(xin)
    xl = x.astype(np.longdouble)
    for which, ref in ((0, 1 / np.sqrt(xl)), (1, 1 / (xl * np.sqrt(xl))), (2, 1 / xl)):
        genga.genga_phase_mathcheck(len(x), which, xin, out)
        assert _ulp_err(out.cpu().numpy(), ref) <= 2.0, which
    xs = -x[:1000]
    genga.genga_phase_mathcheck(len(xs), 2, dev(xs), out)
    assert _ulp_err(out.cpu().numpy()[:1000], 1 / xs.astype(np.longdouble)) <= 2.0


def _state2048(seed=2):
    d = ics.disk2048(seed)
    p = O.params(G=d["G"], m0=d["m0"], dt=d["dt"], order=4)
    return d, p


def test_rcrit_matches_oracle():
    d, p = _state2048()
    n = len(d["m"])
    alive = np.ones(n, np.int32); alive[[5, 77]] = 0
    ref = O.rcrit(p, 6.0, d["m"], alive, d["x"], d["v"])
    rc = dev(np.zeros(n))
    genga.genga_phase_rcrit(n, d["G"], d["m0"], 3.0, 0.4, 6.0, dev(d["m"]), dev(alive), soa(d["x"]), soa(d["v"]), rc)
    got = rc.cpu().numpy()
    np.testing.assert_allclose(got[alive == 1], ref[alive == 1], rtol=2e-15)
    assert np.all(got[alive == 0] == 0.0)


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 100, 2048])
@pytest.mark.parametrize("kmode,precise", [(0, 0), (1, 0), (0, 1)])
def test_kick_accelerations_and_precheck_match_oracle(n, kmode, precise):
    d, p = _state2048()
    p.kmode = kmode
    rng = np.random.default_rng(n)
    sel = np.sort(rng.choice(2048, n, replace=False))
    m, x, v = d["m"][sel], d["x"][sel], d["v"][sel]
    alive = np.ones(n, np.int32)
    if n > 10:
        alive[rng.choice(n, 2, replace=False)] = 0
    rc = O.rcrit(p, 6.0, m, alive, x, v) * (1.0 if n > 200 else 25.0)  # small sets: force near pairs
    ref_a = O.accel_B(p, m, alive, x, rc)
    ref_c = O.precheck(p, alive, x, rc)
    a = dev(np.zeros((3, n)))
    cap = max(1, n * (n - 1) // 2)
    cand = dev(np.zeros(2 * cap, np.int32))
    cnt = genga.genga_phase_kick(n, d["G"], 3.0, kmode, precise, dev(m), dev(alive), soa(x), dev(rc), a, cand, cap)
    got_c = cand.cpu().numpy()[: 2 * cnt].reshape(-1, 2)
    assert cnt == len(ref_c)
    np.testing.assert_array_equal(got_c, ref_c)
    got_a = aos(a)
    scale = np.abs(ref_a).max() if n > 1 else 1.0
    np.testing.assert_allclose(got_a, ref_a, rtol=0, atol=1e-13 * scale)
    if n >= 100:
        assert cnt > 0  # the transition zone was exercised


@pytest.mark.parametrize("dt", [6.0, -10.2144862, 0.0])
def test_kepler_drift_matches_oracle(dt):
    d, p = _state2048()
    n = 2048
    x, v = d["x"].copy(), d["v"].copy()
    # add a few eccentric and unbound orbits
    x[:3] = [[0.3, 0.0, 0.0], [4.0, 1.0, 0.2], [1.0, 0.0, 0.0]]
    v[:3] = [[0.0, 0.0400, 0.0], [0.0, 0.0030, 0.001], [0.0, 0.0300, 0.0]]
    alive = np.ones(n, np.int32)
    X, V, fail = soa(x), soa(v), dev(np.zeros(n, np.int32))
    genga.genga_phase_kepler(n, d["G"] * d["m0"], dt, 30, dev(alive), X, V, fail)
    gx, gv = aos(X), aos(V)
    assert fail.cpu().numpy().sum() == 0
    for i in range(n):
        rx, rv, st, _ = O.kepler_drift(d["G"] * d["m0"], x[i], v[i], dt)
        assert st == 0
        assert np.linalg.norm(gx[i] - rx) <= 1e-13 * np.linalg.norm(rx)
        assert np.linalg.norm(gv[i] - rv) <= 1e-13 * np.linalg.norm(rv)


@pytest.mark.parametrize("tau", [6.0, -10.2144862])
def test_encounter_list_is_bit_exact(tau):
    d, p = _state2048()
    n = 2048
    alive = np.ones(n, np.int32); alive[11] = 0
    rc = O.rcrit(p, 6.0, d["m"], alive, d["x"], d["v"]) * 2.0
    cand = O.precheck(p, alive, d["x"], rc)
    x1, v1 = d["x"].copy(), d["v"].copy()
    for i in range(n):
        x1[i], v1[i], st, _ = O.kepler_drift(d["G"] * d["m0"], d["x"][i], d["v"][i], tau)
    ref = O.encounters(alive, d["x"], d["v"], x1, v1, rc, cand, tau)
    assert len(ref) > 50
    cap = len(cand) + 1
    out = dev(np.zeros(2 * cap, np.int32))
    cnt = genga.genga_phase_encounters(n, dev(alive), soa(d["x"]), soa(d["v"]), soa(x1), soa(v1), dev(rc),
                                       dev(cand.reshape(-1)), len(cand), tau, out, cap)
    np.testing.assert_array_equal(out.cpu().numpy()[: 2 * cnt].reshape(-1, 2), ref)


@pytest.mark.parametrize("npairs", [0, 1, 300, 3000])
def test_groups_match_oracle(npairs):
    n = 2048
    rng = np.random.default_rng(npairs)
    pairs = set()
    while len(pairs) < npairs:
        i, j = sorted(rng.choice(n, 2, replace=False))
        pairs.add((int(i), int(j)))
    pairs = np.array(sorted(pairs), np.int32).reshape(-1, 2)
    single = np.zeros(n, np.int32); single[[0, 2047, 1000]] = 1
    ref = O.groups(n, pairs, single)
    gs, mem = dev(np.zeros(n + 1, np.int32)), dev(np.zeros(n, np.int32))
    ng = genga.genga_phase_groups(n, dev(pairs.reshape(-1)) if npairs else None, npairs, dev(single), gs, mem)
    gsh, memh = gs.cpu().numpy(), mem.cpu().numpy()
    got = [memh[gsh[k]:gsh[k + 1]] for k in range(ng)]
    assert len(got) == len(ref)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)


def _cluster_groups(seed, ngroups=40, per=(2, 5)):
    """Bodies in tight, separated clumps around 1 AU so that each clump is one encounter group."""
    rng = np.random.default_rng(seed)
    xs, vs, ms, groups = [], [], [], []
    k = 0
    for g in range(ngroups):
        sz = int(rng.integers(per[0], per[1] + 1))
        ang = 2 * np.pi * g / ngroups
        c = np.array([np.cos(ang), np.sin(ang), 0.0])
        vc = np.sqrt(ics.G_GAUSS) * np.array([-np.sin(ang), np.cos(ang), 0.0])
        idx = []
        for _ in range(sz):
            xs.append(c + rng.normal(0, 0.004, 3))
            vs.append(vc + rng.normal(0, 2e-4, 3))
            ms.append(np.exp(rng.uniform(np.log(1e-9), np.log(3e-7))))
            idx.append(k)
            k += 1
        groups.append(idx)
    return np.array(xs), np.array(vs), np.array(ms), groups


@pytest.mark.parametrize("kmode", [0, 1])
def test_bs_groups_match_oracle(kmode):
    x, v, m, groups = _cluster_groups(7)
    n = len(m)
    R = ics.radius_from_mass(m)
    alive = np.ones(n, np.int32)
    p = O.params(G=ics.G_GAUSS, m0=1.0, kmode=kmode)
    rc = np.full(n, 0.02)
    tau = 6.0
    ref_x, ref_v = x.copy(), v.copy()
    for gi in groups:
        out = O.bs_group(p, gi, tau, m, R, alive, ref_x, ref_v, rc)
        assert out["status"] == 0
        ref_x, ref_v = out["x"], out["v"]
    gstart = np.concatenate([[0], np.cumsum([len(g) for g in groups])]).astype(np.int32)
    members = np.concatenate(groups).astype(np.int32)
    X, V, M, RR, AL = soa(x), soa(v), dev(m), dev(R), dev(alive)
    st, U = genga.genga_phase_bs(n, ics.G_GAUSS, 1.0, tau, 1e-12, 8, 30, kmode, 1, len(groups), dev(gstart),
                                 dev(members), dev(rc), M, RR, AL, X, V)
    assert st == 0 and U == 0.0
    np.testing.assert_allclose(aos(X), ref_x, rtol=0, atol=1e-11 * np.abs(ref_x).max())
    np.testing.assert_allclose(aos(V), ref_v, rtol=0, atol=1e-11 * np.abs(ref_v).max())


def _clumps(sizes, seed, spread=0.004, R=None):
    """One tight clump per entry of sizes (each one encounter group), spaced around 1 AU."""
    rng = np.random.default_rng(seed)
    xs, vs, ms, groups, k = [], [], [], [], 0
    for g, sz in enumerate(sizes):
        ang = 2 * np.pi * g / len(sizes)
        c = np.array([np.cos(ang), np.sin(ang), 0.0])
        vc = np.sqrt(ics.G_GAUSS) * np.array([-np.sin(ang), np.cos(ang), 0.0])
        xs.append(c + rng.normal(0, spread, (sz, 3)) * [1.0, 1.0, 0.2])
        vs.append(vc + rng.normal(0, 2e-5, (sz, 3)))
        ms.append(np.exp(rng.uniform(np.log(1e-10), np.log(1e-9), sz)))
        groups.append(list(range(k, k + sz)))
        k += sz
    m = np.concatenate(ms)
    Rr = ics.radius_from_mass(m) * 1e-3 if R is None else np.full(len(m), R)
    return np.vstack(xs), np.vstack(vs), m, Rr, groups


def _bs_phase_vs_oracle(x, v, m, R, groups, kmode=0, tau=6.0):
    n = len(m)
    alive = np.ones(n, np.int32)
    p = O.params(G=ics.G_GAUSS, m0=1.0, kmode=kmode)
    rc = np.full(n, 0.02)
    ref = dict(x=x.copy(), v=v.copy(), m=m.copy(), R=R.copy(), alive=alive.copy(), U=0.0, steps=0, coll=0)
    for gi in groups:
        out = O.bs_group(p, gi, tau, ref["m"], ref["R"], ref["alive"], ref["x"], ref["v"], rc)
        assert out["status"] == 0
        for k in ("x", "v", "m", "R", "alive"):
            ref[k] = out[k]
        ref["U"] += out["U"]
        ref["steps"] += out["bs_steps"]
        ref["coll"] += len(out["collisions"])
    gstart = np.concatenate([[0], np.cumsum([len(g) for g in groups])]).astype(np.int32)
    members = np.concatenate(groups).astype(np.int32)
    X, V, M, RR, AL = soa(x), soa(v), dev(m), dev(R), dev(alive)
    st, U = genga.genga_phase_bs(n, ics.G_GAUSS, 1.0, tau, 1e-12, 8, 30, kmode, 1, len(groups), dev(gstart),
                                 dev(members), dev(rc), M, RR, AL, X, V)
    assert st == 0, st
    np.testing.assert_array_equal(AL.cpu().numpy(), ref["alive"])
    np.testing.assert_allclose(M.cpu().numpy(), ref["m"], rtol=1e-15)
    np.testing.assert_allclose(RR.cpu().numpy(), ref["R"], rtol=1e-14)
    live = ref["alive"] == 1
    np.testing.assert_allclose(aos(X)[live], ref["x"][live], rtol=0, atol=1e-11 * np.abs(ref["x"]).max())
    np.testing.assert_allclose(aos(V)[live], ref["v"][live], rtol=0, atol=1e-11 * np.abs(ref["v"]).max())
    return ref, U


@pytest.mark.parametrize("sizes,spread", [((3, 12, 40, 100), 0.004), ((33, 64, 65, 128), 0.004), ((200,), 0.004),
                                          ((400,), 0.004), ((1000,), 0.03)])
def test_bs_large_groups_match_oracle(sizes, spread):
    """Groups above 32 members run on the grid-wide BS kernel (the paper's split path above 128
    members, Sect. 3.2); with the one-CTA and cluster kernels beside them for the smaller groups.
    The 65- and 128-member clumps need 3 and 4 substeps, the 400-member one 10 (halvings and
    doublings of H on the device)."""
    x, v, m, R, groups = _clumps(sizes, seed=sum(sizes), spread=spread)
    ref, U = _bs_phase_vs_oracle(x, v, m, R, groups)
    assert ref["coll"] == 0 and U == 0.0


@pytest.mark.parametrize("tau", [6.0, 0.05])
def test_bs_cluster_group_sizes_match_oracle(tau):
    """Groups of 5..32 members on the cluster kernel: up to 8 members one term per lane, above that
    every pair once (Newton's third law) with 8, 4 or 2 threads per member component in the sums
    (up to 10, 21 and 32 members). At tau = 0.05 d the groups converge at low levels, which the
    kernel tests together at level 4 before testing each level as it completes."""
    x, v, m, R, groups = _clumps((5, 8, 9, 10, 11, 16, 21, 22, 32), seed=77)
    ref, U = _bs_phase_vs_oracle(x, v, m, R, groups, tau=tau)
    assert ref["coll"] == 0 and U == 0.0


def test_bs_pairs_needing_several_substeps_match_oracle():
    """Tight pairs whose first attempt fails (1, 2 and 9 substeps in the oracle): the one-CTA kernel
    runs the attempt at H/2 beside the one at H in the lanes a pair leaves idle and takes it exactly
    when the serial control would try it next, so the result is the serial algorithm's."""
    x, v, m, R, groups = _clumps((2, 2, 2, 2, 1), seed=4, spread=0.0002)
    ref, U = _bs_phase_vs_oracle(x, v, m, R, groups)
    assert ref["steps"] >= 12


def test_bs_cluster_group_mergers_match_oracle():
    """Contacts and mergers inside groups of 12 and 20 members on the cluster kernel (2 and 6 in the
    oracle)."""
    x, v, m, Rr, groups = _clumps((12, 20), seed=9, spread=0.001, R=3e-4)
    ref, U = _bs_phase_vs_oracle(x, v, m, Rr, groups)
    assert ref["coll"] >= 4
    assert U == pytest.approx(ref["U"], rel=1e-9)


@pytest.mark.parametrize("R", [1e-4, 3e-4])
def test_bs_large_group_mergers_match_oracle(R):
    """Mergers inside a 150-member group on the grid-wide kernel: 2 (R = 1e-4 AU) and 27 (3e-4 AU)
    contacts, merged in ascending pair order as in the oracle."""
    x, v, m, Rr, groups = _clumps((150,), seed=5, R=R)
    ref, U = _bs_phase_vs_oracle(x, v, m, Rr, groups)
    assert ref["coll"] >= 2
    assert U == pytest.approx(ref["U"], rel=1e-9)


def test_bs_merger_matches_oracle():
    m = np.array([4e-7, 1e-7, 2e-7])
    R = np.array([2e-5, 1e-5, 1e-5])
    x = np.array([[1.0, 0.0, 0.0], [1.0, 0.002, 0.0], [1.0, -0.01, 0.001]])
    v = np.array([[0.0, 0.0172, 0.0], [0.0, 0.0172 - 0.001, 0.0], [0.0005, 0.0172, 0.0]])
    alive = np.ones(3, np.int32)
    p = O.params(G=ics.G_GAUSS, m0=1.0)
    rc = np.full(3, 0.05)
    ref = O.bs_group(p, [0, 1, 2], 6.0, m, R, alive, x, v, rc)
    assert len(ref["collisions"]) == 1
    X, V, M, RR, AL = soa(x), soa(v), dev(m), dev(R), dev(alive)
    st, U = genga.genga_phase_bs(3, ics.G_GAUSS, 1.0, 6.0, 1e-12, 8, 30, 0, 1, 1, dev(np.array([0, 3], np.int32)),
                                 dev(np.arange(3, dtype=np.int32)), dev(rc), M, RR, AL, X, V)
    np.testing.assert_array_equal(AL.cpu().numpy(), ref["alive"])
    np.testing.assert_allclose(M.cpu().numpy(), ref["m"], rtol=1e-15)
    np.testing.assert_allclose(RR.cpu().numpy(), ref["R"], rtol=1e-14)
    assert U == pytest.approx(ref["U"], rel=1e-9)
    live = ref["alive"] == 1
    np.testing.assert_allclose(aos(X)[live], ref["x"][live], rtol=0, atol=1e-11)
    np.testing.assert_allclose(aos(V)[live], ref["v"][live], rtol=0, atol=1e-11)


def test_energy_matches_oracle():
    d, p = _state2048()
    n = 2048
    alive = np.ones(n, np.int32); alive[[3, 4]] = 0
    ref = O.energy(p, d["m"], alive, d["x"], d["v"])
    E = genga.genga_phase_energy(n, d["G"], d["m0"], dev(d["m"]), dev(alive), soa(d["x"]), soa(d["v"]))
    assert E == pytest.approx(ref, rel=1e-13)
