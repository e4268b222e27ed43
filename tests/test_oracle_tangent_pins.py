"""Pins of the oracle tangent map (forward-mode derivatives of the hybrid step, merging off).

The tangent oracle is pinned to things other than itself:
  * its values are the C oracle's trajectory (same inputs, same decisions);
  * its derivatives are central finite differences of the C oracle (h = 1e-7 relative for x and v,
    1e-4 for masses);
  * on encounter-free steps (K = 1 for every pair, so the critical radii drop out) the step is a
    composition of exact Hamiltonian flows (Sect. 2.2), hence symplectic in the canonical
    democratic heliocentric coordinates (x_i, p_i = m_i v_i barycentric): J^T Omega J = Omega.
"""
import numpy as np
import pytest

import oracle as O
from oracle import tangent as TG

G = 0.01720209895 ** 2


def _circular(x):
    v = np.zeros_like(x)
    for i in range(len(x)):
        r = np.linalg.norm(x[i])
        v[i] = np.sqrt(G / r) * np.array([-x[i, 1], x[i, 0], 0.0]) / r
    return v


def flyby():
    """A hyperbolic close pass (0.02 AU start, ~1e-3 AU/day relative) that BS integrates over a few
    steps, plus a distant third body."""
    m = np.array([3e-6, 1e-6, 2e-6])
    x = np.array([[1.0, 0.0, 0.0], [1.0, -0.02, 0.002], [-0.3, 1.5, 0.01]])
    v = _circular(x)
    v[1] += [0.0005, 0.0012, 0.0]
    return m, x, v


def quiet():
    """Four bodies far apart: no candidate pair, K = 1 throughout."""
    m = np.array([3e-6, 1e-5, 2e-6, 5e-6])
    x = np.array([[1.0, 0.0, 0.0], [0.0, 1.6, 0.01], [-2.4, 0.3, -0.02], [0.4, -3.3, 0.05]])
    v = _circular(x)
    v[0] *= 1.01
    return m, x, v


def _oracle_state(p, m, x, v, steps):
    s = O.Sim(p, m, np.zeros(len(m)), x, v)
    s.step(steps)
    st = s.state()
    stats = s.stats()
    s.close()
    return np.concatenate([st["x"].ravel(), st["v"].ravel()]), stats


@pytest.mark.parametrize("order", [2, 4])
def test_tangent_values_follow_the_oracle(order):
    m, x, v = flyby()
    p = O.params(G=G, m0=1.0, dt=6.0, order=order, collisions=0)
    ref, stats = _oracle_state(p, m, x, v, 8)
    T = TG.TangentSim(p, m, x, v, directions=np.zeros((7 * len(m), 1)))
    T.step(8)
    xh, vh = T.state()
    got = np.concatenate([xh.ravel(), vh.ravel()])
    assert stats["bs_steps"] > 0
    assert sum(len(q[1]) for seqs in T.bs_sequences for q in seqs) == stats["bs_steps"]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("order", [2, 4])
def test_tangent_matches_central_differences_of_the_oracle(order):
    m, x, v = flyby()
    n = len(m)
    steps = 6
    p = O.params(G=G, m0=1.0, dt=6.0, order=order, collisions=0)
    T = TG.TangentSim(p, m, x, v)
    T.step(steps)
    J = T.jacobian()
    assert sum(len(q[1]) for seqs in T.bs_sequences for q in seqs) > 0
    base = np.concatenate([x.ravel(), v.ravel(), m])
    scale = np.concatenate([np.repeat(np.linalg.norm(x, axis=1), 3), np.repeat(np.linalg.norm(v, axis=1), 3), m])
    f0, _ = _oracle_state(p, m, x, v, steps)
    for k in range(7 * n):
        # h = 1e-7 relative for x and v; masses barely move the O(1) outputs, so a mass step that
        # small would be lost in rounding: 1e-4 relative there (the map is nearly linear in m)
        h = (1e-7 if k < 6 * n else 1e-4) * scale[k]
        cols = []
        for sgn in (1.0, -1.0):
            b = base.copy()
            b[k] += sgn * h
            out, _ = _oracle_state(p, b[6 * n:], b[:3 * n].reshape(n, 3), b[3 * n:6 * n].reshape(n, 3), steps)
            cols.append(out)
        fd = (cols[0] - cols[1]) / (2.0 * h)
        noise = 4.0 * np.finfo(float).eps * np.abs(f0).max() * np.sqrt(6 * n) / h  # rounding floor of the quotient
        # masses: the close pass amplifies the rounding of the outputs, and a mass column can be
        # small (a distant body); a missing or wrong term would still be off by O(1)
        rel = 1e-6 if k < 6 * n else 1e-3
        err = np.linalg.norm(fd - J[:, k])
        assert err <= rel * np.linalg.norm(J[:, k]) + noise, (k, err, np.linalg.norm(J[:, k]), noise)


def test_encounter_free_step_is_symplectic():
    m, x, v = quiet()
    n = len(m)
    p = O.params(G=G, m0=1.0, dt=6.0, order=4, collisions=0)
    dirs = np.zeros((7 * n, 6 * n))
    dirs[:6 * n, :6 * n] = np.eye(6 * n)  # x and v only; masses fixed
    T = TG.TangentSim(p, m, x, v, directions=dirs)
    T.step(5)
    assert all(len(seqs) == 0 for seqs in T.bs_sequences)
    Jh = T.jacobian()
    # heliocentric (x, v_h) -> canonical (x, p = m v_b), v_b = v_h - sum m v_h / (m0 + sum m)
    M = 1.0 + m.sum()
    Cv = np.zeros((3 * n, 3 * n))
    for i in range(n):
        for j in range(n):
            Cv[3 * i:3 * i + 3, 3 * j:3 * j + 3] = m[i] * ((i == j) - m[j] / M) * np.eye(3)
    C = np.block([[np.eye(3 * n), np.zeros((3 * n, 3 * n))], [np.zeros((3 * n, 3 * n)), Cv]])
    J = C @ Jh @ np.linalg.inv(C)
    Om = np.block([[np.zeros((3 * n, 3 * n)), np.eye(3 * n)], [-np.eye(3 * n), np.zeros((3 * n, 3 * n))]])
    R = J.T @ Om @ J - Om
    # entries of J^T Omega J scale with |J|^2 in the mixed units: normalise per entry
    scale = np.abs(J.T) @ np.abs(Om) @ np.abs(J)
    assert np.max(np.abs(R) / np.maximum(scale, 1e-300)) <= 1e-11
