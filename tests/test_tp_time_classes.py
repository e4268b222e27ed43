"""Midpoint times of a test particle's attempt pair (H and H/2, levels k = 1..8 with n_k = 2k
substeps, Sect. 3.2): the rule by which the GPU evaluates each planet position only once per set of
bit-identical times.

Entry (hf, k, m) lies at t0 + m h_k with h_k = He / 2k rounded (He = H / 2^hf), or at t0 + He when
m = 2k. Writing 2k = o 2^e and m = mo 2^a (o, mo odd), h_k is round(H / o) 2^-(e + hf), so m h_k is
determined by (o, mo, a - e - hf): entries with equal keys have equal times, bit for bit, both when
the product is rounded before the addition and when the two fuse into one rounding. These tests
check the rule on IEEE doubles (and exact rational arithmetic for the fused form); the library
re-checks its own classes at initialisation.
"""
from fractions import Fraction

import numpy as np
import pytest

LEVELS = 8


def _key(hf, k, m):
    if m == 0:
        return (0, 0, 0)
    if m == 2 * k:
        return (1, 1, -hf)
    o, e = 2 * k, 0
    while o % 2 == 0:
        o //= 2
        e += 1
    mo, a = m, 0
    while mo % 2 == 0:
        mo //= 2
        a += 1
    return (o, mo, a - e - hf)


def _classes():
    cls = {}
    for hf in (0, 1):
        for k in range(1, LEVELS + 1):
            for m in range(2 * k + 1):
                cls.setdefault(_key(hf, k, m), []).append((hf, k, m))
    return cls


def _time(t0, H, hf, k, m, fused):
    He = 0.5 * H if hf else H
    if m == 2 * k:
        return t0 + He
    hk = He / (2 * k)
    if fused:  # one rounding of t0 + m hk, exactly
        return float(Fraction(t0) + Fraction(m) * Fraction(hk))
    return t0 + m * hk


def test_class_count():
    cls = _classes()
    assert sum(len(v) for v in cls.values()) == 2 * sum(2 * k + 1 for k in range(1, LEVELS + 1)) == 160
    assert len(cls) == 76


@pytest.mark.parametrize("fused", [False, True])
def test_members_share_their_time_bitwise(fused):
    rng = np.random.default_rng(7)
    cls = _classes()
    trials = 400 if fused else 4000
    for t in range(trials):
        H = float(rng.uniform(-10, 10) * 10.0 ** rng.integers(-4, 2))
        t0 = 0.0 if t % 3 == 0 else float(rng.uniform(-6, 6))
        for key, members in cls.items():
            times = {np.float64(_time(t0, H, *mem, fused)).tobytes() for mem in members}
            assert len(times) == 1, (H, t0, key, members)


def test_distinct_keys_can_differ():
    """The classes are not coarser than the times: some pair of different keys gives different
    times for a generic H (a sanity check that the test above is not vacuous)."""
    cls = _classes()
    H, t0 = 6.0 * 0.7310585786300049, 1.25
    reps = {key: _time(t0, H, *members[0], False) for key, members in cls.items()}
    assert len(set(reps.values())) > 60
