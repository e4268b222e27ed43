"""Pins of the literal higher-order prechecker (Sect. 2.3: each substep runs the full scheme "but
not the prechecker"). With precheck_substeps = 0 only the closing kick of a full step prechecks,
and its candidates serve the encounter search of every substep of the next step. CPU only.

The premise is that the step-start candidates (r < pc * rcrit) already contain every pair that can
come within rcrit during the next step. It is checked against the per-substep prechecker on the
disk workloads: every encounter confirmed in any substep must be among the candidates of the
preceding full step; any miss is reported."""
import numpy as np
import pytest

import oracle as O
from paper_1404_2324_gb300 import ics


def _misses(d, order, steps):
    """Encounters found by the per-substep prechecker that the step-start candidates lack."""
    p = O.params(G=d["G"], m0=d["m0"], dt=d["dt"], order=order)
    s = O.Sim(p, d["m"], d["R"], d["x"], d["v"])
    nsub = len(O.substep_weights(order))
    missed, total = [], 0
    for it in range(steps):
        cand = {tuple(c) for c in s.candidates()}
        s.step(1)
        for js in range(nsub):
            for pair in map(tuple, s.encounters(js)):
                total += 1
                if pair not in cand:
                    missed.append((it + 1, js, pair))
    s.close()
    return missed, total


@pytest.mark.parametrize("seed,order", [(1, 4), (2, 4), (3, 6)])
def test_step_start_candidates_contain_every_substep_encounter_disk32(seed, order):
    missed, total = _misses(ics.disk32(seed), order, 300)
    print(f"disk32 seed {seed} order {order}: {total} substep encounters, {len(missed)} outside the step-start candidates")
    assert total > 0 and not missed, missed[:5]


def test_step_start_candidates_contain_every_substep_encounter_disk2048():
    missed, total = _misses(ics.disk2048(2, order=4), 4, 5)
    print(f"disk2048 order 4: {total} substep encounters, {len(missed)} outside the step-start candidates")
    assert total > 100 and not missed, missed[:5]


@pytest.mark.parametrize("order", [4, 6])
def test_literal_prechecker_changes_nothing_but_the_candidates(order):
    """Where no encounter is missed, the literal variant takes the same encounter decisions, and the
    oracle's kicks are the plain all-pairs definition, so the runs agree bit for bit; the literal
    variant records fewer candidate sets (one per step instead of one per substep)."""
    d = ics.disk32(1)
    runs = []
    for ps in (1, 0):
        p = O.params(G=d["G"], m0=d["m0"], dt=d["dt"], order=order, precheck_substeps=ps)
        s = O.Sim(p, d["m"], d["R"], d["x"], d["v"])
        s.step(300)
        runs.append((s.state(), s.stats()))
        s.close()
    (a, sa), (b, sb) = runs
    np.testing.assert_array_equal(a["x"], b["x"])
    np.testing.assert_array_equal(a["v"], b["v"])
    assert sa["encounters"] == sb["encounters"] > 0
    assert sb["candidates"] < sa["candidates"]
