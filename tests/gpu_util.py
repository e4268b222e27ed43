"""Helpers shared by the GPU parity tests: array marshalling and paired GPU / oracle runs."""
import numpy as np

import oracle as O
from paper_1404_2324_gb300 import genga


def torch():
    import torch as t
    return t


def dev(a, dtype=None):
    t = torch()
    a = np.ascontiguousarray(a)
    if dtype is None:
        dtype = t.float64 if a.dtype.kind == "f" else t.int32
    return t.tensor(a, dtype=dtype, device="cuda")


def soa(x):
    """[n,3] host array -> [3,n] contiguous device tensor (component-major SoA)."""
    return dev(np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1, 3).T))


def aos(t):
    return t.detach().cpu().numpy().reshape(3, -1).T.copy()


def with_central(d):
    m = np.concatenate([[d["m0"]], d["m"]])
    R = np.concatenate([[0.0], d["R"]])
    x = np.vstack([np.zeros(3), d["x"]])
    v = np.vstack([np.zeros(3), d["v"]])
    return m, R, x, v


def pair_sims(d, order, steps=0, **params):
    """A GPU simulation and an oracle simulation of the same input, both advanced `steps` steps."""
    m, R, x, v = with_central(d)
    gp = genga.genga_default_params()
    op = O.params(G=d["G"], m0=d["m0"], dt=d["dt"], order=order)
    for k, val in params.items():
        setattr(gp, k, val)
        if hasattr(op, k):
            setattr(op, k, val)
    g = genga.Genga(m, R, x, v, d["G"], d["dt"], order, params=gp if params else None)
    o = O.Sim(op, d["m"], d["R"], d["x"], d["v"])
    if steps:
        g.step(steps)
        o.step(steps)
    return g, o


def rel_state_error(g, o):
    """Max over live bodies of |dx|/|x| and |dv|/|v| (heliocentric), and the live-flag agreement."""
    gs, os_ = g.state(), o.state()
    same_alive = np.array_equal(gs["alive"][1:], os_["alive"])
    live = os_["alive"] == 1
    ex = np.linalg.norm(gs["x"][1:][live] - os_["x"][live], axis=1) / np.linalg.norm(os_["x"][live], axis=1)
    ev = np.linalg.norm(gs["v"][1:][live] - os_["v"][live], axis=1) / np.linalg.norm(os_["v"][live], axis=1)
    return max(ex.max(), ev.max()), same_alive


def oracle_sensitivity(d, order, steps, trials=3, eps=1e-15, **params):
    """How far the oracle itself moves after `steps` steps when its initial positions are perturbed
    by eps (relative, random directions): the rounding amplification of the system's close passes.
    Returns the largest relative state change over `trials` perturbations."""
    op = O.params(G=d["G"], m0=d["m0"], dt=d["dt"], order=order)
    for k, val in params.items():
        if hasattr(op, k):
            setattr(op, k, val)
    base = O.Sim(op, d["m"], d["R"], d["x"], d["v"])
    base.step(steps)
    a = base.state()
    base.close()
    live = a["alive"] == 1
    worst = 0.0
    for k in range(trials):
        rng = np.random.default_rng(1000 + k)
        x = d["x"] * (1.0 + eps * rng.standard_normal(d["x"].shape))
        o = O.Sim(op, d["m"], d["R"], x, d["v"])
        o.step(steps)
        b = o.state()
        o.close()
        both = live & (b["alive"] == 1)
        ex = np.linalg.norm(a["x"][both] - b["x"][both], axis=1) / np.linalg.norm(a["x"][both], axis=1)
        ev = np.linalg.norm(a["v"][both] - b["v"][both], axis=1) / np.linalg.norm(a["v"][both], axis=1)
        worst = max(worst, ex.max(), ev.max())
    return worst
