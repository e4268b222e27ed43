"""Tangent map of the hybrid symplectic step -- TEST INFRASTRUCTURE ONLY.

Forward-mode derivatives of the oracle's step (Grimm & Stadel 2014, Sect. 2.1-2.3 and 3.2) with
perfect merging switched off. Every quantity is a dual number: its value and its derivatives along
a fixed set of input directions. The arithmetic repeats, step for step, what the C oracle does:
critical radii (Eq. rcrit) at the start of each full step, the kick weighted by K (Eq. Hb), the
Sun drifts (Eq. Hc), the universal-variable Kepler drift (Eq. fg, Newton on the universal Kepler
equation), the Hermite encounter test on the candidates of the previous closing kick, groups,
Bulirsch-Stoer of every group in the field of H_A (n_k = 2k, Neville extrapolation in h^2) and the
Yoshida composition for 4th order (Sect. 2.3).

Every decision -- the branch of K, the prechecker, the encounter test, Newton's stopping rule, the
BS acceptance -- is taken on the values alone, so the result is the derivative of the map with
those decisions frozen: the map the adjoint differentiates. The discrete parts that carry no
derivative (Hermite minimum, grouping) call the C oracle's own routines.

Inputs and outputs use the public convention: heliocentric positions and velocities, masses of
the orbiting bodies; the central mass m0 is a fixed parameter.

Only tests may import this module. It shares no code with the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np

from . import encounters as _encounters, groups as _groups, precheck as _precheck

_MAXSUB = 7


class D:
    """Dual number: value v and derivative vector d (one entry per input direction)."""

    __slots__ = ("v", "d")

    def __init__(self, v, d):
        self.v = float(v)
        self.d = d

    # arithmetic ----------------------------------------------------------------------------
    def __add__(self, o):
        if isinstance(o, D):
            return D(self.v + o.v, self.d + o.d)
        return D(self.v + o, self.d)

    __radd__ = __add__

    def __sub__(self, o):
        if isinstance(o, D):
            return D(self.v - o.v, self.d - o.d)
        return D(self.v - o, self.d)

    def __rsub__(self, o):
        return D(o - self.v, -self.d)

    def __neg__(self):
        return D(-self.v, -self.d)

    def __mul__(self, o):
        if isinstance(o, D):
            return D(self.v * o.v, self.d * o.v + o.d * self.v)
        return D(self.v * o, self.d * o)

    __rmul__ = __mul__

    def __truediv__(self, o):
        if isinstance(o, D):
            q = self.v / o.v
            return D(q, (self.d - o.d * q) / o.v)
        return D(self.v / o, self.d / o)

    def __rtruediv__(self, o):
        q = o / self.v
        return D(q, self.d * (-q / self.v))

    def __repr__(self):
        return f"D({self.v!r})"


def const(x, ndir):
    return D(x, np.zeros(ndir))


def val(a):
    return a.v if isinstance(a, D) else float(a)


def dsqrt(a: D) -> D:
    r = math.sqrt(a.v)
    return D(r, a.d * (0.5 / r)) if r > 0.0 else D(0.0, a.d * 0.0)


def dcbrt(a: D) -> D:
    c = float(np.cbrt(a.v))
    # d cbrt(a) = cbrt(a) / (3 a); at a = 0 the branch that uses it never wins (Hill radius 0)
    return D(c, a.d * (c / (3.0 * a.v))) if a.v != 0.0 else D(0.0, a.d * 0.0)


def dot3(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


# -------------------------------------------------------------------------------------- Sect. 2.1
def changeover(r: D, rc: D):
    """K(r) with y = (r - 0.1 rc)/(0.9 rc); 0 for y <= 0, 1 for y >= 1 (branch on values)."""
    y = (r - 0.1 * rc) / (0.9 * rc)
    if y.v <= 0.0:
        return 0.0
    if y.v >= 1.0:
        return 1.0
    return y * y / (2.0 * y * y - 2.0 * y + 1.0)


def changeover_dr(r: D, rc: D):
    y = (r - 0.1 * rc) / (0.9 * rc)
    if y.v <= 0.0 or y.v >= 1.0:
        return 0.0
    dd = 2.0 * y * y - 2.0 * y + 1.0
    return 2.0 * y * (1.0 - y) / (dd * dd) / (0.9 * rc)


def weight_B(r2: D, rc: D, kmode: int):
    if r2.v >= rc.v * rc.v:
        return 1.0
    r = dsqrt(r2)
    w = changeover(r, rc)
    if kmode == 1:
        w = w - r * changeover_dr(r, rc)
    return w


def rc_pair(rc, i, j):
    return rc[i] if rc[i].v > rc[j].v else rc[j]


def rcrit(p, m, x, v, tau_abs):
    """Eq. rcrit: max(n1 R_H, n2 tau |v|), R_H = a (m/(3 m0))^(1/3), a from 1/a = 2/|x| - |v|^2/mu
    (|x| if unbound)."""
    mu = p.G * p.m0
    out = []
    for i in range(len(m)):
        r = dsqrt(dot3(x[i], x[i]))
        v2 = dot3(v[i], v[i])
        inva = 2.0 / r - v2 / mu
        a = 1.0 / inva if inva.v > 0.0 else r
        a1 = p.n1 * (a * dcbrt(m[i] / (3.0 * p.m0)))
        a2 = p.n2 * tau_abs * dsqrt(v2)
        out.append(a1 if a1.v > a2.v else a2)
    return out


# -------------------------------------------------------------------------------------- Sect. 2.2
def accel_B(p, m, x, rc):
    """Kick acceleration: sum over j != i of G m_j W_B(r_ij) (x_j - x_i)/r_ij^3 (Eq. Hb)."""
    n = len(m)
    a = []
    for i in range(n):
        acc = [0.0, 0.0, 0.0]
        for j in range(n):
            if j == i:
                continue
            d = [x[j][c] - x[i][c] for c in range(3)]
            r2 = dot3(d, d)
            w = weight_B(r2, rc_pair(rc, i, j), p.kmode)
            r = dsqrt(r2)
            f = p.G * m[j] * w / (r2 * r)
            acc = [acc[c] + f * d[c] for c in range(3)]
        a.append(acc)
    return a


def momentum(m, v):
    P = [0.0, 0.0, 0.0]
    for i in range(len(m)):
        P = [P[c] + m[i] * v[i][c] for c in range(3)]
    return P


def sun_drift(p, x, P, h):
    f = h / p.m0
    return [[x[i][c] + f * P[c] for c in range(3)] for i in range(len(x))]


def stumpff(z: D):
    """c0..c3 by argument quartering, series of c2 and c3, and the quadrupling identities."""
    nred = 0
    while abs(z.v) > 0.1 and nred < 200:
        z = z * 0.25
        nred += 1
    t2, s2 = 0.5, 0.5
    t3, s3 = 1.0 / 6.0, 1.0 / 6.0
    for k in range(1, 13):
        t2 = t2 * (-1.0 * z) / ((2.0 * k + 1.0) * (2.0 * k + 2.0))
        s2 = s2 + t2
        t3 = t3 * (-1.0 * z) / ((2.0 * k + 2.0) * (2.0 * k + 3.0))
        s3 = s3 + t3
    c2, c3 = s2, s3
    c1 = 1.0 - z * c3
    c0 = 1.0 - z * c2
    for _ in range(nred):
        c3 = (c2 + c0 * c3) * 0.25
        c2 = 0.5 * c1 * c1
        c1 = c0 * c1
        c0 = 2.0 * c0 * c0 - 1.0
    return c0, c1, c2, c3


def kepler_drift(mu, x, v, dt, maxit):
    """Eq. fg in universal variables: Newton on F(s) = r0 s c1 + u s^2 c2 + mu s^3 c3 - dt from
    s = dt/r0 with the oracle's stopping rule (on values), then Gauss' f and g. Returns (x, v, ok)."""
    r0 = dsqrt(dot3(x, x))
    v2 = dot3(v, v)
    u = dot3(x, v)
    beta = 2.0 * mu / r0 - v2
    s = dt / r0
    ds_prev = math.inf
    ok = False
    for _ in range(maxit):
        c0, c1, c2, c3 = stumpff(beta * s * s)
        F = r0 * s * c1 + u * s * s * c2 + mu * s * s * s * c3 - dt
        Fp = r0 * c0 + u * s * c1 + mu * s * s * c2
        ds = F / Fp
        s = s - ds
        if not math.isfinite(s.v):
            break
        if abs(ds.v) <= 4.0 * np.finfo(float).eps * abs(s.v):
            ok = True
            break
        if abs(ds.v) <= 1e-10 * abs(s.v) and abs(ds.v) >= 0.5 * ds_prev:
            ok = True
            break
        ds_prev = abs(ds.v)
    if not ok:
        return x, v, False
    c0, c1, c2, c3 = stumpff(beta * s * s)
    r = r0 * c0 + u * s * c1 + mu * s * s * c2
    f = 1.0 - (mu / r0) * s * s * c2
    g = dt - mu * s * s * s * c3
    fd = -(mu / (r * r0)) * s * c1
    gd = 1.0 - (mu / r) * s * s * c2
    return [f * x[c] + g * v[c] for c in range(3)], [fd * x[c] + gd * v[c] for c in range(3)], True


# -------------------------------------------------------------------------------------- Sect. 3.2
def _bs_deriv(p, m, rc, idx, y):
    """H_A restricted to the group: dx/dt = v, dv/dt = -G m0 x/|x|^3 + sum G m_p W_A (x_p - x_q)/r^3,
    W_A = 1 - W_B."""
    out = []
    for q, iq in enumerate(idx):
        yq = y[q]
        r2 = dot3(yq[:3], yq[:3])
        r = dsqrt(r2)
        f = p.G * p.m0 / (r2 * r)
        a = [-1.0 * f * yq[c] for c in range(3)]
        for s_, is_ in enumerate(idx):
            if s_ == q:
                continue
            d = [y[s_][c] - yq[c] for c in range(3)]
            pr2 = dot3(d, d)
            wa = 1.0 - weight_B(pr2, rc_pair(rc, iq, is_), p.kmode)
            if val(wa) == 0.0:
                continue
            pr = dsqrt(pr2)
            fp = p.G * m[is_] * wa / (pr2 * pr)
            a = [a[c] + fp * d[c] for c in range(3)]
        out.append([yq[3], yq[4], yq[5], a[0], a[1], a[2]])
    return out


def _mmid(p, m, rc, idx, y, dy0, H, nsub):
    h = H / nsub
    za = [list(yq) for yq in y]
    zb = [[y[q][e] + h * dy0[q][e] for e in range(6)] for q in range(len(y))]
    for _ in range(1, nsub):
        f = _bs_deriv(p, m, rc, idx, zb)
        nz = [[za[q][e] + 2.0 * h * f[q][e] for e in range(6)] for q in range(len(y))]
        za, zb = zb, nz
    f = _bs_deriv(p, m, rc, idx, zb)
    return [[0.5 * (zb[q][e] + za[q][e] + h * f[q][e]) for e in range(6)] for q in range(len(y))]


def _bs_attempt(p, m, rc, idx, y, H):
    dy0 = _bs_deriv(p, m, rc, idx, y)
    sc = []
    for yq in y:
        sx = math.sqrt(sum(yq[c].v ** 2 for c in range(3))) or np.finfo(float).tiny
        sv = math.sqrt(sum(yq[c].v ** 2 for c in range(3, 6))) or np.finfo(float).tiny
        sc.append([sx] * 3 + [sv] * 3)
    T = {}
    for k in range(1, p.bs_kmax + 1):
        T[(k, 1)] = _mmid(p, m, rc, idx, y, dy0, H, 2 * k)
        for j in range(1, k):
            fac = (k / (k - j)) ** 2 - 1.0
            T[(k, j + 1)] = [[T[(k, j)][q][e] + (T[(k, j)][q][e] - T[(k - 1, j)][q][e]) / fac for e in range(6)]
                             for q in range(len(y))]
        if k >= 2:
            err = 0.0
            for q in range(len(y)):
                for e in range(6):
                    ee = abs(T[(k, k)][q][e].v - T[(k, k - 1)][q][e].v) / sc[q][e]
                    if not ee <= err:
                        err = ee
            if err <= p.bs_eps:
                return T[(k, k)], k
    return None, 0


def bs_group(p, m, rc, idx, x, v, tau):
    """BS of one group over tau from (x, v) of its members (the oracle's controller: halve on
    failure, double after acceptance). Returns the members' (x, v) and the accepted (H, k) list."""
    y = [list(x[i]) + list(v[i]) for i in idx]
    rem, H, halvings = tau, tau, 0
    seq = []
    while rem != 0.0:
        if abs(H) > abs(rem):
            H = rem
        yn, k = _bs_attempt(p, m, rc, idx, y, H)
        if k == 0:
            H *= 0.5
            halvings += 1
            if halvings > p.bs_max_halvings:
                raise RuntimeError("BS failed")
            continue
        halvings = 0
        seq.append((H, k))
        y = yn
        rem -= H
        H *= 2.0
    return [yq[:3] for yq in y], [yq[3:] for yq in y], seq


# -------------------------------------------------------------------------------------- Sect. 2.3
def substep_weights(order):
    if order == 4:
        c = 2.0 ** (1.0 / 3.0)
        return [1.0 / (2.0 - c), -c / (2.0 - c), 1.0 / (2.0 - c)]
    if order == 6:
        w1, w2, w3 = -1.17767998417887, 0.235573213359357, 0.784513610477560
        w0 = 1.0 - 2.0 * (w1 + w2 + w3)
        return [w3, w2, w1, w0, w1, w2, w3]
    return [1.0]


def _values(x):
    return np.array([[c.v for c in xi] for xi in x])


class TangentSim:
    """Tangent-linear integration of one system. x, v (heliocentric, shape (n, 3)) and m (n) are
    the inputs; ``directions`` (shape (7n, ndir)) are the input perturbations, ordered x (3n, body
    major), v (3n), m (n). ``jacobian()`` returns d(x, v)_final / d(directions)."""

    def __init__(self, p, m, xh, vh, directions=None):
        n = len(m)
        self.p = p
        self.n = n
        if directions is None:
            directions = np.eye(7 * n)
        directions = np.asarray(directions, dtype=np.float64)
        nd = directions.shape[1]
        self.nd = nd
        X = [[D(xh[i][c], directions[3 * i + c].copy()) for c in range(3)] for i in range(n)]
        V = [[D(vh[i][c], directions[3 * n + 3 * i + c].copy()) for c in range(3)] for i in range(n)]
        M = [D(m[i], directions[6 * n + i].copy()) for i in range(n)]
        # heliocentric -> democratic: v_b = v_h - sum m v_h / (m0 + sum m)
        Mtot = p.m0 + sum(M[1:], M[0]) if n else const(p.m0, nd)
        Ph = momentum(M, V)
        self.x = X
        self.v = [[V[i][c] - Ph[c] / Mtot for c in range(3)] for i in range(n)]
        self.m = M
        rc = rcrit(p, M, self.x, self.v, abs(p.dt))
        self.a = accel_B(p, M, self.x, rc)
        self.cand = _precheck(p, np.ones(n, np.int32), _values(self.x), np.array([r.v for r in rc]))
        self.bs_sequences = []

    def _substep(self, tau, rc):
        p, n = self.p, self.n
        h = 0.5 * tau
        v = [[self.v[i][c] + h * self.a[i][c] for c in range(3)] for i in range(n)]
        x = sun_drift(p, self.x, momentum(self.m, v), h)
        x0, v0 = x, v
        mu = p.G * p.m0
        x1, v1, fail = [], [], np.zeros(n, np.int32)
        for i in range(n):
            xi, vi, ok = kepler_drift(mu, x0[i], v0[i], tau, p.kepler_maxit)
            x1.append(xi)
            v1.append(vi)
            fail[i] = 0 if ok else 1
        rcv = np.array([r.v for r in rc])
        enc = _encounters(np.ones(n, np.int32), _values(x0), _values(v0), _values(x1), _values(v1), rcv,
                          self.cand, tau)
        seqs = []
        for idx in _groups(n, enc, fail):
            xs, vs, seq = bs_group(p, self.m, rc, list(idx), x0, v0, tau)
            for q, i in enumerate(idx):
                x1[i], v1[i] = xs[q], vs[q]
            seqs.append((list(idx), seq))
        self.bs_sequences.append(seqs)
        x = sun_drift(p, x1, momentum(self.m, v1), h)
        self.a = accel_B(p, self.m, x, rc)
        self.v = [[v1[i][c] + h * self.a[i][c] for c in range(3)] for i in range(n)]
        self.x = x
        self.cand = _precheck(p, np.ones(n, np.int32), _values(x), rcv)

    def step(self, nsteps=1):
        p = self.p
        for _ in range(nsteps):
            rc = rcrit(p, self.m, self.x, self.v, abs(p.dt))
            self.a = accel_B(p, self.m, self.x, rc)
            for w in substep_weights(p.order):
                self._substep(w * p.dt, rc)

    def state(self):
        """Heliocentric (x, v) values, shape (n, 3) each: v_h = v_b + P/m0."""
        P = momentum(self.m, self.v)
        xh = _values(self.x)
        vh = np.array([[(self.v[i][c] + P[c] / self.p.m0).v for c in range(3)] for i in range(self.n)])
        return xh, vh

    def jacobian(self):
        """d(x_h, v_h)_final / d(directions): shape (6n, ndir), rows x (body major), then v."""
        P = momentum(self.m, self.v)
        rows = [self.x[i][c].d for i in range(self.n) for c in range(3)]
        rows += [(self.v[i][c] + P[c] / self.p.m0).d for i in range(self.n) for c in range(3)]
        return np.array(rows)
