"""CPU FP64 oracle of the GENGA hybrid symplectic step -- TEST INFRASTRUCTURE ONLY.

The oracle (``genga_oracle.c``) is a plain, slow restatement of Grimm & Stadel (2014), Sect. 2
and 3.2, used to check the CUDA library. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package. It shares
no code with the CUDA sources and never imports the product package's binding.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "genga_oracle.c")
_HDR = os.path.join(_HERE, "genga_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_OMP_PATH = os.path.join(_OUT_DIR, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

CFLAGS = ["-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]

ST_KEPLER_FALLBACK = 1
ST_BS_FAILED = 2
ST_REUSE_VIOLATION = 4
ST_CAPACITY = 8

STAT_NAMES = ["steps", "substeps", "candidates", "encounters", "groups", "bs_steps",
              "kepler_fallbacks", "collisions", "reuse_violations", "kepler_iterations",
              "status_bits", "ejections"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) into oracle/_build/liboracle.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def build_omp(force: bool = False):
    """The same source built with OpenMP (the pair sums split over bodies; results are bit-identical
    to the plain build), for timing the oracle on all host cores. Returns the path, or None where the
    compiler has no OpenMP."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_OMP_PATH) or os.path.getmtime(_OMP_PATH) < newest:
        tmp = _OMP_PATH + f".{os.getpid()}.tmp"
        res = subprocess.run(["gcc", *CFLAGS, "-fopenmp", "-o", tmp, _SRC, "-lm"], capture_output=True)
        if res.returncode != 0:
            return None
        os.replace(tmp, _OMP_PATH)
    return _OMP_PATH


class Params(C.Structure):
    _fields_ = [("G", C.c_double), ("m0", C.c_double), ("dt", C.c_double), ("order", C.c_int),
                ("kmode", C.c_int), ("n1", C.c_double), ("n2", C.c_double), ("pc", C.c_double),
                ("bs_eps", C.c_double), ("bs_kmax", C.c_int), ("bs_max_halvings", C.c_int),
                ("kepler_maxit", C.c_int), ("collisions", C.c_int), ("rcut", C.c_double), ("rcut_sun", C.c_double),
                ("precheck_substeps", C.c_int)]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_P = C.POINTER(Params)


def lib_omp():
    """The OpenMP build (see build_omp), or None."""
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            path = build_omp()
            if path is None:
                return None
            _lib_omp = _declare(C.CDLL(path))
    return _lib_omp


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _declare(C.CDLL(build()))
    return _lib


def _declare(L):
    """Argument and result types of the oracle's C functions on the loaded library L."""
    sig = {
        "orc_default_params": (None, [_P]),
        "orc_changeover": (C.c_double, [C.c_double, C.c_double]),
        "orc_changeover_dr": (C.c_double, [C.c_double, C.c_double]),
        "orc_weight_B": (C.c_double, [C.c_double, C.c_double, C.c_int]),
        "orc_rcrit": (None, [C.c_int, _P, C.c_double, _D, _I, _D, _D, _D]),
        "orc_accel_B": (None, [C.c_int, _P, _D, _I, _D, _D, _D]),
        "orc_precheck": (C.c_int, [C.c_int, _P, _I, _D, _D, _I, C.c_int]),
        "orc_momentum": (None, [C.c_int, _D, _I, _D, _D]),
        "orc_sun_drift": (None, [C.c_int, _P, _I, _D, _D, C.c_double]),
        "orc_stumpff": (None, [C.c_double, _D]),
        "orc_kepler_drift": (C.c_int, [C.c_double, _D, _D, C.c_double, C.c_int, _I]),
        "orc_hermite_min": (C.c_double, [_D, _D, _D, _D, C.c_double]),
        "orc_encounters": (C.c_int, [C.c_int, _I, _D, _D, _D, _D, _D, _I, C.c_int,
                                     C.c_double, _I, C.c_int]),
        "orc_groups": (C.c_int, [C.c_int, _I, C.c_int, _I, _I, _I]),
        "orc_energy": (C.c_double, [C.c_int, _P, _D, _I, _D, _D]),
        "orc_bs_group": (C.c_int, [C.c_int, _P, C.c_int, _I, C.c_double, _D, _D, _I, _D,
                                   _D, _D, _D, _I, _I, C.c_int, _I]),
        "orc_bs_group_rec": (C.c_int, [C.c_int, _P, C.c_int, _I, C.c_double, _D, _D, _I, _D,
                                       _D, _D, _D, _I, _I, C.c_int, _I, _D, _D, C.c_int, _I]),
        "orc_get_collision_records": (C.c_int, [C.c_void_p, _D, C.c_int]),
        "orc_set_spin": (None, [C.c_void_p, _D]),
        "orc_get_spin": (None, [C.c_void_p, _D]),
        "orc_substep_weights": (C.c_int, [C.c_int, _D]),
        "orc_create": (C.c_void_p, [C.c_int, _P, _D, _D, _D, _D]),
        "orc_free": (None, [C.c_void_p]),
        "orc_step": (C.c_int, [C.c_void_p, C.c_int]),
        "orc_get_state": (None, [C.c_void_p, _D, _D, _D, _D, _I]),
        "orc_get_internal": (None, [C.c_void_p, _D, _D, _D, _D]),
        "orc_get_energy": (C.c_double, [C.c_void_p, _D]),
        "orc_get_candidates": (C.c_int, [C.c_void_p, _I, C.c_int]),
        "orc_get_encounters": (C.c_int, [C.c_void_p, C.c_int, _I, C.c_int]),
        "orc_get_groups": (C.c_int, [C.c_void_p, C.c_int, _I, _I, C.c_int]),
        "orc_get_stats": (None, [C.c_void_p, C.POINTER(C.c_longlong), C.c_int]),
        "orc_get_collisions": (C.c_int, [C.c_void_p, _I, C.c_int]),
        "orc_get_ejections": (C.c_int, [C.c_void_p, _D, C.c_int]),
        "orc_tp_get_ejections": (C.c_int, [C.c_void_p, _D, C.c_int]),
        "orc_tp_create": (C.c_void_p, [C.c_int, _P, _D, _D, _D, _D, C.c_int, _D, _D, _D]),
        "orc_tp_free": (None, [C.c_void_p]),
        "orc_tp_step": (C.c_int, [C.c_void_p, C.c_int]),
        "orc_tp_get_state": (None, [C.c_void_p, _D, _D, _D, _I, _D, _D, _I]),
        "orc_tp_get_stats": (None, [C.c_void_p, C.POINTER(C.c_longlong), C.c_int]),
        "orc_tp_get_encounters": (C.c_int, [C.c_void_p, C.c_int, _I, C.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def params(**kw) -> Params:
    p = Params()
    lib().orc_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_D)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_I)


def _dout(n):
    a = np.zeros(n, dtype=np.float64)
    return a, a.ctypes.data_as(_D)


def _iout(n):
    a = np.zeros(n, dtype=np.int32)
    return a, a.ctypes.data_as(_I)


# ---------------------------------------------------------------- phase routines
def changeover(r, rc):
    return lib().orc_changeover(float(r), float(rc))


def changeover_dr(r, rc):
    return lib().orc_changeover_dr(float(r), float(rc))


def weight_B(r2, rc, kmode=0):
    return lib().orc_weight_B(float(r2), float(rc), int(kmode))


def rcrit(p: Params, tau_abs, m, alive, x, v):
    n = len(m)
    m, pm = _d(m); al, pa = _i(alive); x, px = _d(x); v, pv = _d(v)
    rc, prc = _dout(n)
    lib().orc_rcrit(n, C.byref(p), float(tau_abs), pm, pa, px, pv, prc)
    return rc


def accel_B(p: Params, m, alive, x, rc):
    n = len(m)
    m, pm = _d(m); al, pa = _i(alive); x, px = _d(x); rc, prc = _d(rc)
    a, pa_out = _dout(3 * n)
    lib().orc_accel_B(n, C.byref(p), pm, pa, px, prc, pa_out)
    return a.reshape(n, 3)


def precheck(p: Params, alive, x, rc):
    n = len(alive)
    al, pa = _i(alive); x, px = _d(x); rc, prc = _d(rc)
    cap = max(1, n * (n - 1) // 2)
    out, po = _iout(2 * cap)
    cnt = lib().orc_precheck(n, C.byref(p), pa, px, prc, po, cap)
    return out[: 2 * cnt].reshape(cnt, 2)


def momentum(m, alive, v):
    m, pm = _d(m); al, pa = _i(alive); v, pv = _d(v)
    P, pP = _dout(3)
    lib().orc_momentum(len(m), pm, pa, pv, pP)
    return P


def sun_drift(p: Params, alive, x, P, h):
    n = len(alive)
    al, pa = _i(alive)
    x = np.array(x, dtype=np.float64)
    P, pP = _d(P)
    lib().orc_sun_drift(n, C.byref(p), pa, x.ctypes.data_as(_D), pP, float(h))
    return x


def stumpff(z):
    c, pc = _dout(4)
    lib().orc_stumpff(float(z), pc)
    return c


def kepler_drift(mu, x, v, dt, maxit=30):
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    it = C.c_int(0)
    st = lib().orc_kepler_drift(float(mu), x.ctypes.data_as(_D), v.ctypes.data_as(_D), float(dt),
                                int(maxit), C.byref(it))
    return x, v, st, it.value


def hermite_min(dx0, dv0, dx1, dv1, tau):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (dx0, dv0, dx1, dv1)]
    return lib().orc_hermite_min(*[a.ctypes.data_as(_D) for a in arrs], float(tau))


def encounters(alive, x0, v0, x1, v1, rc, cand, tau):
    n = len(alive)
    al, pa = _i(alive)
    x0, p0 = _d(x0); v0, pv0 = _d(v0); x1, p1 = _d(x1); v1, pv1 = _d(v1); rc, prc = _d(rc)
    cand = np.ascontiguousarray(np.asarray(cand, dtype=np.int32).reshape(-1, 2))
    pc = cand.ctypes.data_as(_I)
    cap = max(1, len(cand))
    out, po = _iout(2 * cap)
    cnt = lib().orc_encounters(n, pa, p0, pv0, p1, pv1, prc, pc, len(cand), float(tau), po, cap)
    return out[: 2 * cnt].reshape(cnt, 2)


def groups(n, pairs, single=None):
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    s = np.zeros(n, np.int32) if single is None else np.asarray(single, np.int32)
    s, ps = _i(s)
    gs, pgs = _iout(n + 1)
    mem, pm = _iout(max(n, 1))
    ng = lib().orc_groups(n, pairs.ctypes.data_as(_I), len(pairs), ps, pgs, pm)
    return [mem[gs[k]:gs[k + 1]].copy() for k in range(ng)]


def energy(p: Params, m, alive, x, v):
    m, pm = _d(m); al, pa = _i(alive); x, px = _d(x); v, pv = _d(v)
    return lib().orc_energy(len(m), C.byref(p), pm, pa, px, pv)


CREC = 24  # doubles per collision report (orc_get_collision_records)


def bs_group(p: Params, idx, tau, m, R, alive, x, v, rc, spin=None):
    """BS-integrate the group idx over tau; returns (x, v, m, R, alive, U, status, collisions, spin,
    records). spin [n, 3] (None: zero) is updated by mergers; records are the collision reports."""
    n = len(m)
    idx, pidx = _i(idx)
    m = np.array(m, np.float64); R = np.array(R, np.float64)
    alive = np.array(alive, np.int32); x = np.array(x, np.float64); v = np.array(v, np.float64)
    sp = np.zeros((n, 3)) if spin is None else np.array(spin, np.float64).reshape(n, 3)
    rc, prc = _d(rc)
    U = C.c_double(0.0)
    nc = C.c_int(0)
    coll, pcoll = _iout(2 * max(n, 1))
    rec, prec = _dout(CREC * max(n, 1))
    nrec = C.c_int(0)
    steps = C.c_int(0)
    st = lib().orc_bs_group_rec(n, C.byref(p), len(idx), pidx, float(tau), m.ctypes.data_as(_D),
                                R.ctypes.data_as(_D), alive.ctypes.data_as(_I), x.ctypes.data_as(_D),
                                v.ctypes.data_as(_D), prc, C.byref(U), C.byref(nc), pcoll, n,
                                C.byref(steps), sp.ctypes.data_as(_D), prec, n, C.byref(nrec))
    return dict(x=x, v=v, m=m, R=R, alive=alive, U=U.value, status=st,
                collisions=coll[: 2 * nc.value].reshape(-1, 2), bs_steps=steps.value, spin=sp,
                records=rec[: CREC * nrec.value].reshape(-1, CREC))


def substep_weights(order):
    """The oracle's composition weights (Sect. 2.3): substep j of a full step has length w[j] tau."""
    w, pw = _dout(7)
    k = lib().orc_substep_weights(int(order), pw)
    return w[:k].copy()


# ---------------------------------------------------------------- whole simulation
class Sim:
    """Main-mode simulation on the oracle (n orbiting bodies, central mass in params)."""

    def __init__(self, p: Params, m, R, xh, vh, omp: bool = False):
        self.p = p
        self.n = len(m)
        self._L = lib_omp() if omp else lib()
        if self._L is None:
            raise RuntimeError("the OpenMP build of the oracle is unavailable")
        m, pm = _d(m); R, pR = _d(R); xh, px = _d(xh); vh, pv = _d(vh)
        self._h = self._L.orc_create(self.n, C.byref(p), pm, pR, px, pv)
        if not self._h:
            raise RuntimeError("orc_create failed")

    def close(self):
        if getattr(self, "_h", None):
            self._L.orc_free(self._h)
            self._h = None

    __del__ = close

    def step(self, nsteps=1) -> int:
        return self._L.orc_step(self._h, int(nsteps))

    def state(self):
        n = self.n
        x, px = _dout(3 * n); v, pv = _dout(3 * n); m, pm = _dout(n); R, pR = _dout(n)
        al, pa = _iout(n)
        self._L.orc_get_state(self._h, px, pv, pm, pR, pa)
        return dict(x=x.reshape(n, 3), v=v.reshape(n, 3), m=m, R=R, alive=al)

    def internal(self):
        n = self.n
        x, px = _dout(3 * n); v, pv = _dout(3 * n); a, pa = _dout(3 * n); rc, prc = _dout(n)
        self._L.orc_get_internal(self._h, px, pv, pa, prc)
        return dict(x=x.reshape(n, 3), v=v.reshape(n, 3), a=a.reshape(n, 3), rc=rc)

    def energy(self):
        U = C.c_double(0.0)
        E = self._L.orc_get_energy(self._h, C.byref(U))
        return E, U.value

    def candidates(self):
        cnt = self._L.orc_get_candidates(self._h, None, 0)
        out, po = _iout(2 * max(cnt, 1))
        self._L.orc_get_candidates(self._h, po, cnt)
        return out[: 2 * cnt].reshape(cnt, 2)

    def encounters(self, substep=-1):
        cnt = self._L.orc_get_encounters(self._h, substep, None, 0)
        out, po = _iout(2 * max(cnt, 1))
        self._L.orc_get_encounters(self._h, substep, po, cnt)
        return out[: 2 * cnt].reshape(cnt, 2)

    def groups(self, substep=-1):
        n = self.n
        gs, pgs = _iout(n + 1)
        mem, pm = _iout(max(n, 1))
        ng = self._L.orc_get_groups(self._h, substep, pgs, pm, n)
        return [mem[gs[k]:gs[k + 1]].copy() for k in range(ng)]

    def stats(self):
        arr = (C.c_longlong * 12)()
        self._L.orc_get_stats(self._h, arr, 12)
        return dict(zip(STAT_NAMES, list(arr)))

    def collisions(self):
        cnt = self._L.orc_get_collisions(self._h, None, 0)
        out, po = _iout(2 * max(cnt, 1))
        self._L.orc_get_collisions(self._h, po, cnt)
        return out[: 2 * cnt].reshape(-1, 2)

    def ejections(self):
        """Removed bodies (Sect. 3.2, Ejections): rows of body index, step, heliocentric x[3], v[3]."""
        return _ejections(self._L.orc_get_ejections, self._h)

    def collision_records(self):
        """Collision reports (Sect. 3.2): rows of CREC doubles, see orc_get_collision_records."""
        cnt = self._L.orc_get_collision_records(self._h, None, 0)
        out, po = _dout(CREC * max(cnt, 1))
        self._L.orc_get_collision_records(self._h, po, cnt)
        return out[: CREC * cnt].reshape(cnt, CREC)

    def set_spin(self, spin):
        sp, psp = _d(np.asarray(spin, np.float64).reshape(self.n, 3))
        self._L.orc_set_spin(self._h, psp)

    def spin(self):
        sp, psp = _dout(3 * self.n)
        self._L.orc_get_spin(self._h, psp)
        return sp.reshape(self.n, 3)


def _ejections(fn, h):
    cnt = fn(h, None, 0)
    out, po = _dout(8 * max(cnt, 1))
    fn(h, po, cnt)
    return out[: 8 * cnt].reshape(cnt, 8)


TP_STAT_NAMES = ["tp_candidates", "tp_encounters", "tp_bs_steps", "tp_removed", "tp_bs_failed", "tp_ejected", "u6", "u7"]


class TPSim:
    """Test-particle mode on the oracle: massive bodies (<= 32) plus massless test particles."""

    def __init__(self, p: Params, m, R, xh, vh, xt, vt, Rt=None):
        self.p = p
        self.n = len(m)
        self.nt = len(xt)
        m, pm = _d(m); R, pR = _d(R); xh, px = _d(xh); vh, pv = _d(vh)
        xt, pxt = _d(xt); vt, pvt = _d(vt)
        Rt, pRt = _d(np.zeros(self.nt) if Rt is None else Rt)
        self._h = lib().orc_tp_create(self.n, C.byref(p), pm, pR, px, pv, self.nt, pxt, pvt, pRt)
        if not self._h:
            raise RuntimeError("orc_tp_create failed")

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_tp_free(self._h)
            self._h = None

    __del__ = close

    def step(self, nsteps=1):
        return lib().orc_tp_step(self._h, int(nsteps))

    def state(self):
        n, nt = self.n, self.nt
        x, px = _dout(3 * n); v, pv = _dout(3 * n); m, pm = _dout(n); al, pa = _iout(n)
        xt, pxt = _dout(3 * nt); vt, pvt = _dout(3 * nt); at, pat = _iout(nt)
        lib().orc_tp_get_state(self._h, px, pv, pm, pa, pxt, pvt, pat)
        return dict(x=x.reshape(n, 3), v=v.reshape(n, 3), m=m, alive=al, xt=xt.reshape(nt, 3), vt=vt.reshape(nt, 3),
                    tp_alive=at)

    def stats(self):
        arr = (C.c_longlong * 8)()
        lib().orc_tp_get_stats(self._h, arr, 8)
        return dict(zip(TP_STAT_NAMES, list(arr)))

    def ejections(self):
        """Removed planets, as Sim.ejections (removed particles: tp_alive and stats()["tp_ejected"])."""
        return _ejections(lib().orc_tp_get_ejections, self._h)

    def encounters(self, substep=-1):
        cnt = lib().orc_tp_get_encounters(self._h, substep, None, 0)
        out, po = _iout(2 * max(cnt, 1))
        lib().orc_tp_get_encounters(self._h, substep, po, cnt)
        return out[: 2 * cnt].reshape(cnt, 2)
