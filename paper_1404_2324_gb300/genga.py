"""ctypes binding of libgenga (include/genga.h), same names as the C ABI.

Argument marshalling only: host arrays are numpy float64/int32, device arrays are torch CUDA
tensors whose data pointers are passed through. Every computation runs in the CUDA library; when
the library cannot be loaded the binding raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

GENGA_OK = 0
GENGA_EINVAL = -1
GENGA_ECUDA = -2
GENGA_ENOMEM = -3
GENGA_ECAP = -4
GENGA_ESIZE = -5
ST_KEPLER_FALLBACK = 1
ST_BS_FAILED = 2
ST_REUSE_FULLKICK = 4
ST_GROUP_TOO_LARGE = 8
ST_RECORD_OVERFLOW = 32
ST_UNION_ROUNDS = 16
ST_EJECT_OVERFLOW = 64
ST_GRID_TIMEOUT = 128
ST_COLL_OVERFLOW = 256
COUNTER_NAMES = ["steps", "candidates", "encounters", "groups", "bs_steps", "kepler_fallbacks",
                 "mergers", "full_kicks"]


class GengaError(RuntimeError):
    pass


class genga_params(C.Structure):
    _fields_ = [("n1", C.c_double), ("n2", C.c_double), ("pc", C.c_double), ("bs_eps", C.c_double),
                ("bs_kmax", C.c_int), ("bs_max_halvings", C.c_int), ("kepler_maxit", C.c_int),
                ("kmode", C.c_int), ("collisions", C.c_int), ("precise_div", C.c_int),
                ("rcut", C.c_double), ("rcut_sun", C.c_double), ("nmin", C.c_int), ("precheck_substeps", C.c_int)]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_V = C.c_void_p

_SIGS = {
    "genga_default_params": (C.c_int, [C.POINTER(genga_params)]),
    "genga_init": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, _D, _D, _D, _D, C.c_double, C.c_double,
                             C.c_int, C.c_int]),
    "genga_set_params": (C.c_int, [_V, C.POINTER(genga_params)]),
    "genga_set_stream": (C.c_int, [_V, _V]),
    "genga_step": (C.c_int, [_V, C.c_int]),
    "genga_sync": (C.c_int, [_V]),
    "genga_set_state": (C.c_int, [_V, _D, _D]),
    "genga_get_state": (C.c_int, [_V, _D, _D, _D, _D, _I]),
    "genga_energy": (C.c_int, [_V, _D, _D]),
    "genga_encounters": (C.c_int, [_V, C.c_int, _I, C.c_int, _I]),
    "genga_ejections": (C.c_int, [_V, _D, C.c_int, _I]),
    "genga_collisions": (C.c_int, [_V, _D, C.c_int, _I]),
    "genga_batch_schedule": (C.c_int, [_V, _I, _I, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "genga_batch_set_schedule": (C.c_int, [_V, C.c_int]),
    "genga_fp64_probe": (C.c_int, [C.c_int, _D, C.POINTER(C.c_float), _V]),
    "genga_tp_encounters": (C.c_int, [_V, _I, C.c_int, _I]),
    "genga_batch_encounters": (C.c_int, [_V, _I, C.c_int, _I]),
    "genga_set_spin": (C.c_int, [_V, _D]),
    "genga_get_spin": (C.c_int, [_V, _D]),
    "genga_status": (C.c_int, [_V, _I, C.POINTER(C.c_longlong)]),
    "genga_free": (None, [_V]),
    "genga_set_profiling": (C.c_int, [_V, C.c_int]),
    "genga_kick_time": (C.c_int, [_V, C.POINTER(C.c_float), _I]),
    "genga_launch_count": (C.c_int, [_V, _I]),
    "genga_phase_rcrit": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                    _V, _V, _V, _V, _V, _V]),
    "genga_phase_kick": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, _V, _V, _V, _V, _V,
                                   _V, C.c_int, _I, _V]),
    "genga_phase_kepler": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_int, _V, _V, _V, _V, _V]),
    "genga_phase_encounters": (C.c_int, [C.c_int, _V, _V, _V, _V, _V, _V, _V, C.c_int, C.c_double, _V,
                                         C.c_int, _I, _V]),
    "genga_phase_groups": (C.c_int, [C.c_int, _V, C.c_int, _V, _V, _V, _I, _V]),
    "genga_phase_bs": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int,
                                 C.c_int, C.c_int, C.c_int, _V, _V, _V, _V, _V, _V, _V, _V, _D, _V]),
    "genga_phase_energy": (C.c_int, [C.c_int, C.c_double, C.c_double, _V, _V, _V, _V, _D, _V]),
    "genga_phase_mathcheck": (C.c_int, [C.c_int, C.c_int, _V, _V, _V]),
    "genga_adj_init": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, _D, C.c_double, C.c_double, C.c_int,
                                 C.c_int]),
    "genga_adj_set_stream": (C.c_int, [_V, _V]),
    "genga_adj_forward": (C.c_int, [_V, C.c_int, _V, _V, _V, _V, _V]),
    "genga_adj_backward": (C.c_int, [_V, _V, _V, _V, _V, _V]),
    "genga_adj_status": (C.c_int, [_V, _I]),
    "genga_adj_sync": (C.c_int, [_V]),
    "genga_adj_free": (None, [_V]),
    "genga_init_tp": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, _D, _D, _D, _D, C.c_double, C.c_double, C.c_int,
                                C.c_int, _D, _D, _D]),
    "genga_get_state_tp": (C.c_int, [_V, _D, _D, _I]),
    "genga_tp_status": (C.c_int, [_V, C.POINTER(C.c_longlong)]),
    "genga_init_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, _I, _D, _D, _D, _D, _D, C.c_double,
                                   C.c_double, C.c_int, C.c_int]),
    "genga_batch_info": (C.c_int, [_V, _I, _I, _I]),
    "genga_batch_set_kick": (C.c_int, [_V, C.c_int, C.c_int]),
    "genga_get_state_batch": (C.c_int, [_V, _D, _D, _D, _D, _I]),
    "genga_set_state_batch": (C.c_int, [_V, _D, _D]),
    "genga_energy_batch": (C.c_int, [_V, _D, _D]),
    "genga_kick_noalloc": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, _V, _V, _V, _V, _V,
                                     _V, C.c_int, _V, _V]),
}

EXPORTED = sorted(_SIGS)


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Loads libgenga.so (building it first if needed); raises GengaError if that fails."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise GengaError(f"libgenga not built: {path}")
            L = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise GengaError(f"{what} failed with code {rc}")
    return rc


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _ip(a: np.ndarray):
    return a.ctypes.data_as(_I)


def _tp(t):
    """Device pointer of a contiguous torch CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise GengaError("phase arguments must be contiguous CUDA tensors")
    return C.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------------------------------ C names
def genga_default_params() -> genga_params:
    p = genga_params()
    _check(lib().genga_default_params(C.byref(p)), "genga_default_params")
    return p


def genga_init(masses, radii, x, v, G, dt, order=2, mode=0):
    """Returns an opaque context handle; arrays are host (numpy), central mass at index 0."""
    m = np.ascontiguousarray(masses, np.float64)
    R = np.ascontiguousarray(radii, np.float64)
    xx = np.ascontiguousarray(x, np.float64).reshape(-1)
    vv = np.ascontiguousarray(v, np.float64).reshape(-1)
    n = len(m)
    if len(R) != n or len(xx) != 3 * n or len(vv) != 3 * n:
        raise GengaError("genga_init: array sizes disagree")
    h = C.c_void_p()
    _check(lib().genga_init(C.byref(h), n, _dp(m), _dp(R), _dp(xx), _dp(vv), float(G), float(dt), int(order),
                            int(mode)), "genga_init")
    return h


def genga_set_params(ctx, p: genga_params):
    return _check(lib().genga_set_params(ctx, C.byref(p)), "genga_set_params")


def genga_set_stream(ctx, stream=None):
    return _check(lib().genga_set_stream(ctx, None if stream is None else C.c_void_p(stream.cuda_stream)),
                  "genga_set_stream")


def genga_step(ctx, n_steps=1):
    return _check(lib().genga_step(ctx, int(n_steps)), "genga_step")


def genga_sync(ctx):
    return _check(lib().genga_sync(ctx), "genga_sync")


def genga_set_state(ctx, x, v):
    xx = np.ascontiguousarray(x, np.float64).reshape(-1)
    vv = np.ascontiguousarray(v, np.float64).reshape(-1)
    return _check(lib().genga_set_state(ctx, _dp(xx), _dp(vv)), "genga_set_state")


def genga_get_state(ctx, n, x=None, v=None, m=None, R=None, alive=None):
    """Fills (or allocates) host arrays x, v [n,3], m, R [n], alive [n]; returns them as a dict."""
    x = np.empty((n, 3)) if x is None else x
    v = np.empty((n, 3)) if v is None else v
    m = np.empty(n) if m is None else m
    R = np.empty(n) if R is None else R
    alive = np.empty(n, np.int32) if alive is None else alive
    _check(lib().genga_get_state(ctx, _dp(x), _dp(v), _dp(m), _dp(R), _ip(alive)), "genga_get_state")
    return dict(x=x, v=v, m=m, R=R, alive=alive)


def genga_energy(ctx):
    E, U = C.c_double(), C.c_double()
    _check(lib().genga_energy(ctx, C.byref(E), C.byref(U)), "genga_energy")
    return E.value, U.value


def genga_encounters(ctx, substep=-1):
    cnt = C.c_int(0)
    rc = lib().genga_encounters(ctx, int(substep), None, 0, C.byref(cnt))
    if rc not in (GENGA_OK, GENGA_ECAP):
        _check(rc, "genga_encounters")
    out = np.zeros(2 * max(cnt.value, 1), np.int32)
    _check(lib().genga_encounters(ctx, int(substep), _ip(out), cnt.value, C.byref(cnt)), "genga_encounters")
    return out[: 2 * cnt.value].reshape(-1, 2)


def genga_status(ctx):
    code = C.c_int(0)
    det = (C.c_longlong * 8)()
    _check(lib().genga_status(ctx, C.byref(code), det), "genga_status")
    return code.value, dict(zip(COUNTER_NAMES, list(det)))


def genga_set_profiling(ctx, on=True):
    return _check(lib().genga_set_profiling(ctx, int(bool(on))), "genga_set_profiling")


def genga_kick_time(ctx):
    ms, n = C.c_float(0.0), C.c_int(0)
    _check(lib().genga_kick_time(ctx, C.byref(ms), C.byref(n)), "genga_kick_time")
    return ms.value, n.value


def genga_launch_count(ctx):
    k = C.c_int(0)
    _check(lib().genga_launch_count(ctx, C.byref(k)), "genga_launch_count")
    return k.value


def genga_free(ctx):
    if ctx:
        lib().genga_free(ctx)


# ------------------------------------------------------------------------------------ test particles
def genga_init_tp(masses, radii, x, v, G, dt, order, xt, vt, Rt=None):
    m = np.ascontiguousarray(masses, np.float64)
    R = np.ascontiguousarray(radii, np.float64)
    xx = np.ascontiguousarray(x, np.float64).reshape(-1)
    vv = np.ascontiguousarray(v, np.float64).reshape(-1)
    xtt = np.ascontiguousarray(xt, np.float64).reshape(-1)
    vtt = np.ascontiguousarray(vt, np.float64).reshape(-1)
    ntp = len(xtt) // 3
    Rtt = None if Rt is None else np.ascontiguousarray(Rt, np.float64)
    h = C.c_void_p()
    _check(lib().genga_init_tp(C.byref(h), len(m), _dp(m), _dp(R), _dp(xx), _dp(vv), float(G), float(dt), int(order),
                               ntp, _dp(xtt), _dp(vtt), None if Rtt is None else _dp(Rtt)), "genga_init_tp")
    return h


def genga_get_state_tp(ctx, n_tp):
    xt, vt, al = np.empty((n_tp, 3)), np.empty((n_tp, 3)), np.empty(n_tp, np.int32)
    _check(lib().genga_get_state_tp(ctx, _dp(xt), _dp(vt), _ip(al)), "genga_get_state_tp")
    return dict(xt=xt, vt=vt, tp_alive=al)


def genga_tp_status(ctx):
    d = (C.c_longlong * 5)()
    _check(lib().genga_tp_status(ctx, d), "genga_tp_status")
    return dict(zip(["tp_candidates", "tp_encounters", "tp_bs_steps", "tp_removed", "tp_ejected"], list(d)))


def genga_ejections(ctx):
    """Ejection records (Sect. 3.2): rows of body index, step, heliocentric x[3], v[3]."""
    n = C.c_int(0)
    _check(lib().genga_ejections(ctx, None, 0, C.byref(n)), "genga_ejections")
    out = np.zeros((max(n.value, 1), 8))
    _check(lib().genga_ejections(ctx, out.ctypes.data_as(_D), n.value, C.byref(n)), "genga_ejections")
    return out[: min(n.value, 4096)]


CREC = 24  # doubles per collision report


def genga_collisions(ctx):
    """Collision reports (Sect. 3.2): rows of step, substep, time, i, j, x_i, v_i, spin_i, x_j, v_j,
    spin_j, survivor (see include/genga.h)."""
    n = C.c_int(0)
    _check(lib().genga_collisions(ctx, None, 0, C.byref(n)), "genga_collisions")
    out = np.zeros((max(n.value, 1), CREC))
    _check(lib().genga_collisions(ctx, out.ctypes.data_as(_D), n.value, C.byref(n)), "genga_collisions")
    return out[: min(n.value, 4096)]


def _pairs(fn, ctx, name):
    n = C.c_int(0)
    rc = fn(ctx, None, 0, C.byref(n))
    if rc not in (0, -4):
        _check(rc, name)
    out = np.zeros((max(n.value, 1), 2), np.int32)
    _check(fn(ctx, out.ctypes.data_as(_I), n.value, C.byref(n)), name)
    return out[: n.value]


def genga_tp_encounters(ctx):
    """(particle, planet) encounter pairs of the last substep; planets numbered with the central mass at 0."""
    return _pairs(lib().genga_tp_encounters, ctx, "genga_tp_encounters")


def genga_batch_encounters(ctx):
    """Encounter pairs of every system in the last substep, flat caller indices (i < j)."""
    return _pairs(lib().genga_batch_encounters, ctx, "genga_batch_encounters")


def genga_fp64_probe(iters=1 << 16, stream=None):
    """Measured FP64 throughput of the device in TFLOP/s (and the probe launch's ms)."""
    tf, ms = C.c_double(0.0), C.c_float(0.0)
    _check(lib().genga_fp64_probe(int(iters), C.byref(tf), C.byref(ms), _stream_ptr(stream)), "genga_fp64_probe")
    return tf.value, ms.value


def genga_batch_schedule(ctx):
    """The batched schedule chosen at init: persistent launch or step graph, and the timings."""
    p, k = C.c_int(0), C.c_int(0)
    mg, mp = C.c_float(0.0), C.c_float(0.0)
    _check(lib().genga_batch_schedule(ctx, C.byref(p), C.byref(k), C.byref(mg), C.byref(mp)), "genga_batch_schedule")
    return dict(persistent=p.value, ctas=k.value, ms_graph=mg.value, ms_persistent=mp.value)


def genga_batch_set_schedule(ctx, persistent):
    _check(lib().genga_batch_set_schedule(ctx, int(persistent)), "genga_batch_set_schedule")


def genga_set_spin(ctx, spin):
    sp = np.ascontiguousarray(spin, np.float64)
    _check(lib().genga_set_spin(ctx, sp.ctypes.data_as(_D)), "genga_set_spin")


def genga_get_spin(ctx, nrows):
    out = np.zeros((nrows, 3))
    _check(lib().genga_get_spin(ctx, out.ctypes.data_as(_D)), "genga_get_spin")
    return out


# ------------------------------------------------------------------------------------ batched mode
def genga_init_batch(offsets, m0, masses, radii, x, v, G, dt, order=2, steps_per_launch=100):
    off = np.ascontiguousarray(offsets, np.int32)
    m0a = np.ascontiguousarray(m0, np.float64)
    m = np.ascontiguousarray(masses, np.float64)
    R = np.ascontiguousarray(radii, np.float64)
    xx = np.ascontiguousarray(x, np.float64).reshape(-1)
    vv = np.ascontiguousarray(v, np.float64).reshape(-1)
    nsys = len(off) - 1
    if len(m0a) != nsys or len(m) != off[-1] or len(xx) != 3 * len(m) or len(vv) != 3 * len(m) or len(R) != len(m):
        raise GengaError("genga_init_batch: array sizes disagree")
    h = C.c_void_p()
    _check(lib().genga_init_batch(C.byref(h), nsys, _ip(off), _dp(m0a), _dp(m), _dp(R), _dp(xx), _dp(vv), float(G),
                                  float(dt), int(order), int(steps_per_launch)), "genga_init_batch")
    return h


def genga_batch_set_kick(ctx, split, block):
    _check(lib().genga_batch_set_kick(ctx, int(split), int(block)), "genga_batch_set_kick")


def genga_batch_info(ctx):
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    _check(lib().genga_batch_info(ctx, C.byref(a), C.byref(b), C.byref(c)), "genga_batch_info")
    return a.value, b.value, c.value


def genga_get_state_batch(ctx, n):
    x, v, m, R = np.empty((n, 3)), np.empty((n, 3)), np.empty(n), np.empty(n)
    alive = np.empty(n, np.int32)
    _check(lib().genga_get_state_batch(ctx, _dp(x), _dp(v), _dp(m), _dp(R), _ip(alive)), "genga_get_state_batch")
    return dict(x=x, v=v, m=m, R=R, alive=alive)


def genga_set_state_batch(ctx, x, v):
    xx = np.ascontiguousarray(x, np.float64).reshape(-1)
    vv = np.ascontiguousarray(v, np.float64).reshape(-1)
    return _check(lib().genga_set_state_batch(ctx, _dp(xx), _dp(vv)), "genga_set_state_batch")


def genga_energy_batch(ctx, nsys):
    E = np.empty(nsys)
    U = C.c_double()
    _check(lib().genga_energy_batch(ctx, _dp(E), C.byref(U)), "genga_energy_batch")
    return E, U.value


# ------------------------------------------------------------------------------------ phases
def genga_phase_rcrit(n, G, m0, n1, n2, tau_abs, m, alive, x, v, rc, stream=None):
    return _check(lib().genga_phase_rcrit(n, G, m0, n1, n2, tau_abs, _tp(m), _tp(alive), _tp(x), _tp(v), _tp(rc),
                                          _stream_ptr(stream)), "genga_phase_rcrit")


def genga_phase_kick(n, G, pc, kmode, precise_div, m, alive, x, rc, a, cand, cap, stream=None):
    cnt = C.c_int(0)
    rc_ = lib().genga_phase_kick(n, G, pc, kmode, precise_div, _tp(m), _tp(alive), _tp(x), _tp(rc), _tp(a),
                                 _tp(cand), int(cap), C.byref(cnt), _stream_ptr(stream))
    _check(rc_, "genga_phase_kick")
    return cnt.value


def genga_phase_kepler(n, mu, dt, maxit, alive, x, v, fail, stream=None):
    return _check(lib().genga_phase_kepler(n, mu, dt, maxit, _tp(alive), _tp(x), _tp(v), _tp(fail),
                                           _stream_ptr(stream)), "genga_phase_kepler")


def genga_phase_encounters(n, alive, x0, v0, x1, v1, rc, cand, ncand, tau, out, cap, stream=None):
    cnt = C.c_int(0)
    _check(lib().genga_phase_encounters(n, _tp(alive), _tp(x0), _tp(v0), _tp(x1), _tp(v1), _tp(rc), _tp(cand),
                                        int(ncand), float(tau), _tp(out), int(cap), C.byref(cnt),
                                        _stream_ptr(stream)), "genga_phase_encounters")
    return cnt.value


def genga_phase_groups(n, pairs, npairs, single, group_start, members, stream=None):
    ng = C.c_int(0)
    _check(lib().genga_phase_groups(n, _tp(pairs), int(npairs), _tp(single), _tp(group_start), _tp(members),
                                    C.byref(ng), _stream_ptr(stream)), "genga_phase_groups")
    return ng.value


def genga_phase_bs(n, G, m0, tau, bs_eps, bs_kmax, bs_max_halvings, kmode, collisions, ngroups, group_start,
                   members, rc, m, R, alive, x, v, stream=None):
    U = C.c_double(0.0)
    st = lib().genga_phase_bs(n, G, m0, tau, bs_eps, bs_kmax, bs_max_halvings, kmode, collisions, ngroups,
                              _tp(group_start), _tp(members), _tp(rc), _tp(m), _tp(R), _tp(alive), _tp(x), _tp(v),
                              C.byref(U), _stream_ptr(stream))
    _check(st, "genga_phase_bs")
    return st, U.value


def genga_phase_energy(n, G, m0, m, alive, x, v, stream=None):
    E = C.c_double(0.0)
    _check(lib().genga_phase_energy(n, G, m0, _tp(m), _tp(alive), _tp(x), _tp(v), C.byref(E),
                                    _stream_ptr(stream)), "genga_phase_energy")
    return E.value


def genga_phase_mathcheck(n, which, inp, out, stream=None):
    return _check(lib().genga_phase_mathcheck(n, which, _tp(inp), _tp(out), _stream_ptr(stream)),
                  "genga_phase_mathcheck")


def genga_kick_noalloc(n, G, pc, kmode, precise_div, m, alive, x, rc, a, cand, cap, ncand, stream=None):
    """The kick phase without device allocation; ncand is a one-element int32 CUDA tensor."""
    return _check(lib().genga_kick_noalloc(n, G, pc, kmode, precise_div, _tp(m), _tp(alive), _tp(x), _tp(rc), _tp(a),
                                           _tp(cand), int(cap), _tp(ncand), _stream_ptr(stream)),
                  "genga_kick_noalloc")


# ------------------------------------------------------------------------------------ convenience
class Genga:
    """One simulation on the GPU (main mode). Host arrays include the central mass at index 0."""

    def __init__(self, masses, radii, x, v, G, dt, order=2, params: genga_params | None = None):
        self.n = len(masses)
        self.ctx = genga_init(masses, radii, x, v, G, dt, order)
        if params is not None:
            genga_set_params(self.ctx, params)

    def close(self):
        if getattr(self, "ctx", None):
            genga_free(self.ctx)
            self.ctx = None

    __del__ = close

    def step(self, n=1):
        genga_step(self.ctx, n)

    def sync(self):
        return genga_sync(self.ctx)

    def state(self):
        return genga_get_state(self.ctx, self.n)

    def set_state(self, x, v):
        genga_set_state(self.ctx, x, v)

    def energy(self):
        return genga_energy(self.ctx)

    def encounters(self, substep=-1):
        return genga_encounters(self.ctx, substep)

    def status(self):
        return genga_status(self.ctx)

    def collisions(self):
        return genga_collisions(self.ctx)

    def spin(self):
        return genga_get_spin(self.ctx, self.n)

    def set_spin(self, spin):
        genga_set_spin(self.ctx, spin)
