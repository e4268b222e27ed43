"""Independent two-body propagator used to pin the Kepler drift.

Classical route: Cartesian state -> orbital elements -> mean (or hyperbolic mean) anomaly
advanced linearly in time -> Kepler's equation solved for the eccentric (hyperbolic) anomaly
-> Cartesian state. It shares nothing with the universal-variable f/g solver under test.
"""
import numpy as np


def _solve_elliptic(M, e):
    E = M if e < 0.8 else np.pi * np.sign(M) if M != 0 else 0.0
    for _ in range(100):
        dE = (E - e * np.sin(E) - M) / (1.0 - e * np.cos(E))
        E -= dE
        if abs(dE) < 1e-16 * max(1.0, abs(E)):
            break
    return E


def _solve_hyperbolic(M, e):
    F = np.arcsinh(M / e)
    for _ in range(200):
        dF = (e * np.sinh(F) - F - M) / (e * np.cosh(F) - 1.0)
        F -= dF
        if abs(dF) < 1e-16 * max(1.0, abs(F)):
            break
    return F


def propagate(mu, x, v, dt):
    x = np.asarray(x, float)
    v = np.asarray(v, float)
    r = np.linalg.norm(x)
    h = np.cross(x, v)
    evec = np.cross(v, h) / mu - x / r
    e = np.linalg.norm(evec)
    eps = 0.5 * v @ v - mu / r
    a = -mu / (2.0 * eps)
    P = evec / e
    Q = np.cross(h, P) / np.linalg.norm(h)
    if e < 1.0:
        n = np.sqrt(mu / a ** 3)
        cosE = (1.0 - r / a) / e
        sinE = (x @ v) / (e * np.sqrt(mu * a))
        E0 = np.arctan2(sinE, cosE)
        M1 = E0 - e * np.sin(E0) + n * dt
        M1 = (M1 + np.pi) % (2 * np.pi) - np.pi
        E1 = _solve_elliptic(M1, e)
        b = np.sqrt(1.0 - e * e)
        r1 = a * (1.0 - e * np.cos(E1))
        x1 = a * (np.cos(E1) - e) * P + a * b * np.sin(E1) * Q
        v1 = np.sqrt(mu * a) / r1 * (-np.sin(E1) * P + b * np.cos(E1) * Q)
    else:
        aa = -a
        n = np.sqrt(mu / aa ** 3)
        coshF = (1.0 + r / aa) / e
        sinhF = (x @ v) / (e * np.sqrt(mu * aa))
        F0 = np.arcsinh(sinhF)
        del coshF
        M1 = e * np.sinh(F0) - F0 + n * dt
        F1 = _solve_hyperbolic(M1, e)
        b = np.sqrt(e * e - 1.0)
        r1 = aa * (e * np.cosh(F1) - 1.0)
        x1 = aa * (e - np.cosh(F1)) * P + aa * b * np.sinh(F1) * Q
        v1 = np.sqrt(mu * aa) / r1 * (-np.sinh(F1) * P + b * np.cosh(F1) * Q)
    return x1, v1
