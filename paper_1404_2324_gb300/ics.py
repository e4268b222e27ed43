"""Seeded synthetic initial conditions shaped like the paper's workloads.

This module only draws inputs; it holds none of the integrator's arithmetic. It is the one
piece shared by the CUDA path (bench, tests) and the CPU oracle (tests). The paper's runs use
synthetic planetesimal disks with no public data set (Sect. 4.1, 4.2, 4.3); these recipes
stand in for them:

* ``disk32``     -- 32 bodies, m log-uniform [1e-8, 1e-6] Msun, a U[0.5, 1.5] AU,
                    e ~ Rayleigh(0.01), i ~ Rayleigh(0.005 rad), angles U[0, 2 pi).
* ``disk2048``   -- 2048 bodies, the same shapes over a U[0.5, 4] AU, masses rescaled to a total
                    of 2 Earth masses.
* ``tp_disk``    -- 8 planets (m log-uniform [1e-7, 1e-3], a log-spaced 0.4-30 AU, e, i
                    Rayleigh(0.01)) plus massless test particles (a U[0.3, 5], e U[0, 0.3],
                    i U[0, 0.2]).
* ``batch``      -- many independent systems, N_s ~ U{4..64} bodies including the star;
                    planets m log-uniform [1e-7, 1e-4], a U[0.1, 5], e ~ Rayleigh(0.02),
                    i ~ Rayleigh(0.01).
* ``adj_disks``  -- many independent disks of equal size with the ``disk2048`` shapes, each with
                    2 Earth masses x n/2048 (the differentiable engine's workload).

Radii follow from a bulk density of 2 g/cm^3. Units: AU, day, Msun, G = k^2 (Gaussian).
Orbital elements become heliocentric Cartesian states with mu = G (m0 + m_i); this conversion
belongs to the input recipe, not to the method.
"""
from __future__ import annotations

import numpy as np

K_GAUSS = 0.01720209895
G_GAUSS = K_GAUSS * K_GAUSS  # AU^3 Msun^-1 day^-2
M_EARTH = 3.00349e-6         # Msun
MSUN_G = 1.98847e33          # g
AU_CM = 1.495978707e13       # cm


def radius_from_mass(m, rho_cgs=2.0):
    """Physical radius [AU] of a body of mass m [Msun] and bulk density rho [g/cm^3]."""
    vol = np.asarray(m, dtype=np.float64) * MSUN_G / rho_cgs
    return np.cbrt(3.0 * vol / (4.0 * np.pi)) / AU_CM


def elements_to_cartesian(mu, a, e, inc, node, peri, mean_anom):
    """Heliocentric position and velocity of elliptic orbits (vectorised over bodies)."""
    a = np.asarray(a, np.float64)
    e = np.asarray(e, np.float64)
    M = np.mod(np.asarray(mean_anom, np.float64), 2.0 * np.pi)
    E = M + e * np.sin(M)
    for _ in range(60):  # eccentric anomaly from E - e sin E = M
        dE = (E - e * np.sin(E) - M) / (1.0 - e * np.cos(E))
        E = E - dE
        if np.max(np.abs(dE)) < 1e-15:
            break
    cE, sE = np.cos(E), np.sin(E)
    b = np.sqrt(1.0 - e * e)
    xp = a * (cE - e)
    yp = a * b * sE
    n = np.sqrt(mu / a ** 3)
    edot = n / (1.0 - e * cE)
    vxp = -a * sE * edot
    vyp = a * b * cE * edot
    cO, sO = np.cos(node), np.sin(node)
    cw, sw = np.cos(peri), np.sin(peri)
    ci, si = np.cos(inc), np.sin(inc)
    r11 = cO * cw - sO * sw * ci
    r12 = -cO * sw - sO * cw * ci
    r21 = sO * cw + cO * sw * ci
    r22 = -sO * sw + cO * cw * ci
    r31 = sw * si
    r32 = cw * si
    x = np.stack([r11 * xp + r12 * yp, r21 * xp + r22 * yp, r31 * xp + r32 * yp], axis=-1)
    v = np.stack([r11 * vxp + r12 * vyp, r21 * vxp + r22 * vyp, r31 * vxp + r32 * vyp], axis=-1)
    return x, v


def _disk(rng, n, m_lo, m_hi, a_lo, a_hi, e_sigma, i_sigma, m0=1.0, G=G_GAUSS, total_mass=None):
    m = np.exp(rng.uniform(np.log(m_lo), np.log(m_hi), n))
    if total_mass is not None:
        m *= total_mass / m.sum()
    a = rng.uniform(a_lo, a_hi, n)
    e = np.minimum(rng.rayleigh(e_sigma, n), 0.9)
    inc = rng.rayleigh(i_sigma, n)
    node, peri, M = (rng.uniform(0.0, 2.0 * np.pi, n) for _ in range(3))
    x, v = elements_to_cartesian(G * (m0 + m), a, e, inc, node, peri, M)
    return dict(m0=m0, G=G, m=m, R=radius_from_mass(m), x=x, v=v)


def disk32(seed=1, n=32):
    """Config 'disk32': the 32-body disk (energy-conservation shape of Sect. 4.1)."""
    rng = np.random.default_rng(seed)
    d = _disk(rng, n, 1e-8, 1e-6, 0.5, 1.5, 0.01, 0.005)
    d.update(dt=6.0, order=2, name=f"disk{n}")
    return d


def disk2048(seed=2, n=2048, total_mass=2.0 * M_EARTH, order=4):
    """Config 'disk2048': the 2048-planetesimal disk over 0.5-4 AU (Sect. 4.2 / 4.3 shape)."""
    rng = np.random.default_rng(seed)
    d = _disk(rng, n, 1e-8, 1e-6, 0.5, 4.0, 0.01, 0.005, total_mass=total_mass)
    d.update(dt=6.0, order=order, name=f"disk{n}")
    return d


def tp_disk(seed=3, n_tp=1 << 20, n_planets=8):
    """Config 'tp_disk': planets plus massless test particles (Sect. 3.3 shape)."""
    rng = np.random.default_rng(seed)
    mp = np.exp(rng.uniform(np.log(1e-7), np.log(1e-3), n_planets))
    ap = np.geomspace(0.4, 30.0, n_planets)
    ep = np.minimum(rng.rayleigh(0.01, n_planets), 0.9)
    ip = rng.rayleigh(0.01, n_planets)
    angs = [rng.uniform(0.0, 2.0 * np.pi, n_planets) for _ in range(3)]
    xp, vp = elements_to_cartesian(G_GAUSS * (1.0 + mp), ap, ep, ip, *angs)
    at = rng.uniform(0.3, 5.0, n_tp)
    et = rng.uniform(0.0, 0.3, n_tp)
    it = rng.uniform(0.0, 0.2, n_tp)
    angt = [rng.uniform(0.0, 2.0 * np.pi, n_tp) for _ in range(3)]
    xt, vt = elements_to_cartesian(G_GAUSS, at, et, it, *angt)
    return dict(m0=1.0, G=G_GAUSS, m=mp, R=radius_from_mass(mp), x=xp, v=vp,
                x_tp=xt, v_tp=vt, R_tp=np.zeros(n_tp), dt=6.0, order=2, name="tp_disk")


def batch(seed=4, n_sys=8192, n_lo=4, n_hi=64):
    """Config 'batch': many independent systems of N_s ~ U{n_lo..n_hi} bodies incl. the star."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, n_sys)  # bodies including the star
    nb = ns - 1
    offsets = np.zeros(n_sys + 1, np.int64)
    offsets[1:] = np.cumsum(nb)
    tot = int(offsets[-1])
    m = np.exp(rng.uniform(np.log(1e-7), np.log(1e-4), tot))
    a = rng.uniform(0.1, 5.0, tot)
    e = np.minimum(rng.rayleigh(0.02, tot), 0.9)
    inc = rng.rayleigh(0.01, tot)
    angs = [rng.uniform(0.0, 2.0 * np.pi, tot) for _ in range(3)]
    x, v = elements_to_cartesian(G_GAUSS * (1.0 + m), a, e, inc, *angs)
    return dict(m0=np.ones(n_sys), G=G_GAUSS, m=m, R=radius_from_mass(m), x=x, v=v,
                offsets=offsets, dt=6.0, order=2, name="batch")


def adj_disks(seed=5, n_sys=64, n=256, order=2):
    """Config 'adj_disks': n_sys independent disks of n planetesimals with the 2048-disk shapes
    (0.5-4 AU, e~Rayleigh(0.01), i~Rayleigh(0.005), masses log-uniform 1e-8..1e-6 Msun rescaled to
    2 Earth masses x n/2048 per disk), for the differentiable engine. Arrays [n_sys, n(, 3)]."""
    rng = np.random.default_rng(seed)
    ds = [_disk(rng, n, 1e-8, 1e-6, 0.5, 4.0, 0.01, 0.005, total_mass=2.0 * M_EARTH * n / 2048) for _ in range(n_sys)]
    return dict(m0=np.ones(n_sys), G=G_GAUSS, m=np.stack([d["m"] for d in ds]), x=np.stack([d["x"] for d in ds]),
                v=np.stack([d["v"] for d in ds]), dt=6.0, order=order, name="adj_disks")
