"""Seeded synthetic particle distributions (FP64) for the tree-code force calculation.

This module only draws positions and masses. It holds none of the tree-code's
arithmetic, so both the CUDA path and the CPU oracle may take their inputs
from it.

The paper measures on a Milky Way model (bulge:disc:halo mass 1:1:4, Sec. 3)
whose initial conditions are not available here; the distributions below stand
in for it:

* ``plummer``      -- Plummer sphere, scale radius ``a``, equal masses 1/N,
                      radius from the inverse of the cumulative mass profile
                      r = a (U^{-2/3} - 1)^{-1/2}, redrawn when r > ``rmax``.
* ``clustered``    -- ``n_clusters`` Plummer spheres of equal particle count,
                      scale radii log-uniform in [0.01, 0.1], centres uniform in
                      the unit cube, each truncated at 20 scale radii.
* ``ensemble``     -- independent Plummer systems with N log-uniform in
                      [n_min, n_max] (rounded to an integer).
* ``sphere_disc``  -- half the particles in a uniform sphere of radius 1, half
                      in an exponential disc (surface density ~ exp(-R/0.3),
                      so R ~ Gamma(2, 0.3)) with a sech^2 vertical profile of
                      scale height 0.03.

Only ``Generator.random`` (uniform doubles from PCG64) is used, whose stream is
stable across numpy versions and machines.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["plummer", "clustered", "ensemble", "sphere_disc", "uniform_cube", "sample_indices"]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    cos_t = 2.0 * rng.random(n) - 1.0
    phi = 2.0 * math.pi * rng.random(n)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], axis=1)


def _plummer_radii(rng: np.random.Generator, n: int, a: float, rmax: float) -> np.ndarray:
    r = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        u = rng.random(todo.size)
        u = np.where(u <= 0.0, 1e-300, u)
        rr = a / np.sqrt(np.power(u, -2.0 / 3.0) - 1.0)
        ok = np.isfinite(rr) & (rr <= rmax)
        r[todo[ok]] = rr[ok]
        todo = todo[~ok]
    return r


def plummer(n: int, seed: int = 1, a: float = 1.0, rmax: float = 100.0,
            centre=(0.0, 0.0, 0.0), total_mass: float = 1.0):
    """Plummer sphere: returns (pos float64 [n,3], mass float64 [n]).

    ``rmax`` is in units of the scale radius ``a``.
    """
    rng = _rng(seed)
    r = _plummer_radii(rng, n, a, rmax * a)
    pos = _isotropic(rng, n) * r[:, None] + np.asarray(centre, dtype=np.float64)[None, :]
    mass = np.full(n, total_mass / n)
    return np.ascontiguousarray(pos), mass


def plummer_pv(n: int, seed: int = 1, a: float = 1.0, rmax: float = 100.0):
    """Plummer sphere in equilibrium, G = M = 1: (pos [n,3], vel [n,3], mass [n]).

    Positions as ``plummer``; each speed is q times the local escape speed
    sqrt(2) (r^2 + a^2)^(-1/4), with q drawn from the speed law of the
    isotropic distribution function, g(q) ~ q^2 (1 - q^2)^(7/2), by rejection
    (g < 0.1 on [0, 1]); directions isotropic; total momentum removed.
    """
    pos, mass = plummer(n, seed=seed, a=a, rmax=rmax)
    r2 = np.einsum("ij,ij->i", pos, pos)
    vesc = np.sqrt(2.0) * np.power(r2 + a * a, -0.25)
    q = np.empty(n)
    todo = np.arange(n)
    rng = _rng(seed + 1_000_003)
    while todo.size:
        x = rng.random(todo.size)
        y = 0.1 * rng.random(todo.size)
        ok = y < x * x * np.power(1.0 - x * x, 3.5)
        q[todo[ok]] = x[ok]
        todo = todo[~ok]
    vel = _isotropic(rng, n) * (q * vesc)[:, None]
    vel -= np.average(vel, axis=0, weights=mass)  # zero total momentum
    return pos, np.ascontiguousarray(vel), mass


def clustered(n: int = 4_194_304, n_clusters: int = 64, seed: int = 3,
              rs_min: float = 0.01, rs_max: float = 0.1, trunc: float = 20.0):
    """Sum of Plummer spheres; masses 1/N so each sphere weighs its share."""
    rng = _rng(seed)
    per = np.full(n_clusters, n // n_clusters)
    per[: n - per.sum()] += 1
    log_rs = rng.random(n_clusters) * (math.log(rs_max) - math.log(rs_min)) + math.log(rs_min)
    rs = np.exp(log_rs)
    centres = rng.random((n_clusters, 3))
    parts = []
    for k in range(n_clusters):
        r = _plummer_radii(rng, int(per[k]), float(rs[k]), trunc * float(rs[k]))
        parts.append(_isotropic(rng, int(per[k])) * r[:, None] + centres[k][None, :])
    pos = np.ascontiguousarray(np.concatenate(parts, axis=0))
    return pos, np.full(n, 1.0 / n)


def ensemble(n_sys: int = 256, seed: int = 4, n_min: int = 1024, n_max: int = 65536):
    """List of independent Plummer systems [(pos, mass), ...] with log-uniform N."""
    rng = _rng(seed)
    u = rng.random(n_sys)
    ns = np.rint(np.exp(math.log(n_min) + u * (math.log(n_max) - math.log(n_min)))).astype(np.int64)
    sub = rng.random(n_sys)
    out = []
    for k in range(n_sys):
        s = int(sub[k] * 2**31) + 1000 * k + 17
        out.append(plummer(int(ns[k]), seed=s))
    return out


def sphere_disc(n: int = 1_048_576, seed: int = 5, r_sphere: float = 1.0,
                r_d: float = 0.3, z_d: float = 0.03):
    """Uniform cold sphere (n//2) plus exponential sech^2 disc (rest), equal masses."""
    rng = _rng(seed)
    ns = n // 2
    nd = n - ns
    r = r_sphere * np.cbrt(rng.random(ns))
    sph = _isotropic(rng, ns) * r[:, None]
    u1 = rng.random(nd)
    u2 = rng.random(nd)
    R = -r_d * (np.log1p(-u1) + np.log1p(-u2))
    phi = 2.0 * math.pi * rng.random(nd)
    uz = rng.random(nd)
    uz = np.clip(uz, 1e-15, 1.0 - 1e-15)
    z = z_d * np.arctanh(2.0 * uz - 1.0)
    disc = np.stack([R * np.cos(phi), R * np.sin(phi), z], axis=1)
    pos = np.ascontiguousarray(np.concatenate([sph, disc], axis=0))
    return pos, np.full(n, 1.0 / n)


def _hernquist_radii(rng: np.random.Generator, n: int, a: float, rmax: float) -> np.ndarray:
    # M(<r) / M = r^2 / (r + a)^2  =>  r = a sqrt(u) / (1 - sqrt(u)), truncated at rmax
    umax = (rmax / (rmax + a)) ** 2
    s = np.sqrt(rng.random(n) * umax)
    return a * s / (1.0 - s)


def galaxy(n: int, seed: int = 9, r_d: float = 1.0, z_d: float = 0.1, a_bulge: float = 0.2,
           a_halo: float = 6.0):
    """Disc galaxy stand-in with bulge : disc : halo masses 1 : 1 : 4, equal-mass
    particles (n/6, n/6, 2n/3), total mass 1: Hernquist bulge (scale a_bulge,
    truncated at 10 a_bulge), exponential sech^2 disc (scale length r_d, height
    z_d), Hernquist halo (scale a_halo, truncated at 10 a_halo). Returns
    (pos [n,3], mass [n])."""
    rng = _rng(seed)
    nb = n // 6
    nd = n // 6
    nh = n - nb - nd
    rb = _hernquist_radii(rng, nb, a_bulge, 10 * a_bulge)
    bulge = _isotropic(rng, nb) * rb[:, None]
    u1 = rng.random(nd)
    u2 = rng.random(nd)
    R = -r_d * (np.log1p(-u1) + np.log1p(-u2))
    phi = 2.0 * math.pi * rng.random(nd)
    uz = np.clip(rng.random(nd), 1e-15, 1.0 - 1e-15)
    z = z_d * np.arctanh(2.0 * uz - 1.0)
    disc = np.stack([R * np.cos(phi), R * np.sin(phi), z], axis=1)
    rh = _hernquist_radii(rng, nh, a_halo, 10 * a_halo)
    halo = _isotropic(rng, nh) * rh[:, None]
    pos = np.ascontiguousarray(np.concatenate([bulge, disc, halo], axis=0))
    return pos, np.full(n, 1.0 / n)


def uniform_cube(n: int, seed: int = 7, side: float = 1.0):
    rng = _rng(seed)
    pos = np.ascontiguousarray(rng.random((n, 3)) * side)
    mass = 0.5 + rng.random(n)
    return pos, mass / mass.sum()


def sample_indices(n: int, k: int, seed: int = 11) -> np.ndarray:
    """k distinct particle indices (sorted) drawn uniformly from range(n)."""
    rng = _rng(seed)
    k = min(k, n)
    picked: list = []
    seen: set = set()
    while len(picked) < k:
        for v in np.floor(rng.random(2 * k) * n).astype(np.int64).tolist():
            if v not in seen:
                seen.add(v)
                picked.append(v)
                if len(picked) == k:
                    break
    return np.sort(np.asarray(picked, dtype=np.int64))
