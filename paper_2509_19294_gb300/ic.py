"""Seeded synthetic initial conditions (numpy FP64).

This module is the one piece shared by the oracle tests and the CUDA tests and
benchmark.  It only draws inputs; it holds none of the force, integration or
diagnostic arithmetic.

The paper runs its own initial conditions, which it does not publish (Sec. 4:
102 400 particles over ten time cycles), so every workload here is synthetic:

* ``plummer``            -- Plummer sphere by the Aarseth-Henon-Wielen (1974)
  recipe, in Henon units (G = M = 1, E = -1/4), truncated at 10 Plummer radii,
  equal masses, centre-of-mass frame.
* ``uniform_sphere``     -- uniform-density ball of radius R, at rest.
* ``log_uniform_masses`` -- masses log-uniform on [lo, hi], normalised to total 1.
* ``two_plummer``        -- two Plummer spheres on a head-on approach.
* ``ensemble``           -- independent Plummer clusters of uneven size.

All generators take a seed and use numpy's PCG64; the same seed gives the
same arrays on every machine.  Arrays are returned in the C-ABI layout:
``pos``/``vel`` as ``[3, n]`` float64, ``mass`` as ``[n]`` float64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

HENON_R = 3.0 * math.pi / 16.0          # Plummer scale length in Henon units
HENON_V = math.sqrt(16.0 / (3.0 * math.pi))


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _isotropic(rng, n):
    """n unit vectors, uniform on the sphere, shape [3, n]."""
    cos_t = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t])


def plummer(n: int, seed: int, rmax: float = 10.0, masses=None, centre=True):
    """Plummer sphere, Aarseth-Henon-Wielen sampling, Henon units.

    Radius from the inverted cumulative mass, r = (X^(-2/3) - 1)^(-1/2) in
    Plummer units, redrawn while r > ``rmax``; the speed is q * v_esc with q
    drawn by rejection from g(q) = q^2 (1 - q^2)^(7/2) (bounded by 0.1); the
    directions are isotropic.  Returns (pos, vel, mass).
    """
    rng = _rng(seed)
    r = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        x = rng.uniform(0.0, 1.0, todo.size)
        with np.errstate(divide="ignore", invalid="ignore"):
            rr = 1.0 / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
        ok = np.isfinite(rr) & (rr <= rmax) & (x > 0.0)
        r[todo[ok]] = rr[ok]
        todo = todo[~ok]
    pos = _isotropic(rng, n) * r
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        x4 = rng.uniform(0.0, 1.0, todo.size)
        x5 = rng.uniform(0.0, 1.0, todo.size)
        ok = 0.1 * x5 < x4 * x4 * (1.0 - x4 * x4) ** 3.5
        q[todo[ok]] = x4[ok]
        todo = todo[~ok]
    vesc = math.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    vel = _isotropic(rng, n) * (q * vesc)
    pos *= HENON_R
    vel *= HENON_V
    if masses is None:
        mass = np.full(n, 1.0 / n)
    else:
        mass = np.asarray(masses, dtype=np.float64)
    if centre:
        mt = mass.sum()
        pos -= (pos * mass).sum(axis=1, keepdims=True) / mt
        vel -= (vel * mass).sum(axis=1, keepdims=True) / mt
    return np.ascontiguousarray(pos), np.ascontiguousarray(vel), mass


def log_uniform_masses(n: int, seed: int, lo: float = 0.1, hi: float = 10.0):
    """Masses exp(U(ln lo, ln hi)), normalised to a total of 1."""
    rng = _rng(seed)
    m = np.exp(rng.uniform(math.log(lo), math.log(hi), n))
    return m / m.sum()


def uniform_sphere(n: int, seed: int, radius: float = 1.0, masses=None):
    """Uniform-density ball: r = R U^(1/3), isotropic direction, at rest."""
    rng = _rng(seed)
    r = radius * rng.uniform(0.0, 1.0, n) ** (1.0 / 3.0)
    pos = _isotropic(rng, n) * r
    vel = np.zeros((3, n))
    mass = np.full(n, 1.0 / n) if masses is None else np.asarray(masses, np.float64)
    return np.ascontiguousarray(pos), vel, mass


def two_plummer(n_each: int, seed: int, separation: float = 10.0, v_rel: float = 0.5):
    """Two Plummer spheres of ``n_each`` particles on a head-on approach.

    Each sphere is a unit Henon Plummer model scaled to mass 1/2 (velocities by
    sqrt(1/2), which keeps it in virial equilibrium).  The centres sit at
    x = -separation/2 and +separation/2 and move towards each other with
    relative speed ``v_rel``; the pair is in its centre-of-mass frame.
    """
    pa, va, ma = plummer(n_each, seed * 1000 + 1)
    pb, vb, mb = plummer(n_each, seed * 1000 + 2)
    s = math.sqrt(0.5)
    pa[0] -= 0.5 * separation
    pb[0] += 0.5 * separation
    va *= s
    vb *= s
    va[0] += 0.5 * v_rel
    vb[0] -= 0.5 * v_rel
    pos = np.ascontiguousarray(np.concatenate([pa, pb], axis=1))
    vel = np.ascontiguousarray(np.concatenate([va, vb], axis=1))
    mass = np.concatenate([ma, mb]) * 0.5
    return pos, vel, mass


@dataclass
class Ensemble:
    pos: np.ndarray          # [3, n_total]
    vel: np.ndarray          # [3, n_total]
    mass: np.ndarray         # [n_total]
    offsets: np.ndarray      # [n_clusters + 1] int64
    eps: np.ndarray          # [n_clusters] float64

    @property
    def sizes(self):
        return np.diff(self.offsets)


def ensemble(n_clusters: int, seed: int, n_min: int = 256, n_max: int = 8192,
             eps_coeff: float = 0.01) -> Ensemble:
    """Independent unit Henon Plummer clusters, N_c ~ U{n_min..n_max}.

    Cluster c has softening eps_c = eps_coeff * N_c^(-1/3).  Clusters do not
    interact; each is centred at the origin in its own frame.
    """
    rng = _rng(seed)
    sizes = rng.integers(n_min, n_max + 1, n_clusters)
    offsets = np.zeros(n_clusters + 1, np.int64)
    offsets[1:] = np.cumsum(sizes)
    ps, vs, ms = [], [], []
    for c, nc in enumerate(sizes):
        p, v, m = plummer(int(nc), seed * 100003 + c)
        ps.append(p)
        vs.append(v)
        ms.append(m)
    eps = eps_coeff * sizes.astype(np.float64) ** (-1.0 / 3.0)
    return Ensemble(np.ascontiguousarray(np.concatenate(ps, axis=1)),
                    np.ascontiguousarray(np.concatenate(vs, axis=1)),
                    np.concatenate(ms), offsets, eps)


def sample_rows(n: int, k: int, seed: int):
    """k distinct row indices in [0, n), sorted, always including 0 and n-1."""
    rng = _rng(seed)
    k = min(k, n)
    rows = rng.choice(n, size=k, replace=False)
    rows[0] = 0
    if k > 1:
        rows[1] = n - 1
    return np.unique(rows).astype(np.int64)
