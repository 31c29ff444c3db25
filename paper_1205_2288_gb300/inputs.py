"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds none of the integrator's arithmetic: it only draws initial
conditions, mass spectra, cluster sizes and active-set subsets from a seeded
numpy PCG64 stream. Both the FP64 CPU oracle and the CUDA library receive the
same arrays from here.

Workloads follow the paper's test problems (Sec. 3, Sec. 6): Plummer spheres
in standard N-body units (G = 1, M = 1, E = -1/4), equal masses, Plummer
softening. The paper's own realisations are not published, so seeded Plummer
models stand in for them.
"""
from __future__ import annotations

import math

import numpy as np

# Plummer scale length that puts a Plummer sphere of total mass 1 at total
# energy -1/4 (standard N-body units): E = -(3 pi / 64) G M^2 / a.
_PLUMMER_SCALE = 3.0 * math.pi / 16.0
# The radial mass fraction is cut here so that no particle lands at infinity.
_MASS_CUT = 0.999


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _isotropic(g: np.random.Generator, n: int) -> np.ndarray:
    """Unit vectors uniform on the sphere, shape (n, 3)."""
    cos_t = g.uniform(-1.0, 1.0, n)
    phi = g.uniform(0.0, 2.0 * math.pi, n)
    sin_t = np.sqrt(1.0 - cos_t * cos_t)
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], axis=1)


def plummer(n: int, seed: int = 0, masses: np.ndarray | None = None):
    """Plummer sphere of n bodies in standard N-body units.

    Sampling follows the published recipe of Aarseth, Henon & Wielen (1974):
    radius from the inverted cumulative mass profile, speed from the
    isotropic distribution function by von Neumann rejection on
    g(q) = q^2 (1 - q^2)^(7/2), isotropic directions. The model is then
    scaled from Plummer units (a = 1) to standard units (a = 3 pi / 16) and
    moved to its centre-of-mass frame. The total energy is -1/4 up to the
    O(N^-1/2) sampling noise; no exact rescaling is applied.

    Returns (m, r, v): float64 arrays of shape (n,), (n, 3), (n, 3), with
    r and v in row-major (x, y, z) order per body.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    g = rng(seed)
    if masses is None:
        m = np.full(n, 1.0 / n)
    else:
        m = np.asarray(masses, dtype=np.float64).copy()
        if m.shape != (n,):
            raise ValueError("masses must have shape (n,)")
    x = g.uniform(0.0, _MASS_CUT, n)
    x = np.maximum(x, 1e-10)
    radius = 1.0 / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
    r = radius[:, None] * _isotropic(g, n)
    q = np.empty(n)
    filled = 0
    while filled < n:
        want = n - filled
        xs = g.uniform(0.0, 1.0, 2 * want + 16)
        ys = g.uniform(0.0, 0.1, 2 * want + 16)
        ok = ys < xs * xs * (1.0 - xs * xs) ** 3.5
        take = xs[ok][:want]
        q[filled:filled + take.size] = take
        filled += take.size
    v_esc = math.sqrt(2.0) * (1.0 + radius * radius) ** -0.25
    v = (q * v_esc)[:, None] * _isotropic(g, n)
    r *= _PLUMMER_SCALE
    v *= 1.0 / math.sqrt(_PLUMMER_SCALE)
    mt = m.sum()
    r -= (m[:, None] * r).sum(axis=0) / mt
    v -= (m[:, None] * v).sum(axis=0) / mt
    return m, np.ascontiguousarray(r), np.ascontiguousarray(v)


def salpeter_masses(n: int, seed: int, alpha: float = 2.35,
                    m_lo: float = 0.1, m_hi: float = 10.0) -> np.ndarray:
    """n masses from dN/dm ~ m^-alpha on [m_lo, m_hi] by inverse CDF,
    normalised to total mass 1."""
    g = rng(seed)
    u = g.uniform(0.0, 1.0, n)
    e = 1.0 - alpha
    lo, hi = m_lo ** e, m_hi ** e
    mass = (lo + u * (hi - lo)) ** (1.0 / e)
    return mass / mass.sum()


def ensemble_sizes(n_clusters: int, seed: int, n_lo: int = 64,
                   n_hi: int = 4096) -> np.ndarray:
    """Cluster sizes drawn log-uniform in [n_lo, n_hi], rounded."""
    g = rng(seed)
    s = np.exp(g.uniform(math.log(n_lo), math.log(n_hi), n_clusters))
    return np.clip(np.rint(s).astype(np.int64), n_lo, n_hi)


def ensemble(n_clusters: int = 512, seed: int = 0):
    """Independent Plummer clusters with Salpeter masses and eps_c = 4 / N_c.

    Returns (offsets[n_clusters + 1], m, r, v, eps[n_clusters]); cluster c
    owns bodies offsets[c] .. offsets[c + 1] - 1.
    """
    sizes = ensemble_sizes(n_clusters, seed)
    offsets = np.zeros(n_clusters + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    ms, rs, vs = [], [], []
    for c, nc in enumerate(sizes):
        mc = salpeter_masses(int(nc), seed=1_000_003 * (seed + 1) + 2 * c)
        m, r, v = plummer(int(nc), seed=1_000_003 * (seed + 1) + 2 * c + 1,
                          masses=mc)
        ms.append(m)
        rs.append(r)
        vs.append(v)
    eps = 4.0 / sizes.astype(np.float64)
    return (offsets, np.concatenate(ms), np.concatenate(rs),
            np.concatenate(vs), eps)


def active_subset(n: int, n_act: int, seed: int) -> np.ndarray:
    """Ascending int32 indices of a uniform random subset of size n_act."""
    if not 0 <= n_act <= n:
        raise ValueError("n_act out of range")
    g = rng(seed)
    idx = g.choice(n, size=n_act, replace=False)
    return np.sort(idx).astype(np.int32)
