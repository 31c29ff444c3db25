"""Pins of the seeded input recipes (reading R13 and the ensemble recipe).

Each generator is checked against the closed-form distribution it claims
to sample, with Kolmogorov-Smirnov tests at a fixed seed: the Plummer
cumulative mass profile M(<r) = r^3 / (r^2 + a^2)^(3/2) (truncated at
0.999, a = 3 pi / 16), the Plummer speed distribution
g(q) ~ q^2 (1 - q^2)^(7/2) of q = v / v_esc(r), isotropy, the Salpeter
power law, log-uniform cluster sizes; plus the frames and normalisations
the workloads rely on.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from paper_1205_2288_gb300 import inputs

A = 3.0 * math.pi / 16.0
CUT = 0.999


@pytest.fixture(scope="module")
def big():
    return inputs.plummer(20000, 11)


def test_plummer_frame_and_masses(big):
    m, r, v = big
    assert m.shape == (20000,) and np.all(m == 1.0 / 20000)
    np.testing.assert_allclose((m[:, None] * r).sum(0), 0.0, atol=1e-14)
    np.testing.assert_allclose((m[:, None] * v).sum(0), 0.0, atol=1e-14)
    assert r.flags.c_contiguous and v.flags.c_contiguous


def test_plummer_cumulative_mass_profile(big):
    m, r, v = big
    rad = np.linalg.norm(r, axis=1)   # COM shift is O(N^-1/2) of a

    def cdf(x):
        return np.minimum((x ** 3 / (x * x + A * A) ** 1.5) / CUT, 1.0)
    assert stats.kstest(rad, cdf).pvalue > 1e-3


def test_plummer_mass_cut(big):
    """The radial mass fraction is cut at 0.999: no body lies beyond the
    radius enclosing that fraction, and the shell between the radii
    enclosing 0.99 and 0.999 holds its share (0.009 / 0.999) of the bodies,
    which the cumulative profile alone does not resolve at this n."""
    m, r, v = big
    rad = np.linalg.norm(r, axis=1)

    def radius_of(x):                  # inverse of the Plummer mass profile
        return A / math.sqrt(x ** (-2.0 / 3.0) - 1.0)
    # the move to the centre-of-mass frame is O(N^-1/2) of the rms radius
    # (~0.01 here); 0.1 bounds it
    assert rad.max() <= radius_of(CUT) + 0.1
    n = rad.size
    p = (CUT - 0.99) / CUT
    outer = np.sum(rad > radius_of(0.99))
    assert abs(outer - n * p) < 5 * math.sqrt(n * p * (1 - p)) + 2


def test_plummer_speed_distribution_and_isotropy(big):
    m, r, v = big
    rad = np.linalg.norm(r, axis=1) / A           # Plummer units
    speed = np.linalg.norm(v, axis=1) * math.sqrt(A)
    q = speed / (math.sqrt(2.0) * (1.0 + rad * rad) ** -0.25)
    assert q.max() < 1.0 + 1e-6                  # bound (COM shift aside)
    # CDF of g(q) = q^2 (1 - q^2)^(7/2) tabulated on a fine grid
    grid = np.linspace(0.0, 1.0, 20001)
    tab = integrate.cumulative_trapezoid(grid ** 2 * (1 - grid ** 2) ** 3.5,
                                         grid, initial=0.0)
    tab /= tab[-1]
    assert stats.kstest(np.clip(q, 0.0, 1.0),
                        lambda x: np.interp(x, grid, tab)).pvalue > 1e-3
    # isotropy of positions and velocities
    for w in (r, v):
        u = w / np.linalg.norm(w, axis=1)[:, None]
        assert np.abs(u.mean(0)).max() < 0.03
        assert abs((u[:, 2] ** 2).mean() - 1.0 / 3.0) < 0.01


def test_plummer_is_seeded_and_deterministic():
    a = inputs.plummer(100, 4)
    b = inputs.plummer(100, 4)
    c = inputs.plummer(100, 5)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    assert not np.array_equal(a[1], c[1])
    m = inputs.salpeter_masses(100, 3)
    mm, rr, vv = inputs.plummer(100, 4, masses=m)
    np.testing.assert_array_equal(mm, m)
    np.testing.assert_allclose((m[:, None] * rr).sum(0), 0.0, atol=1e-15)


def test_salpeter_power_law():
    alpha, lo, hi = 2.35, 0.1, 10.0
    m = inputs.salpeter_masses(20000, 7)
    assert abs(m.sum() - 1.0) < 1e-12
    # undo the normalisation: the ratio to the smallest mass is scale-free
    raw = m / m.min() * lo
    e = 1.0 - alpha

    def cdf(x):
        x = np.clip(x, lo, hi)
        return (x ** e - lo ** e) / (hi ** e - lo ** e)
    # the smallest sample sits at lo only up to sampling noise; test the
    # shape on the normalised values rescaled by the theoretical mean
    mean_th = (e / (e + 1.0)) * (hi ** (e + 1) - lo ** (e + 1)) / (
        hi ** e - lo ** e)
    x = m * 20000 * mean_th
    assert stats.kstest(x, cdf).pvalue > 1e-3
    assert raw.max() / raw.min() <= hi / lo * (1 + 1e-9)


def test_ensemble_sizes_log_uniform_and_recipe():
    s = inputs.ensemble_sizes(4000, 9)
    assert s.min() >= 64 and s.max() <= 4096
    u = (np.log(s) - math.log(64)) / (math.log(4096) - math.log(64))
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    off, m, r, v, eps = inputs.ensemble(12, seed=2)
    sizes = np.diff(off)
    assert off[0] == 0 and off[-1] == m.shape[0] == r.shape[0]
    np.testing.assert_array_equal(eps, 4.0 / sizes)
    for c in range(12):
        sl = slice(off[c], off[c + 1])
        assert abs(m[sl].sum() - 1.0) < 1e-12
        np.testing.assert_allclose((m[sl, None] * r[sl]).sum(0), 0.0,
                                   atol=1e-14)


def test_active_subset():
    idx = inputs.active_subset(1000, 137, 3)
    assert idx.dtype == np.int32 and idx.shape == (137,)
    assert np.all(np.diff(idx) > 0) and idx.min() >= 0 and idx.max() < 1000
    assert inputs.active_subset(10, 0, 1).shape == (0,)
    np.testing.assert_array_equal(inputs.active_subset(10, 10, 1),
                                  np.arange(10))
    with pytest.raises(ValueError):
        inputs.active_subset(10, 11, 1)
