"""Pins of the oracle's pairwise force, potential and step criterion
(Sec. 2 Eq. 3 with Plummer softening, Sec. 3) against closed forms,
symmetry and Newton's third law."""
import math

import numpy as np
import pytest

from paper_1205_2288_gb300 import inputs


def test_two_body_closed_form(orc):
    # body 0 at origin, body 1 at (x, y, z); eps > 0
    m = np.array([0.3, 0.7])
    d = np.array([0.3, -0.4, 1.2])
    r = np.stack([np.zeros(3), d])
    v = np.array([[0.1, 0.2, -0.3], [-0.5, 0.4, 0.6]])
    eps = 0.25
    a, phi, q = orc.forces(m, r, v, eps)
    s2 = d @ d + eps ** 2
    s = math.sqrt(s2)
    # a_0 points at body 1 with magnitude m_1 |d| / s^3
    np.testing.assert_allclose(a[0], m[1] * d / s ** 3, rtol=1e-14)
    np.testing.assert_allclose(a[1], -m[0] * d / s ** 3, rtol=1e-14)
    np.testing.assert_allclose(phi, [-m[1] / s, -m[0] / s], rtol=1e-14)
    w = v[1] - v[0]
    coll = (w @ w) / s2           # (|v_ij| / s)^2
    ff = [m[1] / s ** 3, m[0] / s ** 3]   # (|r_ij| / |a_ij|)^-1
    np.testing.assert_allclose(q, [max(coll, ff[0]), max(coll, ff[1])],
                               rtol=1e-14)


def test_time_step_estimate_matches_eq3(orc):
    # Eq. 3 read with the softened distance: eta * min(s/|v|, sqrt(s^3/m))
    m = np.array([1.0, 1e-3])
    d = np.array([2.0, 0.0, 0.0])
    r = np.stack([np.zeros(3), d])
    for speed in (0.0, 0.01, 3.0):
        v = np.array([[0.0, 0, 0], [0, speed, 0]])
        eps = 0.1
        _, _, q = orc.forces(m, r, v, eps)
        s = math.sqrt(4.0 + eps ** 2)
        coll = s / speed if speed > 0 else math.inf
        free_fall = math.sqrt(s ** 3 / m[1])
        eta = 0.02
        assert eta / math.sqrt(q[0]) == pytest.approx(
            eta * min(coll, free_fall), rel=1e-14)


def _cube(edge):
    h = edge / 2
    return np.array([[sx * h, sy * h, sz * h] for sx in (-1, 1)
                     for sy in (-1, 1) for sz in (-1, 1)])


@pytest.mark.parametrize("eps", [0.0, 0.05, 0.7])
def test_cube_vertices_closed_form(orc, eps):
    edge, mass = 0.8, 0.125
    r = _cube(edge)
    m = np.full(8, mass)
    v = np.zeros((8, 3))
    a, phi, q = orc.forces(m, r, v, eps)
    # neighbours: 3 at edge, 3 at edge*sqrt2, 1 at edge*sqrt3
    e2 = edge ** 2
    s1, s2, s3 = (math.sqrt(e2 + eps ** 2), math.sqrt(2 * e2 + eps ** 2),
                  math.sqrt(3 * e2 + eps ** 2))
    comp = mass * edge * (1 / s1 ** 3 + 2 / s2 ** 3 + 1 / s3 ** 3)
    # each component points back toward the centre
    np.testing.assert_allclose(a, -np.sign(r) * comp, rtol=1e-13)
    np.testing.assert_allclose(phi, -mass * (3 / s1 + 3 / s2 + 1 / s3),
                               rtol=1e-13)
    np.testing.assert_allclose(q, mass / s1 ** 3, rtol=1e-13)


def test_centre_of_symmetric_shell(orc):
    # a test body at the centre of the cube feels no force; its potential
    # is -M / sqrt(R^2 + eps^2)
    r = np.vstack([_cube(1.0), np.zeros(3)])
    m = np.concatenate([np.full(8, 0.1), [0.5]])
    v = np.zeros((9, 3))
    eps = 0.03
    a, phi, q = orc.forces(m, r, v, eps, idx=np.array([8], np.int32))
    R2 = 3 * 0.25
    assert np.abs(a).max() < 1e-15
    assert phi[0] == pytest.approx(-0.8 / math.sqrt(R2 + eps ** 2), rel=1e-14)
    assert q[0] == pytest.approx(0.1 / (R2 + eps ** 2) ** 1.5, rel=1e-14)


def test_far_field_monopole(orc):
    # a distant test body sees the cluster as a point mass M
    m, r, v = inputs.plummer(512, seed=3)
    D = np.array([3000.0, -4000.0, 12000.0])
    r2 = np.vstack([r, D])
    m2 = np.concatenate([m, [0.0]])
    v2 = np.vstack([v, np.zeros(3)])
    a, phi, _ = orc.forces(m2, r2, v2, 0.0, idx=np.array([512], np.int32))
    dist = np.linalg.norm(D)
    # dipole vanishes (centre-of-mass frame): relative error O((R/D)^2)
    np.testing.assert_allclose(a[0], -D / dist ** 3, rtol=1e-5)
    assert phi[0] == pytest.approx(-1.0 / dist, rel=1e-5)


@pytest.mark.parametrize("eps", [0.0, 0.01])
def test_newton_third_law(orc, eps):
    m, r, v = inputs.plummer(400, seed=5)
    m = m * np.linspace(0.5, 1.5, 400)
    a, phi, _ = orc.forces(m, r, v, eps)
    net = (m[:, None] * a).sum(axis=0)
    scale = (m[:, None] * np.abs(a)).sum()
    assert np.abs(net).max() < 1e-14 * scale
    # potential energy from phi equals the pair sum of energy_of
    _, ep = orc.energy_of(m, r, v, eps)
    assert 0.5 * float(m @ phi) == pytest.approx(ep, rel=1e-13)


def test_self_term_skipped_with_zero_softening(orc):
    m, r, v = inputs.plummer(64, seed=1)
    a, phi, q = orc.forces(m, r, v, 0.0)
    assert np.isfinite(a).all() and np.isfinite(phi).all()
    assert np.isfinite(q).all()


def test_active_subset_matches_full(orc):
    m, r, v = inputs.plummer(300, seed=2)
    a, phi, q = orc.forces(m, r, v, 0.01)
    idx = inputs.active_subset(300, 37, seed=9)
    a2, phi2, q2 = orc.forces(m, r, v, 0.01, idx=idx)
    np.testing.assert_array_equal(a2, a[idx])
    np.testing.assert_array_equal(phi2, phi[idx])
    np.testing.assert_array_equal(q2, q[idx])


def test_energy_two_body_and_plummer(orc):
    m = np.array([0.25, 0.75])
    r = np.array([[0.0, 0, 0], [0.6, 0.8, 0]])
    v = np.array([[0.0, 1.0, 0], [2.0, 0, 0]])
    ek, ep = orc.energy_of(m, r, v, 0.0)
    assert ek == pytest.approx(0.5 * 0.25 * 1.0 + 0.5 * 0.75 * 4.0, rel=1e-15)
    assert ep == pytest.approx(-0.25 * 0.75 / 1.0, rel=1e-15)
    # standard units: K = 1/4, W = -1/2 up to O(N^-1/2) sampling noise
    n = 4096
    ks, ws = [], []
    for seed in range(4):
        m, r, v = inputs.plummer(n, seed)
        ek, ep = orc.energy_of(m, r, v, 0.0)
        ks.append(ek)
        ws.append(ep)
    assert abs(np.mean(ks) - 0.25) < 2.0 / math.sqrt(n)
    assert abs(np.mean(ws) + 0.5) < 2.0 / math.sqrt(n)
    assert abs(np.mean(2 * np.array(ks) / np.abs(ws)) - 1) < 4.0 / math.sqrt(n)


@pytest.mark.parametrize("eps", [0.0, 0.05])
def test_brute_force_in_forty_digits(orc, eps):
    """The FP64 sums against the same sums in 40-digit arithmetic on the
    exact values of the inputs (N = 48, unequal masses): a_i within 1e-14
    of the scale of its terms, phi_i and q_i within 1e-14 relative."""
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 40
    n = 48
    m = inputs.salpeter_masses(n, 5)
    _, r, v = inputs.plummer(n, 6, masses=m)
    a, phi, q = orc.forces(m, r, v, eps)
    M = [mp.mpf(float(x)) for x in m]
    R = [[mp.mpf(float(x)) for x in row] for row in r]
    V = [[mp.mpf(float(x)) for x in row] for row in v]
    e2 = mp.mpf(eps) ** 2
    for i in range(n):
        ax, ph, qq, scale = [mp.mpf(0)] * 3, mp.mpf(0), mp.mpf(0), mp.mpf(0)
        for j in range(n):
            if j == i:
                continue
            d = [R[j][c] - R[i][c] for c in range(3)]
            w = [V[j][c] - V[i][c] for c in range(3)]
            s2 = d[0] ** 2 + d[1] ** 2 + d[2] ** 2 + e2
            s = mp.sqrt(s2)
            f = M[j] / (s2 * s)
            ax = [ax[c] + f * d[c] for c in range(3)]
            ph -= M[j] / s
            qq = max(qq, (w[0] ** 2 + w[1] ** 2 + w[2] ** 2) / s2, f)
            scale += M[j] / s2
        for c in range(3):
            assert abs(a[i, c] - float(ax[c])) <= 1e-14 * float(scale)
        assert abs(phi[i] - float(ph)) <= 1e-14 * abs(float(ph))
        assert abs(q[i] - float(qq)) <= 1e-14 * float(qq)
