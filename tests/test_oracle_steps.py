"""Pins of the oracle's block-level rule (Eq. 4), first-pass step choice,
the symmetrisation scheme (Alg. 1 and its prose) and the time-symmetric
interpolation, on hand-worked cases.

Ticks: k_max = 10 gives 1024 ticks per time unit; k_min = 3 caps steps at
2^-3 = 128 ticks."""
import numpy as np
import pytest

KMIN, KMAX = 3, 10


@pytest.mark.parametrize("x,ticks,uf", [
    (1.0, 128, 0),          # capped at dt_max = 2^-3
    (0.125, 128, 0),        # exact power of two is its own level
    (0.1249, 64, 0),        # just below -> next level down
    (0.0625, 64, 0),
    (0.0624999, 32, 0),
    (3.0 / 1024, 2, 0),     # 2^-9 <= 0.00293 < 2^-8
    (2.0 ** -10, 1, 0),
    (0.999 * 2.0 ** -10, 1, 1),   # below dt_min: clamped and counted
    (float("inf"), 128, 0),
    (0.0, 1, 1),
])
def test_level(orc, x, ticks, uf):
    assert orc.level_ticks(x, KMIN, KMAX) == (ticks, uf)


@pytest.mark.parametrize("tau,d,dts,want", [
    (0, 8, 1.0, 16),        # growth limited to 2 d
    (24, 8, 1.0, 8),        # 24 is not a multiple of 16: stay commensurate
    (24, 8, 3.0 / 1024, 2),  # unlimited decrease in the first pass
    (4, 4, 1.0, 4),
    (0, 128, 1.0, 128),     # already at dt_max
    (96, 32, 0.05, 32),     # L(0.05) = 2^-5 = 32 ticks
])
def test_forward_step(orc, tau, d, dts, want):
    assert orc.forward_step(tau, d, dts, KMIN, KMAX)[0] == want


# (tau, d, dts, dte(tau + 2d), dte(tau + d), expected), worked from Alg. 1:
# even time -> try 2d, then d, else d/2; odd time -> try d, else d/2;
# a candidate c passes when c <= level((dts + dte(tau + c)) / 2).
SYM_CASES = [
    # even (32 % 32 == 0): avg(0.05, 0.04) = 0.045 -> 32 ticks >= 2d
    (32, 16, 0.05, 0.04, 0.05, 32),
    # even: avg(0.05, 0.01) = 0.03 -> 16 < 32; keep: avg(0.05, 0.03) -> 32
    (32, 16, 0.05, 0.01, 0.03, 16),
    # even: level(0.012) = 8 ticks rejects 32 and 16 -> halve
    (32, 16, 0.012, 0.012, 0.012, 8),
    # odd (48 % 64 != 0): no doubling even though it would pass
    (48, 32, 1.0, 1.0, 1.0, 32),
    # odd, keeping fails -> halve
    (48, 16, 0.01, 1.0, 0.01, 8),
    # even at dt_max: 2d exceeds dt_max and is not tried
    (256, 128, 1.0, 1.0, 1.0, 128),
    # the criterion averages start and end: a tiny end estimate alone
    # does not veto doubling when the mean still allows it
    (0, 16, 0.1, 0.001, 0.02, 32),
    # ... but a tiny start estimate with a tiny end estimate does
    (0, 16, 0.001, 0.001, 0.001, 8),
    # halving is untested: from 16 to 8 even though 8 also fails
    (0, 16, 0.0001, 0.0001, 0.0001, 8),
]


@pytest.mark.parametrize("tau,d,dts,e2,e1,want", SYM_CASES)
def test_symmetric_step(orc, tau, d, dts, e2, e1, want):
    got, uf = orc.symmetric_step(tau, d, dts, e2, e1, KMIN, KMAX)
    assert got == want
    assert uf == 0


def test_symmetric_step_changes_at_most_2x_and_stays_commensurate(orc):
    g = np.random.default_rng(7)
    for _ in range(2000):
        lvl = int(g.integers(0, 8))
        d = 1 << lvl
        tau = d * int(g.integers(0, 64))
        dts, e2, e1 = 10.0 ** g.uniform(-4, 0, 3)
        c, _ = orc.symmetric_step(tau, d, dts, e2, e1, KMIN, KMAX)
        assert c in (max(d // 2, 1), d, 2 * d)
        assert tau % c == 0
        assert c <= 128
        if c == 2 * d:
            assert tau % (2 * d) == 0   # doubling only at even times


def _cubic(t, coef):
    c0, c1, c2, c3 = coef
    r = c0 + c1 * t + c2 * t ** 2 + c3 * t ** 3
    v = c1 + 2 * c2 * t + 3 * c3 * t ** 2
    a = 2 * c2 + 6 * c3 * t
    return r, v, a


def test_hermite_reproduces_cubics(orc):
    g = np.random.default_rng(3)
    coef = [g.normal(size=3) for _ in range(4)]
    ta, tb = 1000, 1064
    T = lambda k: k / 2.0 ** KMAX
    ra, va, aa = _cubic(T(ta), coef)
    rb, vb, ab = _cubic(T(tb), coef)
    for t in (1000, 1001, 1017, 1032, 1050, 1063, 1064):
        r, v = orc.hermite(ta, tb, t, KMAX, ra, va, aa, rb, vb, ab)
        rt, vt, _ = _cubic(T(t), coef)
        np.testing.assert_allclose(r, rt, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(v, vt, rtol=1e-12, atol=1e-12)
    r, v = orc.hermite(ta, tb, ta, KMAX, ra, va, aa, rb, vb, ab)
    np.testing.assert_array_equal(r, ra)
    np.testing.assert_array_equal(v, va)


def test_hermite_is_time_symmetric(orc):
    g = np.random.default_rng(4)
    ra, va, aa, rb, vb, ab = (g.normal(size=3) for _ in range(6))
    for t in (3, 7, 11):
        r1, v1 = orc.hermite(0, 16, t, KMAX, ra, va, aa, rb, vb, ab)
        # the same interval walked backwards: ends swapped, h negated
        r2, v2 = orc.hermite(16, 0, t, KMAX, rb, vb, ab, ra, va, aa)
        np.testing.assert_allclose(r1, r2, rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(v1, v2, rtol=1e-14, atol=1e-15)


def test_hermite_error_is_fourth_order(orc):
    # on r = sin(t) the interpolation error falls ~16x per halving of h
    errs = []
    for span in (64, 32, 16):
        ta, tb = 300, 300 + span
        T = lambda k: k / 2.0 ** KMAX * 8
        h_fac = 8.0   # stretch time so that sin is well resolved
        def state(k):
            t = T(k)
            return (np.array([np.sin(t)] * 3), np.array([np.cos(t)] * 3) * h_fac,
                    -np.array([np.sin(t)] * 3) * h_fac ** 2)
        ra, va, aa = state(ta)
        rb, vb, ab = state(tb)
        r, _ = orc.hermite(ta, tb, ta + span // 2, KMAX, ra, va, aa, rb, vb, ab)
        errs.append(abs(r[0] - np.sin(T(ta + span // 2))))
    assert 12 < errs[0] / errs[1] < 20
    assert 12 < errs[1] / errs[2] < 20
