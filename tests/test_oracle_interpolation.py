"""Pin of the oracle's time-symmetric interpolation in passes >= 1 (Sec. 2:
in the iterations of an era, a body that is not active is placed at the
block time from the data the previous pass stored, not by Eq. 2 from its
own step start; reading R6 takes the cubic Hermite interpolant between the
previous pass's two records that bracket the block time).

What fixes the expected values is the mathematics of that interpolant, not
the oracle: on one step [t_a, t_b] of a slow body, the predicted positions
at the many fast block times inside it lie on one cubic in time whose value
and slope at t_b are the previous pass's end record r_b, v_b (and r_a, v_a
at t_a); the predicted velocities lie on one cubic with value v_b and slope
a_b at t_b. Eq. 2 from the step start makes the velocity linear, ending at
v_a + a_a h instead of v_b, so a pass that does not interpolate fails here
(the mutation check plants exactly that mistake).

The system is a tight, eccentric equal-mass binary with a lighter body
outside it: the binary takes steps of ~2^-18 that change along its orbit
(so the passes of an era differ), the outer body steps of 2^-9, so each
outer step holds hundreds of fast block times.
"""
import numpy as np

import oracle

K_MAX = 20


def two_level_system():
    m = np.array([0.5, 0.5, 0.1])
    d = 0.01
    # 0.4 of the circular speed (G = 1): an eccentric binary
    v_orb = 0.4 * np.sqrt(0.5 * (d / 2) / d ** 2)
    r = np.array([[-d / 2, 0.0, 0.0], [d / 2, 0.0, 0.0], [0.3, 0.2, 0.1]])
    v = np.array([[0.0, -v_orb, 0.0], [0.0, v_orb, 0.0], [0.05, 0.9, -0.1]])
    return m, r, v


def run_traced(n_iter=3):
    m, r, v = two_level_system()
    s = oracle.Sim(m, r, v, eps=1e-4, eta=0.02, dt_max=1 / 8, n_iter=n_iter,
                   era_mode=0, era_log2=3, k_max=K_MAX, trace_body=2)
    start = s.state()
    s.run(0.125)
    tr = s.trace()
    s.close()
    return start, tr


def first_step(tr, pass_):
    """The outer body's first step of one pass: its end record (t_b, r, v,
    a) and the predictions (t, r, v) at the block times before it."""
    sel = tr["pass_"] == pass_
    kind, tau = tr["kind"][sel], tr["tau"][sel]
    k_end = int(np.flatnonzero(kind == 1)[0])
    end = (int(tau[k_end]), tr["r"][sel][k_end], tr["v"][sel][k_end],
           tr["a"][sel][k_end])
    inside = np.arange(k_end)
    return end, (tau[inside], tr["r"][sel][inside], tr["v"][sel][inside])


def cubic_fit(x, y):
    """Least-squares cubic in x (per column); returns the polynomial
    coefficients, highest degree first."""
    return [np.polyfit(x, y[:, c], 3) for c in range(y.shape[1])]


def val(cs, x):
    return np.array([np.polyval(c, x) for c in cs])


def slope(cs, x):
    return np.array([np.polyval(np.polyder(c), x) for c in cs])


def test_pass_one_predictions_are_the_hermite_cubic_of_pass_zero_records():
    start, tr = run_traced()
    ra, va, aa = start["r"][2], start["v"][2], start["a"][2]
    (tb, rb, vb, ab), _ = first_step(tr, 0)
    # pass 1: predictions inside pass 0's first outer step (0, t_b)
    sel = (tr["pass_"] == 1) & (tr["kind"] == 0) & (tr["tau"] < tb)
    t, rp, vp = tr["tau"][sel], tr["r"][sel], tr["v"][sel]
    assert len(t) >= 100
    h = tb * 2.0 ** -K_MAX
    x = t / tb
    cr, cv = cubic_fit(x, rp), cubic_fit(x, vp)
    # the fit is exact: the predictions are one cubic to rounding
    scale_r = np.abs(rp).max()
    assert np.abs(np.array([np.polyval(c, x) for c in cr]).T - rp).max() \
        < 1e-13 * scale_r
    # its ends are the previous pass's records (value and slope)
    np.testing.assert_allclose(val(cr, 0.0), ra, rtol=0, atol=1e-12)
    np.testing.assert_allclose(val(cr, 1.0), rb, rtol=0, atol=1e-12)
    np.testing.assert_allclose(slope(cr, 0.0) / h, va, rtol=0, atol=1e-9)
    np.testing.assert_allclose(slope(cr, 1.0) / h, vb, rtol=0, atol=1e-9)
    np.testing.assert_allclose(val(cv, 0.0), va, rtol=0, atol=1e-12)
    np.testing.assert_allclose(val(cv, 1.0), vb, rtol=0, atol=1e-12)
    np.testing.assert_allclose(slope(cv, 0.0) / h, aa, rtol=0, atol=1e-8)
    np.testing.assert_allclose(slope(cv, 1.0) / h, ab, rtol=0, atol=1e-8)
    # Eq. 2 from the step start would end elsewhere: the pin distinguishes
    assert np.abs((va + aa * h) - vb).max() > 1e3 * 1e-12


def test_each_outer_step_uses_its_own_bracketing_records():
    """Inside every one of the outer body's pass-0 steps [t_k, t_k+1], the
    pass-1 predictions are the cubic through records k and k + 1 (not a
    neighbouring pair)."""
    start, tr = run_traced()
    sel0 = (tr["pass_"] == 0) & (tr["kind"] == 1)
    t_rec = np.concatenate([[0], tr["tau"][sel0]])
    r_rec = np.vstack([start["r"][2], tr["r"][sel0]])
    v_rec = np.vstack([start["v"][2], tr["v"][sel0]])
    assert len(t_rec) >= 4
    for k in range(3):
        ta, tb = t_rec[k], t_rec[k + 1]
        sel = ((tr["pass_"] == 1) & (tr["kind"] == 0) & (tr["tau"] > ta)
               & (tr["tau"] < tb))
        t, rp, vp = tr["tau"][sel], tr["r"][sel], tr["v"][sel]
        assert len(t) >= 20
        x = (t - ta) / (tb - ta)
        cr, cv = cubic_fit(x, rp), cubic_fit(x, vp)
        for c, y in ((cr, r_rec), (cv, v_rec)):
            np.testing.assert_allclose(val(c, 0.0), y[k], rtol=0, atol=1e-12)
            np.testing.assert_allclose(val(c, 1.0), y[k + 1], rtol=0,
                                       atol=1e-12)


def test_body_without_bracketing_records_uses_eq2():
    """A slow far body whose step (dt_max = 1/8) overshoots the era (1/16)
    waits behind the era end: its previous-pass data is the era-start
    record alone, so in every pass it is placed by Eq. 2 from its own state
    (a quadratic in time), not held at the record."""
    m, r, v = two_level_system()
    m = np.append(m, 1e-3)
    r = np.vstack([r, [40.0, -10.0, 5.0]])
    v = np.vstack([v, [0.0, 0.02, 0.01]])
    s = oracle.Sim(m, r, v, eps=1e-4, eta=0.02, dt_max=1 / 8, n_iter=3,
                   era_mode=0, era_log2=4, k_max=K_MAX, trace_body=3)
    st = s.state()
    assert st["dt"][3] == 2 ** (K_MAX - 3)
    s.run(1 / 16)
    tr = s.trace()
    s.close()
    assert (tr["kind"] == 0).all() and set(tr["pass_"]) == {0, 1, 2}
    h = tr["tau"] * 2.0 ** -K_MAX
    ra, va, aa = st["r"][3], st["v"][3], st["a"][3]
    want_r = ra + va * h[:, None] + 0.5 * aa * h[:, None] ** 2
    np.testing.assert_allclose(tr["r"], want_r, rtol=0, atol=1e-14)
    np.testing.assert_allclose(tr["v"], va + aa * h[:, None], rtol=0,
                               atol=1e-14)


def test_later_passes_interpolate_the_pass_before_them():
    """Pass 2 interpolates pass 1's records, not pass 0's: its predictions
    inside pass 1's first outer step end on pass 1's record."""
    start, tr = run_traced(n_iter=3)
    (tb1, rb1, vb1, _), _ = first_step(tr, 1)
    (tb0, rb0, vb0, _), _ = first_step(tr, 0)
    sel = (tr["pass_"] == 2) & (tr["kind"] == 0) & (tr["tau"] < tb1)
    t, rp, vp = tr["tau"][sel], tr["r"][sel], tr["v"][sel]
    assert len(t) >= 100
    x = t / tb1
    cr, cv = cubic_fit(x, rp), cubic_fit(x, vp)
    np.testing.assert_allclose(val(cr, 1.0), rb1, rtol=0, atol=1e-13)
    np.testing.assert_allclose(val(cv, 1.0), vb1, rtol=0, atol=1e-13)
    # pass 1's record differs from pass 0's at the same time, by far more
    # than the fit's rounding: matching pass 1 is a real distinction
    assert tb1 == tb0
    assert np.abs(vb1 - vb0).max() > 1e-11


def test_first_pass_uses_eq2_from_the_step_start():
    """Pass 0 has no stored data: its predictions are Eq. 2 from the step
    start, a quadratic in position and a line in velocity."""
    start, tr = run_traced()
    ra, va, aa = start["r"][2], start["v"][2], start["a"][2]
    (tb, _, _, _), (t, rp, vp) = first_step(tr, 0)
    h = t * 2.0 ** -K_MAX
    want_r = ra + va * h[:, None] + 0.5 * aa * h[:, None] ** 2
    want_v = va + aa * h[:, None]
    np.testing.assert_allclose(rp, want_r, rtol=0, atol=1e-14)
    np.testing.assert_allclose(vp, want_v, rtol=0, atol=1e-14)
