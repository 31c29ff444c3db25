"""Pins of the oracle's use of the previous pass's records (readings R6, R8).

R6: a body that is not active in a pass >= 1 is predicted from its
previous-pass records — the record itself at an exact hit, the cubic
Hermite between the two records that bracket the block time, Eq. 2 from
its own state where the records do not bracket it. R8: the previous pass's
step estimate between two records is linear in time, the fallback outside.

Pinned by brute force on small record sets, by values exact in binary, and
by a cubic trajectory: Hermite interpolation reproduces a cubic exactly, so
only the correct bracketing pair gives the exact position and velocity.
"""
import numpy as np
import pytest

import oracle

K_MAX = 20


def test_hist_find_is_the_last_record_at_or_before_t():
    rng = np.random.default_rng(1)
    for _ in range(50):
        tau = np.unique(rng.integers(0, 200, size=rng.integers(1, 12)))
        for t in range(-2, 205, 3):
            want = max((k for k in range(len(tau)) if tau[k] <= t), default=-1)
            assert oracle.hist_find(tau, t) == want


def test_step_estimate_between_records_is_linear_in_time():
    tau = np.array([0, 4, 8], np.int64)
    dts = np.array([1.0, 2.0, 3.0])
    for t, want in ((0, 1.0), (1, 1.25), (2, 1.5), (4, 2.0), (6, 2.5),
                    (8, 3.0)):
        assert oracle.hist_dts_at(tau, dts, t, -7.0) == want
    # non-uniform spacing, decreasing estimate
    tau = np.array([0, 2, 10], np.int64)
    dts = np.array([4.0, 8.0, 0.0])
    assert oracle.hist_dts_at(tau, dts, 6, -7.0) == 4.0
    assert oracle.hist_dts_at(tau, dts, 3, -7.0) == 7.0


def test_step_estimate_outside_the_records_is_the_fallback():
    tau = np.array([4, 8], np.int64)
    dts = np.array([1.0, 3.0])
    assert oracle.hist_dts_at(tau, dts, 3, -7.0) == -7.0
    assert oracle.hist_dts_at(tau, dts, 9, -7.0) == -7.0
    assert oracle.hist_dts_at(tau[:1], dts[:1], 4, -7.0) == 1.0
    assert oracle.hist_dts_at(tau[:1], dts[:1], 5, -7.0) == -7.0


def cubic(t):
    """A cubic trajectory per component, its velocity and acceleration."""
    c = np.array([[0.5, -1.0, 2.0], [1.5, 0.25, -0.5], [-0.75, 2.0, 1.0],
                  [0.3, -0.6, 0.9]])
    r = c[0] + c[1] * t + c[2] * t ** 2 + c[3] * t ** 3
    v = c[1] + 2 * c[2] * t + 3 * c[3] * t ** 2
    a = 2 * c[2] + 6 * c[3] * t
    return r, v, a


def records(ticks):
    tau = np.array(ticks, np.int64)
    t = tau * 2.0 ** -K_MAX
    rva = [cubic(x) for x in t]
    return (tau, np.array([x[0] for x in rva]), np.array([x[1] for x in rva]),
            np.array([x[2] for x in rva]))


def test_prediction_interpolates_between_the_bracketing_records():
    q = 1 << 12
    tau, r, v, a = records([0, 3 * q, 8 * q, 9 * q, 16 * q])
    own = (np.full(3, 99.0), np.zeros(3), np.zeros(3))  # never used here
    for tn in (1 * q, 5 * q, 8 * q + q // 2, 12 * q, 15 * q + 7):
        rp, vp = oracle.predict_prev(tau, r, v, a, 0, *own, tn, K_MAX)
        rx, vx, _ = cubic(tn * 2.0 ** -K_MAX)
        np.testing.assert_allclose(rp, rx, rtol=0, atol=1e-14)
        np.testing.assert_allclose(vp, vx, rtol=0, atol=1e-14)
        # and it is the Hermite of exactly that pair
        k = oracle.hist_find(tau, tn)
        hr, hv = oracle.hermite(tau[k], tau[k + 1], tn, K_MAX, r[k], v[k],
                                a[k], r[k + 1], v[k + 1], a[k + 1])
        np.testing.assert_array_equal(rp, hr)
        np.testing.assert_array_equal(vp, hv)


def test_prediction_at_a_record_is_the_record():
    q = 1 << 12
    tau, r, v, a = records([0, 3 * q, 8 * q])
    own = (np.full(3, 99.0), np.zeros(3), np.zeros(3))
    for k in range(3):
        rp, vp = oracle.predict_prev(tau, r, v, a, 0, *own, tau[k], K_MAX)
        np.testing.assert_array_equal(rp, r[k])
        np.testing.assert_array_equal(vp, v[k])


@pytest.mark.parametrize("where", ["before", "after", "none"])
def test_prediction_outside_the_records_is_taylor_from_own_state(where):
    q = 1 << 12
    tau, r, v, a = records([4 * q, 8 * q])
    if where == "none":
        tau, r, v, a = tau[:0], r[:0], v[:0], a[:0]
    tj = 2 * q if where == "before" else 8 * q
    tn = tj + (1 << 19)            # h = 1/2
    rj = np.array([1.0, -2.0, 0.5])
    vj = np.array([2.0, 4.0, -1.0])
    aj = np.array([4.0, -8.0, 2.0])
    if where == "before":
        tn = 3 * q                 # before the first record
        h = (tn - tj) * 2.0 ** -K_MAX
        want_r = rj + vj * h + 0.5 * aj * h * h
        want_v = vj + aj * h
    else:
        # r + v h + a h^2 / 2 and v + a h at h = 1/2, exact in binary
        want_r = np.array([1.0 + 1.0 + 0.5, -2.0 + 2.0 - 1.0,
                           0.5 - 0.5 + 0.25])
        want_v = np.array([4.0, 0.0, 0.0])
    rp, vp = oracle.predict_prev(tau, r, v, a, tj, rj, vj, aj, tn, K_MAX)
    np.testing.assert_array_equal(rp, want_r)
    np.testing.assert_array_equal(vp, want_v)
