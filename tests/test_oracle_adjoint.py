"""Pins of the oracle's frozen-schedule adjoint (reading R14).

The replay is pinned to the integrator: a first-pass-only run (n_iter = 1)
uses Taylor prediction everywhere, so replaying its logged schedule must
reproduce its state bit for bit. The reverse mode is pinned by central
finite differences of the replay (error falling as h^2 until roundoff), by
exact translation and boost invariances of the N-body equations, and by
special cases (an empty schedule, a body that never moves).
"""
import numpy as np
import pytest

import oracle
from paper_1205_2288_gb300 import inputs

K_MAX = 20


def schedule_of(m, r, v, *, eps, eta, t_end, n_iter=3, era_log2=3,
                dt_max=1 / 8, era_mode=0):
    s = oracle.Sim(m, r, v, eps=eps, eta=eta, dt_max=dt_max, n_iter=n_iter,
                   era_mode=era_mode, era_log2=era_log2, k_max=K_MAX, log=True)
    s.run(t_end)
    return s


def loss_of(m, r, v, eps, sched):
    rT, _ = oracle.replay(m, r, v, eps, K_MAX, sched)
    return oracle.loss_msr(m, rT)[0]


@pytest.mark.parametrize("era_mode,shared", [(0, False), (1, False), (0, True)])
def test_replay_of_first_pass_schedule_is_the_integrator(era_mode, shared):
    m = inputs.salpeter_masses(96, 3)
    _, r, v = inputs.plummer(96, 4, masses=m)
    kw = dict(eps=0.02, eta=0.03, t_end=0.125, n_iter=1, era_mode=era_mode)
    if shared:   # one shared step: plain velocity Verlet
        kw.update(dt_max=2.0 ** -6, era_log2=6)
    s = schedule_of(m, r, v, **kw)
    st = s.state()
    sched = oracle.final_pass(s.schedule(), 0)
    if era_mode == 0 and not shared:
        # fixed era 1/8 == t_end: the whole run is one era
        rT, vT = oracle.replay(m, r, v, kw["eps"], K_MAX, sched)
        np.testing.assert_array_equal(rT, st["r"])
        np.testing.assert_array_equal(vT, st["v"])
    # every era's schedule, chained, gives the state at the end of the run
    full = s.schedule()
    off = np.concatenate([[0], np.cumsum(full["n_act"])])
    parts = [np.sort(full["idx"][off[k]:off[k + 1]])
             for k in range(len(full["tau"]))]
    chain = (full["tau"], np.concatenate(
        [[0], np.cumsum([len(p) for p in parts])]).astype(np.int64),
        np.concatenate(parts).astype(np.int32))
    rT, vT = oracle.replay(m, r, v, kw["eps"], K_MAX, chain)
    np.testing.assert_array_equal(rT, st["r"])
    np.testing.assert_array_equal(vT, st["v"])


@pytest.fixture(scope="module")
def case():
    """64 bodies, off-centre so that the translation pin is of order one,
    final pass of a three-pass era of 1/8."""
    m = inputs.salpeter_masses(64, 8)
    _, r, v = inputs.plummer(64, 9, masses=m)
    r = r + np.array([0.3, -0.2, 0.5])
    v = v + np.array([0.05, 0.1, -0.02])
    eps = 0.01
    s = schedule_of(m, r, v, eps=eps, eta=0.02, t_end=0.125)
    sched = oracle.final_pass(s.schedule(), 0)
    L, gr, gv, gm = oracle.loss_grad(m, r, v, eps, K_MAX, sched)
    return dict(m=m, r=r, v=v, eps=eps, sched=sched, L=L, gr=gr, gv=gv, gm=gm)


def fd(case, which, d, h):
    args = dict(m=case["m"], r=case["r"], v=case["v"])
    p, q = dict(args), dict(args)
    p[which] = args[which] + h * d
    q[which] = args[which] - h * d
    lp = loss_of(p["m"], p["r"], p["v"], case["eps"], case["sched"])
    lq = loss_of(q["m"], q["r"], q["v"], case["eps"], case["sched"])
    return (lp - lq) / (2 * h)


@pytest.mark.parametrize("which", ["r", "v", "m"])
def test_gradient_matches_central_differences(case, which):
    g = case["g" + which]
    rng = np.random.default_rng({"r": 1, "v": 2, "m": 3}[which])
    for _ in range(3):
        d = rng.standard_normal(g.shape)
        an = float((g * d).sum())
        err = abs(fd(case, which, d, 1e-5) - an)
        assert err <= 2e-8 * abs(an) + 1e-12, (which, err, an)


def test_central_difference_error_falls_as_h_squared(case):
    """Truncation error of the central difference is O(h^2): a gradient
    with a missing term would leave an h-independent error."""
    rng = np.random.default_rng(4)
    d = rng.standard_normal(case["gr"].shape)
    an = float((case["gr"] * d).sum())
    e3 = abs(fd(case, "r", d, 1e-3) - an)
    e4 = abs(fd(case, "r", d, 1e-4) - an)
    assert e4 < e3 / 30, (e3, e4)


@pytest.mark.parametrize("coord", [(0, 0), (17, 2), (63, 1)])
def test_single_coordinates(case, coord):
    i, c = coord
    for which in ("r", "v"):
        d = np.zeros_like(case["r"])
        d[i, c] = 1.0
        an = case["g" + which][i, c]
        assert abs(fd(case, which, d, 1e-5) - an) <= 1e-7 * abs(an) + 1e-10
    d = np.zeros_like(case["m"])
    d[i] = 1.0
    an = case["gm"][i]
    assert abs(fd(case, "m", d, 1e-6) - an) <= 1e-7 * abs(an) + 1e-10


def test_translation_and_boost_invariance(case):
    """Shifting every r0 by c shifts every final position by c; boosting
    every v0 by w shifts it by w T. Hence sum_i dL/dr0_i = 2 R_cm(T) and
    sum_i dL/dv0_i = 2 T R_cm(T) for the mass-weighted loss."""
    m, eps, sched = case["m"], case["eps"], case["sched"]
    rT, _ = oracle.replay(m, case["r"], case["v"], eps, K_MAX, sched)
    T = sched[0][-1] * 2.0 ** -K_MAX
    rcm2 = 2 * (m[:, None] * rT).sum(0) / m.sum()
    assert np.abs(rcm2).max() > 0.1
    np.testing.assert_allclose(case["gr"].sum(0), rcm2, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(case["gv"].sum(0), T * rcm2, rtol=1e-11,
                               atol=1e-13)


def test_loss_partials():
    """L = sum m |r|^2 / sum m: two bodies at +-x give |x|^2; the partials
    follow from the quotient rule."""
    m = np.array([1.0, 3.0])
    r = np.array([[1.0, 2.0, 2.0], [0.0, 0.0, 1.0]])
    L, g_r, g_m = oracle.loss_msr(m, r)
    assert L == (9.0 + 3.0) / 4.0
    np.testing.assert_array_equal(g_r, 2 * m[:, None] * r / 4.0)
    np.testing.assert_array_equal(g_m, (np.array([9.0, 1.0]) - L) / 4.0)


def test_empty_schedule_and_idle_body():
    m, r, v = inputs.plummer(12, 5)
    empty = (np.zeros(0, np.int64), np.zeros(1, np.int64), np.zeros(0, np.int32))
    rT, vT = oracle.replay(m, r, v, 0.05, K_MAX, empty)
    np.testing.assert_array_equal(rT, r)
    np.testing.assert_array_equal(vT, v)
    gr_T = np.ones_like(r)
    gv_T = np.full_like(v, 2.0)
    g_r0, g_v0, g_m = oracle.replay_vjp(m, r, v, 0.05, K_MAX, empty, gr_T, gv_T)
    np.testing.assert_array_equal(g_r0, gr_T)
    np.testing.assert_array_equal(g_v0, gv_T)
    np.testing.assert_array_equal(g_m, 0.0)
    # body 0 never moves: its final state is its initial state, and it
    # still pulls on the others
    steps = np.array([1 << 14, 1 << 15], np.int64)
    act = np.array([1, 2, 3, 1, 2, 3, 4], np.int32)
    sched = (steps, np.array([0, 3, 7], np.int64), act)
    rT, vT = oracle.replay(m, r, v, 0.05, K_MAX, sched)
    np.testing.assert_array_equal(rT[0], r[0])
    np.testing.assert_array_equal(rT[5:], r[5:])
    gr_T = np.zeros_like(r)
    gr_T[1] = 1.0
    g_r0, g_v0, g_m = oracle.replay_vjp(m, r, v, 0.05, K_MAX, sched, gr_T,
                                        np.zeros_like(v))
    assert np.abs(g_r0[0]).max() > 0 and g_m[0] != 0   # it pulls on body 1
    # a loss on the idle body alone sees only its own initial position
    gr_T = np.zeros_like(r)
    gr_T[0] = [1.0, -2.0, 0.5]
    g_r0, g_v0, g_m = oracle.replay_vjp(m, r, v, 0.05, K_MAX, sched, gr_T,
                                        np.zeros_like(v))
    np.testing.assert_array_equal(g_r0, gr_T)
    np.testing.assert_array_equal(g_v0, 0.0)
    np.testing.assert_array_equal(g_m, 0.0)
