"""Pins of the oracle's adjoint through every pass of one era (reading R14
extended to the symmetrised passes, with the Hermite interpolation of the
previous pass's records).

The forward replay of all passes on their logged schedules reproduces the
integrator's era bit for bit; one pass reduces to the single-pass adjoint;
central differences of the multi-pass replay match the gradient (error
falling as h^2); translation and boost invariance hold exactly (the Hermite
interpolation reproduces a uniform shift and a uniform boost).
"""
import numpy as np
import pytest

import oracle
from paper_1205_2288_gb300 import inputs

K_MAX = 20


def integrate(m, r, v, t_end, **kw):
    s = oracle.Sim(m, r, v, log=True, k_max=K_MAX, **kw)
    s.run(t_end)
    return s


@pytest.mark.parametrize("n_iter,era_mode", [(3, 0), (5, 0), (3, 1)])
def test_multi_pass_replay_is_the_integrator(n_iter, era_mode):
    m = inputs.salpeter_masses(80, 21)
    _, r, v = inputs.plummer(80, 22, masses=m)
    kw = dict(eps=0.02, eta=0.03, dt_max=1 / 8, era_mode=era_mode,
              era_log2=3, n_iter=n_iter)
    s = integrate(m, r, v, 0.125, **kw)
    eras = s.eras()
    if era_mode == 1:
        # the first era of a dynamic run, integrated on its own
        s = integrate(m, r, v, eras[1][0] * 2.0 ** -K_MAX, **kw)
    passes = oracle.era_passes(s.schedule(), 0)
    assert len(passes) == n_iter
    rT, vT = oracle.era_replay(m, r, v, 0.02, K_MAX, passes)
    np.testing.assert_array_equal(rT, s.state()["r"])
    np.testing.assert_array_equal(vT, s.state()["v"])


@pytest.fixture(scope="module")
def era_case():
    """A long era (one time unit, eta = 0.3, 73 steps a pass), where the
    earlier passes carry ~5e-5 of the gradient through the records the
    later passes interpolate, well above the central differences' error."""
    m = inputs.salpeter_masses(48, 3)
    _, r, v = inputs.plummer(48, 4, masses=m)
    r = r + np.array([0.3, -0.2, 0.1])
    v = v + np.array([0.05, -0.1, 0.02])
    eps = 0.02
    s = integrate(m, r, v, 1.0, eps=eps, eta=0.3, dt_max=1 / 8,
                  era_mode=0, era_log2=0, n_iter=3)
    passes = oracle.era_passes(s.schedule(), 0)
    rT, _ = oracle.era_replay(m, r, v, eps, K_MAX, passes)
    L, grT, gmL = oracle.loss_msr(m, rT)
    gr, gv, gm = oracle.era_replay_vjp(m, r, v, eps, K_MAX, passes, grT,
                                       np.zeros_like(grT))
    return dict(m=m, r=r, v=v, eps=eps, passes=passes, rT=rT, L=L, gr=gr,
                gv=gv, gm=gm + gmL)


def loss(c, m, r, v):
    rT, _ = oracle.era_replay(m, r, v, c["eps"], K_MAX, c["passes"])
    return oracle.loss_msr(m, rT)[0]


def fd(c, which, d, h):
    args = dict(m=c["m"], r=c["r"], v=c["v"])
    p, q = dict(args), dict(args)
    p[which] = args[which] + h * d
    q[which] = args[which] - h * d
    return (loss(c, **p) - loss(c, **q)) / (2 * h)


@pytest.mark.parametrize("which", ["r", "v", "m"])
def test_gradient_matches_central_differences(era_case, which):
    c = era_case
    g = c["g" + which]
    rng = np.random.default_rng({"r": 5, "v": 6, "m": 7}[which])
    h = 1e-6 if which == "m" else 1e-5
    for _ in range(2):
        d = rng.standard_normal(g.shape)
        an = float((g * d).sum())
        # relative to the scale |g| |d| (a single directional derivative
        # can be small by cancellation)
        scale = np.linalg.norm(g) * np.linalg.norm(d)
        assert abs(fd(c, which, d, h) - an) <= 1e-8 * scale


def test_difference_error_falls_as_h_squared(era_case):
    c = era_case
    d = np.random.default_rng(8).standard_normal(c["gr"].shape)
    an = float((c["gr"] * d).sum())
    e3 = abs(fd(c, "r", d, 1e-3) - an)
    e4 = abs(fd(c, "r", d, 1e-4) - an)
    assert e4 < e3 / 30, (e3, e4)


def test_translation_and_boost_invariance(era_case):
    c = era_case
    T = c["passes"][-1][0][-1] * 2.0 ** -K_MAX
    rcm2 = 2 * (c["m"][:, None] * c["rT"]).sum(0) / c["m"].sum()
    assert np.abs(rcm2).max() > 0.1
    np.testing.assert_allclose(c["gr"].sum(0), rcm2, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(c["gv"].sum(0), T * rcm2, rtol=1e-11,
                               atol=1e-13)


def test_one_pass_is_the_single_pass_adjoint(era_case):
    c = era_case
    one = [c["passes"][0]]
    rng = np.random.default_rng(9)
    gr_T = rng.standard_normal(c["r"].shape)
    gv_T = rng.standard_normal(c["r"].shape)
    a = oracle.era_replay_vjp(c["m"], c["r"], c["v"], c["eps"], K_MAX, one,
                              gr_T, gv_T)
    b = oracle.replay_vjp(c["m"], c["r"], c["v"], c["eps"], K_MAX, one[0],
                          gr_T, gv_T)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_earlier_passes_contribute(era_case):
    """The final pass alone (its schedule replayed with Taylor prediction,
    reading R14 proper) is a different function: the records of the
    earlier passes carry part of the gradient."""
    c = era_case
    L1, grT1, gmL1 = oracle.loss_msr(
        c["m"], oracle.replay(c["m"], c["r"], c["v"], c["eps"], K_MAX,
                              c["passes"][-1])[0])
    g1 = oracle.replay_vjp(c["m"], c["r"], c["v"], c["eps"], K_MAX,
                           c["passes"][-1], grT1, np.zeros_like(grT1))[0]
    diff = np.abs(g1 - c["gr"]).max() / np.abs(c["gr"]).max()
    assert 1e-6 < diff < 1e-2


# ---------------------------------------------------------------------
# Across eras: each era starts from the state the era before it left, a
# body whose step overshot the era end waiting behind it (Sec. 3).
# ---------------------------------------------------------------------

def waiting_system():
    """A Plummer sphere plus one far, slow body whose step (dt_max = 1/8)
    overshoots every era of 1/16: it waits behind two era ends out of
    three, so later eras start from bodies at different ticks."""
    m = inputs.salpeter_masses(40, 13)
    _, r, v = inputs.plummer(40, 14, masses=m)
    m = np.append(m, 2e-3)
    r = np.vstack([r, [30.0, -8.0, 4.0]])
    v = np.vstack([v, [0.0, 0.03, 0.01]])
    return m, r, v


@pytest.mark.parametrize("era_mode", [0, 1])
def test_eras_replay_is_the_integrator(era_mode):
    m, r, v = waiting_system()
    s = integrate(m, r, v, 0.5, eps=0.02, eta=0.05, dt_max=1 / 8,
                  era_mode=era_mode, era_log2=4, n_iter=3)
    sched = s.schedule()
    n_eras = len(np.unique(sched["era"]))
    assert n_eras >= 3
    eras = [oracle.era_passes(sched, k) for k in range(n_eras)]
    (rT, vT, aT, tauT), starts = oracle.eras_replay(m, r, v, 0.02, K_MAX,
                                                    eras)
    st = s.state()
    np.testing.assert_array_equal(rT, st["r"])
    np.testing.assert_array_equal(vT, st["v"])
    np.testing.assert_array_equal(aT, st["a"])
    np.testing.assert_array_equal(tauT, st["tau"])
    # with fixed eras of 1/16 some era starts with the far body (step 1/8)
    # behind the era's start tick (dynamic eras grow to its step)
    if era_mode == 0:
        first_ticks = [e[0][0][0] for e in eras[1:]]
        assert any(t0[-1] < ft - (1 << 16)
                   for (_, _, _, t0), ft in zip(starts[1:], first_ticks))


@pytest.fixture(scope="module")
def eras_case():
    m, r, v = waiting_system()
    s = integrate(m, r, v, 0.25, eps=0.02, eta=0.05, dt_max=1 / 8,
                  era_mode=0, era_log2=4, n_iter=3)
    sched = s.schedule()
    eras = [oracle.era_passes(sched, k)
            for k in range(len(np.unique(sched["era"])))]
    (rT, _, _, _), starts = oracle.eras_replay(m, r, v, 0.02, K_MAX, eras)
    L, grT, gmL = oracle.loss_msr(m, rT)
    gr, gv, gm = oracle.eras_replay_vjp(m, r, v, 0.02, K_MAX, eras, grT,
                                        np.zeros_like(grT))
    return dict(m=m, r=r, v=v, eras=eras, starts=starts, rT=rT, gr=gr,
                gv=gv, gm=gm + gmL)


def eras_loss(c, m, r, v):
    (rT, _, _, _), _ = oracle.eras_replay(m, r, v, 0.02, K_MAX, c["eras"])
    return oracle.loss_msr(m, rT)[0]


@pytest.mark.parametrize("which", ["r", "v", "m"])
def test_eras_gradient_matches_central_differences(eras_case, which):
    c = eras_case
    g = c["g" + which]
    rng = np.random.default_rng({"r": 15, "v": 16, "m": 17}[which])
    # (the loss through several eras is strongly curved: h = 1e-5 leaves a
    # truncation error of ~1e-7 relative, falling as h^2)
    h = 1e-6
    for _ in range(2):
        d = rng.standard_normal(g.shape)
        args = dict(m=c["m"], r=c["r"], v=c["v"])
        p, q = dict(args), dict(args)
        p[which] = args[which] + h * d
        q[which] = args[which] - h * d
        fd = (eras_loss(c, **p) - eras_loss(c, **q)) / (2 * h)
        an = float((g * d).sum())
        scale = np.linalg.norm(g) * np.linalg.norm(d)
        assert abs(fd - an) <= 1e-8 * scale, (which, fd, an)


def test_eras_difference_error_falls_as_h_squared(eras_case):
    c = eras_case
    d = np.random.default_rng(20).standard_normal(c["gr"].shape)
    an = float((c["gr"] * d).sum())

    def fd(h):
        return (eras_loss(c, c["m"], c["r"] + h * d, c["v"])
                - eras_loss(c, c["m"], c["r"] - h * d, c["v"])) / (2 * h)
    e4 = abs(fd(1e-4) - an)
    e5 = abs(fd(1e-5) - an)
    assert e5 < e4 / 30, (e4, e5)


def test_state_start_acceleration_cotangent(eras_case):
    """The cotangent of an era's start accelerations (what the era before
    it hands on) against central differences of that era's replay."""
    c = eras_case
    k = len(c["eras"]) - 1
    r0, v0, a0, tau0 = c["starts"][k]
    passes = c["eras"][k]
    m = c["m"]

    def L(a):
        rT = oracle.era_replay_state(m, r0, v0, a, tau0, 0.02, K_MAX,
                                     passes)[0]
        return oracle.loss_msr(m, rT)[0]
    rT = oracle.era_replay_state(m, r0, v0, a0, tau0, 0.02, K_MAX, passes)[0]
    _, grT, _ = oracle.loss_msr(m, rT)
    g = oracle.era_replay_state_vjp(m, r0, v0, a0, tau0, 0.02, K_MAX, passes,
                                    grT, None, None)
    ga = g[2]
    assert np.abs(ga).max() > 0
    d = np.random.default_rng(18).standard_normal(a0.shape)
    h = 1e-6
    fd = (L(a0 + h * d) - L(a0 - h * d)) / (2 * h)
    an = float((ga * d).sum())
    assert abs(fd - an) <= 1e-7 * np.linalg.norm(ga) * np.linalg.norm(d)


def test_eras_translation_and_boost_invariance(eras_case):
    c = eras_case
    T = c["eras"][-1][-1][0][-1] * 2.0 ** -K_MAX
    rcm2 = 2 * (c["m"][:, None] * c["rT"]).sum(0) / c["m"].sum()
    np.testing.assert_allclose(c["gr"].sum(0), rcm2, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(c["gv"].sum(0), T * rcm2, rtol=1e-10,
                               atol=1e-12)


def test_one_era_chain_is_the_era_adjoint(eras_case):
    c = eras_case
    one = c["eras"][:1]
    rng = np.random.default_rng(19)
    gr_T = rng.standard_normal(c["r"].shape)
    gv_T = rng.standard_normal(c["r"].shape)
    a = oracle.eras_replay_vjp(c["m"], c["r"], c["v"], 0.02, K_MAX, one,
                               gr_T, gv_T)
    b = oracle.era_replay_vjp(c["m"], c["r"], c["v"], 0.02, K_MAX, one[0],
                              gr_T, gv_T)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
