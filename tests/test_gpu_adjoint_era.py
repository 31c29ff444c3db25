"""Parity of the CUDA adjoint through every pass of one era
(tsbts_adjoint_init_era) with the FP64 oracle's (orc_era_replay,
orc_era_replay_vjp): reading R14 extended to the symmetrised passes of
Sec. 2, where a pass after the first places each body that is not active
from the previous pass's records (the record on an exact hit, the cubic
Hermite between the bracketing records, else Eq. 2).

FP64 with ascending-j force sums replays all passes bit for bit (and so
reproduces the integrator's era); the reverse sweep sums its pair terms in
another order than the oracle, so gradients are held to a relative bound.
Checkpointed, taped, graph and stream runs are bit-identical. At the full
size (Plummer n = 8192, eps = 0.01, one era 0..1/4, three passes) the FP64
gradient is checked against central differences of the FP64 replay.
"""
import numpy as np
import pytest

import oracle
from paper_1205_2288_gb300 import inputs, tsbts

pytestmark = pytest.mark.gpu

K_MAX = 20


@pytest.fixture(scope="module", autouse=True)
def need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def rel(a, b):
    """max |a - b| over max |b|"""
    return float(np.abs(a - b).max() / np.abs(b).max())


def oracle_era(m, r, v, *, eps, eta, t_end, era_log2, n_iter, era_mode=0):
    s = oracle.Sim(m, r, v, eps=eps, eta=eta, dt_max=1 / 8, n_iter=n_iter,
                   era_mode=era_mode, era_log2=era_log2, k_max=K_MAX,
                   log=True)
    s.run(t_end)
    st = s.state()
    passes = oracle.era_passes(s.schedule(), 0)
    s.close()
    return passes, st


@pytest.fixture(scope="module")
def case600():
    """n = 600 Salpeter-mass Plummer sphere, one fixed era of 1/2 with three
    passes (eta = 0.1): ~570 block steps a pass, most bodies placed from the
    previous pass's records at most steps. The earlier passes carry ~4e-7
    of the loss gradient (relative), thousands of times the parity bound."""
    m = inputs.salpeter_masses(600, 31)
    _, r, v = inputs.plummer(600, 32, masses=m)
    r = r + np.array([0.2, -0.1, 0.3])
    eps = 0.01
    passes, st = oracle_era(m, r, v, eps=eps, eta=0.1, t_end=0.5,
                            era_log2=1, n_iter=3)
    rT, vT = oracle.era_replay(m, r, v, eps, K_MAX, passes)
    L, g_rT, g_mL = oracle.loss_msr(m, rT)
    gr, gv, gm = oracle.era_replay_vjp(m, r, v, eps, K_MAX, passes, g_rT,
                                       np.zeros_like(g_rT))
    return dict(m=m, r=r, v=v, eps=eps, passes=passes, st=st, rT=rT, vT=vT,
                L=L, gr=gr, gv=gv, gm=gm + g_mL)


def test_case_has_three_long_passes(case600):
    p = case600["passes"]
    assert len(p) == 3
    assert min(len(x[0]) for x in p) > 500


def test_fp64_era_replay_bit_exact(case600):
    c = case600
    with tsbts.Adjoint(600, c["eps"], passes=c["passes"]) as adj:
        rT, vT = adj.forward(c["m"], c["r"], c["v"])
        st = adj.stats()
    np.testing.assert_array_equal(rT, c["rT"])
    np.testing.assert_array_equal(vT, c["vT"])
    # and so the integrator's state at the era end
    np.testing.assert_array_equal(rT, c["st"]["r"])
    np.testing.assert_array_equal(vT, c["st"]["v"])
    assert st["passes"] == 3
    assert st["steps"] == sum(len(x[0]) for x in c["passes"])


@pytest.mark.parametrize("K", [0, 1, 7, 50, 100000])
def test_fp64_era_loss_gradient_matches_oracle(case600, K):
    c = case600
    with tsbts.Adjoint(600, c["eps"], passes=c["passes"],
                       checkpoint_every=K) as adj:
        L, gr, gv, gm = adj.loss_grad(c["m"], c["r"], c["v"])
        st = adj.stats()
    assert abs(L / c["L"] - 1) < 1e-14
    assert rel(gr, c["gr"]) < 1e-10, rel(gr, c["gr"])
    assert rel(gv, c["gv"]) < 1e-10, rel(gv, c["gv"])
    assert rel(gm, c["gm"]) < 1e-10, rel(gm, c["gm"])
    n_steps = [len(x[0]) for x in c["passes"]]
    if K == 0 or K >= sum(n_steps):
        assert st["checkpoints"] == 0
    else:
        # segments of K steps within each pass
        assert st["checkpoints"] == sum(-(-s // K) for s in n_steps)


def test_fp64_era_general_vjp_matches_oracle(case600):
    c = case600
    rng = np.random.default_rng(11)
    gr_T = rng.standard_normal((600, 3))
    gv_T = rng.standard_normal((600, 3))
    want = oracle.era_replay_vjp(c["m"], c["r"], c["v"], c["eps"], K_MAX,
                                 c["passes"], gr_T, gv_T)
    with tsbts.Adjoint(600, c["eps"], passes=c["passes"]) as adj:
        adj.forward(c["m"], c["r"], c["v"])
        got = adj.vjp(gr_T, gv_T)
        # a second reverse sweep of the same forward replay
        again = adj.vjp(gr_T, gv_T)
    for a, b in zip(got, want):
        assert rel(a, b) < 1e-10, rel(a, b)
    for a, b in zip(again, got):
        np.testing.assert_array_equal(a, b)


def test_earlier_passes_change_the_gradient(case600):
    """The gradient through every pass differs from the final pass's alone
    by far more than the parity bound: the records the last pass
    interpolates carry part of it."""
    c = case600
    with tsbts.Adjoint(600, c["eps"], c["passes"][-1]) as adj:
        L1, gr1, gv1, gm1 = adj.loss_grad(c["m"], c["r"], c["v"])
    assert rel(gr1, c["gr"]) > 1e-7
    assert rel(gv1, c["gv"]) > 1e-7


def test_one_pass_era_is_the_plain_adjoint(case600):
    c = case600
    last = c["passes"][-1]
    out = []
    with tsbts.Adjoint(600, c["eps"], last) as adj:
        out.append(adj.loss_grad(c["m"], c["r"], c["v"]))
    with tsbts.Adjoint(600, c["eps"], passes=[last]) as adj:
        out.append(adj.loss_grad(c["m"], c["r"], c["v"]))
    assert out[0][0] == out[1][0]
    for a, b in zip(out[0][1:], out[1][1:]):
        np.testing.assert_array_equal(a, b)


def test_mixed_era_gradient_within_fp32_accuracy(case600):
    c = case600
    with tsbts.Adjoint(600, c["eps"], passes=c["passes"],
                       precision=tsbts.TSBTS_MIXED) as adj:
        rT, _ = adj.forward(c["m"], c["r"], c["v"])
        L, gr, gv, gm = adj.loss_grad(c["m"], c["r"], c["v"])
    assert np.abs(rT - c["rT"]).max() < 1e-6
    assert abs(L / c["L"] - 1) < 1e-7
    for a, b in ((gr, c["gr"]), (gv, c["gv"]), (gm, c["gm"])):
        assert rel(a, b) < 1e-4, rel(a, b)


def test_era_checkpoints_graphs_and_streams_agree(case600):
    c = case600
    out = []
    for K in (0, 5, 64):
        for graph_steps in (0, 32):
            with tsbts.Adjoint(600, c["eps"], passes=c["passes"],
                               checkpoint_every=K, graph_steps=graph_steps,
                               precision=tsbts.TSBTS_MIXED) as adj:
                out.append(adj.loss_grad(c["m"], c["r"], c["v"]))
                again = adj.loss_grad(c["m"], c["r"], c["v"])
            for a, b in zip(again, out[-1]):
                np.testing.assert_array_equal(a, b)
    for o in out[1:]:
        assert o[0] == out[0][0]
        for a, b in zip(o[1:], out[0][1:]):
            np.testing.assert_array_equal(a, b)


def test_dynamic_era_and_five_passes():
    """A dynamic first era (Alg. 3) and a fixed era with five passes, small
    enough for the oracle's reverse mode to run in a moment."""
    m = inputs.salpeter_masses(96, 7)
    _, r, v = inputs.plummer(96, 8, masses=m)
    for kw in (dict(era_mode=1, n_iter=3), dict(era_mode=0, n_iter=5)):
        passes, _ = oracle_era(m, r, v, eps=0.02, eta=0.03, t_end=0.125,
                               era_log2=3, **kw)
        assert len(passes) == kw["n_iter"]
        rng = np.random.default_rng(len(passes))
        gr_T = rng.standard_normal((96, 3))
        gv_T = rng.standard_normal((96, 3))
        want_r, want_v = oracle.era_replay(m, r, v, 0.02, K_MAX, passes)
        want = oracle.era_replay_vjp(m, r, v, 0.02, K_MAX, passes, gr_T,
                                     gv_T)
        with tsbts.Adjoint(96, 0.02, passes=passes,
                           checkpoint_every=4) as adj:
            rT, vT = adj.forward(m, r, v)
            got = adj.vjp(gr_T, gv_T)
        np.testing.assert_array_equal(rT, want_r)
        np.testing.assert_array_equal(vT, want_v)
        for a, b in zip(got, want):
            assert rel(a, b) < 1e-10, (kw, rel(a, b))


def test_hand_made_passes_with_ragged_sets():
    """Passes built by hand: bodies active in one pass and not the next, a
    body that never moves, record hits on the exact tick, bodies past their
    last record (Eq. 2), and single-body steps."""
    n = 37
    m, r, v = inputs.plummer(n, 3)
    q = 1 << 14
    passes = []
    for p in range(3):
        steps = np.array([q, 2 * q, 3 * q, 4 * q + p * 256, 6 * q], np.int64)
        sets = [np.arange(0, n - 1, 2), np.array([n - 2]),
                np.arange(p, n - 1, 3), np.arange(n - 1),
                np.arange(1, n - 1, 2 + p)]
        off = np.concatenate([[0], np.cumsum([len(x) for x in sets])])
        passes.append((steps, off.astype(np.int64),
                       np.concatenate(sets).astype(np.int32)))
    rng = np.random.default_rng(2)
    gr_T = rng.standard_normal((n, 3))
    want_r, want_v = oracle.era_replay(m, r, v, 0.05, K_MAX, passes)
    want = oracle.era_replay_vjp(m, r, v, 0.05, K_MAX, passes, gr_T,
                                 np.zeros_like(gr_T))
    for prec in (tsbts.TSBTS_FP64, tsbts.TSBTS_MIXED):
        for K in (0, 2):
            with tsbts.Adjoint(n, 0.05, passes=passes, precision=prec,
                               checkpoint_every=K) as adj:
                rT, vT = adj.forward(m, r, v)
                got = adj.vjp(gr_T)
            if prec == tsbts.TSBTS_FP64:
                np.testing.assert_array_equal(rT, want_r)
                np.testing.assert_array_equal(vT, want_v)
            tol = 1e-10 if prec == tsbts.TSBTS_FP64 else 1e-4
            for a, b in zip(got, want):
                assert rel(a, b) < tol, (prec, K, rel(a, b))


def test_era_schedule_errors():
    m, r, v = inputs.plummer(8, 1)
    one = (np.array([4, 8], np.int64), np.array([0, 1, 2], np.int64),
           np.array([0, 1], np.int32))
    empty = (np.zeros(0, np.int64), np.zeros(1, np.int64),
             np.zeros(0, np.int32))
    back = (np.array([8, 4], np.int64), np.array([0, 1, 2], np.int64),
            np.array([0, 1], np.int32))
    for passes, what in (([one, empty], "empty pass"),
                         ([one, back], "ticks within a pass")):
        cfg = tsbts.tsbts_config_default()
        ctx = tsbts.tsbts_create(cfg)
        try:
            with pytest.raises(tsbts.TsbtsError) as e:
                tsbts.tsbts_adjoint_init_era(ctx, 8, 0.01, passes)
            assert e.value.code == tsbts.TSBTS_ERR_ARG, what
        finally:
            tsbts.tsbts_destroy(ctx)
    # ticks restart in every pass: the same ticks twice are fine
    with tsbts.Adjoint(8, 0.01, passes=[one, one]) as adj:
        rT, _ = adj.forward(m, r, v)
    want, _ = oracle.era_replay(m, r, v, 0.01, K_MAX, [one, one])
    np.testing.assert_array_equal(rT, want)


@pytest.fixture(scope="module")
def config5_era():
    """Plummer n = 8192, eps = 0.01, eta = 0.01, one era 0..1/4 (fixed era
    2^-2, dt_max = 1/8, three passes): every pass's schedule from the mixed
    GPU integrator."""
    m, r, v = inputs.plummer(8192, 0)
    sim = tsbts.Simulation(m, r, v, eps=0.01, eta=0.01, dt_max=1 / 8,
                           n_iter=3, era_mode=0, era_log2=2,
                           precision=tsbts.TSBTS_MIXED)
    sim.schedule_log(40_000_000)
    sim.step_era(0.25)
    passes = tsbts.era_pass_schedules(sim.schedule(), 0)
    sim.close()
    assert len(passes) == 3
    return dict(m=m, r=r, v=v, passes=passes)


def test_config5_era_fp64_gradient_matches_central_differences(config5_era):
    c = config5_era
    rng = np.random.default_rng(13)
    with tsbts.Adjoint(8192, 0.01, passes=c["passes"], checkpoint_every=64,
                       exact_order=0) as adj:
        L, gr, gv, gm = adj.loss_grad(c["m"], c["r"], c["v"])

        def loss(m, r, v):
            rT, _ = adj.forward(m, r, v)
            return float((m * (rT * rT).sum(1)).sum() / m.sum())
        h = 1e-6
        for which, g in (("r", gr), ("v", gv), ("m", gm)):
            d = rng.standard_normal(g.shape)
            args = dict(m=c["m"], r=c["r"], v=c["v"])
            p, q = dict(args), dict(args)
            p[which] = args[which] + h * d
            q[which] = args[which] - h * d
            fd = (loss(**p) - loss(**q)) / (2 * h)
            an = float((g * d).sum())
            assert abs(fd - an) <= 1e-6 * abs(an), (which, fd, an)
    c["fp64"] = (L, gr, gv, gm)


def test_config5_era_mixed_gradient_tracks_fp64(config5_era):
    c = config5_era
    if "fp64" not in c:
        pytest.skip("needs the FP64 gradient")
    with tsbts.Adjoint(8192, 0.01, passes=c["passes"],
                       precision=tsbts.TSBTS_MIXED) as adj:
        L, gr, gv, gm = adj.loss_grad(c["m"], c["r"], c["v"])
        st = adj.stats()
    L0, gr0, gv0, gm0 = c["fp64"]
    assert abs(L / L0 - 1) < 1e-7
    for a, b in ((gr, gr0), (gv, gv0), (gm, gm0)):
        assert rel(a, b) < 1e-4, rel(a, b)
    assert st["passes"] == 3
    assert st["pairs_backward"] == 2 * (st["entries"] + 8192) * 8192


def test_torch_autograd_through_every_pass():
    import torch
    from paper_1205_2288_gb300 import autograd as ag
    m, r, v = inputs.plummer(10, 8)
    passes, _ = oracle_era(m, r, v, eps=0.05, eta=0.2, t_end=2.0 ** -5,
                           era_log2=5, n_iter=3)
    dev = torch.device("cuda:0")
    adj = ag.make_adjoint(10, 0.05, passes=passes)
    try:
        t = lambda x: torch.tensor(x, dtype=torch.float64, device=dev,
                                   requires_grad=True)
        r0, v0, m0 = t(r), t(v), t(m)
        assert torch.autograd.gradcheck(lambda a, b, c: ag.replay(adj, a, b, c),
                                        (r0, v0, m0), eps=1e-6, atol=1e-7,
                                        rtol=1e-5)
    finally:
        adj.close()


# ---------------------------------------------------------------------
# Across eras: each era replayed from the state (r, v, a, tick) the era
# before it left, bodies whose step overshot the era end waiting behind it
# (Sec. 3); reverse mode chained era by era.
# ---------------------------------------------------------------------

def waiting_system(n, seed):
    """A Plummer sphere plus one far, slow body whose step (dt_max = 1/8)
    overshoots the eras of 1/16: later eras start with bodies at different
    ticks."""
    m = inputs.salpeter_masses(n, seed)
    _, r, v = inputs.plummer(n, seed + 1, masses=m)
    m = np.append(m, 2e-3)
    r = np.vstack([r, [30.0, -8.0, 4.0]])
    v = np.vstack([v, [0.0, 0.03, 0.01]])
    return m, r, v


@pytest.fixture(scope="module")
def eras_case():
    m, r, v = waiting_system(300, 41)
    s = oracle.Sim(m, r, v, eps=0.02, eta=0.05, dt_max=1 / 8, n_iter=3,
                   era_mode=0, era_log2=4, k_max=K_MAX, log=True)
    s.run(0.25)
    st = s.state()
    sched = s.schedule()
    s.close()
    eras = [oracle.era_passes(sched, k)
            for k in range(len(np.unique(sched["era"])))]
    (rT, vT, aT, tauT), starts = oracle.eras_replay(m, r, v, 0.02, K_MAX,
                                                    eras)
    L, g_rT, g_mL = oracle.loss_msr(m, rT)
    gr, gv, gm = oracle.eras_replay_vjp(m, r, v, 0.02, K_MAX, eras, g_rT,
                                        np.zeros_like(g_rT))
    return dict(m=m, r=r, v=v, eras=eras, starts=starts, st=st, rT=rT,
                vT=vT, aT=aT, tauT=tauT, L=L, gr=gr, gv=gv, gm=gm + g_mL)


def test_eras_case_has_waiting_bodies(eras_case):
    c = eras_case
    assert len(c["eras"]) == 4
    n = len(c["m"])
    # eras 1 and 3 start with the far body (and a few outer ones) still at
    # the tick before the era start; era 2 starts synchronised
    for k, waits in ((1, True), (2, False), (3, True)):
        tau0 = c["starts"][k][3]
        era_start = min(p[0][0] for p in c["eras"][k]) >> 16 << 16
        assert (tau0[n - 1] < era_start) == waits
        assert ((tau0 < era_start).sum() > 1) == waits


def test_fp64_state_replay_and_vjp_per_era(eras_case):
    c = eras_case
    rng = np.random.default_rng(21)
    n = len(c["m"])
    for k in (1, 3):
        r0, v0, a0, tau0 = c["starts"][k]
        passes = c["eras"][k]
        want = oracle.era_replay_state(c["m"], r0, v0, a0, tau0, 0.02, K_MAX,
                                       passes)
        g = [rng.standard_normal((n, 3)) for _ in range(3)]
        want_g = oracle.era_replay_state_vjp(c["m"], r0, v0, a0, tau0, 0.02,
                                             K_MAX, passes, *g)
        for K in (0, 6):
            with tsbts.Adjoint(n, 0.02, passes=passes,
                               checkpoint_every=K) as adj:
                got = adj.forward_state(c["m"], r0, v0, a0, tau0)
                got_g = adj.vjp_state(*g)
            for a, b in zip(got, want):
                np.testing.assert_array_equal(a, b)
            for a, b in zip(got_g, want_g):
                assert rel(a, b) < 1e-10, (k, K, rel(a, b))


def test_lone_pass_state_replay(eras_case):
    """One pass from a general start state (the plain block-step adjoint of
    a later era's final pass)."""
    c = eras_case
    n = len(c["m"])
    r0, v0, a0, tau0 = c["starts"][2]
    one = [c["eras"][2][-1]]
    want = oracle.era_replay_state(c["m"], r0, v0, a0, tau0, 0.02, K_MAX, one)
    gr = np.random.default_rng(22).standard_normal((n, 3))
    want_g = oracle.era_replay_state_vjp(c["m"], r0, v0, a0, tau0, 0.02,
                                         K_MAX, one, gr, None, gr)
    with tsbts.Adjoint(n, 0.02, one[0]) as adj:
        got = adj.forward_state(c["m"], r0, v0, a0, tau0)
        got_g = adj.vjp_state(gr, None, gr)
    for a, b in zip(got, want):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(got_g, want_g):
        assert rel(a, b) < 1e-10, rel(a, b)


def test_fp64_eras_adjoint_matches_oracle(eras_case):
    c = eras_case
    n = len(c["m"])
    with tsbts.ErasAdjoint(n, 0.02, c["eras"]) as ea:
        rT, vT, aT, tauT = ea.forward(c["m"], c["r"], c["v"])
        L, gr, gv, gm = ea.loss_grad(c["m"], c["r"], c["v"])
    for a, b in ((rT, c["rT"]), (vT, c["vT"]), (aT, c["aT"]),
                 (tauT, c["tauT"]), (rT, c["st"]["r"]), (tauT, c["st"]["tau"])):
        np.testing.assert_array_equal(a, b)
    assert abs(L / c["L"] - 1) < 1e-14
    for a, b in ((gr, c["gr"]), (gv, c["gv"]), (gm, c["gm"])):
        assert rel(a, b) < 1e-10, rel(a, b)


def test_mixed_eras_adjoint_within_fp32_accuracy(eras_case):
    c = eras_case
    n = len(c["m"])
    with tsbts.ErasAdjoint(n, 0.02, c["eras"],
                           precision=tsbts.TSBTS_MIXED) as ea:
        L, gr, gv, gm = ea.loss_grad(c["m"], c["r"], c["v"])
    assert abs(L / c["L"] - 1) < 1e-7
    for a, b in ((gr, c["gr"]), (gv, c["gv"]), (gm, c["gm"])):
        assert rel(a, b) < 1e-4, rel(a, b)


def test_state_start_errors(eras_case):
    c = eras_case
    n = len(c["m"])
    r0, v0, a0, tau0 = c["starts"][1]
    passes = c["eras"][1]
    first = min(p[0][0] for p in passes)
    with tsbts.Adjoint(n, 0.02, passes=passes) as adj:
        late = tau0.copy()
        late[0] = first
        for bad, what in (((a0, late), "tick at a block tick"),
                          ((a0, tau0 - tau0.max() - 1), "negative tick")):
            with pytest.raises(tsbts.TsbtsError) as e:
                adj.forward_state(c["m"], r0, v0, *bad)
            assert e.value.code == tsbts.TSBTS_ERR_ARG, what
        ctx = adj.ctx
        with pytest.raises(tsbts.TsbtsError) as e:
            tsbts._check(tsbts.lib().tsbts_adjoint_forward_state(
                ctx, c["m"].ctypes.data, r0.ctypes.data, v0.ctypes.data,
                None, tau0.ctypes.data, None, None, None, None, 0), ctx)
        assert e.value.code == tsbts.TSBTS_ERR_ARG
        # still usable
        got = adj.forward_state(c["m"], r0, v0, a0, tau0)
    want = oracle.era_replay_state(c["m"], r0, v0, a0, tau0, 0.02, K_MAX,
                                   passes)
    np.testing.assert_array_equal(got[0], want[0])


def test_gpu_schedule_eras_gradient_matches_central_differences():
    """Four eras of a Plummer n = 2048 run (plus a far, waiting body) from
    the FP64 GPU integrator's own schedule log: the gradient across the
    eras against central differences of the FP64 replay."""
    m, r, v = waiting_system(2048, 51)
    n = len(m)
    sim = tsbts.Simulation(m, r, v, eps=0.01, eta=0.02, dt_max=1 / 8,
                           n_iter=3, era_mode=0, era_log2=4)
    sim.schedule_log(20_000_000)
    sim.step_era(0.25)
    st = sim.state()
    eras = [tsbts.era_pass_schedules(sim.schedule(), k) for k in range(4)]
    sim.close()
    rng = np.random.default_rng(23)
    with tsbts.ErasAdjoint(n, 0.01, eras) as ea:
        rT = ea.forward(m, r, v)[0]
        np.testing.assert_array_equal(rT, st["r"])
        L, gr, gv, gm = ea.loss_grad(m, r, v)

        def loss(m_, r_, v_):
            x = ea.forward(m_, r_, v_)[0]
            return float((m_ * (x * x).sum(1)).sum() / m_.sum())
        h = 1e-6
        for which, g in (("r", gr), ("v", gv), ("m", gm)):
            d = rng.standard_normal(g.shape)
            args = dict(m_=m, r_=r, v_=v)
            p, q = dict(args), dict(args)
            p[which + "_"] = args[which + "_"] + h * d
            q[which + "_"] = args[which + "_"] - h * d
            fd = (loss(**p) - loss(**q)) / (2 * h)
            an = float((g * d).sum())
            assert abs(fd - an) <= 1e-6 * np.linalg.norm(g) * \
                np.linalg.norm(d), (which, fd, an)
