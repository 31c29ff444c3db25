"""Parity of the CUDA frozen-schedule adjoint (tsbts_adjoint_*) with the
FP64 oracle (replay and reverse mode of reading R14).

FP64 with ascending-j force sums replays the schedule bit for bit. The
reverse sweep sums its pair terms in another order than the oracle, so its
gradients are held to a relative bound; checkpointed and fully taped
sweeps are bit-identical. The mixed path is held to the FP32 pair-term
accuracy. At the full size (Plummer n = 8192, eps = 0.01, one era 0..1/4)
the FP64 gradient is checked against central differences of the FP64
replay, and the mixed gradient against the FP64 one.
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


def oracle_schedule(m, r, v, *, eps, eta=0.02, t_end=0.125, era_log2=3,
                    n_iter=3):
    s = oracle.Sim(m, r, v, eps=eps, eta=eta, dt_max=1 / 8, n_iter=n_iter,
                   era_mode=0, era_log2=era_log2, k_max=K_MAX, log=True)
    s.run(t_end)
    return oracle.final_pass(s.schedule(), 0)


def rel(a, b):
    """max |a - b| over max |b|"""
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def case600():
    m = inputs.salpeter_masses(600, 31)
    _, r, v = inputs.plummer(600, 32, masses=m)
    r = r + np.array([0.2, -0.1, 0.3])
    eps = 0.01
    sched = oracle_schedule(m, r, v, eps=eps)
    L, gr, gv, gm = oracle.loss_grad(m, r, v, eps, K_MAX, sched)
    rT, vT = oracle.replay(m, r, v, eps, K_MAX, sched)
    return dict(m=m, r=r, v=v, eps=eps, sched=sched, L=L, gr=gr, gv=gv,
                gm=gm, rT=rT, vT=vT)


def test_fp64_replay_bit_exact(case600):
    c = case600
    with tsbts.Adjoint(600, c["eps"], c["sched"]) as adj:
        rT, vT = adj.forward(c["m"], c["r"], c["v"])
    np.testing.assert_array_equal(rT, c["rT"])
    np.testing.assert_array_equal(vT, c["vT"])


@pytest.mark.parametrize("K", [0, 1, 7, 50])
def test_fp64_loss_gradient_matches_oracle(case600, K):
    c = case600
    with tsbts.Adjoint(600, c["eps"], c["sched"], checkpoint_every=K) as adj:
        L, gr, gv, gm = adj.loss_grad(c["m"], c["r"], c["v"])
        st = adj.stats()
    assert abs(L / c["L"] - 1) < 1e-14
    assert rel(gr, c["gr"]) < 1e-10, rel(gr, c["gr"])
    assert rel(gv, c["gv"]) < 1e-10, rel(gv, c["gv"])
    assert rel(gm, c["gm"]) < 1e-10, rel(gm, c["gm"])
    n_steps = len(c["sched"][0])
    if K == 0 or K >= n_steps:
        assert st["checkpoints"] == 0
        assert st["tape_entries"] == st["entries"]
    else:
        assert st["checkpoints"] == -(-n_steps // K)
        assert st["tape_entries"] < st["entries"]
        # recomputed forward steps are counted in the reverse sweep
        assert st["pairs_backward"] == (3 * st["entries"] + 2 * 600) * 600


def test_checkpointing_is_bit_identical(case600):
    c = case600
    out = []
    for K in (0, 3, 64):
        with tsbts.Adjoint(600, c["eps"], c["sched"], checkpoint_every=K,
                           precision=tsbts.TSBTS_MIXED) as adj:
            out.append(adj.loss_grad(c["m"], c["r"], c["v"]))
    for o in out[1:]:
        assert o[0] == out[0][0]
        for a, b in zip(o[1:], out[0][1:]):
            np.testing.assert_array_equal(a, b)


def test_graph_and_stream_launches_agree(case600):
    c = case600
    out = []
    for K in (0, 16):
        for graph_steps in (0, 32):
            with tsbts.Adjoint(600, c["eps"], c["sched"], checkpoint_every=K,
                               precision=tsbts.TSBTS_MIXED,
                               graph_steps=graph_steps) as adj:
                out.append(adj.loss_grad(c["m"], c["r"], c["v"]))
                # a second call replays the captured graphs
                again = adj.loss_grad(c["m"], c["r"], c["v"])
                st = adj.stats()
            for a, b in zip(again[1:], out[-1][1:]):
                np.testing.assert_array_equal(a, b)
            assert st["kernel_launches"] > 0
    for o in out[1:]:
        for a, b in zip(o[1:], out[0][1:]):
            np.testing.assert_array_equal(a, b)


def test_fp64_general_vjp_matches_oracle(case600):
    c = case600
    rng = np.random.default_rng(5)
    gr_T = rng.standard_normal((600, 3))
    gv_T = rng.standard_normal((600, 3))
    want = oracle.replay_vjp(c["m"], c["r"], c["v"], c["eps"], K_MAX,
                             c["sched"], gr_T, gv_T)
    with tsbts.Adjoint(600, c["eps"], c["sched"]) as adj:
        adj.forward(c["m"], c["r"], c["v"])
        got = adj.vjp(gr_T, gv_T)
        # only a velocity cotangent
        got_v = adj.vjp(None, gv_T)
    for a, b in zip(got, want):
        assert rel(a, b) < 1e-10, rel(a, b)
    want_v = oracle.replay_vjp(c["m"], c["r"], c["v"], c["eps"], K_MAX,
                               c["sched"], np.zeros_like(gr_T), gv_T)
    for a, b in zip(got_v, want_v):
        assert rel(a, b) < 1e-10


def test_mixed_gradient_within_fp32_accuracy(case600):
    c = case600
    with tsbts.Adjoint(600, c["eps"], c["sched"],
                       precision=tsbts.TSBTS_MIXED) as adj:
        rT, vT = adj.forward(c["m"], c["r"], c["v"])
        L, gr, gv, gm = adj.loss_grad(c["m"], c["r"], c["v"])
    assert np.abs(rT - c["rT"]).max() < 1e-6
    assert abs(L / c["L"] - 1) < 1e-7
    for a, b in ((gr, c["gr"]), (gv, c["gv"]), (gm, c["gm"])):
        assert rel(a, b) < 1e-4, rel(a, b)


def test_ragged_sizes_and_tiny_sets():
    """n not a multiple of any tile, single-body steps, every body at once."""
    for n in (1, 2, 37, 129):
        m, r, v = inputs.plummer(max(n, 2), 40 + n)
        m, r, v = m[:n], r[:n], v[:n]
        steps = np.array([1 << 12, 1 << 13, 3 << 12, 1 << 14], np.int64)
        sets = [np.arange(n), np.array([n - 1]), np.arange(0, n, 2),
                np.arange(n)]
        off = np.concatenate([[0], np.cumsum([len(x) for x in sets])])
        sched = (steps, off.astype(np.int64),
                 np.concatenate(sets).astype(np.int32))
        rng = np.random.default_rng(n)
        gr_T = rng.standard_normal((n, 3))
        want_rT, want_vT = oracle.replay(m, r, v, 0.05, K_MAX, sched)
        want = oracle.replay_vjp(m, r, v, 0.05, K_MAX, sched, gr_T,
                                 np.zeros_like(gr_T))
        for prec in (tsbts.TSBTS_FP64, tsbts.TSBTS_MIXED):
            with tsbts.Adjoint(n, 0.05, sched, precision=prec) as adj:
                rT, vT = adj.forward(m, r, v)
                got = adj.vjp(gr_T)
            if prec == tsbts.TSBTS_FP64:
                np.testing.assert_array_equal(rT, want_rT)
                np.testing.assert_array_equal(vT, want_vT)
            tol = 1e-10 if prec == tsbts.TSBTS_FP64 else 1e-4
            for a, b in zip(got, want):
                if np.abs(b).max() == 0:
                    assert np.abs(a).max() == 0
                else:
                    assert rel(a, b) < tol, (n, prec, rel(a, b))


def test_empty_schedule_and_idle_body():
    m, r, v = inputs.plummer(12, 5)
    empty = (np.zeros(0, np.int64), np.zeros(1, np.int64),
             np.zeros(0, np.int32))
    with tsbts.Adjoint(12, 0.05, empty) as adj:
        rT, vT = adj.forward(m, r, v)
        g_r0, g_v0, g_m = adj.vjp(np.ones((12, 3)), np.full((12, 3), 2.0))
    np.testing.assert_array_equal(rT, r)
    np.testing.assert_array_equal(vT, v)
    np.testing.assert_array_equal(g_r0, 1.0)
    np.testing.assert_array_equal(g_v0, 2.0)
    np.testing.assert_array_equal(g_m, 0.0)
    sched = (np.array([1 << 14, 1 << 15], np.int64),
             np.array([0, 3, 7], np.int64),
             np.array([1, 2, 3, 1, 2, 3, 4], np.int32))
    gr_T = np.zeros((12, 3))
    gr_T[0] = [1.0, -2.0, 0.5]
    with tsbts.Adjoint(12, 0.05, sched) as adj:
        adj.forward(m, r, v)
        g_r0, g_v0, g_m = adj.vjp(gr_T)
    np.testing.assert_array_equal(g_r0, gr_T)
    np.testing.assert_array_equal(g_v0, 0.0)
    np.testing.assert_array_equal(g_m, 0.0)


def test_schedule_and_state_errors():
    m, r, v = inputs.plummer(8, 1)
    bad = [
        ((np.array([4, 4], np.int64), np.array([0, 1, 2]), np.array([0, 1])),
         "ticks"),
        ((np.array([0], np.int64), np.array([0, 1]), np.array([0])), "zero"),
        ((np.array([4], np.int64), np.array([0, 0]), np.zeros(0)), "empty"),
        ((np.array([4], np.int64), np.array([0, 1]), np.array([8])), "range"),
        ((np.array([4], np.int64), np.array([0, 2]), np.array([3, 3])),
         "repeat"),
    ]
    for sched, what in bad:
        cfg = tsbts.tsbts_config_default()
        ctx = tsbts.tsbts_create(cfg)
        try:
            with pytest.raises(tsbts.TsbtsError) as e:
                tsbts.tsbts_adjoint_init(ctx, 8, 0.01, sched)
            assert e.value.code == tsbts.TSBTS_ERR_ARG, what
        finally:
            tsbts.tsbts_destroy(ctx)
    good = (np.array([4], np.int64), np.array([0, 2], np.int64),
            np.array([1, 3], np.int32))
    with tsbts.Adjoint(8, 0.01, good) as adj:
        with pytest.raises(tsbts.TsbtsError) as e:
            adj.vjp(np.ones((8, 3)))
        assert e.value.code == tsbts.TSBTS_ERR_STATE
        r2 = r.copy()
        r2[2, 0] = np.inf
        with pytest.raises(tsbts.TsbtsError) as e:
            adj.forward(m, r2, v)
        assert e.value.code == tsbts.TSBTS_ERR_NONFINITE


def test_torch_autograd_replay_and_loss():
    import torch
    from paper_1205_2288_gb300 import autograd as ag
    m, r, v = inputs.plummer(10, 8)
    sched = oracle_schedule(m, r, v, eps=0.05, eta=0.2, t_end=2.0 ** -5,
                            era_log2=5)
    dev = torch.device("cuda:0")
    adj = ag.make_adjoint(10, 0.05, sched)
    try:
        t = lambda x: torch.tensor(x, dtype=torch.float64, device=dev,
                                   requires_grad=True)
        r0, v0, m0 = t(r), t(v), t(m)

        def f(r0, v0, m0):
            rT, vT = ag.replay(adj, r0, v0, m0)
            return rT, vT
        assert torch.autograd.gradcheck(f, (r0, v0, m0), eps=1e-6,
                                        atol=1e-7, rtol=1e-5)
        # the fused loss agrees with the loss of the differentiable replay
        L = ag.era_loss(adj, r0, v0, m0)
        L.backward()
        g1 = [x.grad.clone() for x in (r0, v0, m0)]
        for x in (r0, v0, m0):
            x.grad = None
        rT, _ = ag.replay(adj, r0, v0, m0)
        L2 = (m0 * (rT * rT).sum(1)).sum() / m0.sum()
        L2.backward()
        assert abs(L.item() - L2.item()) <= 1e-14 * abs(L.item())
        for a, x in zip(g1, (r0, v0, m0)):
            torch.testing.assert_close(a, x.grad, rtol=1e-10, atol=1e-13)
        # a backward after another forward replays its own inputs again
        for x in (r0, v0, m0):
            x.grad = None
        rT, vT = ag.replay(adj, r0, v0, m0)
        (rT.sum() + vT.sum()).backward()
        want = [x.grad.clone() for x in (r0, v0, m0)]
        for x in (r0, v0, m0):
            x.grad = None
        rT, vT = ag.replay(adj, r0, v0, m0)
        ag.replay(adj, r0.detach() + 0.1, v0.detach(), m0.detach())
        (rT.sum() + vT.sum()).backward()
        for a, x in zip(want, (r0, v0, m0)):
            torch.testing.assert_close(x.grad, a, rtol=0, atol=0)
    finally:
        adj.close()


@pytest.fixture(scope="module")
def config5():
    """Plummer n = 8192, eps = 0.01, eta = 0.01, one era 0..1/4 (fixed era
    2^-2, dt_max = 1/8, three passes); the final pass's schedule from the
    mixed GPU integrator."""
    m, r, v = inputs.plummer(8192, 0)
    sim = tsbts.Simulation(m, r, v, eps=0.01, eta=0.01, dt_max=1 / 8,
                           n_iter=3, era_mode=0, era_log2=2,
                           precision=tsbts.TSBTS_MIXED)
    sim.schedule_log(40_000_000)
    sim.step_era(0.25)
    sched = tsbts.final_pass_schedule(sim.schedule(), 0)
    sim.close()
    return dict(m=m, r=r, v=v, sched=sched)


def test_config5_fp64_gradient_matches_central_differences(config5):
    c = config5
    rng = np.random.default_rng(9)
    # j-split FP64 sums: deterministic, so central differences of the
    # replay are exact up to FP64 rounding and truncation
    with tsbts.Adjoint(8192, 0.01, c["sched"], checkpoint_every=64,
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


def test_config5_mixed_gradient_tracks_fp64(config5):
    c = config5
    if "fp64" not in c:
        pytest.skip("needs the FP64 gradient")
    with tsbts.Adjoint(8192, 0.01, c["sched"],
                       precision=tsbts.TSBTS_MIXED) as adj:
        L, gr, gv, gm = adj.loss_grad(c["m"], c["r"], c["v"])
        st = adj.stats()
    L0, gr0, gv0, gm0 = c["fp64"]
    assert abs(L / L0 - 1) < 1e-7
    for a, b in ((gr, gr0), (gv, gv0), (gm, gm0)):
        assert rel(a, b) < 1e-4, rel(a, b)
    assert st["pairs_backward"] == 2 * (st["entries"] + 8192) * 8192
