"""Parity of the CUDA integrator (Alg. 2, Alg. 3) with the FP64 oracle,
through the C ABI (tsbts_init / tsbts_step_era / tsbts_energy /
tsbts_state / tsbts_schedule_*).

FP64 with ascending-j sums reproduces the oracle bit for bit: the block
schedule (block times, active sets, new steps), the final state and the
energy. The mixed path is held to the energy bar: its relative energy
error at most twice the oracle's (plus a floor at the FP32 force noise).
"""
import numpy as np
import pytest

from paper_1205_2288_gb300 import inputs, tsbts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def run_pair(orc, m, r, v, t_end, *, log=True, gpu_kw=None, **kw):
    """Run the oracle and the GPU on the same inputs and settings."""
    gpu_kw = gpu_kw or {}
    o = orc.Sim(m, r, v, log=log, **kw)
    e0 = o.energy()
    o.run(t_end)
    g = tsbts.Simulation(m, r, v, **kw, **gpu_kw)
    g0 = g.energy()
    if log:
        g.schedule_log(4_000_000)
    g.step_era(t_end)
    return o, g, e0, g0


def sorted_schedule(s):
    """Active bodies sorted by index within each block step."""
    off = np.concatenate([[0], np.cumsum(s["n_act"])]).astype(np.int64)
    idx = s["idx"].copy()
    dt = s["dt"].copy()
    for k in range(len(off) - 1):
        a, b = off[k], off[k + 1]
        o = np.argsort(idx[a:b], kind="stable")
        idx[a:b] = idx[a:b][o]
        dt[a:b] = dt[a:b][o]
    return idx, dt


def assert_same_schedule(o, g):
    so, sg = o.schedule(), g.schedule()
    assert sg["dropped"] == 0
    for key in ("era", "pass_", "tau", "n_act"):
        np.testing.assert_array_equal(so[key], sg[key], err_msg=key)
    gi, gd = sorted_schedule(sg)
    np.testing.assert_array_equal(so["idx"], gi)
    np.testing.assert_array_equal(so["dt"], gd)


def assert_same_state(o, g):
    so, sg = o.state(), g.state()
    for key in ("r", "v", "a", "tau", "dt"):
        np.testing.assert_array_equal(so[key], sg[key], err_msg=key)


CFG1 = dict(eps=0.01, eta=0.01, dt_max=1 / 8, n_iter=3, era_mode=0,
            era_log2=3, k_max=20)


def test_config1_plummer256_bit_exact(orc):
    """Plummer n = 256, eps = 0.01, eta = 0.01, dt = 2^-k (k = 3..20),
    fixed era 1/8, three passes, t = 0..1, FP64."""
    m, r, v = inputs.plummer(256, 0)
    o, g, e0, g0 = run_pair(orc, m, r, v, 1.0, **CFG1)
    assert g0 == e0
    assert_same_schedule(o, g)
    assert_same_state(o, g)
    assert g.energy() == o.energy()
    st = g.stats()
    ost = o.stats()
    assert st["block_steps"] == ost["block_steps"]
    assert st["interactions"] == ost["interactions"]
    assert st["eras"] == 8 and st["passes"] == 24


@pytest.mark.parametrize("graph_steps", [0, 2, 64])
def test_launch_modes_agree(orc, graph_steps):
    m, r, v = inputs.plummer(128, 3)
    kw = dict(CFG1, eta=0.03)
    o, g, _, _ = run_pair(orc, m, r, v, 0.25, gpu_kw=dict(graph_steps=graph_steps),
                          **kw)
    assert_same_schedule(o, g)
    assert_same_state(o, g)


@pytest.mark.parametrize("n_iter", [1, 2, 5])
def test_iteration_counts(orc, n_iter):
    m, r, v = inputs.plummer(200, 5)
    kw = dict(CFG1, eta=0.05, n_iter=n_iter)
    o, g, _, _ = run_pair(orc, m, r, v, 0.25, **kw)
    assert_same_schedule(o, g)
    assert_same_state(o, g)


def test_dynamic_era_bit_exact(orc):
    """Alg. 3 (eras from the device's block-time extrema and R11), ragged
    n. Bodies excluded by an era end are covered by the fixed-era resume
    test, where the era is shorter than the largest step."""
    m, r, v = inputs.plummer(1000, 7)
    kw = dict(eps=1 / 256, eta=0.02, dt_max=1 / 8, n_iter=3, era_mode=1,
              era_log2=3, k_max=20)
    o, g, _, _ = run_pair(orc, m, r, v, 0.375, **kw)
    assert o.stats()["eras"] == g.stats()["eras"]
    assert_same_schedule(o, g)
    assert_same_state(o, g)
    assert g.energy() == o.energy()


def test_unequal_masses_and_shared_step(orc):
    m = inputs.salpeter_masses(300, 11)
    _, r, v = inputs.plummer(300, 12, masses=m)
    kw = dict(eps=4 / 300, eta=0.02, dt_max=1 / 16, n_iter=3, era_mode=0,
              era_log2=4, k_max=20)
    o, g, _, _ = run_pair(orc, m, r, v, 0.25, **kw)
    assert_same_schedule(o, g)
    assert_same_state(o, g)
    # shared step k_min = k_max: every body active at every block step
    kw = dict(eps=0.02, eta=0.1, dt_max=2.0 ** -7, n_iter=3, era_mode=0,
              era_log2=3, k_max=7)
    o, g, _, _ = run_pair(orc, m, r, v, 0.25, **kw)
    assert_same_state(o, g)
    assert (g.schedule()["n_act"] == 300).all()


def test_history_growth_reruns_the_era(orc):
    """An era longer than the history buffer holds: the engine grows the
    buffers and re-runs the era; the result is unchanged."""
    m, r, v = inputs.plummer(2048, 13)
    kw = dict(eps=0.01, eta=0.05, dt_max=1 / 8, n_iter=2, era_mode=0,
              era_log2=0, k_max=20)
    o, g, _, _ = run_pair(orc, m, r, v, 1.0, log=False, **kw)
    assert g.stats()["era_restarts"] >= 1
    assert_same_state(o, g)
    # only the kept run of a re-run era is counted
    assert g.stats()["block_steps"] == o.stats()["block_steps"]
    assert g.stats()["interactions"] == o.stats()["interactions"]
    assert g.stats()["passes"] == o.stats()["passes"]


def test_fp64_jsplit_path_tracks_oracle(orc):
    """FP64 with the j-split (summation order differs from the oracle)."""
    m, r, v = inputs.plummer(1500, 17)
    kw = dict(eps=0.01, eta=0.02, dt_max=1 / 8, n_iter=3, era_mode=1,
              era_log2=3, k_max=20)
    o, g, e0, g0 = run_pair(orc, m, r, v, 0.125, log=False,
                            gpu_kw=dict(exact_order=0), **kw)
    E0 = sum(e0)
    de_o = abs(sum(o.energy()) / E0 - 1)
    de_g = abs(sum(g.energy()) / E0 - 1)
    assert de_g <= 2 * de_o + 1e-12
    np.testing.assert_allclose(g.state()["r"], o.state()["r"], atol=1e-9)


@pytest.mark.parametrize("era_mode", [0, 1])
def test_mixed_precision_energy_within_twice_oracle(orc, era_mode):
    m, r, v = inputs.plummer(2048, 21)
    kw = dict(eps=1 / 256, eta=0.01, dt_max=1 / 8, n_iter=3,
              era_mode=era_mode, era_log2=3, k_max=20)
    o, g, e0, _ = run_pair(orc, m, r, v, 0.25, log=False,
                           gpu_kw=dict(precision=tsbts.TSBTS_MIXED), **kw)
    E0 = sum(e0)
    de_o = abs(sum(o.energy()) / E0 - 1)
    de_g = abs(sum(g.energy()) / E0 - 1)
    assert de_g <= 2 * de_o + 1e-7, (de_g, de_o)
    # the trajectories stay close over a quarter time unit
    assert np.abs(g.state()["r"] - o.state()["r"]).max() < 1e-4


def test_argument_and_state_errors():
    m, r, v = inputs.plummer(16, 0)
    cfg = tsbts.tsbts_config_default()
    ctx = tsbts.tsbts_create(cfg)
    try:
        with pytest.raises(tsbts.TsbtsError) as e:
            tsbts.tsbts_step_era(ctx, 0.5)
        assert e.value.code == tsbts.TSBTS_ERR_STATE
        for bad in (dict(eps=-1.0), dict(eta=0.0), dict(dt_max=0.3),
                    dict(dt_max=2.0)):
            kw = dict(eps=0.01, eta=0.01, dt_max=0.125)
            kw.update(bad)
            with pytest.raises(tsbts.TsbtsError) as e:
                tsbts.tsbts_init(ctx, m, r, v, **kw)
            assert e.value.code == tsbts.TSBTS_ERR_ARG
        tsbts.tsbts_init(ctx, m, r, v, 0.01, 0.01, 0.125)
        with pytest.raises(tsbts.TsbtsError) as e:
            tsbts.tsbts_step_era(ctx, 1.0 / 3.0)   # not on the tick grid
        assert e.value.code == tsbts.TSBTS_ERR_ARG
        tsbts.tsbts_step_era(ctx, 0.125)
        with pytest.raises(tsbts.TsbtsError) as e:
            tsbts.tsbts_step_era(ctx, 0.0625)      # in the past
        assert e.value.code == tsbts.TSBTS_ERR_ARG
        assert tsbts.tsbts_state(ctx, 16)["t"] == 0.125
    finally:
        tsbts.tsbts_destroy(ctx)
    # non-finite input is rejected and poisons the context
    ctx = tsbts.tsbts_create(cfg)
    try:
        r2 = r.copy()
        r2[3, 1] = np.nan
        with pytest.raises(tsbts.TsbtsError) as e:
            tsbts.tsbts_init(ctx, m, r2, v, 0.01, 0.01, 0.125)
        assert e.value.code == tsbts.TSBTS_ERR_NONFINITE
        with pytest.raises(tsbts.TsbtsError) as e:
            tsbts.tsbts_init(ctx, m, r, v, 0.01, 0.01, 0.125)
        assert e.value.code == tsbts.TSBTS_ERR_STATE
    finally:
        tsbts.tsbts_destroy(ctx)


def test_repeatable_and_deterministic():
    m, r, v = inputs.plummer(3000, 23)
    out = []
    for _ in range(2):
        g = tsbts.Simulation(m, r, v, eps=0.01, eta=0.02, dt_max=1 / 8,
                             precision=tsbts.TSBTS_MIXED, era_mode=1)
        g.step_era(0.0625)
        out.append(g.state())
        g.close()
    for key in ("r", "v", "a", "tau", "dt"):
        np.testing.assert_array_equal(out[0][key], out[1][key])


@pytest.mark.parametrize("graph_steps", [0, 16])
def test_force_timing_counts_real_steps(orc, graph_steps):
    """With timing on, every block step's force launch is timed once and
    the results do not change."""
    m, r, v = inputs.plummer(512, 29)
    kw = dict(CFG1, eta=0.03)
    o = orc.Sim(m, r, v, **kw)
    o.run(0.25)
    g = tsbts.Simulation(m, r, v, graph_steps=graph_steps, **kw)
    g.set_timing(1)
    g.step_era(0.25)
    st = g.stats()
    assert st["force_launches"] == st["block_steps"] == o.stats()["block_steps"]
    assert st["force_interactions"] == st["interactions"]
    assert st["force_ms"] > 0
    assert st["kernel_launches"] >= 3 * st["block_steps"]
    assert_same_state(o, g)
    g.close()
    # a sample: every third chunk of steps is timed, the rest run without
    # events; the results stay the same
    g = tsbts.Simulation(m, r, v, graph_steps=graph_steps, **kw)
    g.set_timing(3)
    g.step_era(0.25)
    st = g.stats()
    assert 0 < st["force_launches"] < st["block_steps"]
    assert 0 < st["force_interactions"] < st["interactions"]
    assert st["force_ms"] > 0
    assert_same_state(o, g)
    g.close()


@pytest.mark.parametrize("era_mode,tol", [(0, 1e9), (1, 1e9), (0, 1e-6),
                                          (1, 1e-300)])
def test_converged_iteration_bit_exact(orc, era_mode, tol):
    """Reading R15 (converged iteration): an era stops after pass p >= 1
    once pass p took the same block steps as pass p - 1 and its end
    positions are within conv_tol of them, at most n_iter passes. In FP64
    the GPU takes the same decisions as the oracle, era by era: the same
    passes, schedule and state, bit for bit. tol = 1e9 lets the schedule
    decide; 1e-300 cannot be met, so every pass runs."""
    m, r, v = inputs.plummer(160, 41)
    kw = dict(eps=0.02, eta=0.05, dt_max=1 / 8, n_iter=6, era_mode=era_mode,
              era_log2=3, k_max=20, conv_tol=tol)
    o, g, _, _ = run_pair(orc, m, r, v, 0.375, **kw)
    assert g.stats()["passes"] == o.stats()["passes"]
    if tol == 1e-300:
        assert o.stats()["passes"] == 6 * o.stats()["eras"]
    assert_same_schedule(o, g)
    assert_same_state(o, g)
    assert g.energy() == o.energy()


def test_shared_step_converges_after_two_passes():
    """Every body active at every step: pass 1 repeats pass 0 exactly, so
    with any tolerance the era stops after two passes and the state is the
    one-pass state (as the oracle's pin shows)."""
    m, r, v = inputs.plummer(40, 2)
    kw = dict(eps=0.05, eta=0.1, dt_max=2.0 ** -7, era_mode=0, era_log2=4,
              k_max=7)
    a = tsbts.Simulation(m, r, v, n_iter=6, conv_tol=1e-300, **kw)
    a.step_era(0.25)
    b = tsbts.Simulation(m, r, v, n_iter=1, **kw)
    b.step_era(0.25)
    st = a.stats()
    assert st["passes"] == 2 * st["eras"]
    sa, sb = a.state(), b.state()
    for key in ("r", "v", "a", "tau", "dt"):
        np.testing.assert_array_equal(sa[key], sb[key])


def test_pass_step_limit_gives_timeout_and_poisons():
    """The host watchdog of the block-step loop: a pass that takes more
    block steps than max_pass_steps stops with TSBTS_ERR_TIMEOUT (no GPU
    wait is involved: the loop's chunks return and the host counts them),
    the context refuses further calls, and a new context on the same
    device runs normally."""
    m, r, v = inputs.plummer(256, 3)
    kw = dict(eps=0.01, eta=0.01, dt_max=1 / 8, n_iter=3, era_mode=0,
              era_log2=3, k_max=20)
    g = tsbts.Simulation(m, r, v, max_pass_steps=8, graph_steps=16, **kw)
    with pytest.raises(tsbts.TsbtsError) as e:
        g.step_era(0.125)
    assert e.value.code == tsbts.TSBTS_ERR_TIMEOUT
    with pytest.raises(tsbts.TsbtsError) as e:
        g.energy()
    assert e.value.code == tsbts.TSBTS_ERR_STATE
    g.close()
    ok = tsbts.Simulation(m, r, v, **kw)
    ok.step_era(0.125)
    assert ok.stats()["block_steps"] > 8
    ok.close()


def test_step_underflow_count_matches_oracle(orc):
    """Reading R10: steps below 2^-k_max are clamped to one tick and
    counted; with k_max = 8 a tight Plummer cluster underflows, and the
    GPU counts the same clamps as the oracle (FP64, bit-exact run)."""
    m, r, v = inputs.plummer(96, 12)
    kw = dict(eps=0.002, eta=0.05, dt_max=1 / 8, n_iter=3, era_mode=0,
              era_log2=3, k_max=8)
    o, g, _, _ = run_pair(orc, m, r, v, 0.25, **kw)
    assert o.stats()["underflow"] > 0
    assert g.stats()["dt_underflow"] == o.stats()["underflow"]
    assert_same_state(o, g)
