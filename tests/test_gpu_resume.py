"""Resume at an era end through the C ABI (tsbts_state +
tsbts_step_estimates, then tsbts_set_state): a run stopped at an era end
and restarted in a new context continues bit for bit like the
uninterrupted run (era ends carry the whole state, Alg. 2 steps 2 and 10),
and in FP64 it stays bit-identical to the oracle's resumed run.
"""
import numpy as np
import pytest

from paper_1205_2288_gb300 import inputs, tsbts

pytestmark = pytest.mark.gpu

K_MAX = 20
KEYS = ("r", "v", "a", "tau", "dt")


@pytest.fixture(scope="module", autouse=True)
def need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def era_end(orc, m, r, v, t2, **kw):
    o = orc.Sim(m, r, v, log=True, k_max=K_MAX, **kw)
    o.run(t2)
    _, te = o.eras()
    return int(te[(len(te) - 1) // 2]) * 2.0 ** -K_MAX, o


@pytest.mark.parametrize("precision,n,era_mode", [
    (tsbts.TSBTS_FP64, 256, 1),
    (tsbts.TSBTS_FP64, 300, 0),
    (tsbts.TSBTS_MIXED, 1000, 1),
])
def test_resume_continues_bit_for_bit(orc, precision, n, era_mode):
    m = inputs.salpeter_masses(n, 41)
    _, r, v = inputs.plummer(n, 42, masses=m)
    kw = dict(eps=0.02, eta=0.03, dt_max=1 / 8, n_iter=3, era_mode=era_mode,
              era_log2=4)
    t2 = 0.25
    t1, o_full = era_end(orc, m, r, v, t2, **kw)
    assert 0 < t1 < t2
    gk = dict(kw, k_max=K_MAX, precision=precision)
    full = tsbts.Simulation(m, r, v, **gk)
    full.step_era(t2)
    head = tsbts.Simulation(m, r, v, **gk)
    head.step_era(t1)
    ck = head.checkpoint()
    assert ck["t"] == t1
    rng = np.random.default_rng(5)
    tail = tsbts.Simulation(2 * m, r + rng.standard_normal(r.shape),
                            v + rng.standard_normal(v.shape), **gk)
    tail.set_state(ck)
    assert tail.energy() == head.energy()
    back = tail.checkpoint()
    for key in KEYS + ("m", "dts", "t"):
        np.testing.assert_array_equal(back[key], ck[key], err_msg=key)
    tail.step_era(t2)
    a, b = full.state(), tail.state()
    for key in KEYS:
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)
    assert tail.energy() == full.energy()
    if precision == tsbts.TSBTS_FP64:
        # the step estimates at the resume point and the end state are the
        # oracle's, bit for bit
        o_head = orc.Sim(m, r, v, k_max=K_MAX, **kw)
        o_head.run(t1)
        np.testing.assert_array_equal(ck["dts"], o_head.state()["dts"])
        so = o_full.state()
        for key in KEYS:
            np.testing.assert_array_equal(so[key], b[key], err_msg=key)
    for s in (full, head, tail):
        s.close()


def test_bad_states_are_refused_and_change_nothing():
    m, r, v = inputs.plummer(64, 3)
    g = tsbts.Simulation(m, r, v, eps=0.02, eta=0.03, dt_max=1 / 8,
                         era_mode=0, era_log2=4, k_max=K_MAX)
    g.step_era(1 / 16)
    ck = g.checkpoint()
    T = 2 ** K_MAX // 16
    cases = []
    for key, i, val in (("dt", 3, 3), ("dt", 4, 0), ("dt", 5, 2 ** K_MAX),
                        ("dts", 6, 0.0), ("dts", 7, np.nan)):
        bad = {k: np.copy(x) for k, x in ck.items()}
        bad[key][i] = val
        cases.append(bad)
    for tau, dt in ((T - 1, 4), (T + 1, 1), (T - 1, 1)):
        bad = {k: np.copy(x) for k, x in ck.items()}
        bad["tau"][9], bad["dt"][9] = tau, dt
        cases.append(bad)
    bad = {k: np.copy(x) for k, x in ck.items()}
    bad["r"][2, 1] = np.inf
    cases.append(bad)
    bad = dict(ck, t=ck["t"] + 2.0 ** -30)
    cases.append(bad)
    for bad in cases:
        with pytest.raises(tsbts.TsbtsError) as e:
            g.set_state(bad)
        assert e.value.code == tsbts.TSBTS_ERR_ARG
    after = g.checkpoint()
    for key in KEYS + ("m", "dts", "t"):
        np.testing.assert_array_equal(after[key], ck[key], err_msg=key)
    g.step_era(1 / 8)  # the context is still usable
    g.close()
