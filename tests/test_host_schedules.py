"""Host helpers of the binding that need no GPU: splitting a schedule log
into the passes of an era (the adjoint's input) and concatenating passes
into the C ABI's layout. Each is checked against the oracle's own parser of
the same log format (written separately, in oracle/__init__.py) on a log
the oracle integrator writes, and on the properties the C ABI requires."""
import numpy as np
import pytest

import oracle
from paper_1205_2288_gb300 import inputs, tsbts


@pytest.fixture(scope="module")
def log():
    m, r, v = inputs.plummer(60, 3)
    s = oracle.Sim(m, r, v, eps=0.02, eta=0.05, dt_max=1 / 8, n_iter=3,
                   era_mode=1, era_log2=3, k_max=20, log=True)
    s.run(0.25)
    out = s.schedule()
    n_eras = len(np.unique(out["era"]))
    s.close()
    assert n_eras >= 2
    return out, n_eras


def same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(np.asarray(x), np.asarray(y))


def test_era_pass_schedules_match_the_oracles_parser(log):
    sched, n_eras = log
    for k in range(n_eras):
        ours = tsbts.era_pass_schedules(sched, k)
        theirs = oracle.era_passes(sched, k)
        assert len(ours) == len(theirs) == 3
        for a, b in zip(ours, theirs):
            same(a, b)


def test_final_pass_schedule_matches_the_oracles_parser(log):
    sched, n_eras = log
    for k in range(n_eras):
        same(tsbts.final_pass_schedule(sched, k), oracle.final_pass(sched, k))


def test_era_schedule_layout(log):
    """Concatenated passes: pass_off counts steps, step_off runs on across
    the passes, every step non-empty, ticks increasing within each pass,
    bodies ascending within each step; the same layout as the oracle's."""
    sched, _ = log
    passes = tsbts.era_pass_schedules(sched, 0)
    pass_off, tau, off, act = tsbts.era_schedule(passes)
    assert pass_off[0] == 0 and pass_off[-1] == len(tau) == len(off) - 1
    assert off[0] == 0 and off[-1] == len(act)
    assert (np.diff(off) > 0).all()
    for p in range(len(passes)):
        t = tau[pass_off[p]:pass_off[p + 1]]
        assert t[0] > 0 and (np.diff(t) > 0).all()
        np.testing.assert_array_equal(t, passes[p][0])
    for s in range(len(tau)):
        assert (np.diff(act[off[s]:off[s + 1]]) > 0).all()
    keep, _ = oracle._era_args(passes)
    o_tau, o_pass_off, o_off, o_act = keep
    for a, b in ((pass_off, o_pass_off), (tau, o_tau), (off, o_off),
                 (act, o_act)):
        np.testing.assert_array_equal(a, b)


def test_era_schedule_rejects_bad_passes():
    good = (np.array([4, 8]), np.array([0, 1, 2]), np.array([0, 1]))
    with pytest.raises(ValueError):
        tsbts.era_schedule([good, (np.array([4]), np.array([1, 2]),
                                   np.array([0]))])
    with pytest.raises(ValueError):
        tsbts.era_schedule([(np.array([4, 8]), np.array([0, 1]),
                             np.array([0]))])
