"""Pins of the oracle's converged iteration (the paper fixes the pass count;
an era that stops iterating once a pass repeats the previous one extends
reading R15).

With conv_tol > 0 an era stops after pass p >= 1 when pass p took the same
block steps as pass p - 1 and its era-end positions are within conv_tol of
pass p - 1's; n_iter bounds the passes.
"""
import numpy as np

import oracle
from paper_1205_2288_gb300 import inputs


def run(m, r, v, t_end, **kw):
    s = oracle.Sim(m, r, v, log=True, **kw)
    s.run(t_end)
    return s


def passes_schedules(sched, era):
    """Per pass of one era: the list of (block time, sorted active set)."""
    off = np.concatenate([[0], np.cumsum(sched["n_act"])])
    out = {}
    for k in np.flatnonzero(sched["era"] == era):
        p = int(sched["pass_"][k])
        out.setdefault(p, []).append(
            (int(sched["tau"][k]),
             tuple(np.sort(sched["idx"][off[k]:off[k + 1]]))))
    return [out[p] for p in sorted(out)]


def test_shared_step_converges_after_the_second_pass():
    """Every body is active at every step, so pass 1 repeats pass 0
    exactly (Taylor prediction, the same steps): the era stops after two
    passes and its state is the one-pass state."""
    m, r, v = inputs.plummer(40, 2)
    kw = dict(eps=0.05, eta=0.1, dt_max=2.0 ** -7, era_mode=0, era_log2=4,
              k_max=7)
    a = run(m, r, v, 0.25, n_iter=6, conv_tol=1e-300, **kw)
    b = run(m, r, v, 0.25, n_iter=1, **kw)
    st = a.stats()
    assert st["passes"] == 2 * st["eras"]
    for key in ("r", "v", "a", "tau", "dt"):
        np.testing.assert_array_equal(a.state()[key], b.state()[key])


def test_stops_at_the_first_repeated_schedule():
    m, r, v = inputs.plummer(120, 6)
    kw = dict(eps=0.02, eta=0.05, dt_max=1 / 8, era_mode=0, era_log2=3,
              k_max=20)
    fixed = run(m, r, v, 0.125, n_iter=6, **kw)
    sch = passes_schedules(fixed.schedule(), 0)
    want = next((p + 1 for p in range(1, len(sch)) if sch[p] == sch[p - 1]),
                len(sch))
    # a tolerance the positions always meet: the schedule decides
    conv = run(m, r, v, 0.125, n_iter=6, conv_tol=1e9, **kw)
    assert conv.stats()["passes"] == want
    ref = run(m, r, v, 0.125, n_iter=want, **kw)
    for key in ("r", "v", "a", "tau", "dt"):
        np.testing.assert_array_equal(conv.state()[key], ref.state()[key])


def test_tight_tolerance_runs_every_pass():
    m, r, v = inputs.plummer(120, 6)
    kw = dict(eps=0.02, eta=0.05, dt_max=1 / 8, era_mode=1, era_log2=3,
              k_max=20, n_iter=4)
    conv = run(m, r, v, 0.125, conv_tol=1e-300, **kw)
    fixed = run(m, r, v, 0.125, **kw)
    assert conv.stats()["passes"] == fixed.stats()["passes"]
    for key in ("r", "v", "tau", "dt"):
        np.testing.assert_array_equal(conv.state()[key], fixed.state()[key])
