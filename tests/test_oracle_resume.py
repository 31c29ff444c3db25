"""Pins of the oracle's resume at an era end (checkpoint/resume; era ends are
the method's synchronisation points, Alg. 2 steps 2 and 10).

An era starts from (m, r, v, a, dts, tau, dt) and the system time: its
first pass predicts with Eq. 2 alone and later passes interpolate records of
the same era. So an integration stopped at an era end and restarted from
that state in a new simulation must continue bit for bit like the
uninterrupted run, whatever the new simulation was created from.
"""
import numpy as np
import pytest

import oracle
from paper_1205_2288_gb300 import inputs

K_MAX = 20
KEYS = ("r", "v", "a", "tau", "dt", "dts")


def make(m, r, v, **kw):
    return oracle.Sim(m, r, v, log=True, k_max=K_MAX, **kw)


def cluster(n=96, seed=31):
    m = inputs.salpeter_masses(n, seed)
    _, r, v = inputs.plummer(n, seed + 1, masses=m)
    return m, r, v


CASES = {
    "fixed": dict(eps=0.02, eta=0.03, dt_max=1 / 8, era_mode=0, era_log2=4,
                  n_iter=3),
    "dynamic": dict(eps=0.02, eta=0.03, dt_max=1 / 16, era_mode=1, n_iter=3),
    "converged": dict(eps=0.02, eta=0.03, dt_max=1 / 16, era_mode=1, n_iter=5,
                      conv_tol=1e-12),
}


def era_ends(sim):
    _, te = sim.eras()
    return [int(t) * 2.0 ** -K_MAX for t in te]


def steps_after(sched, t_ticks):
    keep = sched["tau"] > t_ticks
    off = np.concatenate([[0], np.cumsum(sched["n_act"])])
    idx = [np.sort(sched["idx"][off[k]:off[k + 1]])
           for k in np.flatnonzero(keep)]
    return sched["pass_"][keep], sched["tau"][keep], idx


@pytest.mark.parametrize("case", sorted(CASES))
def test_resume_continues_bit_for_bit(case):
    kw = CASES[case]
    m, r, v = cluster()
    t2 = 0.25
    full = make(m, r, v, **kw)
    full.run(t2)
    ends = era_ends(full)
    t1 = ends[(len(ends) - 1) // 2]
    assert 0 < t1 < t2
    head = make(m, r, v, **kw)
    head.run(t1)
    st = head.state()
    # created from other bodies: set_state must replace all of them
    rng = np.random.default_rng(4)
    tail = make(2 * m, r + rng.standard_normal(r.shape),
                v - rng.standard_normal(v.shape), **kw)
    tail.set_state(t1, m, st)
    back = tail.state()
    for k in KEYS:
        np.testing.assert_array_equal(back[k], st[k], err_msg=k)
    np.testing.assert_array_equal(tail.energy(), head.energy())
    tail.run(t2)
    a, b = full.state(), tail.state()
    for k in KEYS:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    assert full.energy() == tail.energy()
    # the same block steps after the resume point, pass by pass
    sa = steps_after(full.schedule(), int(t1 * 2 ** K_MAX))
    sb = steps_after(tail.schedule(), int(t1 * 2 ** K_MAX))
    np.testing.assert_array_equal(sa[0], sb[0])
    np.testing.assert_array_equal(sa[1], sb[1])
    assert len(sa[2]) == len(sb[2]) > 0
    for x, y in zip(sa[2], sb[2]):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("case", ["fixed", "dynamic"])
def test_era_end_states_are_resumable(case):
    """Every era end of a run satisfies what set_state demands (steps powers
    of two up to dt_max, body times multiples of their steps, tau <= t <
    tau + dt). With a fixed era shorter than the largest step, bodies whose
    step overshoots the era end wait behind it."""
    m, r, v = cluster(64, 7)
    kw = CASES[case]
    probe = make(m, r, v, **kw)
    probe.run(0.25)
    dt_max_t = int(kw["dt_max"] * 2 ** K_MAX)
    waiting = 0
    for t in era_ends(probe)[:6]:
        s = make(m, r, v, **kw)
        s.run(t)
        st = s.state()
        T = int(t * 2 ** K_MAX)
        dt, tau = st["dt"], st["tau"]
        assert np.all((dt >= 1) & (dt <= dt_max_t) & ((dt & (dt - 1)) == 0))
        assert np.all(tau % dt == 0)
        assert np.all((tau <= T) & (T < tau + dt))
        assert np.all(st["dts"] > 0)
        waiting += int(np.sum(tau < T))
        s.set_state(t, m, st)  # accepted as it is
    assert waiting > 0 or case != "fixed"


@pytest.mark.parametrize("field,index,value", [
    ("dt", 3, 3),          # not a power of two
    ("dt", 5, 0),
    ("dt", 0, 2 ** K_MAX),  # above dt_max = 1/8
    ("tau", 2, "plus1"),    # not a multiple of its step
    ("tau", 4, "ahead"),    # ahead of the system time
    ("tau", 6, "behind"),   # its next time is not after the system time
    ("r", 1, np.nan),
    ("a", 7, np.inf),
    ("dts", 8, 0.0),
    ("dts", 9, np.nan),
])
def test_states_that_cannot_end_an_era_are_refused(field, index, value):
    m, r, v = cluster(32, 11)
    kw = CASES["fixed"]
    s = make(m, r, v, **kw)
    s.run(1 / 16)
    T = 2 ** K_MAX // 16
    st = s.state()
    bad = {k: x.copy() for k, x in st.items()}
    if value == "plus1":
        # tau <= T < tau + dt holds; only the multiple of the step fails
        bad["dt"][index] = 4
        bad["tau"][index] = T - 1
    elif value == "ahead":
        bad["dt"][index] = 1
        bad["tau"][index] = T + 1
    elif value == "behind":
        bad["dt"][index] = 1
        bad["tau"][index] = T - 1
    elif field in ("r", "a"):
        bad[field][index, 0] = value
    else:
        bad[field][index] = value
    with pytest.raises(ValueError):
        s.set_state(1 / 16, m, bad)
    after = s.state()
    for k in KEYS:
        np.testing.assert_array_equal(after[k], st[k], err_msg=k)
    with pytest.raises(ValueError):
        s.set_state(1 / 16 + 2.0 ** -30, m, st)  # not a whole tick
