"""Pins of the oracle's integrator (Eq. 1-2, Alg. 1-3) against closed forms,
a textbook integrator it must reduce to, conservation laws, schedule
invariants and the paper's qualitative claims about iteration."""
import math

import numpy as np
import pytest

from paper_1205_2288_gb300 import inputs


def sim(orc, m, r, v, **kw):
    base = dict(eps=0.01, eta=0.05, dt_max=1 / 16, n_iter=3, era_mode=0,
                era_log2=4, k_max=20)
    base.update(kw)
    return orc.Sim(m, r, v, **base)


def kepler_solution(t, a, e, M):
    """Relative orbit x(t), v(t) of a Kepler ellipse starting at pericentre,
    from Kepler's equation solved by Newton iteration."""
    n = math.sqrt(M / a ** 3)
    Mean = n * t
    E = Mean if e < 0.8 else math.pi
    for _ in range(60):
        E -= (E - e * math.sin(E) - Mean) / (1 - e * math.cos(E))
    x = a * (math.cos(E) - e)
    y = a * math.sqrt(1 - e * e) * math.sin(E)
    Edot = n / (1 - e * math.cos(E))
    vx = -a * math.sin(E) * Edot
    vy = a * math.sqrt(1 - e * e) * math.cos(E) * Edot
    return np.array([x, y, 0.0]), np.array([vx, vy, 0.0])


def two_body(e, a=1.0, m1=0.5, m2=0.5):
    M = m1 + m2
    x, vx = kepler_solution(0.0, a, e, M)
    m = np.array([m1, m2])
    r = np.stack([-m2 / M * x, m1 / M * x])
    v = np.stack([-m2 / M * vx, m1 / M * vx])
    return m, r, v


@pytest.mark.parametrize("n_iter", [1, 3])
def test_kepler_eccentric_orbit(orc, n_iter):
    """Two bodies on an e = 0.5 ellipse with eps = 0 follow the closed-form
    Kepler orbit; the energy equals -m1 m2 / (2a)."""
    m, r, v = two_body(0.5)
    s = sim(orc, m, r, v, eps=0.0, eta=0.005, n_iter=n_iter)
    ek, ep = s.energy()
    assert ek + ep == pytest.approx(-0.125, rel=1e-14)
    t_end = round(2 * math.pi * 1024) / 1024  # one period, on the tick grid
    s.run(t_end)
    st = s.state()
    assert (st["tau"] == st["tau"][0]).all()
    x_num = st["r"][1] - st["r"][0]
    x_ref, v_ref = kepler_solution(t_end, 1.0, 0.5, 1.0)
    assert np.linalg.norm(x_num - x_ref) < 2e-4
    assert np.linalg.norm(st["v"][1] - st["v"][0] - v_ref) < 4e-4
    ek, ep = s.energy()
    assert abs((ek + ep + 0.125) / 0.125) < 1e-5


def test_circular_orbit_second_order(orc):
    """Shared step (k_min = k_max): the phase error after t = 1 falls 4x per
    halving of the step (second order)."""
    errs = []
    for k in (6, 7, 8):
        m, r, v = two_body(0.0)
        s = sim(orc, m, r, v, eps=0.0, dt_max=2.0 ** -k, n_iter=1, k_max=k,
                era_log2=0)
        s.run(1.0)
        st = s.state()
        x_ref, _ = kepler_solution(1.0, 1.0, 0.0, 1.0)
        errs.append(np.linalg.norm(st["r"][1] - st["r"][0] - x_ref))
    assert 3.5 < errs[0] / errs[1] < 4.5
    assert 3.5 < errs[1] / errs[2] < 4.5


def velocity_verlet(m, r, v, eps, h, steps):
    """Textbook kick-drift-kick velocity Verlet with Plummer softening."""
    def acc(x):
        d = x[None, :, :] - x[:, None, :]
        s2 = (d ** 2).sum(-1) + eps ** 2
        np.fill_diagonal(s2, np.inf)
        return (m[None, :, None] * d / s2[:, :, None] ** 1.5).sum(axis=1)
    r, v = r.copy(), v.copy()
    a = acc(r)
    for _ in range(steps):
        r = r + v * h + 0.5 * a * h * h
        a_new = acc(r)
        v = v + 0.5 * (a + a_new) * h
        a = a_new
    return r, v


@pytest.mark.parametrize("n_iter", [1, 3])
def test_shared_step_reduces_to_velocity_verlet(orc, n_iter):
    m, r, v = inputs.plummer(32, seed=4)
    k = 7
    s = sim(orc, m, r, v, eps=0.05, dt_max=2.0 ** -k, k_max=k, era_log2=3,
            n_iter=n_iter)
    s.run(0.5)
    st = s.state()
    rr, vv = velocity_verlet(m, r, v, 0.05, 2.0 ** -k, 64)
    np.testing.assert_allclose(st["r"], rr, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(st["v"], vv, rtol=1e-11, atol=1e-12)


def test_shared_step_conserves_momentum_and_reverses(orc):
    m, r, v = inputs.plummer(48, seed=6)
    m = m * np.linspace(0.3, 1.7, 48)
    kw = dict(eps=0.02, dt_max=2.0 ** -8, k_max=8, era_log2=3)
    s = sim(orc, m, r, v, **kw)
    s.run(1.0)
    st = s.state()
    p0 = (m[:, None] * v).sum(0)
    p1 = (m[:, None] * st["v"]).sum(0)
    assert np.abs(p1 - p0).max() < 1e-14
    back = sim(orc, m, st["r"], -st["v"], **kw)
    back.run(1.0)
    sb = back.state()
    np.testing.assert_allclose(sb["r"], r, atol=1e-10)
    np.testing.assert_allclose(-sb["v"], v, atol=1e-10)




def test_block_schedule_invariants(orc):
    m, r, v = inputs.plummer(64, seed=2)
    kmax = 20
    s = sim(orc, m, r, v, eta=0.1, log=True, k_max=kmax)
    s.run(0.5)
    log = s.schedule()
    dt_max = 2 ** (kmax - 4)
    off = np.concatenate([[0], np.cumsum(log["n_act"])])
    last_tau = np.zeros(64, np.int64)
    cur_dt = None
    saved = None
    prev_key = None
    nxt = {}
    for k in range(len(log["tau"])):
        era, pas, tn = int(log["era"][k]), int(log["pass_"][k]), int(log["tau"][k])
        key = (era, pas)
        if key != prev_key:
            if pas == 0:
                saved = last_tau.copy()
            else:
                last_tau = saved.copy()
            prev_key = key
            nxt = {}
        idx = log["idx"][off[k]:off[k + 1]]
        dts = log["dt"][off[k]:off[k + 1]]
        assert np.all(np.diff(idx) > 0)
        for i, c in zip(idx, dts):
            i, c = int(i), int(c)
            d = tn - last_tau[i]
            # body steps exactly at the end of its previous step
            assert nxt.get(i, tn) == tn
            assert c & (c - 1) == 0 and 1 <= c <= dt_max
            assert tn % c == 0
            if pas == 0:
                assert c <= 2 * d
            else:
                assert c in (d // 2, d, 2 * d) or (d == 1 and c == 1)
                if c == 2 * d:
                    assert tn % (2 * d) == 0
            last_tau[i] = tn
            nxt[i] = tn + c
    # no body is skipped: every body steps at least once per pass
    assert s.stats()["passes"] == 3 * s.stats()["eras"]


def test_single_iteration_is_the_first_pass(orc):
    """One iteration is the plain block step scheme: the first era of a
    1-pass run equals the first pass of a 3-pass run (Sec. 6)."""
    m, r, v = inputs.plummer(64, seed=8)
    s1 = sim(orc, m, r, v, n_iter=1, log=True)
    s3 = sim(orc, m, r, v, n_iter=3, log=True)
    s1.run(1 / 16)
    s3.run(1 / 16)
    l1, l3 = s1.schedule(), s3.schedule()
    first = l3["pass_"] == 0
    np.testing.assert_array_equal(l1["tau"], l3["tau"][first])
    np.testing.assert_array_equal(l1["n_act"], l3["n_act"][first])
    n1 = int(l1["n_act"].sum())
    np.testing.assert_array_equal(l1["idx"], l3["idx"][:n1])
    np.testing.assert_array_equal(l1["dt"], l3["dt"][:n1])


def test_iteration_improves_reversibility_and_energy(orc):
    """Sec. 6: with equal eta, three iterations beat one. Forward 0 -> 1,
    velocities flipped, forward again: the symmetrised scheme returns
    closer to the start, on every seed, and conserves energy better."""
    worse_rev, worse_e = 0, 0
    for seed in range(4):
        m, r, v = inputs.plummer(64, seed)
        ret, de = {}, {}
        for it in (1, 3):
            s = sim(orc, m, r, v, eta=0.1, n_iter=it)
            e0 = sum(s.energy())
            s.run(1.0)
            de[it] = abs(sum(s.energy()) / e0 - 1)
            st = s.state()
            b = sim(orc, m, st["r"], -st["v"], eta=0.1, n_iter=it)
            b.run(1.0)
            ret[it] = np.abs(b.state()["r"] - r).max()
            assert np.isfinite(ret[it]) and np.isfinite(de[it])
        worse_rev += not ret[3] < ret[1]
        worse_e += not de[3] < de[1]
    assert worse_rev == 0
    assert worse_e == 0


def test_dynamic_era_rules(orc):
    """Alg. 3: an era is last minus first block time, clamped to
    [dt_max / 8, dt_max] and rounded up to a power of two (R11); bodies
    whose next time passes the era end wait for a later era (Sec. 4)."""
    m, r, v = inputs.plummer(96, seed=1)
    kmax = 20
    kw = dict(eta=0.02, era_mode=1, dt_max=1 / 8, k_max=kmax)
    s = sim(orc, m, r, v, log=True, **kw)
    s.run(0.5)
    assert np.isfinite(s.state()["r"]).all()
    ts, te = s.eras()
    L = te - ts
    dtm = 2 ** (kmax - 3)
    assert ts[0] == 0 and te[-1] == 2 ** (kmax - 1)
    assert np.all(ts[1:] == te[:-1])
    # every era but a last one cut short by t_end is a power of two
    assert np.all((L[:-1] & (L[:-1] - 1)) == 0)
    assert np.all(L[:-1] >= dtm // 8) and np.all(L <= dtm)
    log = s.schedule()
    for e in range(len(ts)):
        sel = log["era"] == e
        assert np.all(log["tau"][sel] > ts[e]) and np.all(log["tau"][sel] <= te[e])
    # the rule itself, era by era, from the state at each era start
    # (integrating to an era end reproduces the same eras)
    probe = sim(orc, m, r, v, **kw)
    shorter = 0
    for k in range(len(ts) - 1):
        probe.run(int(ts[k]) * 2.0 ** -kmax)
        st = probe.state()
        nxt = st["tau"] + st["dt"]
        span = min(max(int(nxt.max() - nxt.min()), dtm // 8), dtm)
        want = 1
        while want < span:
            want *= 2
        assert L[k] == want, (k, span, L[k])
        shorter += int(want < dtm)
    assert len(ts) > 2 and shorter > 0


def test_t_end_must_be_on_tick_grid(orc):
    m, r, v = inputs.plummer(8, seed=0)
    s = sim(orc, m, r, v, k_max=10)
    with pytest.raises(ValueError):
        s.run(1.0 / 3.0)
