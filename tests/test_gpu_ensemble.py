"""Ensembles of independent clusters (tsbts_init_ensemble): every cluster,
integrated together with the others on the GPU, must match the FP64 oracle
run on that cluster alone. With FP64 ascending-j sums each cluster's block
schedule, state and energy are bit-identical; mixed precision is held to
the energy bar of the single-system tests."""
import numpy as np
import pytest

from paper_1205_2288_gb300 import inputs, tsbts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def make_clusters(sizes, seed):
    ms, rs, vs = [], [], []
    for c, n in enumerate(sizes):
        m = inputs.salpeter_masses(n, seed=1000 * seed + 2 * c)
        m, r, v = inputs.plummer(n, seed=1000 * seed + 2 * c + 1, masses=m)
        ms.append(m)
        rs.append(r)
        vs.append(v)
    off = np.zeros(len(sizes) + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    eps = 4.0 / np.asarray(sizes, np.float64)
    return off, np.concatenate(ms), np.concatenate(rs), np.concatenate(vs), eps


KW = dict(eta=0.02, dt_max=1 / 8, n_iter=3, era_log2=3, k_max=20)


def oracle_clusters(orc, off, m, r, v, eps, t_end, era_mode=0, **kw):
    out = []
    for c in range(len(off) - 1):
        a, b = off[c], off[c + 1]
        s = orc.Sim(m[a:b], r[a:b], v[a:b], eps=eps[c], era_mode=era_mode,
                    **kw)
        e0 = s.energy()
        s.run(t_end)
        out.append((s.state(), e0, s.energy(), s.stats()))
    return out


def test_ensemble_fp64_bit_exact_per_cluster(orc):
    sizes = [64, 100, 37, 300, 77, 512, 1]
    off, m, r, v, eps = make_clusters(sizes, seed=1)
    ref = oracle_clusters(orc, off, m, r, v, eps, 0.25, **KW)
    g = tsbts.Ensemble(off, m, r, v, eps=eps, **KW)
    ek0, ep0 = g.cluster_energy()
    g.step_era(0.25)
    st = g.state()
    ek, ep = g.cluster_energy()
    for c in range(len(sizes)):
        a, b = off[c], off[c + 1]
        so, e0, e1, _ = ref[c]
        for key in ("r", "v", "a", "tau", "dt"):
            np.testing.assert_array_equal(st[key][a:b], so[key],
                                          err_msg=f"cluster {c} {key}")
        assert (ek0[c], ep0[c]) == e0
        assert (ek[c], ep[c]) == e1
    # interactions: every cluster's own n_act * N_c, summed
    assert g.stats()["interactions"] == sum(x[3]["interactions"] for x in ref)
    assert g.stats()["kernel_launches"] > 0


def test_single_cluster_ensemble_equals_single_system():
    off, m, r, v, eps = make_clusters([200], seed=2)
    e = tsbts.Ensemble(off, m, r, v, eps=eps, **KW)
    s = tsbts.Simulation(m, r, v, eps=float(eps[0]), **KW)
    e.step_era(0.25)
    s.step_era(0.25)
    a, b = e.state(), s.state()
    for key in ("r", "v", "a", "tau", "dt"):
        np.testing.assert_array_equal(a[key], b[key])
    assert e.stats()["block_steps"] == s.stats()["block_steps"]


@pytest.mark.parametrize("graph_steps", [0, 32])
def test_ensemble_mixed_energy_and_trajectories(orc, graph_steps):
    sizes = [64, 500, 1500, 200, 3000, 90]
    off, m, r, v, eps = make_clusters(sizes, seed=3)
    kw = dict(KW, eta=0.01)
    ref = oracle_clusters(orc, off, m, r, v, eps, 0.125, **kw)
    g = tsbts.Ensemble(off, m, r, v, eps=eps, precision=tsbts.TSBTS_MIXED,
                       graph_steps=graph_steps, **kw)
    ek0, ep0 = g.cluster_energy()
    g.step_era(0.125)
    ek, ep = g.cluster_energy()
    st = g.state()
    for c in range(len(sizes)):
        a, b = off[c], off[c + 1]
        so, e0, e1, _ = ref[c]
        E0 = sum(e0)
        de_o = abs(sum(e1) / E0 - 1)
        de_g = abs((ek[c] + ep[c]) / (ek0[c] + ep0[c]) - 1)
        assert de_g <= 2 * de_o + 1e-7, (c, de_g, de_o)
        assert np.abs(st["r"][a:b] - so["r"]).max() < 1e-4


def test_ensemble_argument_errors():
    off, m, r, v, eps = make_clusters([10, 20], seed=4)
    cfg = tsbts.tsbts_config_default()
    ctx = tsbts.tsbts_create(cfg)
    try:
        bad = off.copy()
        bad[1] = 0     # an empty cluster
        with pytest.raises(tsbts.TsbtsError) as e:
            tsbts.tsbts_init_ensemble(ctx, bad, m, r, v, eps, 0.02, 1 / 8)
        assert e.value.code == tsbts.TSBTS_ERR_ARG
        with pytest.raises(tsbts.TsbtsError) as e:
            tsbts.tsbts_init_ensemble(ctx, off, m, r, v, -eps, 0.02, 1 / 8)
        assert e.value.code == tsbts.TSBTS_ERR_ARG
    finally:
        tsbts.tsbts_destroy(ctx)
    # every cluster would need its own pass count: refused
    cfg.conv_tol = 1e-6
    ctx = tsbts.tsbts_create(cfg)
    try:
        with pytest.raises(tsbts.TsbtsError) as e:
            tsbts.tsbts_init_ensemble(ctx, off, m, r, v, eps, 0.02, 1 / 8)
        assert e.value.code == tsbts.TSBTS_ERR_ARG
    finally:
        tsbts.tsbts_destroy(ctx)


def scaled_clusters(sizes, scales, seed):
    """Clusters of different sizes and radii (virial scaling: r by s, v by
    s^-1/2), so that their block steps and dynamic eras differ."""
    off, m, r, v, eps = make_clusters(sizes, seed)
    for c, s in enumerate(scales):
        a, b = off[c], off[c + 1]
        r[a:b] *= s
        v[a:b] /= np.sqrt(s)
    return off, m, r, v, eps


KWD = dict(eta=0.02, dt_max=1 / 8, n_iter=3, dyn_min_log2=3, k_max=20)


@pytest.mark.parametrize("graph_steps", [0, 32])
def test_ensemble_dynamic_eras_fp64_bit_exact_per_cluster(orc, graph_steps):
    """Dynamic eras (Alg. 3) taken by every cluster on its own bodies: each
    cluster's state and energies are those of the oracle's lone run of it
    with the dynamic era, bit for bit, although the clusters take
    different numbers of eras of different lengths."""
    sizes = [24, 100, 257, 64, 500, 1]
    off, m, r, v, eps = scaled_clusters(sizes, [1.0, 0.3, 1.0, 3.0, 1.5,
                                                1.0], seed=9)
    ref = []
    for c in range(len(sizes)):
        a, b = off[c], off[c + 1]
        s = orc.Sim(m[a:b], r[a:b], v[a:b], eps=eps[c], era_mode=1, **KWD)
        e0 = s.energy()
        s.run(0.25)   # the same two calls as below: era ends at 0.25 too
        s.run(0.375)
        ref.append((s.state(), e0, s.energy(), s.stats()))
    g = tsbts.Ensemble(off, m, r, v, eps=eps, era_mode=1,
                       graph_steps=graph_steps, **KWD)
    ek0, ep0 = g.cluster_energy()
    g.step_era(0.25)
    g.step_era(0.375)
    st = g.state()
    ek, ep = g.cluster_energy()
    for c in range(len(sizes)):
        a, b = off[c], off[c + 1]
        so, e0, e1, _ = ref[c]
        for key in ("r", "v", "a", "tau", "dt"):
            np.testing.assert_array_equal(st[key][a:b], so[key],
                                          err_msg=f"cluster {c} {key}")
        assert (ek0[c], ep0[c]) == e0
        assert (ek[c], ep[c]) == e1
    eras = [x[3]["eras"] for x in ref]
    assert len(set(eras)) > 1, eras
    assert g.stats()["interactions"] == sum(x[3]["interactions"] for x in ref)
    assert st["t"] == 0.375


def config4_subset(count=32, seed=7):
    """A seeded subset of the 512-cluster workload (sizes log-uniform in
    [64, 4096], Salpeter masses, eps_c = 4 / N_c): the clusters' own
    bodies, offsets and softenings."""
    off, m, r, v, eps = inputs.ensemble(512, seed=0)
    pick = np.sort(np.random.default_rng(seed).choice(512, count,
                                                      replace=False))
    sizes = np.diff(off)[pick]
    sub_off = np.zeros(count + 1, np.int64)
    sub_off[1:] = np.cumsum(sizes)
    take = np.concatenate([np.arange(off[c], off[c + 1]) for c in pick])
    return sub_off, m[take], r[take], v[take], eps[pick]


KW4 = dict(eta=0.01, dt_max=1 / 8, n_iter=3, era_log2=3, k_max=20)


def test_config4_subset_fp64_bit_exact(orc):
    """32 clusters of the 512-cluster configuration, FP64 with ascending-j
    sums, over t = 0..1/64: every cluster's state and energy are the
    oracle's, bit for bit."""
    off, m, r, v, eps = config4_subset()
    assert np.diff(off).max() > 1000 and np.diff(off).min() < 200
    orc.set_threads(16)
    ref = oracle_clusters(orc, off, m, r, v, eps, 1 / 64, **KW4)
    g = tsbts.Ensemble(off, m, r, v, eps=eps, exact_order=1, **KW4)
    g.step_era(1 / 64)
    st = g.state()
    ek, ep = g.cluster_energy()
    for c in range(len(off) - 1):
        a, b = off[c], off[c + 1]
        so, _, e1, _ = ref[c]
        for key in ("r", "v", "a", "tau", "dt"):
            np.testing.assert_array_equal(st[key][a:b], so[key],
                                          err_msg=f"cluster {c} {key}")
        assert (ek[c], ep[c]) == e1
    assert g.stats()["interactions"] == sum(x[3]["interactions"] for x in ref)


def test_config4_subset_mixed_energy_bar(orc):
    """The same clusters in mixed precision: each cluster's relative energy
    error within twice the oracle's (plus the FP32 force-noise floor)."""
    off, m, r, v, eps = config4_subset()
    orc.set_threads(16)
    ref = oracle_clusters(orc, off, m, r, v, eps, 1 / 64, **KW4)
    g = tsbts.Ensemble(off, m, r, v, eps=eps, precision=tsbts.TSBTS_MIXED,
                       **KW4)
    ek0, ep0 = g.cluster_energy()
    g.step_era(1 / 64)
    ek, ep = g.cluster_energy()
    for c in range(len(off) - 1):
        _, e0, e1, _ = ref[c]
        de_o = abs(sum(e1) / sum(e0) - 1.0)
        de_g = abs((ek[c] + ep[c]) / (ek0[c] + ep0[c]) - 1.0)
        assert de_g <= 2 * de_o + 1e-7, (c, de_g, de_o)


def test_ensemble_dynamic_eras_mixed_energy(orc):
    """Mixed precision with every cluster's own dynamic eras: each cluster's
    relative energy error within twice its oracle run's (+1e-7)."""
    sizes = [64, 300, 1000, 128]
    off, m, r, v, eps = scaled_clusters(sizes, [1.0, 0.5, 1.0, 2.0], seed=11)
    kw = dict(KWD, eta=0.01)
    ref = oracle_clusters(orc, off, m, r, v, eps, 0.125, era_mode=1, **kw)
    g = tsbts.Ensemble(off, m, r, v, eps=eps, era_mode=1,
                       precision=tsbts.TSBTS_MIXED, **kw)
    ek0, ep0 = g.cluster_energy()
    g.step_era(0.125)
    ek, ep = g.cluster_energy()
    for c in range(len(sizes)):
        _, e0, e1, _ = ref[c]
        de_o = abs(sum(e1) / sum(e0) - 1)
        de_g = abs((ek[c] + ep[c]) / (ek0[c] + ep0[c]) - 1)
        assert de_g <= 2 * de_o + 1e-7, (c, de_g, de_o)
