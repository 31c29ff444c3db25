"""tsbts_force_static: the stand-alone force for callers that cannot
allocate device memory (their device memory belongs to another allocator,
or they must not call cudaMalloc/cudaFree, which can synchronise the
device). Its scratch is a fixed array inside the library.

Checked through the C ABI on two calls in a row, against tsbts_force,
which allocates its own scratch, and against the FP64 oracle's forces: the
FP64 path with ascending-j sums must agree bit for bit with both, the mixed
path within the force tolerance of the other GPU tests (every a_i within
1e-6 of sum_j m_j / s_ij^2, phi 1e-6, q 2e-6). The largest case fills the
fixed array exactly (n = n_act = 65536).
This file is collected last so that a run stopping at the first failure
has run every other test first; it also passes on its own.
"""
import numpy as np
import pytest

import oracle
from paper_1205_2288_gb300 import inputs, tsbts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    return torch


def _call(torch, fn, precision, m, r, v, eps, idx):
    dev = "cuda:0"
    tm, tr, tv = (torch.from_numpy(np.ascontiguousarray(x)).to(dev)
                  for x in (m, r, v))
    ti = torch.from_numpy(np.ascontiguousarray(idx, np.int32)).to(dev)
    na = len(idx)
    a = torch.full((na, 3), float("nan"), dtype=torch.float64, device=dev)
    phi = torch.full((na,), float("nan"), dtype=torch.float64, device=dev)
    q = torch.full((na,), float("nan"), dtype=torch.float64, device=dev)
    fn(precision, tm, tr, tv, eps, ti, a, phi, q)
    torch.cuda.synchronize()
    return a.cpu().numpy(), phi.cpu().numpy(), q.cpu().numpy()


def _scale(m, r, eps, idx):
    out = np.zeros(len(idx))
    for k, i in enumerate(idx):
        d2 = ((r - r[i]) ** 2).sum(1) + eps ** 2
        w = m / d2
        w[i] = 0.0
        out[k] = w.sum()
    return out


@pytest.mark.parametrize("n,n_act,seed", [(5000, 777, 0), (3001, 3001, 1),
                                          (40000, 64, 2),
                                          (65536, 65536, 3)])
def test_static_scratch_matches_allocating_entry(torch_cuda, n, n_act, seed):
    m, r, v = inputs.plummer(n, seed)
    eps = 0.01
    idx = inputs.active_subset(n, n_act, seed + 10)
    # the oracle on a sample of the active bodies (all of them when small)
    pick = np.arange(n_act) if n_act <= 1024 else \
        np.sort(np.random.default_rng(seed).choice(n_act, 256, replace=False))
    oracle.set_threads(8)
    want = oracle.forces(m, r, v, eps, idx[pick])
    scale_pick = _scale(m, r, eps, idx[pick])
    for precision in (tsbts.TSBTS_FP64, tsbts.TSBTS_MIXED):
        ref = _call(torch_cuda, tsbts.tsbts_force, precision, m, r, v, eps,
                    idx)
        # two calls in a row share the array: the second must not see
        # anything left by the first
        for _ in range(2):
            got = _call(torch_cuda, tsbts.tsbts_force_static, precision, m, r,
                        v, eps, idx)
            for x in got:
                assert np.isfinite(x).all()
            sub = [x[pick] for x in got]
            if precision == tsbts.TSBTS_FP64 and n <= 8192:
                for g, w in zip(got, ref):
                    np.testing.assert_array_equal(g, w)
                for g, w in zip(sub, want):
                    np.testing.assert_array_equal(g, w)
            elif precision == tsbts.TSBTS_FP64:
                scale = _scale(m, r, eps, idx) if n_act <= 8192 else None
                if scale is not None:
                    assert (np.abs(got[0] - ref[0]).max(1)
                            / scale).max() < 1e-13
                np.testing.assert_allclose(got[1], ref[1], rtol=1e-13)
                np.testing.assert_array_equal(got[2], ref[2])
                assert (np.abs(sub[0] - want[0]).max(1)
                        / scale_pick).max() < 1e-13
                np.testing.assert_allclose(sub[1], want[1], rtol=1e-13)
                np.testing.assert_allclose(sub[2], want[2], rtol=1e-14)
            else:
                if n_act <= 8192:
                    scale = _scale(m, r, eps, idx)
                    assert (np.abs(got[0] - ref[0]).max(1)
                            / scale).max() < 1e-6
                np.testing.assert_allclose(got[1], ref[1], rtol=1e-6)
                np.testing.assert_allclose(got[2], ref[2], rtol=2e-6)
                assert (np.abs(sub[0] - want[0]).max(1)
                        / scale_pick).max() < 1e-6
                np.testing.assert_allclose(sub[1], want[1], rtol=1e-6)
                np.testing.assert_allclose(sub[2], want[2], rtol=2e-6)


@pytest.mark.parametrize("n,n_act", [(65537, 1), (65536, 65537)])
def test_static_scratch_rejects_sizes_beyond_its_limit(torch_cuda, n, n_act):
    torch = torch_cuda
    dev = "cuda:0"
    m = torch.zeros(n, dtype=torch.float64, device=dev)
    r = torch.zeros(n, 3, dtype=torch.float64, device=dev)
    idx = torch.zeros(n_act, dtype=torch.int32, device=dev)
    a = torch.zeros(n_act, 3, dtype=torch.float64, device=dev)
    p = torch.zeros(n_act, dtype=torch.float64, device=dev)
    with pytest.raises(tsbts.TsbtsError) as e:
        tsbts.tsbts_force_static(tsbts.TSBTS_MIXED, m, r, r, 0.01, idx, a, p,
                                 p)
    assert e.value.code == tsbts.TSBTS_ERR_ARG
