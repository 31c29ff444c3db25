"""tsbts_force_static: the stand-alone force for callers that cannot
allocate device memory (their device memory belongs to another allocator,
or they must not call cudaMalloc/cudaFree, which can synchronise the
device). Its scratch is a fixed array inside the library.

Checked through the C ABI against tsbts_force, which allocates its own
scratch, on two calls in a row: the FP64 path with ascending-j sums must
agree bit for bit, the mixed path within the force tolerance of the other
GPU tests (every a_i within 1e-6 of sum_j m_j / s_ij^2, phi 1e-6, q 2e-6).
This file is collected last so that a run stopping at the first failure
has run every other test first; it also passes on its own.
"""
import numpy as np
import pytest

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
                                          (40000, 64, 2)])
def test_static_scratch_matches_allocating_entry(torch_cuda, n, n_act, seed):
    m, r, v = inputs.plummer(n, seed)
    eps = 0.01
    idx = inputs.active_subset(n, n_act, seed + 10)
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
            if precision == tsbts.TSBTS_FP64 and n <= 8192:
                for g, w in zip(got, ref):
                    np.testing.assert_array_equal(g, w)
            elif precision == tsbts.TSBTS_FP64:
                scale = _scale(m, r, eps, idx)
                assert (np.abs(got[0] - ref[0]).max(1) / scale).max() < 1e-13
                np.testing.assert_allclose(got[1], ref[1], rtol=1e-13)
                np.testing.assert_array_equal(got[2], ref[2])
            else:
                scale = _scale(m, r, eps, idx)
                assert (np.abs(got[0] - ref[0]).max(1) / scale).max() < 1e-6
                np.testing.assert_allclose(got[1], ref[1], rtol=1e-6)
                np.testing.assert_allclose(got[2], ref[2], rtol=2e-6)


def test_static_scratch_rejects_sizes_beyond_its_limit(torch_cuda):
    torch = torch_cuda
    n = 65537
    m = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    r = torch.zeros(n, 3, dtype=torch.float64, device="cuda:0")
    idx = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    a = torch.zeros(1, 3, dtype=torch.float64, device="cuda:0")
    p = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    with pytest.raises(tsbts.TsbtsError) as e:
        tsbts.tsbts_force_static(tsbts.TSBTS_MIXED, m, r, r, 0.01, idx, a, p,
                                 p)
    assert e.value.code == tsbts.TSBTS_ERR_ARG
