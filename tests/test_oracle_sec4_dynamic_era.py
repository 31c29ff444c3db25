"""The oracle against the paper's Sec. 4 comparison of dynamic and fixed
eras (Alg. 3 with reading R11).

The paper integrates ten 100-body Plummer models with a dynamic era and
with a fixed era equal to the largest step (1/64), three passes each, and
finds the dynamic era's energy errors in the same range and modestly
smaller (smaller in 70% of the 100-body runs; larger in 45% of all its
runs). Seeded realisations stand in for the unpublished ones, and the run
is shortened to 100 time units so that it fits the CPU suite. Asserted: the
dynamic era's largest relative energy error is at most the fixed era's for
at least half of the seeds, and their ratio averages (geometrically) below
1.2. Measured on these seeds: 7 of 10, mean ratio 0.90 (at 1000 time
units: mean ratio 0.72). Rounding the era down instead of up (the other
reading of Alg. 3) gives 1 of 10 and 1.58 (at 1000 time units, dynamic
errors 2.5 to 10 times the fixed ones).
"""
import concurrent.futures as cf
import json
import math
import multiprocessing as mp
import os

import numpy as np
import pytest

pytestmark = pytest.mark.slow

with open(os.path.join(os.path.dirname(__file__), "golden",
                       "sec4_dynamic_era.json")) as _f:
    PAPER = json.load(_f)
T_END = 100
SEED0 = 2000


def max_energy_error(seed, era_mode, t_end=T_END):
    import oracle
    from paper_1205_2288_gb300 import inputs
    oracle.set_threads(1)  # one process per run
    m, r, v = inputs.plummer(PAPER["n_bodies"], SEED0 + seed)
    era_log2 = round(-math.log2(PAPER["fixed_era"]))
    s = oracle.Sim(m, r, v, eps=PAPER["eps_plummer"], eta=PAPER["eta"],
                   dt_max=PAPER["dt_max"], n_iter=PAPER["n_iter"],
                   era_mode=era_mode, era_log2=era_log2, k_max=20)
    e0 = sum(s.energy())
    worst = 0.0
    for t in range(1, t_end + 1):
        s.run(float(t))
        worst = max(worst, abs(sum(s.energy()) - e0) / abs(e0))
    return worst


def ratios(t_end):
    seeds = range(PAPER["n_realisations"])
    jobs = [(seed, mode, t_end) for seed in seeds for mode in (0, 1)]
    with cf.ProcessPoolExecutor(max_workers=min(len(jobs), os.cpu_count()),
                                mp_context=mp.get_context("spawn")) as ex:
        out = dict(zip(jobs, ex.map(max_energy_error, *zip(*jobs))))
    fixed = np.array([out[(s, 0, t_end)] for s in seeds])
    dyn = np.array([out[(s, 1, t_end)] for s in seeds])
    return dyn, fixed


def test_dynamic_era_errors_in_the_range_of_the_fixed_era():
    dyn, fixed = ratios(T_END)
    ratio = dyn / fixed
    assert np.sum(dyn <= fixed) >= len(fixed) / 2, ratio
    assert math.exp(np.mean(np.log(ratio))) < 1.2, ratio


@pytest.mark.skipif(os.environ.get("TSBTS_LONG") != "1",
                    reason="long run: set TSBTS_LONG=1")
def test_over_the_papers_full_span():
    """The paper's 1000 time units (~40 min of CPU time, six minutes on
    eight cores): dynamic no worse than fixed for at least half of the
    seeds and modestly better on average (measured: 7 of 10, geometric-mean
    ratio 0.72)."""
    dyn, fixed = ratios(PAPER["t_end"])
    ratio = dyn / fixed
    assert np.sum(dyn <= fixed) >= len(fixed) / 2, ratio
    assert math.exp(np.mean(np.log(ratio))) < 1.0, ratio
