"""The oracle against the paper's Sec. 3 experiment (Figs. 1 and 2): 100-body
Plummer models in standard units, eta = 0.1, eps = 0.01, dt_max = 1/64,
integrated for 1000 time units with a fixed era.

The paper finds that with an era of 0.25 time units three passes let the
relative energy error grow steadily, while five passes keep it small. Its
realisations are not published, so five seeded ones stand in for them and
only the comparison is asserted: for every seed the largest error over the
run with five passes is below the one with three, and on average several
times below. (Measured on these seeds: three passes 0.057-0.22, five
passes 0.008-0.032; the paper's figures show at most 0.035 and 0.008.)

About half an hour of CPU time, spread over processes (six minutes on
eight cores); it runs only with TSBTS_LONG=1 in the environment.
"""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest

pytestmark = [
    pytest.mark.slow,
    pytest.mark.skipif(os.environ.get("TSBTS_LONG") != "1",
                       reason="long run: set TSBTS_LONG=1"),
]

T_END = 1000
ERA_LOG2 = 2  # era 0.25


def max_energy_error(seed, n_iter):
    import oracle
    from paper_1205_2288_gb300 import inputs
    m, r, v = inputs.plummer(100, 1000 + seed)
    s = oracle.Sim(m, r, v, eps=0.01, eta=0.1, dt_max=1 / 64, n_iter=n_iter,
                   era_mode=0, era_log2=ERA_LOG2, k_max=20)
    e0 = sum(s.energy())
    worst = 0.0
    for t in range(1, T_END + 1):
        s.run(float(t))
        worst = max(worst, abs(sum(s.energy()) - e0) / abs(e0))
    return worst


def test_five_passes_hold_the_error_that_three_let_grow():
    jobs = [(seed, k) for seed in range(5) for k in (3, 5)]
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=min(len(jobs), os.cpu_count()),
                                mp_context=ctx) as ex:
        out = dict(zip(jobs, ex.map(max_energy_error, *zip(*jobs))))
    three = np.array([out[(s, 3)] for s in range(5)])
    five = np.array([out[(s, 5)] for s in range(5)])
    assert np.all(five < three), (three, five)
    assert three.mean() > 3 * five.mean(), (three, five)
