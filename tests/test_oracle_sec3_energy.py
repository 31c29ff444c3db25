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
import json
import multiprocessing as mp
import os

import numpy as np
import pytest

pytestmark = [
    pytest.mark.slow,
    pytest.mark.skipif(os.environ.get("TSBTS_LONG") != "1",
                       reason="long run: set TSBTS_LONG=1"),
]

# the paper's setup and reported figures (numbers only, cited in the file)
with open(os.path.join(os.path.dirname(__file__), "golden",
                       "sec3_energy_experiment.json")) as _f:
    PAPER = json.load(_f)
T_END = PAPER["t_end"]
ERA = PAPER["linear_growth_with_3_iterations_at_era"]
ERA_LOG2 = 2
assert 2.0 ** -ERA_LOG2 == ERA


def max_energy_error(seed, n_iter):
    import oracle
    from paper_1205_2288_gb300 import inputs
    oracle.set_threads(1)  # one process per run
    m, r, v = inputs.plummer(PAPER["n_bodies"], 1000 + seed)
    s = oracle.Sim(m, r, v, eps=PAPER["eps_plummer"], eta=PAPER["eta"],
                   dt_max=PAPER["dt_max"], n_iter=n_iter, era_mode=0,
                   era_log2=ERA_LOG2, k_max=20)
    e0 = sum(s.energy())
    worst = 0.0
    for t in range(1, T_END + 1):
        s.run(float(t))
        worst = max(worst, abs(sum(s.energy()) - e0) / abs(e0))
    return worst


def test_five_passes_hold_the_error_that_three_let_grow():
    seeds = range(PAPER["n_realisations"])
    jobs = [(seed, k) for seed in seeds for k in (3, 5)]
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=min(len(jobs), os.cpu_count()),
                                mp_context=ctx) as ex:
        out = dict(zip(jobs, ex.map(max_energy_error, *zip(*jobs))))
    three = np.array([out[(s, 3)] for s in seeds])
    five = np.array([out[(s, 5)] for s in seeds])
    w = PAPER["worst_relative_energy_error"]
    print(f"worst |dE/E|, 3 passes: {three} (paper {w['n_iter_3']['value']});"
          f" 5 passes: {five} (paper < {w['n_iter_5']['bound']})")
    assert np.all(five < three), (three, five)
    assert three.mean() > 3 * five.mean(), (three, five)
