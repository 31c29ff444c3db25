"""Writes oracle_plummer16384_t1.json: the FP64 oracle's run of the benchmark
workload over its whole span, so that the benchmark can hold both GPU paths
to the accuracy bar of the headline metric (relative energy error at most
twice the oracle's) at the end of the timed integration, not on a sample.

Workload: Plummer n = 16384, equal masses, seed 0, eps = 1/256,
eta = 0.01, dt = 2^-k (k = 3..20), dynamic era (Alg. 3), three passes per
era (Alg. 2), t = 0..1. The energy is the Sec. 3 diagnostic (kinetic plus
softened potential at the system time).

It calls only the oracle and the seeded input generator; the oracle sums in
a fixed order with correctly rounded operations, so the numbers do not
depend on the machine or the thread count. About an hour on eight cores.

Run from the repository root:
    python tests/golden/make_plummer16384_golden.py [threads]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(
    os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1205_2288_gb300 import inputs  # noqa: E402

CONFIG = dict(n=16384, seed=0, eps=1.0 / 256.0, eta=0.01, dt_max=0.125,
              n_iter=3, era_mode=1, era_log2=3, dyn_min_log2=3, k_max=20,
              t_end=1.0)


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    oracle.set_threads(threads)
    c = dict(CONFIG)
    n, seed, t_end = c.pop("n"), c.pop("seed"), c.pop("t_end")
    m, r, v = inputs.plummer(n, seed)
    s = oracle.Sim(m, r, v, **c)
    e0 = s.energy()
    t0 = time.perf_counter()
    s.run(t_end)
    sec = time.perf_counter() - t0
    e1 = s.energy()
    st = s.stats()
    ts, te = s.eras()
    s.close()
    E0, E1 = e0[0] + e0[1], e1[0] + e1[1]
    out = {
        "config": CONFIG,
        "energy_0": [x.hex() for x in e0],
        "energy_t": [x.hex() for x in e1],
        "dE_E": abs(E1 / E0 - 1.0),
        "block_steps": st["block_steps"],
        "interactions": st["interactions"],
        "init_interactions": st["init_interactions"],
        "eras": st["eras"],
        "passes": st["passes"],
        "dt_underflow": st["underflow"],
        "era_starts_ticks": [int(x) for x in ts],
        "era_ends_ticks": [int(x) for x in te],
        "oracle_seconds": sec,
        "oracle_threads": threads,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        "oracle_plummer16384_t1.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
