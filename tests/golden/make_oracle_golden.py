"""Writes oracle_era_run.json: a frozen end state of the FP64 oracle, so that
any later change to the oracle's arithmetic shows up as a failing test
(tests/test_oracle_golden.py) and has to be justified by the passage of
the paper it follows.

It calls only the oracle and the seeded input generator. The inputs are
stored too, so the check does not depend on the generator. Doubles are
stored as hexadecimal floats (exact).

Run from the repository root: python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(
    os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1205_2288_gb300 import inputs  # noqa: E402

CASES = {
    # dynamic era (Alg. 3), three passes, unequal masses
    "dynamic_3pass": dict(n=32, seed=71, eps=0.02, eta=0.03, dt_max=0.125,
                          n_iter=3, era_mode=1, era_log2=3, k_max=20,
                          t_end=0.25),
    # fixed era of 1/16, five passes
    "fixed_5pass": dict(n=24, seed=72, eps=0.05, eta=0.05, dt_max=0.0625,
                        n_iter=5, era_mode=0, era_log2=4, k_max=20,
                        t_end=0.1875),
}


def hexes(a):
    return [float(x).hex() for x in a.reshape(-1)]


def run(case):
    c = dict(case)
    n, seed, t_end = c.pop("n"), c.pop("seed"), c.pop("t_end")
    m = inputs.salpeter_masses(n, seed)
    _, r, v = inputs.plummer(n, seed + 1, masses=m)
    return m, r, v, t_end, c


def main():
    out = {}
    for name, case in CASES.items():
        m, r, v, t_end, kw = run(case)
        s = oracle.Sim(m, r, v, **kw)
        e0 = s.energy()
        s.run(t_end)
        st = s.state()
        stats = s.stats()
        out[name] = {
            "config": dict(kw, t_end=t_end),
            "m": hexes(m), "r": hexes(r), "v": hexes(v),
            "energy_0": [x.hex() for x in e0],
            "energy_t": [x.hex() for x in s.energy()],
            "r_t": hexes(st["r"]), "v_t": hexes(st["v"]), "a_t": hexes(st["a"]),
            "dts_t": hexes(st["dts"]),
            "tau_t": [int(x) for x in st["tau"]],
            "dt_t": [int(x) for x in st["dt"]],
            "block_steps": stats["block_steps"],
            "interactions": stats["interactions"],
            "passes": stats["passes"],
        }
        s.close()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        "oracle_era_run.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
