"""The library's dynamic-era length (csrc/era_rule.h, host arithmetic the
engine calls between eras) checked on the CPU: against the rule as the
paper's Alg. 3 with reading R11 states it, on random inputs and at the
edges, and against the era lengths the oracle actually takes, from the
states at its era starts (the oracle implements the rule separately)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1205_2288_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1205_2288_gb300", "csrc")
K_MAX = 20

HARNESS = r"""
#include <cstdio>
#include "era_rule.h"
int main() {
  long long first, last, dtmax;
  int dml;
  while (std::scanf("%lld %lld %lld %d", &first, &last, &dtmax, &dml) == 4)
    std::printf("%lld\n", tsbts_dynamic_era_ticks(first, last, dtmax, dml));
  return 0;
}
"""


@pytest.fixture(scope="module")
def era_rule(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("era_rule")
    src, exe = d / "h.cpp", d / "h"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, str(src), "-o",
                    str(exe)], check=True)

    def call(rows):
        text = "".join(f"{a} {b} {c} {k}\n" for a, b, c, k in rows)
        out = subprocess.run([str(exe)], input=text, capture_output=True,
                             text=True, check=True).stdout
        return [int(x) for x in out.split()]
    return call


def rule(first, last, dt_max, dyn_min_log2):
    """Alg. 3 (R11): last - first, clamped to [dt_max 2^-dyn_min_log2 (at
    least one tick), dt_max], then the smallest power of two that long."""
    span = min(max(last - first, max(dt_max >> dyn_min_log2, 1)), dt_max)
    p = 1
    while p < span:
        p *= 2
    return p


def test_random_and_edge_inputs(era_rule):
    rng = np.random.default_rng(3)
    rows = []
    for _ in range(4000):
        k_min = int(rng.integers(0, 21))
        dt_max = 2 ** (K_MAX - k_min)
        first = int(rng.integers(1, 2 ** 30))
        last = first + int(rng.integers(0, 2 * dt_max + 1))
        rows.append((first, last, dt_max, int(rng.integers(0, 41))))
    for dt_max in (1, 2, 2 ** 17, 2 ** 20):
        for span in (0, 1, dt_max // 2 - 1, dt_max // 2, dt_max // 2 + 1,
                     dt_max - 1, dt_max, dt_max + 1):
            for dml in (0, 3, 40):
                rows.append((100, 100 + max(span, 0), dt_max, dml))
    got = era_rule(rows)
    want = [rule(*r) for r in rows]
    assert got == want


@pytest.mark.parametrize("seed,eta,dt_max", [(1, 0.02, 1 / 8), (4, 0.05, 1 / 4),
                                             (9, 0.01, 1 / 2)])
def test_engine_rule_gives_the_oracles_eras(era_rule, seed, eta, dt_max):
    m, r, v = inputs.plummer(128, seed)
    kw = dict(eps=0.01, eta=eta, dt_max=dt_max, era_mode=1, k_max=K_MAX)
    full = oracle.Sim(m, r, v, **kw)
    full.run(0.5)
    ts, te = full.eras()
    probe = oracle.Sim(m, r, v, **kw)
    rows = []
    for k in range(len(ts) - 1):    # the last era may be cut by t_end
        probe.run(int(ts[k]) * 2.0 ** -K_MAX)
        st = probe.state()
        nxt = st["tau"] + st["dt"]
        rows.append((int(nxt.min()), int(nxt.max()),
                     int(dt_max * 2 ** K_MAX), 3))
    assert len(rows) >= 1
    assert era_rule(rows) == [int(x) for x in (te - ts)[:len(rows)]]
