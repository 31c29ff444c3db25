"""The oracle reproduces its frozen outputs bit for bit (regression guard).

tests/golden/oracle_era_run.json was written by
tests/golden/make_oracle_golden.py, which calls only the oracle. It holds
inputs and end states of two era runs (a dynamic era with three passes; a
fixed era with five). The oracle uses only +, -, *, /, sqrt and ldexp
(correctly rounded) in a fixed order, so the comparison is exact on any
machine. A change to the oracle's arithmetic fails here and must be
justified by the passage of the paper it follows before the file is
rewritten.
"""
import json
import os

import numpy as np
import pytest

import oracle

PATH = os.path.join(os.path.dirname(__file__), "golden", "oracle_era_run.json")
with open(PATH) as _f:
    GOLDEN = json.load(_f)


def unhex(xs, shape=None):
    a = np.array([float.fromhex(x) for x in xs])
    return a.reshape(shape) if shape else a


@pytest.mark.parametrize("name", sorted(GOLDEN))
def test_oracle_matches_frozen_run(name):
    g = GOLDEN[name]
    kw = dict(g["config"])
    t_end = kw.pop("t_end")
    m = unhex(g["m"])
    n = m.shape[0]
    s = oracle.Sim(m, unhex(g["r"], (n, 3)), unhex(g["v"], (n, 3)), **kw)
    assert [x.hex() for x in s.energy()] == g["energy_0"]
    s.run(t_end)
    st = s.state()
    for key in ("r", "v", "a"):
        np.testing.assert_array_equal(st[key], unhex(g[key + "_t"], (n, 3)),
                                      err_msg=key)
    np.testing.assert_array_equal(st["dts"], unhex(g["dts_t"]))
    np.testing.assert_array_equal(st["tau"], g["tau_t"])
    np.testing.assert_array_equal(st["dt"], g["dt_t"])
    assert [x.hex() for x in s.energy()] == g["energy_t"]
    stats = s.stats()
    for key in ("block_steps", "interactions", "passes"):
        assert stats[key] == g[key], key
