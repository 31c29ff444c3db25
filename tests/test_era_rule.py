"""The library's host arithmetic at era boundaries (csrc/era_rule.h),
compiled and checked on the CPU:

* the dynamic era length the engine takes between eras, against the rule
  of Alg. 3 with reading R11 (random and edge inputs) and against the era
  lengths the oracle takes from the states at its era starts;
* the check tsbts_set_state makes before it copies a state, against the
  oracle's own resume check, on states that end an era and on copies of
  them with one value spoiled.
The oracle implements both separately.
"""
import ctypes as C
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

WRAP = r"""
#include "era_rule.h"
extern "C" long long era_len(long long first, long long last,
                             long long dt_max, int dml) {
  return tsbts_dynamic_era_ticks(first, last, dt_max, dml);
}
extern "C" long long first_bad(long long T, long long dt_max, long long n,
                               const double* m, const double* r,
                               const double* v, const double* a,
                               const int64_t* tau, const int64_t* dt,
                               const double* dts) {
  return tsbts_first_bad_body(T, dt_max, n, m, r, v, a, tau, dt, dts);
}
"""

DP = C.POINTER(C.c_double)
LP = C.POINTER(C.c_int64)


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("era_rule")
    src, so = d / "w.cpp", d / "libw.so"
    src.write_text(WRAP)
    subprocess.run([cxx, "-std=c++17", "-O2", "-shared", "-fPIC", "-I", CSRC,
                    str(src), "-o", str(so)], check=True)
    L = C.CDLL(str(so))
    L.era_len.restype = C.c_longlong
    L.era_len.argtypes = [C.c_longlong, C.c_longlong, C.c_longlong, C.c_int]
    L.first_bad.restype = C.c_longlong
    L.first_bad.argtypes = [C.c_longlong, C.c_longlong, C.c_longlong, DP, DP,
                            DP, DP, LP, LP, DP]
    return L


def rule(first, last, dt_max, dyn_min_log2):
    """Alg. 3 (R11): last - first, clamped to [dt_max 2^-dyn_min_log2 (at
    least one tick), dt_max], then the smallest power of two that long."""
    span = min(max(last - first, max(dt_max >> dyn_min_log2, 1)), dt_max)
    p = 1
    while p < span:
        p *= 2
    return p


def test_era_length_on_random_and_edge_inputs(lib):
    rng = np.random.default_rng(3)
    rows = []
    for _ in range(4000):
        dt_max = 2 ** (K_MAX - int(rng.integers(0, 21)))
        first = int(rng.integers(1, 2 ** 30))
        last = first + int(rng.integers(0, 2 * dt_max + 1))
        rows.append((first, last, dt_max, int(rng.integers(0, 41))))
    for dt_max in (1, 2, 2 ** 17, 2 ** 20):
        for span in (0, 1, dt_max // 2 - 1, dt_max // 2, dt_max // 2 + 1,
                     dt_max - 1, dt_max, dt_max + 1):
            for dml in (0, 3, 40):
                rows.append((100, 100 + max(span, 0), dt_max, dml))
    for row in rows:
        assert lib.era_len(*row) == rule(*row), row


@pytest.mark.parametrize("seed,eta,dt_max", [(1, 0.02, 1 / 8), (4, 0.05, 1 / 4),
                                             (9, 0.01, 1 / 2)])
def test_era_length_gives_the_oracles_eras(lib, seed, eta, dt_max):
    m, r, v = inputs.plummer(128, seed)
    kw = dict(eps=0.01, eta=eta, dt_max=dt_max, era_mode=1, k_max=K_MAX)
    full = oracle.Sim(m, r, v, **kw)
    full.run(0.5)
    ts, te = full.eras()
    probe = oracle.Sim(m, r, v, **kw)
    assert len(ts) >= 2
    for k in range(len(ts) - 1):    # the last era may be cut by t_end
        probe.run(int(ts[k]) * 2.0 ** -K_MAX)
        st = probe.state()
        nxt = st["tau"] + st["dt"]
        got = lib.era_len(int(nxt.min()), int(nxt.max()),
                          int(dt_max * 2 ** K_MAX), 3)
        assert got == int(te[k] - ts[k]), k


def first_bad(lib, T, dt_max_t, m, st):
    m = np.ascontiguousarray(m, np.float64)
    r, v, a = (np.ascontiguousarray(st[k], np.float64) for k in "rva")
    tau, dt = (np.ascontiguousarray(st[k], np.int64) for k in ("tau", "dt"))
    dts = np.ascontiguousarray(st["dts"], np.float64)
    p = lambda x, t=DP: x.ctypes.data_as(t)  # noqa: E731
    return lib.first_bad(T, dt_max_t, m.shape[0], p(m), p(r), p(v), p(a),
                         p(tau, LP), p(dt, LP), p(dts))


def test_resume_check_agrees_with_the_oracle(lib):
    m, r, v = inputs.plummer(48, 17)
    kw = dict(eps=0.02, eta=0.03, dt_max=1 / 8, era_mode=0, era_log2=4,
              k_max=K_MAX)
    dt_max_t = 2 ** K_MAX // 8
    s = oracle.Sim(m, r, v, **kw)
    rng = np.random.default_rng(8)
    checked = refused = 0
    for t in (1 / 16, 1 / 8, 3 / 16):
        s.run(t)
        T = int(t * 2 ** K_MAX)
        st = s.state()
        assert first_bad(lib, T, dt_max_t, m, st) == -1
        for _ in range(150):
            bad = {k: np.copy(x) for k, x in st.items()}
            mm = np.copy(m)
            i = int(rng.integers(0, 48))
            kind = int(rng.integers(0, 8))
            if kind == 0:
                bad["dt"][i] = int(rng.choice([0, 3, 6, dt_max_t * 2,
                                               dt_max_t, 1, -4]))
            elif kind == 1:
                bad["tau"][i] = T - int(rng.integers(-3, 9))
            elif kind == 2:
                bad["tau"][i], bad["dt"][i] = (
                    T - int(rng.integers(0, 5)), int(rng.choice([1, 2, 4])))
            elif kind == 3:
                bad["dts"][i] = float(rng.choice([0.0, -1.0, np.nan, np.inf,
                                                  1e-300]))
            elif kind == 4:
                mm[i] = float(rng.choice([np.nan, np.inf, -1.0, 0.0]))
            else:
                key = "rva"[kind - 5]
                bad[key][i, int(rng.integers(0, 3))] = float(
                    rng.choice([np.nan, -np.inf, 1e300, 0.0]))
            got = first_bad(lib, T, dt_max_t, mm, bad)
            probe = oracle.Sim(m, r, v, **kw)
            try:
                probe.set_state(t, mm, bad)
                accepted = True
            except ValueError:
                accepted = False
            probe.close()
            assert (got == -1) == accepted, (kind, i)
            if not accepted:
                assert got == i
                refused += 1
            checked += 1
    assert checked == 450 and 100 < refused < 450
    # spoils that only one condition refuses
    T = int(3 / 16 * 2 ** K_MAX)
    st = s.state()
    for tau, dt in ((0, 2 * dt_max_t),     # step above dt_max only
                    (T + 4, 4),            # ahead of the system time only
                    (T - 4, 4),            # next time not after T only
                    (T - 2, 4),            # off its step grid only
                    (T, 3)):               # not a power of two only
        bad = {k: np.copy(x) for k, x in st.items()}
        bad["tau"][5], bad["dt"][5] = tau, dt
        assert first_bad(lib, T, dt_max_t, m, bad) == 5, (tau, dt)
        with pytest.raises(ValueError):
            s.set_state(3 / 16, m, bad)
