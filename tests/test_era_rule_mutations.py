"""The CPU checks of the library's era-boundary arithmetic
(tests/test_era_rule.py) catch plausible mistakes in csrc/era_rule.h (a
mutation check). Each entry plants one mistake in a copy of the header
under a temporary directory; the checks then run against that copy and
some check must fail (none may error)."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

pytestmark = pytest.mark.slow

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
PKG = "paper_1205_2288_gb300"

# (name, the mistake, anchor, replacement). Dropping the one-tick floor
# of the lower clamp is not among them: the era starts at one tick and only
# doubles, so that mistake changes no result.
MUTANTS = [
    ("rounded_down", "era rounded down to a power of two",
     "while (p2 < e) p2 *= 2;", "while (2 * p2 <= e) p2 *= 2;"),
    ("no_lower_clamp", "era span not clamped below",
     "if (e < lo) e = lo;", ""),
    ("no_upper_clamp", "era span not clamped at dt_max",
     "if (e > dt_max_ticks) e = dt_max_ticks;", ""),
    ("step_not_power_of_two", "steps need not be powers of two",
     "(d & (d - 1)) == 0 && ", ""),
    ("step_above_dt_max", "steps above dt_max accepted",
     "d <= dt_max_ticks && ", ""),
    ("tau_off_grid", "body times off their step grid accepted",
     "ti % d == 0 && ", ""),
    ("body_past_its_next_time", "tau + dt <= T accepted",
     "T - ti < d", "T - ti <= d"),
    ("body_ahead", "tau > T accepted", "ti <= T && ", ""),
    ("dts_zero", "zero step estimate accepted", "dts[i] > 0.0", "dts[i] >= 0.0"),
    ("mass_unchecked", "non-finite mass accepted",
     "std::isfinite(m[i]) && ", ""),
    ("accel_unchecked", "non-finite acceleration accepted",
     " &&\n           std::isfinite(a[3 * (size_t)i + c])", ""),
]


def plant(top, anchor, repl):
    pkg = os.path.join(top, PKG)
    os.makedirs(os.path.join(pkg, "csrc"))
    for f in ("__init__.py", "inputs.py"):
        shutil.copy(os.path.join(ROOT, PKG, f), pkg)
    with open(os.path.join(ROOT, PKG, "csrc", "era_rule.h")) as f:
        src = f.read()
    assert src.count(anchor) == 1, anchor
    with open(os.path.join(pkg, "csrc", "era_rule.h"), "w") as f:
        f.write(src.replace(anchor, repl))
    os.symlink(os.path.join(ROOT, "oracle"), os.path.join(top, "oracle"))
    tdir = os.path.join(top, "tests")
    os.makedirs(tdir)
    for f in ("test_era_rule.py", "conftest.py"):
        shutil.copy(os.path.join(HERE, f), tdir)


def caught(top):
    # one OpenMP thread per copy: the copies run side by side
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(
        [sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
         "tests"], cwd=top, capture_output=True, text=True, timeout=600,
        env=env)
    summary = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else ""
    return (r.returncode == 1 and " failed" in summary
            and "error" not in summary), summary


def test_every_planted_mistake_fails_an_era_rule_check(tmp_path):
    import oracle
    oracle.lib()  # built once here; the copies link to this oracle
    tops = []
    for name, _, anchor, repl in MUTANTS:
        top = str(tmp_path / name)
        plant(top, anchor, repl)
        tops.append(top)
    with cf.ThreadPoolExecutor(max_workers=max(1, (os.cpu_count() or 2) // 2)
                               ) as ex:
        results = list(ex.map(caught, tops))
    missed = [(m[0], m[1], s) for m, (ok, s) in zip(MUTANTS, results)
              if not ok]
    assert not missed, missed
