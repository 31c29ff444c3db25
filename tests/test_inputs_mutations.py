"""The input recipe's pins catch plausible mistakes (a mutation check of
paper_1205_2288_gb300/inputs.py against tests/test_inputs.py).

Each entry plants one mistake in a copy of the generator under a temporary
directory; the input tests then run against that copy and some test must
fail (none may error).
"""
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

# (name, the mistake, anchor, replacement)
MUTANTS = [
    ("radius_exponent", "mass profile inverted with the wrong power",
     "x ** (-2.0 / 3.0)", "x ** (-1.0 / 3.0)"),
    ("mass_cut", "radial mass fraction cut at 0.99",
     "_MASS_CUT = 0.999", "_MASS_CUT = 0.99"),
    ("rejection_exponent", "speed density q^2 (1 - q^2)^(9/2)",
     "(1.0 - xs * xs) ** 3.5", "(1.0 - xs * xs) ** 4.5"),
    ("escape_speed_power", "escape speed with (1 + r^2)^(-1/2)",
     "(1.0 + radius * radius) ** -0.25", "(1.0 + radius * radius) ** -0.5"),
    ("velocity_scale", "velocities scaled up instead of down",
     "v *= 1.0 / math.sqrt(_PLUMMER_SCALE)", "v *= math.sqrt(_PLUMMER_SCALE)"),
    ("radius_scale", "radii scaled by the inverse length",
     "r *= _PLUMMER_SCALE", "r /= _PLUMMER_SCALE"),
    ("hemisphere", "directions on one hemisphere",
     "cos_t = g.uniform(-1.0, 1.0, n)", "cos_t = g.uniform(0.0, 1.0, n)"),
    ("sin_not_sqrt", "sin(theta) without the square root",
     "sin_t = np.sqrt(1.0 - cos_t * cos_t)", "sin_t = 1.0 - cos_t * cos_t"),
    ("no_com_frame", "positions left outside the centre-of-mass frame",
     "    r -= (m[:, None] * r).sum(axis=0) / mt\n", ""),
    ("salpeter_exponent", "inverse CDF with m^-alpha instead of m^(1-alpha)",
     "e = 1.0 - alpha", "e = -alpha"),
    ("sizes_linear", "cluster sizes uniform instead of log-uniform",
     "s = np.exp(g.uniform(math.log(n_lo), math.log(n_hi), n_clusters))",
     "s = g.uniform(n_lo, n_hi, n_clusters)"),
    ("eps_rule", "cluster softening 1/N_c",
     "eps = 4.0 / sizes.astype(np.float64)",
     "eps = 1.0 / sizes.astype(np.float64)"),
    ("subset_unsorted", "active subset left unsorted",
     "return np.sort(idx).astype(np.int32)", "return idx.astype(np.int32)"),
]


def plant(top, anchor, repl):
    pkg = os.path.join(top, PKG)
    os.makedirs(pkg)
    shutil.copy(os.path.join(ROOT, PKG, "__init__.py"), pkg)
    with open(os.path.join(ROOT, PKG, "inputs.py")) as f:
        src = f.read()
    assert src.count(anchor) == 1, anchor
    with open(os.path.join(pkg, "inputs.py"), "w") as f:
        f.write(src.replace(anchor, repl))
    tdir = os.path.join(top, "tests")
    os.makedirs(tdir)
    for f in ("test_inputs.py", "conftest.py"):
        shutil.copy(os.path.join(HERE, f), tdir)


def caught(top):
    r = subprocess.run(
        [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
         "tests"], cwd=top, capture_output=True, text=True, timeout=600)
    summary = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else ""
    return (r.returncode == 1 and " failed" in summary
            and "error" not in summary), summary


def test_every_planted_mistake_fails_an_input_pin(tmp_path):
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
