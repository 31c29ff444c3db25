"""The oracle's pins catch plausible mistakes (a mutation check).

Each entry plants one mistake in a copy of the oracle's C source under a
temporary directory, and the oracle pin tests run against that copy: some
test must fail (and none may error, e.g. on a compile failure). The
mistakes are the ones a reader of the paper might make: a dropped term, a
wrong sign or factor, a wrong bracket, a skipped reset or restore, a
missing check.

tests/test_oracle_golden.py is left out: as a regression guard it would
catch every change to the arithmetic and prove nothing about the pins.
Two passes over the pin tests are long or opt-in (the Sec. 3 experiment,
this file) and are left out as well.
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
SKIP = {"test_oracle_golden.py", "test_oracle_sec3_energy.py",
        "test_oracle_mutations.py"}

# (file, name, the mistake, anchor in the source, replacement)
MUTANTS = [
    ('tsbts_oracle.c', 'hermite_h11_sign', 'Hermite basis h11 with the wrong sign (R6)',
     'const double h11 = x * x * (x - 1.0);',
     'const double h11 = x * x * (1.0 - x);'),
    ('tsbts_oracle.c', 'taylor_half', 'Eq. 2 without the 1/2 on a',
     'rp[c] = r[c] + v[c] * h + 0.5 * a[c] * h * h;',
     'rp[c] = r[c] + v[c] * h + a[c] * h * h;'),
    ('tsbts_oracle.c', 'kick_new_only', 'Eq. 1 kick with the new force only',
     '0.5 * (s->a[3 * i + c] + s->an[3 * k + c]) * h',
     's->an[3 * k + c] * h'),
    ('tsbts_oracle.c', 'sym_min_not_avg', 'Eq. 4 with the minimum instead of the average',
     '2 * d <= orc_level_ticks((dts + dte_2d) / 2.0',
     '2 * d <= orc_level_ticks((dts < dte_2d ? dts : dte_2d)'),
    ('tsbts_oracle.c', 'no_restore_dt', 'a pass restarts without restoring the steps',
     '        memcpy(s->dt, s->dt0, ni);\n        history',
     '        history'),
    ('tsbts_oracle.c', 'dte_fallback_always', 'R8: the previous pass estimate never used',
     'if (k + 1 >= h->len) return fallback;',
     'return fallback;'),
    ('tsbts_oracle.c', 'odd_allows_double', 'Alg. 1 doubling allowed at odd times',
     'const int even = (tau % (2 * d)) == 0;',
     'const int even = 1;'),
    ('tsbts_oracle.c', 'phi_self', 'self pair counted when eps > 0',
     'if (j == i) continue;\n    const double dx = r[3 * j + 0] - r[3 * i + 0];\n    const double dy = r[3 * j + 1] - r[3 * i + 1];\n    const double dz = r[3 * j + 2] - r[3 * i + 2];\n    const double s2 = dx * dx + dy * dy + dz * dz + eps2;\n    const double s = sqrt(s2);',
     'const double dx = r[3 * j + 0] - r[3 * i + 0];\n    const double dy = r[3 * j + 1] - r[3 * i + 1];\n    const double dz = r[3 * j + 2] - r[3 * i + 2];\n    const double s2 = dx * dx + dy * dy + dz * dz + eps2;\n    const double s = sqrt(s2); if (j == i && eps2 == 0) continue;'),
    ('tsbts_oracle.c', 'q_unsoftened_coll', 'R1: unsoftened collision term',
     '/ s2; /* |v_ij|^2/s^2 */',
     '/ (s2 - eps2 + 1e-300); /* |v_ij|^2/s^2 */'),
    ('tsbts_oracle.c', 'dyn_no_pow2', 'Alg. 3 era not rounded to a power of two',
     '  while (p < e) p *= 2;\n  return p;',
     '  return e;'),
    ('tsbts_oracle.c', 'era_rounded_down', 'R11 era rounded down, not up',
     '  while (p < e) p *= 2;',
     '  while (2 * p <= e) p *= 2;'),
    ('tsbts_oracle.c', 'fwd_no_commensurate', 'R9 without commensurability',
     'while (tau % c != 0) c /= 2;',
     ''),
    ('tsbts_oracle.c', 'vpred_half', 'Eq. 2 velocity with a 1/2',
     'vp[c] = v[c] + a[c] * h;',
     'vp[c] = v[c] + 0.5 * a[c] * h;'),
    ('tsbts_oracle.c', 'interp_same_record', 'R6 interpolation between a record and itself',
     'const record* B = &hp->rec[k + 1];\n    orc_hermite',
     'const record* B = &hp->rec[k + 1];\n    A = B; orc_hermite'),
    ('tsbts_oracle.c', 'bracket_off_by_one', 'R6 bracket one record early',
     'const record* A = &hp->rec[k];\n    const record* B = &hp->rec[k + 1];\n    orc_hermite',
     'const record* A = &hp->rec[k > 0 ? k - 1 : k];\n    const record* B = &hp->rec[k > 0 ? k : k + 1];\n    orc_hermite'),
    ('tsbts_oracle.c', 'no_interp', 'passes >= 1 never interpolate',
     'if (pass > 0 && !s->is_act[j]) {',
     'if (0) {'),
    ('tsbts_oracle.c', 'dte_nearest_not_linear', 'R8 nearest record instead of linear',
     'return A->dts + (B->dts - A->dts) * w;',
     'return w < 0.5 ? A->dts : B->dts;'),
    ('tsbts_oracle.c', 'exact_hit_interpolated', 'R6 exact record hit not taken as is',
     'if (k >= 0 && hp->rec[k].tau == tn) {',
     'if (0) {'),
    ('tsbts_oracle.c', 'taylor_outside_uses_record', 'R6 record copied outside the bracket',
     '    taylor(r, v, a, ticks_to_time(tn - tj, k_max), rp, vp);\n  }\n}',
     '    if (k >= 0) { memcpy(rp, hp->rec[k].r, 24); memcpy(vp, hp->rec[k].v, 24); } else taylor(r, v, a, ticks_to_time(tn - tj, k_max), rp, vp);\n  }\n}'),
    ('tsbts_adjoint.c', 'drop_3ld_term_i', 'force VJP without the -3(l.d)d/s^5 term (i side)',
     'gx += m[j] * (lx / s3 - 3.0 * ld * dx / s5);\n      gy += m[j] * (ly / s3 - 3.0 * ld * dy / s5);\n      gz += m[j] * (lz / s3 - 3.0 * ld * dz / s5);\n    }\n    gi',
     'gx += m[j] * (lx / s3);\n      gy += m[j] * (ly / s3);\n      gz += m[j] * (lz / s3);\n    }\n    gi'),
    ('tsbts_adjoint.c', 'j_side_sign', 'force VJP j side with the wrong sign',
     'gp[3 * j] += gx;',
     'gp[3 * j] -= gx;'),
    ('tsbts_adjoint.c', 'mass_sign', 'mass cotangent with the wrong sign',
     'mm += ld / s3;',
     'mm -= ld / s3;'),
    ('tsbts_adjoint.c', 'no_init_force_vjp', 'initial force left out of the reverse sweep',
     'force_vjp(n, m, r0, eps2, n, all, gA, gp, gm);',
     ''),
    ('tsbts_adjoint.c', 'taylor_a_full_h2', 'Eq. 2 adjoint without the 1/2',
     'gA[3 * j + c] += 0.5 * h * h * gp[3 * j + c];',
     'gA[3 * j + c] += h * h * gp[3 * j + c];'),
    ('tsbts_adjoint.c', 'lam_no_half', 'Eq. 1 adjoint without the 1/2',
     'lam[3 * k + c] = gA[3 * i + c] + 0.5 * h * gV[3 * i + c];',
     'lam[3 * k + c] = gA[3 * i + c] + h * gV[3 * i + c];'),
    ('tsbts_adjoint.c', 'gA_active_not_reset', 'acceleration cotangent not reset',
     'gA[3 * i + c] = 0.5 * h * gV[3 * i + c];',
     'gA[3 * i + c] += 0.5 * h * gV[3 * i + c];'),
    ('tsbts_adjoint.c', 'gR_active_not_reset', 'position cotangent not reset',
     'gR[3 * i + c] = 0.0;',
     ''),
    ('tsbts_adjoint.c', 'no_restore_tau', 'tape restore forgets the body time',
     'tau[i] = x->tau;',
     ''),
    ('tsbts_adjoint.c', 'loss_gm_no_L', 'loss mass partial without the quotient term',
     'g_m[i] = (r2 - L) / M;',
     'g_m[i] = r2 / M;'),
    ('tsbts_adjoint.c', 'pred_v_in_fwd', 'replay prediction without the 1/2',
     'r[3 * j + c] + v[3 * j + c] * h + 0.5 * a[3 * j + c] * h * h;',
     'r[3 * j + c] + v[3 * j + c] * h + a[3 * j + c] * h * h;'),
    ('tsbts_adjoint.c', 'self_pair_in_j', 'self pair in the VJP j side',
     'if (i == j) continue;\n      const double lx',
     'const double lx'),
    ('tsbts_adjoint_era.c', 'no_record_injection_r', 'record position cotangents dropped',
     'gR[3 * i + c] += P->grec_r[3 * rec + c];',
     ''),
    ('tsbts_adjoint_era.c', 'no_record_injection_v', 'record velocity cotangents dropped',
     'gV[3 * i + c] += P->grec_v[3 * rec + c];',
     ''),
    ('tsbts_adjoint_era.c', 'hermite_v_weights_swapped', 'Hermite adjoint weights swapped',
     'va[c] += how[j].w[1] * g[c];',
     'va[c] += how[j].w[3] * g[c];'),
    ('tsbts_adjoint_era.c', 'hermite_rb_weight_wrong', 'Hermite adjoint weight of r_b wrong',
     'rb[c] += how[j].w[2] * g[c];',
     'rb[c] += how[j].w[0] * g[c];'),
    ('tsbts_adjoint_era.c', 'no_start_records', 'era-start record cotangents dropped',
     'G0r[3 * b + c] += gR[3 * b + c] + P->grec_r[3 * k + c];',
     'G0r[3 * b + c] += gR[3 * b + c];'),
    ('tsbts_adjoint_era.c', 'exact_hit_dropped', 'exact-hit cotangent dropped',
     'for (int c = 0; c < 3; ++c) q[c] += g[c];',
     ''),
    ('tsbts_adjoint_era.c', 'G0a_missing', 'initial acceleration cotangent dropped',
     'G0a[3 * b + c] += gA[3 * b + c];',
     ''),
    ('tsbts_adjoint_era.c', 'records_ignored_all', 'interpolated predictions treated as Taylor',
     '} else if (how[j].kind == 1) {',
     '} else if (0) {'),
    ('tsbts_adjoint_era.c', 'start_record_tick_zero', 'later era: era-start records at tick 0',
     'P->rec_tau[P->rec_off[b]] = tau0 ? tau0[b] : 0;',
     'P->rec_tau[P->rec_off[b]] = 0;'),
    ('tsbts_adjoint_era.c', 'state_tau_ignored', 'later era: every body restarts at tick 0',
     'X->tau[b] = X->tau0 ? X->tau0[b] : 0;',
     'X->tau[b] = 0;'),
    ('tsbts_adjoint_era.c', 'state_a0_ignored', 'later era: start accelerations recomputed',
     '  if (a0_in) {\n    memcpy(a0, a0_in,',
     '  if (0) {\n    memcpy(a0, a0_in,'),
    ('tsbts_adjoint_era.c', 'ga_T_dropped', 'across eras: final acceleration cotangent dropped',
     'if (ga_T) memcpy(gA, ga_T, n3);',
     ''),
    ('tsbts_adjoint_era.c', 'g_a0_not_returned', 'across eras: start acceleration cotangent lost',
     'if (g_a0) memcpy(g_a0, G0a, n3);',
     'if (g_a0) memset(g_a0, 0, n3);'),
    # (the record-by-record time test alone is not reached in practice:
    # passes with equal record counts have had equal record times in every
    # case tried, so the mistake planted drops the whole schedule test)
    ('tsbts_oracle.c', 'conv_ignores_schedule', 'R15 stop without the schedule test',
     '    if (a->len != b->len) return 0;\n    for (int64_t k = 0; k < a->len; ++k)\n      if (a->rec[k].tau != b->rec[k].tau) return 0;\n',
     ''),
    ('tsbts_oracle.c', 'conv_ignores_positions', 'R15 stop without the position test',
     '      if (!(fabs(s->r[3 * i + c] - s->rlast[3 * i + c]) < s->cfg.conv_tol))\n        return 0;',
     ''),
    ('tsbts_oracle.c', 'set_state_no_dts', 'resume without the step estimates',
     'memcpy(s->dts, dts, n1);',
     ''),
    ('tsbts_oracle.c', 'set_state_no_multiple_check', 'resume accepts tau off its step grid',
     'tau[i] % d != 0 || ',
     ''),
    ('tsbts_oracle.c', 'set_state_no_time', 'resume keeps the old system time',
     '  s->t_sys = t;',
     ''),
]


def pin_tests():
    return sorted(f for f in os.listdir(HERE)
                  if f.startswith("test_oracle_") and f.endswith(".py")
                  and f not in SKIP)


def plant(top, fname, anchor, repl):
    src_dir = os.path.join(ROOT, "oracle")
    dst = os.path.join(top, "oracle")
    os.makedirs(dst)
    for f in os.listdir(src_dir):
        if f.endswith((".c", ".h", ".py")):
            shutil.copy(os.path.join(src_dir, f), dst)
    path = os.path.join(dst, fname)
    with open(path) as f:
        src = f.read()
    assert src.count(anchor) == 1, "anchor not unique in " + fname
    with open(path, "w") as f:
        f.write(src.replace(anchor, repl))
    os.symlink(os.path.join(ROOT, "paper_1205_2288_gb300"),
               os.path.join(top, "paper_1205_2288_gb300"))
    tdir = os.path.join(top, "tests")
    os.makedirs(tdir)
    for f in pin_tests() + ["conftest.py"]:
        shutil.copy(os.path.join(HERE, f), tdir)
    shutil.copytree(os.path.join(HERE, "golden"), os.path.join(tdir, "golden"))


def caught(top, only=None):
    env = dict(os.environ, OMP_NUM_THREADS="2")
    target = os.path.join("tests", only) if only else "tests"
    r = subprocess.run(
        [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
         target], cwd=top, capture_output=True, text=True, env=env,
        timeout=900)
    summary = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else ""
    return r.returncode == 1 and " failed" in summary and "error" not in \
        summary, summary


def test_every_planted_mistake_fails_a_pin(tmp_path):
    tops = []
    for fname, name, _, anchor, repl in MUTANTS:
        top = str(tmp_path / name)
        plant(top, fname, anchor, repl)
        tops.append(top)
    with cf.ThreadPoolExecutor(max_workers=max(1, (os.cpu_count() or 2) // 2)
                               ) as ex:
        results = list(ex.map(caught, tops))
    missed = [(m[1], m[2], s) for m, (ok, s) in zip(MUTANTS, results)
              if not ok]
    assert not missed, missed


# The time-symmetric interpolation of passes >= 1 (R6) was first caught
# only by the multi-pass adjoint replay, a second restatement of the same
# passes. The interpolation pin (test_oracle_interpolation.py) checks the
# passes against the mathematics of the Hermite interpolant; on its own it
# must catch every planted R6 mistake that changes a prediction.
R6_MUTANTS = ("no_interp", "interp_same_record", "bracket_off_by_one",
              "hermite_h11_sign", "taylor_outside_uses_record")


def test_interpolation_pin_alone_catches_the_r6_mistakes(tmp_path):
    chosen = [m for m in MUTANTS if m[1] in R6_MUTANTS]
    assert len(chosen) == len(R6_MUTANTS)
    tops = []
    for fname, name, _, anchor, repl in chosen:
        top = str(tmp_path / name)
        plant(top, fname, anchor, repl)
        tops.append(top)
    with cf.ThreadPoolExecutor(max_workers=max(1, (os.cpu_count() or 2) // 2)
                               ) as ex:
        results = list(ex.map(lambda t: caught(
            t, "test_oracle_interpolation.py"), tops))
    missed = [(m[1], m[2], s) for m, (ok, s) in zip(chosen, results)
              if not ok]
    assert not missed, missed
