"""FP64 CPU oracle of the TSBTS integrator (Kaplan & Saygin, Sec. 2-4).

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the bench's
CPU-baseline leg may import this package. It is built from the plain C in
``tsbts_oracle.c`` (integrator) and ``tsbts_adjoint.c`` (frozen-schedule
replay and its reverse mode) with gcc and shares nothing with the CUDA
library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsbts_oracle.c")
_SRC_ADJ = os.path.join(_HERE, "tsbts_adjoint.c")
_SRC_ERA = os.path.join(_HERE, "tsbts_adjoint_era.c")
_HDR = os.path.join(_HERE, "tsbts_oracle.h")
_LIBDIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

I64 = C.c_int64
I32P = C.POINTER(C.c_int32)
I64P = C.POINTER(C.c_int64)
DP = C.POINTER(C.c_double)


class OrcCfg(C.Structure):
    _fields_ = [("n_iter", C.c_int), ("era_mode", C.c_int),
                ("era_log2", C.c_int), ("k_max", C.c_int),
                ("dyn_min_log2", C.c_int), ("log", C.c_int),
                ("eps", C.c_double), ("eta", C.c_double),
                ("dt_max", C.c_double), ("conv_tol", C.c_double),
                ("trace_body", C.c_int64)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP over bodies)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    newest = max(os.path.getmtime(x) for x in (_SRC, _SRC_ADJ, _SRC_ERA,
                                               _HDR))
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, _SRC_ADJ,
           _SRC_ERA, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_forces.argtypes = [I64, DP, DP, DP, C.c_double, I64, I32P,
                                     DP, DP, DP]
            L.orc_energy_of.argtypes = [I64, DP, DP, DP, C.c_double, DP, DP]
            L.orc_level_ticks.argtypes = [C.c_double, C.c_int, C.c_int, I64P]
            L.orc_level_ticks.restype = I64
            L.orc_forward_step.argtypes = [I64, I64, C.c_double, C.c_int,
                                           C.c_int, I64P]
            L.orc_forward_step.restype = I64
            L.orc_symmetric_step.argtypes = [I64, I64, C.c_double, C.c_double,
                                             C.c_double, C.c_int, C.c_int, I64P]
            L.orc_symmetric_step.restype = I64
            L.orc_hermite.argtypes = [I64, I64, I64, C.c_int, DP, DP, DP, DP,
                                      DP, DP, DP, DP]
            L.orc_create.argtypes = [I64, DP, DP, DP, C.POINTER(OrcCfg)]
            L.orc_create.restype = C.c_void_p
            L.orc_run.argtypes = [C.c_void_p, C.c_double]
            L.orc_run.restype = C.c_int
            L.orc_energy.argtypes = [C.c_void_p, DP, DP]
            L.orc_get_state.argtypes = [C.c_void_p, DP, DP, DP, I64P, I64P, DP]
            L.orc_set_state.argtypes = [C.c_void_p, I64, DP, DP, DP, DP, I64P,
                                        I64P, DP]
            L.orc_set_state.restype = C.c_int
            L.orc_stats.argtypes = [C.c_void_p, I64P]
            L.orc_log_steps.argtypes = [C.c_void_p]
            L.orc_log_steps.restype = I64
            L.orc_log_entries.argtypes = [C.c_void_p]
            L.orc_log_entries.restype = I64
            L.orc_log_get.argtypes = [C.c_void_p, I32P, I32P, I64P, I32P, I32P,
                                      I64P]
            L.orc_era_log.argtypes = [C.c_void_p, I64P, I64P]
            L.orc_era_log.restype = I64
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_trace_get.argtypes = [C.c_void_p, I32P, I32P, I64P, I32P,
                                        DP]
            L.orc_trace_get.restype = I64
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_get_threads.restype = C.c_int
            L.orc_hist_find.argtypes = [I64, I64P, I64]
            L.orc_hist_find.restype = I64
            L.orc_hist_dts_at.argtypes = [I64, I64P, DP, I64, C.c_double]
            L.orc_hist_dts_at.restype = C.c_double
            L.orc_predict_prev.argtypes = [I64, I64P, DP, DP, DP, I64, DP, DP,
                                           DP, I64, C.c_int, DP, DP]
            sched = [I64, I64P, I64P, I32P]
            L.orc_replay.argtypes = [I64, DP, DP, DP, C.c_double, C.c_int,
                                     *sched, DP, DP]
            L.orc_replay_vjp.argtypes = [I64, DP, DP, DP, C.c_double, C.c_int,
                                         *sched, DP, DP, DP, DP, DP]
            era = [I64, I64P, I64P, I64P, I32P]
            L.orc_era_replay.argtypes = [I64, DP, DP, DP, C.c_double,
                                         C.c_int, *era, DP, DP]
            L.orc_era_replay_vjp.argtypes = [I64, DP, DP, DP, C.c_double,
                                             C.c_int, *era, DP, DP, DP, DP,
                                             DP]
            L.orc_era_replay_state.argtypes = [I64, DP, DP, DP, DP, I64P,
                                               C.c_double, C.c_int, *era,
                                               DP, DP, DP, I64P]
            L.orc_era_replay_state_vjp.argtypes = [I64, DP, DP, DP, DP, I64P,
                                                   C.c_double, C.c_int, *era,
                                                   DP, DP, DP, DP, DP, DP,
                                                   DP]
            L.orc_loss_msr.argtypes = [I64, DP, DP, DP, DP]
            L.orc_loss_msr.restype = C.c_double
            _lib = L
    return _lib


def _d(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _p(x, t=DP):
    return x.ctypes.data_as(t)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def forces(m, r, v, eps, idx=None):
    """a (n_act, 3), phi (n_act,), q (n_act,) on bodies idx from all bodies."""
    m, r, v = _d(m), _d(r), _d(v)
    n = m.shape[0]
    idx = np.arange(n, dtype=np.int32) if idx is None else \
        np.ascontiguousarray(idx, dtype=np.int32)
    na = idx.shape[0]
    a = np.zeros((na, 3))
    phi = np.zeros(na)
    q = np.zeros(na)
    lib().orc_forces(n, _p(m), _p(r), _p(v), float(eps), na, _p(idx, I32P),
                     _p(a), _p(phi), _p(q))
    return a, phi, q


def energy_of(m, r, v, eps):
    m, r, v = _d(m), _d(r), _d(v)
    ek, ep = C.c_double(), C.c_double()
    lib().orc_energy_of(m.shape[0], _p(m), _p(r), _p(v), float(eps),
                        C.byref(ek), C.byref(ep))
    return ek.value, ep.value


def level_ticks(x, k_min, k_max):
    uf = C.c_int64(0)
    t = lib().orc_level_ticks(float(x), k_min, k_max, C.byref(uf))
    return int(t), int(uf.value)


def forward_step(tau, d, dts, k_min, k_max):
    uf = C.c_int64(0)
    t = lib().orc_forward_step(int(tau), int(d), float(dts), k_min, k_max,
                               C.byref(uf))
    return int(t), int(uf.value)


def symmetric_step(tau, d, dts, dte_2d, dte_d, k_min, k_max):
    uf = C.c_int64(0)
    t = lib().orc_symmetric_step(int(tau), int(d), float(dts), float(dte_2d),
                                 float(dte_d), k_min, k_max, C.byref(uf))
    return int(t), int(uf.value)


def hermite(ta, tb, t, k_max, ra, va, aa, rb, vb, ab):
    ro, vo = np.zeros(3), np.zeros(3)
    args = [_d(x) for x in (ra, va, aa, rb, vb, ab)]
    lib().orc_hermite(int(ta), int(tb), int(t), int(k_max),
                      *[_p(x) for x in args], _p(ro), _p(vo))
    return ro, vo


def hist_find(tau, t):
    """Index of the last record with tau <= t, or -1 (R6)."""
    tau = np.ascontiguousarray(tau, dtype=np.int64)
    return int(lib().orc_hist_find(tau.shape[0], _p(tau, I64P), int(t)))


def hist_dts_at(tau, dts, t, fallback):
    """Previous pass's step estimate at tick t (R8)."""
    tau = np.ascontiguousarray(tau, dtype=np.int64)
    dts = _d(dts)
    return float(lib().orc_hist_dts_at(tau.shape[0], _p(tau, I64P), _p(dts),
                                       int(t), float(fallback)))


def predict_prev(tau, r, v, a, tj, rj, vj, aj, tn, k_max):
    """Prediction of a non-active body in a pass >= 1 (R6)."""
    tau = np.ascontiguousarray(tau, dtype=np.int64)
    r, v, a = _d(r), _d(v), _d(a)
    rj, vj, aj = _d(rj), _d(vj), _d(aj)
    rp, vp = np.zeros(3), np.zeros(3)
    lib().orc_predict_prev(tau.shape[0], _p(tau, I64P), _p(r), _p(v), _p(a),
                           int(tj), _p(rj), _p(vj), _p(aj), int(tn),
                           int(k_max), _p(rp), _p(vp))
    return rp, vp


def final_pass(sched, era=-1):
    """The block schedule of one era's last pass, from a schedule log:
    (step_tau, step_off, act) with the active bodies ascending per step."""
    eras = np.unique(sched["era"])
    e = eras[era]
    sel = sched["era"] == e
    last = sched["pass_"][sel].max()
    sel &= sched["pass_"] == last
    off = np.concatenate([[0], np.cumsum(sched["n_act"])]).astype(np.int64)
    steps = np.nonzero(sel)[0]
    tau = sched["tau"][steps].astype(np.int64)
    parts = [np.sort(sched["idx"][off[k]:off[k + 1]]) for k in steps]
    step_off = np.concatenate([[0], np.cumsum([len(x) for x in parts])])
    act = np.concatenate(parts) if parts else np.zeros(0, np.int32)
    return (np.ascontiguousarray(tau), step_off.astype(np.int64),
            np.ascontiguousarray(act, dtype=np.int32))


def _sched_args(schedule):
    tau, off, act = schedule
    tau = np.ascontiguousarray(tau, dtype=np.int64)
    off = np.ascontiguousarray(off, dtype=np.int64)
    act = np.ascontiguousarray(act, dtype=np.int32)
    return (tau, off, act), [tau.shape[0], _p(tau, I64P), _p(off, I64P),
                             _p(act, I32P)]


def replay(m, r0, v0, eps, k_max, schedule):
    """Final (r, v) of the Taylor replay of a frozen schedule (R14)."""
    m, r0, v0 = _d(m), _d(r0), _d(v0)
    keep, sa = _sched_args(schedule)
    r, v = np.zeros_like(r0), np.zeros_like(v0)
    lib().orc_replay(m.shape[0], _p(m), _p(r0), _p(v0), float(eps),
                     int(k_max), *sa, _p(r), _p(v))
    return r, v


def replay_vjp(m, r0, v0, eps, k_max, schedule, gr_T, gv_T):
    """Cotangents (g_r0, g_v0, g_m) of the replay for final cotangents."""
    m, r0, v0 = _d(m), _d(r0), _d(v0)
    gr_T, gv_T = _d(gr_T), _d(gv_T)
    keep, sa = _sched_args(schedule)
    g_r0, g_v0, g_m = np.zeros_like(r0), np.zeros_like(v0), np.zeros_like(m)
    lib().orc_replay_vjp(m.shape[0], _p(m), _p(r0), _p(v0), float(eps),
                         int(k_max), *sa, _p(gr_T), _p(gv_T), _p(g_r0),
                         _p(g_v0), _p(g_m))
    return g_r0, g_v0, g_m


def era_passes(sched, era=0):
    """Every pass of one era from a schedule log: a list of
    (step_tau, step_off, act) per pass, active bodies ascending per step."""
    off = np.concatenate([[0], np.cumsum(sched["n_act"])]).astype(np.int64)
    sel = np.flatnonzero(sched["era"] == np.unique(sched["era"])[era])
    out = []
    for p in np.unique(sched["pass_"][sel]):
        steps = sel[sched["pass_"][sel] == p]
        parts = [np.sort(sched["idx"][off[k]:off[k + 1]]) for k in steps]
        so = np.concatenate([[0], np.cumsum([len(x) for x in parts])])
        out.append((sched["tau"][steps].astype(np.int64), so.astype(np.int64),
                    np.concatenate(parts).astype(np.int32)))
    return out


def _era_args(passes):
    tau = np.concatenate([p[0] for p in passes]).astype(np.int64)
    pass_off = np.concatenate([[0], np.cumsum([len(p[0]) for p in passes])])
    offs, base = [], 0
    for i, p in enumerate(passes):
        o = np.asarray(p[1], np.int64) + base
        offs.append(o if i == len(passes) - 1 else o[:-1])
        base = int(o[-1])
    step_off = np.concatenate(offs).astype(np.int64)
    act = np.concatenate([p[2] for p in passes]).astype(np.int32)
    pass_off = np.ascontiguousarray(pass_off, dtype=np.int64)
    keep = (tau, pass_off, step_off, act)
    return keep, [len(passes), _p(pass_off, I64P), _p(tau, I64P),
                  _p(step_off, I64P), _p(act, I32P)]


def era_replay(m, r0, v0, eps, k_max, passes):
    """Last pass's final (r, v) of the multi-pass era replay."""
    m, r0, v0 = _d(m), _d(r0), _d(v0)
    keep, ea = _era_args(passes)
    r, v = np.zeros_like(r0), np.zeros_like(v0)
    lib().orc_era_replay(m.shape[0], _p(m), _p(r0), _p(v0), float(eps),
                         int(k_max), *ea, _p(r), _p(v))
    return r, v


def era_replay_vjp(m, r0, v0, eps, k_max, passes, gr_T, gv_T):
    """Cotangents (g_r0, g_v0, g_m) through every pass of the era."""
    m, r0, v0 = _d(m), _d(r0), _d(v0)
    gr_T, gv_T = _d(gr_T), _d(gv_T)
    keep, ea = _era_args(passes)
    g_r0, g_v0, g_m = np.zeros_like(r0), np.zeros_like(v0), np.zeros_like(m)
    lib().orc_era_replay_vjp(m.shape[0], _p(m), _p(r0), _p(v0), float(eps),
                             int(k_max), *ea, _p(gr_T), _p(gv_T), _p(g_r0),
                             _p(g_v0), _p(g_m))
    return g_r0, g_v0, g_m


def _opt(x, t=DP):
    return None if x is None else _p(x, t)


def era_replay_state(m, r0, v0, a0, tau0, eps, k_max, passes):
    """Multi-pass era replay from a general era-start state (each body at
    tick tau0 with acceleration a0; None: tick 0 and the force at r0):
    the last pass's final (r, v, a, tau)."""
    m, r0, v0 = _d(m), _d(r0), _d(v0)
    a0 = None if a0 is None else _d(a0)
    tau0 = None if tau0 is None else np.ascontiguousarray(tau0, np.int64)
    keep, ea = _era_args(passes)
    r, v, a = np.zeros_like(r0), np.zeros_like(v0), np.zeros_like(r0)
    tau = np.zeros(m.shape[0], np.int64)
    lib().orc_era_replay_state(m.shape[0], _p(m), _p(r0), _p(v0), _opt(a0),
                               _opt(tau0, I64P), float(eps), int(k_max), *ea,
                               _p(r), _p(v), _p(a), _p(tau, I64P))
    return r, v, a, tau


def era_replay_state_vjp(m, r0, v0, a0, tau0, eps, k_max, passes, gr_T,
                         gv_T, ga_T):
    """Cotangents (g_r0, g_v0, g_a0, g_m) of era_replay_state for
    cotangents of its final r, v, a (None: zero)."""
    m, r0, v0 = _d(m), _d(r0), _d(v0)
    a0 = None if a0 is None else _d(a0)
    tau0 = None if tau0 is None else np.ascontiguousarray(tau0, np.int64)
    gs = [None if g is None else _d(g) for g in (gr_T, gv_T, ga_T)]
    keep, ea = _era_args(passes)
    g_r0, g_v0, g_a0 = (np.zeros_like(r0) for _ in range(3))
    g_m = np.zeros_like(m)
    lib().orc_era_replay_state_vjp(m.shape[0], _p(m), _p(r0), _p(v0),
                                   _opt(a0), _opt(tau0, I64P), float(eps),
                                   int(k_max), *ea, *(_opt(g) for g in gs),
                                   _p(g_r0), _p(g_v0), _p(g_a0), _p(g_m))
    return g_r0, g_v0, g_a0, g_m


def eras_replay(m, r0, v0, eps, k_max, eras):
    """Replay of consecutive eras (each a list of passes) from (r0, v0) at
    tick 0: every era starts from the state the era before it left. Returns
    the final (r, v, a, tau) and the era-start states [(r, v, a, tau)]."""
    state = (_d(r0), _d(v0), None, None)
    starts = []
    for passes in eras:
        starts.append(state)
        state = era_replay_state(m, *state, eps, k_max, passes)
    return state, starts


def eras_replay_vjp(m, r0, v0, eps, k_max, eras, gr_T, gv_T, ga_T=None):
    """Adjoint across eras: the cotangents (g_r0, g_v0, g_m) of the
    initial state for cotangents of the final r, v, a, chaining each era's
    reverse mode from the last era to the first."""
    _, starts = eras_replay(m, r0, v0, eps, k_max, eras)
    g = (gr_T, gv_T, ga_T)
    g_m = np.zeros(len(m))
    for passes, st in zip(reversed(eras), reversed(starts)):
        gr, gv, ga, gm = era_replay_state_vjp(m, *st, eps, k_max, passes, *g)
        g_m += gm
        g = (gr, gv, ga)
    return g[0], g[1], g_m


def loss_msr(m, r):
    """L = sum m |r|^2 / sum m with its partials (L, dL/dr, dL/dm)."""
    m, r = _d(m), _d(r)
    g_r, g_m = np.zeros_like(r), np.zeros_like(m)
    L = lib().orc_loss_msr(m.shape[0], _p(m), _p(r), _p(g_r), _p(g_m))
    return L, g_r, g_m


def loss_grad(m, r0, v0, eps, k_max, schedule):
    """The loss of the replayed final positions and its gradient with
    respect to r0, v0 and m (chain rule through orc_replay_vjp)."""
    rT, _ = replay(m, r0, v0, eps, k_max, schedule)
    L, g_rT, g_mL = loss_msr(m, rT)
    g_r0, g_v0, g_m = replay_vjp(m, r0, v0, eps, k_max, schedule, g_rT,
                                 np.zeros_like(g_rT))
    return L, g_r0, g_v0, g_m + g_mL


class Sim:
    """One oracle integration (Alg. 2 / Alg. 3) over seeded inputs."""

    def __init__(self, m, r, v, *, eps, eta, dt_max, n_iter=3, era_mode=0,
                 era_log2=3, k_max=20, dyn_min_log2=3, log=False,
                 conv_tol=0.0, trace_body=-1):
        self.m, r, v = _d(m), _d(r), _d(v)
        self.n = self.m.shape[0]
        self.k_max = k_max
        cfg = OrcCfg(n_iter, era_mode, era_log2, k_max, dyn_min_log2,
                     1 if log else 0, eps, eta, dt_max, conv_tol,
                     int(trace_body))
        self._s = lib().orc_create(self.n, _p(self.m), _p(r), _p(v),
                                   C.byref(cfg))

    def run(self, t_end):
        rc = lib().orc_run(self._s, float(t_end))
        if rc != 0:
            raise ValueError(f"oracle run refused t_end={t_end}")

    def energy(self):
        ek, ep = C.c_double(), C.c_double()
        lib().orc_energy(self._s, C.byref(ek), C.byref(ep))
        return ek.value, ep.value

    def state(self):
        n = self.n
        r, v, a = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
        tau, dt = np.zeros(n, np.int64), np.zeros(n, np.int64)
        dts = np.zeros(n)
        lib().orc_get_state(self._s, _p(r), _p(v), _p(a), _p(tau, I64P),
                            _p(dt, I64P), _p(dts))
        return dict(r=r, v=v, a=a, tau=tau, dt=dt, dts=dts)

    def set_state(self, t, m, st):
        """Resume at an era end: system time t (time units, a whole number
        of ticks), masses m and the fields of state() (r, v, a, tau, dt,
        dts). Raises ValueError (state unchanged) when the state could not
        end an era."""
        tt = float(t) * 2.0 ** self.k_max
        if tt != np.floor(tt):
            raise ValueError("t is not a whole number of ticks")
        n = self.n
        m = _d(m).reshape(n)
        r, v, a = (_d(st[k]).reshape(n, 3) for k in ("r", "v", "a"))
        tau = np.ascontiguousarray(st["tau"], np.int64).reshape(n)
        dt = np.ascontiguousarray(st["dt"], np.int64).reshape(n)
        dts = _d(st["dts"]).reshape(n)
        rc = lib().orc_set_state(self._s, int(tt), _p(m), _p(r), _p(v), _p(a),
                                 _p(tau, I64P), _p(dt, I64P), _p(dts))
        if rc != 0:
            raise ValueError("state cannot end an era")
        self.m = m.copy()

    def stats(self):
        out = np.zeros(7, np.int64)
        lib().orc_stats(self._s, _p(out, I64P))
        keys = ("block_steps", "interactions", "eras", "passes", "underflow",
                "t_sys_ticks", "init_interactions")
        return dict(zip(keys, (int(x) for x in out)))

    def schedule(self):
        L = lib()
        ns, ne = L.orc_log_steps(self._s), L.orc_log_entries(self._s)
        era = np.zeros(ns, np.int32)
        pas = np.zeros(ns, np.int32)
        tau = np.zeros(ns, np.int64)
        nact = np.zeros(ns, np.int32)
        ei = np.zeros(ne, np.int32)
        edt = np.zeros(ne, np.int64)
        L.orc_log_get(self._s, _p(era, I32P), _p(pas, I32P), _p(tau, I64P),
                      _p(nact, I32P), _p(ei, I32P), _p(edt, I64P))
        return dict(era=era, pass_=pas, tau=tau, n_act=nact, idx=ei, dt=edt)

    def trace(self):
        """The traced body's entries (see orc_trace_get): dict of era,
        pass_, tau, kind (0 predicted, 1 corrected) and r, v, a (k, 3)."""
        L = lib()
        k = L.orc_trace_get(self._s, None, None, None, None, None)
        era, pas = np.zeros(k, np.int32), np.zeros(k, np.int32)
        tau, kind = np.zeros(k, np.int64), np.zeros(k, np.int32)
        rva = np.zeros((k, 9))
        L.orc_trace_get(self._s, _p(era, I32P), _p(pas, I32P), _p(tau, I64P),
                        _p(kind, I32P), _p(rva))
        return dict(era=era, pass_=pas, tau=tau, kind=kind, r=rva[:, 0:3],
                    v=rva[:, 3:6], a=rva[:, 6:9])

    def eras(self):
        L = lib()
        ne = L.orc_era_log(self._s, None, None)
        ts, te = np.zeros(ne, np.int64), np.zeros(ne, np.int64)
        L.orc_era_log(self._s, _p(ts, I64P), _p(te, I64P))
        return ts, te

    def close(self):
        if self._s:
            lib().orc_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
