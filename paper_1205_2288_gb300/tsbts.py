"""ctypes binding of the C ABI in include/tsbts.h (libtsbts.so).

The functions below carry the C names and only marshal arguments; every
step of the integrator runs in the CUDA library. There is no CPU fallback:
loading fails loudly when the library cannot be built or loaded, and
``tsbts_create`` fails without a CUDA device.
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np

from . import build as _build

I64 = C.c_int64
I32P = C.POINTER(C.c_int32)
I64P = C.POINTER(C.c_int64)
DP = C.POINTER(C.c_double)
VP = C.c_void_p

TSBTS_OK = 0
TSBTS_ERR_ARG = -1
TSBTS_ERR_CUDA = -2
TSBTS_ERR_NONFINITE = -3
TSBTS_ERR_TIMEOUT = -4
TSBTS_ERR_HISTORY = -6
TSBTS_ERR_STATE = -7
TSBTS_FP64 = 0
TSBTS_MIXED = 1

STATUS_NAMES = {0: "TSBTS_OK", -1: "TSBTS_ERR_ARG", -2: "TSBTS_ERR_CUDA",
                -3: "TSBTS_ERR_NONFINITE", -4: "TSBTS_ERR_TIMEOUT",
                -6: "TSBTS_ERR_HISTORY", -7: "TSBTS_ERR_STATE"}

# every symbol include/tsbts.h declares
EXPORTS = (
    "tsbts_config_default", "tsbts_create", "tsbts_init", "tsbts_init_device",
    "tsbts_step_era", "tsbts_energy", "tsbts_state", "tsbts_get_stats",
    "tsbts_set_timing", "tsbts_schedule_log", "tsbts_schedule_size",
    "tsbts_schedule_get", "tsbts_last_error", "tsbts_destroy", "tsbts_force",
    "tsbts_release_scratch", "tsbts_version", "tsbts_force_static",
    "tsbts_init_ensemble", "tsbts_ensemble_energy", "tsbts_adjoint_init",
    "tsbts_adjoint_forward", "tsbts_adjoint_vjp", "tsbts_adjoint_loss_grad",
    "tsbts_adjoint_get_stats", "tsbts_step_estimates", "tsbts_set_state",
    "tsbts_pipe_peak", "tsbts_adjoint_init_era", "tsbts_adjoint_forward_state",
    "tsbts_adjoint_vjp_state",
)


class tsbts_config(C.Structure):
    _fields_ = [("precision", C.c_int), ("n_iter", C.c_int),
                ("era_mode", C.c_int), ("era_log2", C.c_int),
                ("dyn_min_log2", C.c_int), ("k_max", C.c_int),
                ("exact_order", C.c_int), ("device", C.c_int),
                ("stream", C.c_void_p), ("graph_steps", C.c_int),
                ("conv_tol", C.c_double), ("max_pass_steps", I64)]


class tsbts_stats(C.Structure):
    _fields_ = [("block_steps", I64), ("interactions", I64), ("eras", I64),
                ("passes", I64), ("dt_underflow", I64),
                ("era_restarts", I64), ("history_capacity", I64),
                ("t_sys_ticks", I64), ("force_ms", C.c_double),
                ("force_launches", I64), ("kernel_launches", I64),
                ("force_interactions", I64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class tsbts_adjoint_stats(C.Structure):
    _fields_ = [("steps", I64), ("entries", I64), ("checkpoint_every", I64),
                ("checkpoints", I64), ("tape_entries", I64),
                ("tape_bytes", I64), ("checkpoint_bytes", I64),
                ("device_bytes", I64), ("pairs_forward", I64),
                ("pairs_backward", I64), ("forward_ms", C.c_double),
                ("backward_ms", C.c_double), ("kernel_launches", I64),
                ("passes", I64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TsbtsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.SO


def lib():
    """Load (building first if needed) libtsbts.so and declare signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        L = C.CDLL(_build.build())
        L.tsbts_config_default.argtypes = [C.POINTER(tsbts_config)]
        L.tsbts_config_default.restype = None
        L.tsbts_create.argtypes = [C.POINTER(VP), C.POINTER(tsbts_config)]
        L.tsbts_init.argtypes = [VP, I64, DP, DP, DP, C.c_double, C.c_double,
                                 C.c_double]
        L.tsbts_init_device.argtypes = [VP, I64, VP, VP, VP, C.c_double,
                                        C.c_double, C.c_double]
        L.tsbts_init_ensemble.argtypes = [VP, I64, I64P, DP, DP, DP, DP,
                                          C.c_double, C.c_double]
        L.tsbts_ensemble_energy.argtypes = [VP, DP, DP]
        L.tsbts_step_era.argtypes = [VP, C.c_double, DP]
        L.tsbts_energy.argtypes = [VP, DP, DP, DP]
        L.tsbts_state.argtypes = [VP, DP, DP, DP, DP, DP, I64P, I64P]
        L.tsbts_step_estimates.argtypes = [VP, DP]
        L.tsbts_set_state.argtypes = [VP, C.c_double, DP, DP, DP, DP, I64P,
                                      I64P, DP]
        L.tsbts_get_stats.argtypes = [VP, C.POINTER(tsbts_stats)]
        L.tsbts_set_timing.argtypes = [VP, C.c_int]
        L.tsbts_schedule_log.argtypes = [VP, I64]
        L.tsbts_schedule_size.argtypes = [VP, I64P, I64P, I64P]
        L.tsbts_schedule_get.argtypes = [VP, I32P, I32P, I64P, I32P, I32P,
                                         I64P]
        L.tsbts_last_error.argtypes = [VP]
        L.tsbts_last_error.restype = C.c_char_p
        L.tsbts_destroy.argtypes = [VP]
        L.tsbts_destroy.restype = None
        L.tsbts_force.argtypes = [C.c_int, C.c_int, I64, VP, VP, VP,
                                  C.c_double, I64, VP, VP, VP, VP, VP]
        L.tsbts_force_static.argtypes = [C.c_int, C.c_int, I64, VP, VP, VP,
                                         C.c_double, I64, VP, VP, VP, VP, VP]
        L.tsbts_release_scratch.argtypes = []
        L.tsbts_adjoint_init.argtypes = [VP, I64, C.c_double, I64, I64P,
                                         I64P, I32P, I64]
        L.tsbts_adjoint_init_era.argtypes = [VP, I64, C.c_double, I64, I64P,
                                             I64P, I64P, I32P, I64]
        L.tsbts_adjoint_forward.argtypes = [VP, VP, VP, VP, VP, VP, C.c_int]
        L.tsbts_adjoint_vjp.argtypes = [VP, VP, VP, VP, VP, VP, C.c_int]
        L.tsbts_adjoint_forward_state.argtypes = [VP, VP, VP, VP, VP, VP, VP,
                                                  VP, VP, VP, C.c_int]
        L.tsbts_adjoint_vjp_state.argtypes = [VP, VP, VP, VP, VP, VP, VP, VP,
                                              C.c_int]
        L.tsbts_adjoint_loss_grad.argtypes = [VP, VP, VP, VP, VP, VP, VP, VP,
                                              C.c_int]
        L.tsbts_adjoint_get_stats.argtypes = [VP,
                                              C.POINTER(tsbts_adjoint_stats)]
        L.tsbts_pipe_peak.argtypes = [C.c_int, I64, DP, DP]
        L.tsbts_version.argtypes = []
        L.tsbts_version.restype = C.c_char_p
        _lib = L
        return L


def _p(x, t=DP):
    return x.ctypes.data_as(t)


def _check(code, ctx=None):
    if code != TSBTS_OK:
        msg = ""
        if ctx:
            m = lib().tsbts_last_error(ctx)
            msg = m.decode() if m else ""
        raise TsbtsError(code, msg)


# --- thin wrappers with the C names -------------------------------------

def tsbts_config_default() -> tsbts_config:
    cfg = tsbts_config()
    lib().tsbts_config_default(C.byref(cfg))
    return cfg


def tsbts_create(cfg: tsbts_config):
    h = VP()
    _check(lib().tsbts_create(C.byref(h), C.byref(cfg)))
    return h


def tsbts_init(ctx, m, r, v, eps, eta, dt_max):
    m = np.ascontiguousarray(m, np.float64)
    r = np.ascontiguousarray(r, np.float64)
    v = np.ascontiguousarray(v, np.float64)
    n = m.shape[0]
    if r.shape != (n, 3) or v.shape != (n, 3):
        raise ValueError("r and v must have shape (n, 3)")
    _check(lib().tsbts_init(ctx, n, _p(m), _p(r), _p(v), float(eps),
                            float(eta), float(dt_max)), ctx)


def tsbts_init_device(ctx, m, r, v, eps, eta, dt_max):
    """m, r, v: contiguous float64 CUDA tensors of shape (n,), (n,3), (n,3)."""
    n = m.shape[0]
    _check(lib().tsbts_init_device(ctx, n, m.data_ptr(), r.data_ptr(),
                                   v.data_ptr(), float(eps), float(eta),
                                   float(dt_max)), ctx)


def tsbts_init_ensemble(ctx, offsets, m, r, v, eps, eta, dt_max):
    offsets = np.ascontiguousarray(offsets, np.int64)
    m = np.ascontiguousarray(m, np.float64)
    r = np.ascontiguousarray(r, np.float64)
    v = np.ascontiguousarray(v, np.float64)
    eps = np.ascontiguousarray(eps, np.float64)
    nc = offsets.shape[0] - 1
    if eps.shape != (nc,) or r.shape != (m.shape[0], 3) or \
            v.shape != (m.shape[0], 3):
        raise ValueError("shapes: offsets (nc+1,), eps (nc,), r and v (n, 3)")
    _check(lib().tsbts_init_ensemble(ctx, nc, _p(offsets, I64P), _p(m), _p(r),
                                     _p(v), _p(eps), float(eta),
                                     float(dt_max)), ctx)


def tsbts_ensemble_energy(ctx, n_clusters):
    ek, ep = np.zeros(n_clusters), np.zeros(n_clusters)
    _check(lib().tsbts_ensemble_energy(ctx, _p(ek), _p(ep)), ctx)
    return ek, ep


def tsbts_step_era(ctx, t_end) -> float:
    t = C.c_double()
    _check(lib().tsbts_step_era(ctx, float(t_end), C.byref(t)), ctx)
    return t.value


def tsbts_energy(ctx):
    ek, ep, et = C.c_double(), C.c_double(), C.c_double()
    _check(lib().tsbts_energy(ctx, C.byref(ek), C.byref(ep), C.byref(et)),
           ctx)
    return ek.value, ep.value, et.value


def tsbts_state(ctx, n):
    t = C.c_double()
    m = np.zeros(n)
    r, v, a = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
    tau, dt = np.zeros(n, np.int64), np.zeros(n, np.int64)
    _check(lib().tsbts_state(ctx, C.byref(t), _p(m), _p(r), _p(v), _p(a),
                             _p(tau, I64P), _p(dt, I64P)), ctx)
    return dict(t=t.value, m=m, r=r, v=v, a=a, tau=tau, dt=dt)


def tsbts_step_estimates(ctx, n):
    dts = np.zeros(n)
    _check(lib().tsbts_step_estimates(ctx, _p(dts)), ctx)
    return dts


def tsbts_set_state(ctx, n, t, m, r, v, a, tau, dt, dts):
    m, dts = (np.ascontiguousarray(x, np.float64).reshape(n) for x in (m, dts))
    r, v, a = (np.ascontiguousarray(x, np.float64).reshape(n, 3)
               for x in (r, v, a))
    tau, dt = (np.ascontiguousarray(x, np.int64).reshape(n) for x in (tau, dt))
    _check(lib().tsbts_set_state(ctx, float(t), _p(m), _p(r), _p(v), _p(a),
                                 _p(tau, I64P), _p(dt, I64P), _p(dts)), ctx)


def tsbts_get_stats(ctx) -> dict:
    s = tsbts_stats()
    _check(lib().tsbts_get_stats(ctx, C.byref(s)), ctx)
    return s.as_dict()


def tsbts_set_timing(ctx, period):
    """0/False: off; 1/True: every block step; k > 1: every k-th chunk."""
    _check(lib().tsbts_set_timing(ctx, int(period)), ctx)


def tsbts_schedule_log(ctx, capacity: int):
    _check(lib().tsbts_schedule_log(ctx, int(capacity)), ctx)


def tsbts_schedule_get(ctx):
    L = lib()
    ns, ne, dr = C.c_int64(), C.c_int64(), C.c_int64()
    _check(L.tsbts_schedule_size(ctx, C.byref(ns), C.byref(ne), C.byref(dr)),
           ctx)
    ns, ne = ns.value, ne.value
    era = np.zeros(ns, np.int32)
    pas = np.zeros(ns, np.int32)
    tau = np.zeros(ns, np.int64)
    nact = np.zeros(ns, np.int32)
    ei = np.zeros(ne, np.int32)
    edt = np.zeros(ne, np.int64)
    _check(L.tsbts_schedule_get(ctx, _p(era, I32P), _p(pas, I32P),
                                _p(tau, I64P), _p(nact, I32P), _p(ei, I32P),
                                _p(edt, I64P)), ctx)
    return dict(era=era, pass_=pas, tau=tau, n_act=nact, idx=ei, dt=edt,
                dropped=dr.value)


def tsbts_destroy(ctx):
    if ctx:
        lib().tsbts_destroy(ctx)


def _check_force_tensors(name, m, r, v, idx, a, phi, q):
    """The kernels read and write exactly these shapes and dtypes on the
    current device; anything else is refused before the library is
    called. Index values must lie in [0, n) (not checked here: that would
    synchronise the device on every call)."""
    import torch
    dev = torch.cuda.current_device()
    for t in (m, r, v, idx, a, phi, q):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} takes contiguous CUDA tensors")
        if t.device.index != dev:
            raise ValueError(f"{name}: tensors must be on the current "
                             f"device cuda:{dev}")
    for t in (m, r, v, a, phi, q):
        if t.dtype != torch.float64:
            raise ValueError(f"{name}: m, r, v, a, phi, q must be float64")
    if idx.dtype != torch.int32:
        raise ValueError(f"{name}: idx must be int32")
    n, na = m.shape[0], idx.shape[0]
    if (m.dim() != 1 or tuple(r.shape) != (n, 3) or tuple(v.shape) != (n, 3)
            or idx.dim() != 1 or tuple(a.shape) != (na, 3)
            or tuple(phi.shape) != (na,) or tuple(q.shape) != (na,)):
        raise ValueError(f"{name}: shapes must be m (n,), r and v (n, 3), "
                         "idx (n_act,), a (n_act, 3), phi and q (n_act,)")


def tsbts_force(precision, m, r, v, eps, idx, a, phi, q, exact_order=-1,
                stream=None):
    """Device-pointer force call on torch CUDA tensors (see tsbts.h)."""
    import torch
    _check_force_tensors("tsbts_force", m, r, v, idx, a, phi, q)
    if stream is None:
        stream = torch.cuda.current_stream(m.device).cuda_stream
    _check(lib().tsbts_force(int(precision), int(exact_order), m.shape[0],
                             m.data_ptr(), r.data_ptr(), v.data_ptr(),
                             float(eps), idx.shape[0], idx.data_ptr(),
                             a.data_ptr(), phi.data_ptr(), q.data_ptr(),
                             stream))


def tsbts_force_static(precision, m, r, v, eps, idx, a, phi, q,
                       exact_order=-1, stream=None):
    """tsbts_force without device allocation (see tsbts.h): scratch lives
    in a fixed array inside the library; n, n_act <= 65536."""
    import torch
    _check_force_tensors("tsbts_force_static", m, r, v, idx, a, phi, q)
    if stream is None:
        stream = torch.cuda.current_stream(m.device).cuda_stream
    _check(lib().tsbts_force_static(int(precision), int(exact_order),
                                    m.shape[0], m.data_ptr(), r.data_ptr(),
                                    v.data_ptr(), float(eps), idx.shape[0],
                                    idx.data_ptr(), a.data_ptr(),
                                    phi.data_ptr(), q.data_ptr(), stream))


def tsbts_pipe_peak(kind: int, iters: int):
    """(lane operations per second, ms) of one pipe (see tsbts.h)."""
    ops, ms = C.c_double(), C.c_double()
    _check(lib().tsbts_pipe_peak(int(kind), int(iters), C.byref(ops),
                                 C.byref(ms)))
    return ops.value, ms.value


def tsbts_version() -> str:
    return lib().tsbts_version().decode()


# --- adjoint of a frozen block schedule -----------------------------------

def final_pass_schedule(sched, era=-1):
    """(step_tau, step_off, act) of one era's last pass from a schedule log
    (tsbts_schedule_get), active bodies ascending within each step."""
    eras = np.unique(sched["era"])
    e = eras[era]
    keep = sched["era"] == e
    keep &= sched["pass_"] == sched["pass_"][keep].max()
    off = np.zeros(len(sched["n_act"]) + 1, np.int64)
    np.cumsum(sched["n_act"], out=off[1:])
    steps = np.flatnonzero(keep)
    parts = [np.sort(sched["idx"][off[k]:off[k + 1]]) for k in steps]
    step_off = np.zeros(len(parts) + 1, np.int64)
    np.cumsum([len(x) for x in parts], out=step_off[1:])
    act = (np.concatenate(parts) if parts else np.zeros(0)).astype(np.int32)
    return (np.ascontiguousarray(sched["tau"][steps], dtype=np.int64),
            step_off, act)


def era_pass_schedules(sched, era=0):
    """Every pass of one era from a schedule log (tsbts_schedule_get): a
    list of (step_tau, step_off, act), one per pass in order, active bodies
    ascending within each step."""
    eras = np.unique(sched["era"])
    in_era = sched["era"] == eras[era]
    off = np.zeros(len(sched["n_act"]) + 1, np.int64)
    np.cumsum(sched["n_act"], out=off[1:])
    out = []
    for p in np.unique(sched["pass_"][in_era]):
        steps = np.flatnonzero(in_era & (sched["pass_"] == p))
        parts = [np.sort(sched["idx"][off[k]:off[k + 1]]) for k in steps]
        step_off = np.zeros(len(parts) + 1, np.int64)
        np.cumsum([len(x) for x in parts], out=step_off[1:])
        act = np.concatenate(parts).astype(np.int32)
        out.append((np.ascontiguousarray(sched["tau"][steps], dtype=np.int64),
                    step_off, act))
    return out


def tsbts_adjoint_init(ctx, n, eps, schedule, checkpoint_every=0):
    tau, off, act = (np.ascontiguousarray(schedule[0], np.int64),
                     np.ascontiguousarray(schedule[1], np.int64),
                     np.ascontiguousarray(schedule[2], np.int32))
    if off.shape[0] != tau.shape[0] + 1:
        raise ValueError("step_off must have one more entry than step_tau")
    _check(lib().tsbts_adjoint_init(ctx, int(n), float(eps), tau.shape[0],
                                    _p(tau, I64P), _p(off, I64P),
                                    _p(act, I32P), int(checkpoint_every)), ctx)


def era_schedule(passes):
    """Concatenate per-pass schedules [(step_tau, step_off, act), ...] of
    one era into (pass_off, step_tau, step_off, act) with step_off running
    on across the passes."""
    taus, offs, acts, pass_off, base = [], [], [], [0], 0
    for tau, off, act in passes:
        tau = np.asarray(tau, np.int64)
        off = np.asarray(off, np.int64)
        if off.shape[0] != tau.shape[0] + 1 or off[0] != 0:
            raise ValueError("each pass needs step_off = [0, ...] with one "
                             "more entry than step_tau")
        taus.append(tau)
        offs.append(off[:-1] + base)
        acts.append(np.asarray(act, np.int32))
        base += int(off[-1])
        pass_off.append(pass_off[-1] + tau.shape[0])
    offs.append(np.array([base], np.int64))
    return (np.ascontiguousarray(pass_off, np.int64),
            np.ascontiguousarray(np.concatenate(taus), np.int64),
            np.ascontiguousarray(np.concatenate(offs), np.int64),
            np.ascontiguousarray(np.concatenate(acts), np.int32))


def tsbts_adjoint_init_era(ctx, n, eps, passes, checkpoint_every=0):
    """Adjoint through every pass of one era; passes: one
    (step_tau, step_off, act) per pass, in pass order."""
    pass_off, tau, off, act = era_schedule(passes)
    _check(lib().tsbts_adjoint_init_era(
        ctx, int(n), float(eps), len(passes), _p(pass_off, I64P),
        _p(tau, I64P), _p(off, I64P), _p(act, I32P), int(checkpoint_every)),
        ctx)


def _ptrs(arrays, n, device):
    """Raw pointers of host numpy arrays or CUDA tensors (None -> NULL)."""
    out = []
    for a in arrays:
        if a is None:
            out.append(None)
        elif device:
            if not (a.is_cuda and a.is_contiguous()):
                raise ValueError("device arrays must be contiguous CUDA "
                                 "tensors")
            out.append(a.data_ptr())
        else:
            if a.dtype != np.float64 or not a.flags.c_contiguous:
                raise ValueError("host arrays must be contiguous float64")
            out.append(a.ctypes.data)
    return out


def tsbts_adjoint_forward(ctx, m, r0, v0, r_T=None, v_T=None, device=False):
    """Forward replay; host numpy (default) or CUDA tensors (device=True).
    Host inputs are converted; host outputs are allocated if None."""
    if not device:
        m, r0, v0 = (np.ascontiguousarray(x, np.float64) for x in (m, r0, v0))
        n = m.shape[0]
        r_T = np.zeros((n, 3)) if r_T is None else r_T
        v_T = np.zeros((n, 3)) if v_T is None else v_T
    n = m.shape[0]
    _check(lib().tsbts_adjoint_forward(
        ctx, *_ptrs((m, r0, v0, r_T, v_T), n, device), int(device)), ctx)
    return r_T, v_T


def tsbts_adjoint_vjp(ctx, gr_T, gv_T, g_r0=None, g_v0=None, g_m=None,
                      device=False, n=None):
    if not device:
        gr_T = None if gr_T is None else np.ascontiguousarray(gr_T,
                                                              np.float64)
        gv_T = None if gv_T is None else np.ascontiguousarray(gv_T,
                                                              np.float64)
        n = n if n is not None else (gr_T if gr_T is not None
                                     else gv_T).shape[0]
        g_r0 = np.zeros((n, 3)) if g_r0 is None else g_r0
        g_v0 = np.zeros((n, 3)) if g_v0 is None else g_v0
        g_m = np.zeros(n) if g_m is None else g_m
    _check(lib().tsbts_adjoint_vjp(
        ctx, *_ptrs((gr_T, gv_T, g_r0, g_v0, g_m), n, device), int(device)),
        ctx)
    return g_r0, g_v0, g_m


def tsbts_adjoint_forward_state(ctx, m, r0, v0, a0=None, tau0=None,
                                device=False):
    """Forward replay from a general era-start state (host numpy): body j
    at tick tau0[j] with acceleration a0[j]; a0 None: tick 0 and the force
    at r0. Returns the final (r, v, a, tau)."""
    m, r0, v0 = (np.ascontiguousarray(x, np.float64) for x in (m, r0, v0))
    n = m.shape[0]
    if device:
        raise ValueError("tsbts_adjoint_forward_state takes host arrays")
    a0 = None if a0 is None else np.ascontiguousarray(a0, np.float64)
    tau0 = None if tau0 is None else np.ascontiguousarray(tau0, np.int64)
    for x, shape in ((r0, (n, 3)), (v0, (n, 3)), (a0, (n, 3)), (tau0, (n,))):
        if x is not None and x.shape != shape:
            raise ValueError("start state arrays must be (n, 3) or (n,)")
    r_T, v_T, a_T = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
    tau_T = np.zeros(n, np.int64)
    _check(lib().tsbts_adjoint_forward_state(
        ctx, m.ctypes.data, r0.ctypes.data, v0.ctypes.data,
        None if a0 is None else a0.ctypes.data,
        None if tau0 is None else tau0.ctypes.data, r_T.ctypes.data,
        v_T.ctypes.data, a_T.ctypes.data, tau_T.ctypes.data, 0), ctx)
    return r_T, v_T, a_T, tau_T


def tsbts_adjoint_vjp_state(ctx, n, gr_T=None, gv_T=None, ga_T=None):
    """Reverse mode with cotangents of the final r, v, a (host numpy, None:
    zero): (g_r0, g_v0, g_a0, g_m)."""
    gs = [None if g is None else np.ascontiguousarray(g, np.float64)
          for g in (gr_T, gv_T, ga_T)]
    for g in gs:
        if g is not None and g.shape != (n, 3):
            raise ValueError("cotangents must be (n, 3)")
    out = [np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)]
    _check(lib().tsbts_adjoint_vjp_state(
        ctx, *[None if g is None else g.ctypes.data for g in gs],
        *[x.ctypes.data for x in out], 0), ctx)
    return tuple(out)


def tsbts_adjoint_loss_grad(ctx, m, r0, v0, loss=None, g_r0=None, g_v0=None,
                            g_m=None, device=False):
    """L = sum m |r(T)|^2 / sum m and its gradient (L, g_r0, g_v0, g_m)."""
    if not device:
        m, r0, v0 = (np.ascontiguousarray(x, np.float64) for x in (m, r0, v0))
        n = m.shape[0]
        loss = np.zeros(1) if loss is None else loss
        g_r0 = np.zeros((n, 3)) if g_r0 is None else g_r0
        g_v0 = np.zeros((n, 3)) if g_v0 is None else g_v0
        g_m = np.zeros(n) if g_m is None else g_m
    n = m.shape[0]
    _check(lib().tsbts_adjoint_loss_grad(
        ctx, *_ptrs((m, r0, v0, loss, g_r0, g_v0, g_m), n, device),
        int(device)), ctx)
    return (float(loss[0]) if not device else loss), g_r0, g_v0, g_m


def tsbts_adjoint_get_stats(ctx) -> dict:
    st = tsbts_adjoint_stats()
    _check(lib().tsbts_adjoint_get_stats(ctx, C.byref(st)), ctx)
    return st.as_dict()


# --- convenience wrapper --------------------------------------------------

class Simulation:
    """One TSBTS context: init -> step_era -> energy/state (include/tsbts.h).

    All arrays are numpy float64 on the host; the integration runs on the
    GPU.
    """

    def __init__(self, m, r, v, *, eps, eta, dt_max, precision=TSBTS_FP64,
                 n_iter=3, era_mode=0, era_log2=3, dyn_min_log2=3, k_max=20,
                 exact_order=-1, device=0, stream=None, graph_steps=32,
                 conv_tol=0.0, max_pass_steps=0):
        cfg = tsbts_config_default()
        cfg.conv_tol = conv_tol
        cfg.max_pass_steps = max_pass_steps
        cfg.precision = precision
        cfg.n_iter = n_iter
        cfg.era_mode = era_mode
        cfg.era_log2 = era_log2
        cfg.dyn_min_log2 = dyn_min_log2
        cfg.k_max = k_max
        cfg.exact_order = exact_order
        cfg.device = device
        cfg.stream = stream
        cfg.graph_steps = graph_steps
        self.cfg = cfg
        self.k_max = k_max
        self.n = int(np.asarray(m).shape[0])
        self.ctx = tsbts_create(cfg)
        try:
            tsbts_init(self.ctx, m, r, v, eps, eta, dt_max)
        except Exception:
            tsbts_destroy(self.ctx)
            self.ctx = None
            raise

    def step_era(self, t_end):
        return tsbts_step_era(self.ctx, t_end)

    run = step_era

    def energy(self):
        ek, ep, _ = tsbts_energy(self.ctx)
        return ek, ep

    def state(self):
        return tsbts_state(self.ctx, self.n)

    def checkpoint(self):
        """The state at the system time with the step estimates: what
        set_state needs to resume after an era end."""
        st = tsbts_state(self.ctx, self.n)
        st["dts"] = tsbts_step_estimates(self.ctx, self.n)
        return st

    def set_state(self, ck):
        """Resume from checkpoint() taken at an era end of a run with the
        same configuration and body count."""
        tsbts_set_state(self.ctx, self.n, ck["t"], ck["m"], ck["r"], ck["v"],
                        ck["a"], ck["tau"], ck["dt"], ck["dts"])

    def stats(self):
        return tsbts_get_stats(self.ctx)

    def set_timing(self, period=1):
        tsbts_set_timing(self.ctx, period)

    def schedule_log(self, capacity):
        tsbts_schedule_log(self.ctx, capacity)

    def schedule(self):
        return tsbts_schedule_get(self.ctx)

    def close(self):
        if self.ctx:
            tsbts_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Ensemble(Simulation):
    """Independent clusters integrated together (tsbts_init_ensemble).

    offsets[c] .. offsets[c+1]-1 are cluster c's bodies; eps[c] its
    softening. era_mode 0: one fixed era of 2^-era_log2 for all clusters;
    1: every cluster its own dynamic era (Alg. 3 on its own bodies)."""

    def __init__(self, offsets, m, r, v, *, eps, eta, dt_max,
                 precision=TSBTS_FP64, n_iter=3, era_mode=0, era_log2=3,
                 dyn_min_log2=3, k_max=20, exact_order=-1, device=0,
                 stream=None, graph_steps=32):
        cfg = tsbts_config_default()
        cfg.precision = precision
        cfg.n_iter = n_iter
        cfg.era_mode = era_mode
        cfg.dyn_min_log2 = dyn_min_log2
        cfg.era_log2 = era_log2
        cfg.k_max = k_max
        cfg.exact_order = exact_order
        cfg.device = device
        cfg.stream = stream
        cfg.graph_steps = graph_steps
        self.cfg = cfg
        self.k_max = k_max
        self.n = int(np.asarray(m).shape[0])
        self.n_clusters = int(np.asarray(offsets).shape[0] - 1)
        self.ctx = tsbts_create(cfg)
        try:
            tsbts_init_ensemble(self.ctx, offsets, m, r, v, eps, eta, dt_max)
        except Exception:
            tsbts_destroy(self.ctx)
            self.ctx = None
            raise

    def cluster_energy(self):
        return tsbts_ensemble_energy(self.ctx, self.n_clusters)


class ErasAdjoint:
    """Adjoint across consecutive eras of one run: one Adjoint through
    every pass of each era, era k replayed from the state (r, v, a, tick)
    that era k - 1 left; reverse mode chains the eras last to first.

    eras = [passes of era 0, passes of era 1, ...], each as for
    Adjoint(passes=...) (e.g. era_pass_schedules(log, k)). Keyword
    arguments go to every Adjoint."""

    def __init__(self, n, eps, eras, **kw):
        self.n = int(n)
        self.adj = []
        try:
            for passes in eras:
                self.adj.append(Adjoint(n, eps, passes=passes, **kw))
        except Exception:
            self.close()
            raise

    def forward(self, m, r0, v0):
        """Final (r, v, a, tau) after the last era."""
        state = (r0, v0, None, None)
        for a in self.adj:
            state = a.forward_state(m, *state)
        return state

    def vjp(self, gr_T=None, gv_T=None, ga_T=None):
        """(g_r0, g_v0, g_m) of the initial state for cotangents of the
        last era's final r, v, a; needs forward() first."""
        g = (gr_T, gv_T, ga_T)
        g_m = np.zeros(self.n)
        for a in reversed(self.adj):
            gr, gv, ga, gm = a.vjp_state(*g)
            g_m += gm
            g = (gr, gv, ga)
        return g[0], g[1], g_m

    def loss_grad(self, m, r0, v0):
        """L = sum m |r(T)|^2 / sum m after the last era, with its gradient
        (L, g_r0, g_v0, g_m)."""
        m = np.ascontiguousarray(m, np.float64)
        rT = self.forward(m, r0, v0)[0]
        M = m.sum()
        r2 = (rT * rT).sum(1)
        L = float((m * r2).sum() / M)
        g_r0, g_v0, g_m = self.vjp(2.0 * m[:, None] * rT / M)
        return L, g_r0, g_v0, g_m + (r2 - L) / M

    def stats(self):
        return [a.stats() for a in self.adj]

    def close(self):
        for a in self.adj:
            a.close()
        self.adj = []

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Adjoint:
    """Adjoint of a frozen block schedule (tsbts_adjoint_*): replay of the
    schedule from (m, r0, v0) and reverse-mode gradients.

    schedule = (step_tau, step_off, act) as from final_pass_schedule, or
    passes = a list of such schedules, every pass of one era (the adjoint
    through all of them). checkpoint_every = 0 tapes every step; K > 0
    keeps a checkpoint every K steps and recomputes during the reverse
    sweep. graph_steps = 0 runs plain stream launches; otherwise the
    forward replay and the reverse sweep are each captured once as a CUDA
    graph and replayed."""

    def __init__(self, n, eps, schedule=None, *, passes=None,
                 precision=TSBTS_FP64, k_max=20, checkpoint_every=0,
                 exact_order=-1, device=0, stream=None, graph_steps=32):
        if (schedule is None) == (passes is None):
            raise ValueError("give either schedule or passes")
        cfg = tsbts_config_default()
        cfg.precision = precision
        cfg.k_max = k_max
        cfg.exact_order = exact_order
        cfg.device = device
        cfg.stream = stream
        cfg.graph_steps = graph_steps
        self.n = int(n)
        self.ctx = tsbts_create(cfg)
        try:
            if passes is None:
                tsbts_adjoint_init(self.ctx, n, eps, schedule,
                                   checkpoint_every)
            else:
                tsbts_adjoint_init_era(self.ctx, n, eps, passes,
                                       checkpoint_every)
        except Exception:
            tsbts_destroy(self.ctx)
            self.ctx = None
            raise

    def forward(self, m, r0, v0):
        return tsbts_adjoint_forward(self.ctx, m, r0, v0)

    def vjp(self, gr_T, gv_T=None):
        return tsbts_adjoint_vjp(self.ctx, gr_T, gv_T, n=self.n)

    def loss_grad(self, m, r0, v0):
        return tsbts_adjoint_loss_grad(self.ctx, m, r0, v0)

    def forward_state(self, m, r0, v0, a0=None, tau0=None):
        return tsbts_adjoint_forward_state(self.ctx, m, r0, v0, a0, tau0)

    def vjp_state(self, gr_T=None, gv_T=None, ga_T=None):
        return tsbts_adjoint_vjp_state(self.ctx, self.n, gr_T, gv_T, ga_T)

    def stats(self):
        return tsbts_adjoint_get_stats(self.ctx)

    def close(self):
        if self.ctx:
            tsbts_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
