"""torch.autograd bindings of the frozen-schedule adjoint (tsbts_adjoint_*).

``replay(adj, r0, v0, m)`` returns the replayed final positions and
velocities as a differentiable function of the initial state and masses;
``era_loss(adj, r0, v0, m)`` returns the mass-weighted mean-square radius
of the final positions, with its gradient computed by the library in the
same call. Both run the replay and its reverse mode in the CUDA library on
device pointers of the tensors (float64, contiguous, on the adjoint's
device); nothing is computed by torch but the scaling by the incoming
gradient.

The library keeps the last forward replay's tape or checkpoints inside the
Adjoint. A replay's backward that runs after another forward on the same
Adjoint first replays its own inputs again (recomputation), so it is
always correct; in the usual order (forward, then backward) it reuses the
stored replay.
"""
from __future__ import annotations

import torch

from . import tsbts


def make_adjoint(n, eps, schedule=None, *, passes=None,
                 precision=tsbts.TSBTS_FP64, k_max=20, checkpoint_every=0,
                 device=0):
    """An Adjoint (of one pass's schedule, or of every pass of an era) on
    its own torch stream of `device`; every call first waits for the
    caller's current stream, and returns once its results are written."""
    stream = torch.cuda.Stream(device=device)
    adj = tsbts.Adjoint(n, eps, schedule, passes=passes, precision=precision,
                        k_max=k_max, checkpoint_every=checkpoint_every,
                        device=device, stream=stream.cuda_stream)
    adj.torch_stream = stream
    adj.generation = 0
    return adj


def _order(adj, t):
    """Make the adjoint's stream wait for the work queued on t's device."""
    adj.torch_stream.wait_stream(torch.cuda.current_stream(t.device))


def _check_inputs(*ts):
    for t in ts:
        if t.dtype != torch.float64 or not t.is_cuda:
            raise ValueError("inputs must be float64 CUDA tensors")


class _Replay(torch.autograd.Function):
    @staticmethod
    def forward(ctx, r0, v0, m, adj):
        _check_inputs(r0, v0, m)
        r0, v0, m = r0.contiguous(), v0.contiguous(), m.contiguous()
        r_T = torch.empty_like(r0)
        v_T = torch.empty_like(v0)
        _order(adj, r0)
        tsbts.tsbts_adjoint_forward(adj.ctx, m, r0, v0, r_T, v_T, device=True)
        adj.generation += 1
        ctx.adj = adj
        ctx.generation = adj.generation
        ctx.save_for_backward(r0, v0, m)
        return r_T, v_T

    @staticmethod
    def backward(ctx, gr_T, gv_T):
        adj = ctx.adj
        if adj.generation != ctx.generation:
            # another forward ran since: replay these inputs again
            r0, v0, m = ctx.saved_tensors
            _order(adj, r0)
            tsbts.tsbts_adjoint_forward(adj.ctx, m, r0, v0, None, None,
                                        device=True)
            adj.generation += 1
            ctx.generation = adj.generation
        dev = gr_T.device if gr_T is not None else gv_T.device
        n = adj.n
        g_r0 = torch.empty((n, 3), dtype=torch.float64, device=dev)
        g_v0 = torch.empty((n, 3), dtype=torch.float64, device=dev)
        g_m = torch.empty((n,), dtype=torch.float64, device=dev)
        gr = None if gr_T is None else gr_T.contiguous()
        gv = None if gv_T is None else gv_T.contiguous()
        _order(adj, g_r0)
        tsbts.tsbts_adjoint_vjp(adj.ctx, gr, gv, g_r0, g_v0, g_m, device=True,
                                n=n)
        return g_r0, g_v0, g_m, None


class _EraLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, r0, v0, m, adj):
        _check_inputs(r0, v0, m)
        r0, v0, m = r0.contiguous(), v0.contiguous(), m.contiguous()
        n = adj.n
        loss = torch.empty((1,), dtype=torch.float64, device=r0.device)
        g_r0 = torch.empty((n, 3), dtype=torch.float64, device=r0.device)
        g_v0 = torch.empty((n, 3), dtype=torch.float64, device=r0.device)
        g_m = torch.empty((n,), dtype=torch.float64, device=r0.device)
        _order(adj, r0)
        tsbts.tsbts_adjoint_loss_grad(adj.ctx, m, r0, v0, loss, g_r0, g_v0,
                                      g_m, device=True)
        adj.generation += 1
        ctx.save_for_backward(g_r0, g_v0, g_m)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        g_r0, g_v0, g_m = ctx.saved_tensors
        return g * g_r0, g * g_v0, g * g_m, None


def replay(adj, r0, v0, m):
    """(r_T, v_T) of the frozen-schedule replay, differentiable."""
    return _Replay.apply(r0, v0, m, adj)


def era_loss(adj, r0, v0, m):
    """sum m |r_T|^2 / sum m of the replay, differentiable."""
    return _EraLoss.apply(r0, v0, m, adj)
