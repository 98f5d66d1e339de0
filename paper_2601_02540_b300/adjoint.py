"""Gradients of a gauge-misfit loss with respect to the bathymetry and the
initial water height, through the library's hand-written adjoint kernels.

``GaugeRollout`` is a ``torch.autograd.Function`` mapping (b, h0) to the water
height at a set of gauge nodes after every ``every`` RK4 steps.  The initial
state is at rest (u = v = 0), so the initialization of the auxiliary variables
gives eta0 = h0 and w0 = 0 (eq. (initialization)); the gradient with respect
to h0 is therefore qbar_h + qbar_eta of the initial state.

Forward (K > 0): ``sgn_step`` with a copy of the state kept at the start of
every K-step segment (checkpoint); the last segment runs through
``sgn_step_record`` instead, which keeps the four stage states of each of its
steps, so the backward pass need not recompute it.  Backward: for each
segment, last to first, recompute it from its checkpoint with
``sgn_step_record`` (except the last), then walk its steps backwards with
``sgn_step_vjp``, adding the gauge cotangents to qbar_h at the observation
steps.  The recomputation of the next segment runs on a second CUDA stream
while the current one is walked, so the two overlap on the GPU.

With ``tape`` (K > 0), the recorded segments also keep the tapes of their
stage RHS evaluations (``sgn_step_record_tape``: the intermediate values of
the RHS, written by the stage kernels as they advance the state), and the
walk reads them (``sgn_step_vjp_tape``) instead of evaluating them again:
a step's adjoint then takes five launches instead of nine.  Memory: two
K-step stashes of 20 planes per step, plus with the tape two of 84 planes
per step (4.2 GB and 17.6 GB at 512^2 for K = 100).  ``tape=None`` takes the
tape when it fits in half of the free device memory.  K <= 0 keeps the stage
states of every step during the forward pass instead (no recomputation and
no tape; 84 GB at 512^2 for 2000 steps, which fits in a B300's HBM).

The gauge sampling, the seed injection and the checkpoint copies are small
torch tensor operations; every RHS, stage and adjoint evaluation runs in the
library's kernels.
"""
from __future__ import annotations

import torch

from . import sgn


class GaugeRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, h0, solver: sgn.Solver, dt: float, nsteps: int, every: int,
                gauges: torch.Tensor, K: int, tape: bool | None = None):
        assert solver.prec == "f64", "the adjoint runs in FP64"
        ny, nx = h0.shape
        b = b.detach().to(torch.float64).contiguous()
        solver.set_bathymetry(b)
        q = torch.zeros((5, ny, nx), dtype=torch.float64, device=h0.device)
        q[0] = h0.detach()
        solver.init_aux(q)
        nobs = nsteps // every
        obs = torch.empty((nobs, gauges.numel()), dtype=torch.float64, device=h0.device)
        checkpoints = {}
        stash = tapes = None
        last = 0
        TP = 4 * sgn.TAPE_PLANES
        if K <= 0:
            # keep every step's stage states (no recomputation in the backward pass)
            tape = False
            stash = torch.empty((nsteps, 20, ny, nx), dtype=torch.float64, device=h0.device)
        elif nsteps > 0:
            # the last segment keeps its stage states (stash indexed from its start)
            last = ((nsteps - 1) // K) * K
            if tape is None:
                need = 2 * min(K, nsteps) * (20 + TP) * ny * nx * 8
                tape = need <= 0.5 * torch.cuda.mem_get_info(h0.device)[0]
            stash = torch.empty((nsteps - last, 20, ny, nx), dtype=torch.float64, device=h0.device)
            if tape:
                tapes = torch.empty((nsteps - last, TP, ny, nx), dtype=torch.float64, device=h0.device)
        step = 0
        while step < nsteps:
            if K > 0 and step % K == 0 and step < last:
                checkpoints[step] = q.clone()
            nxt = min(nsteps, (step // every + 1) * every)
            if K > 0:
                nxt = min(nxt, (step // K + 1) * K)
            if K > 0 and step < last:
                solver.step(q, dt, nxt - step)
            else:
                solver.step_record(q, dt, nxt - step, stash[step - last:nxt - last],
                                   tapes[step - last:nxt - last] if tapes is not None else None)
            step = nxt
            if step % every == 0:
                obs[step // every - 1] = q[0].reshape(-1)[gauges]
        ctx.solver, ctx.dt, ctx.nsteps, ctx.every, ctx.K = solver, dt, nsteps, every, K
        ctx.gauges = gauges
        ctx.checkpoints = checkpoints
        ctx.stash = stash
        ctx.tapes = tapes
        ctx.last = last
        ctx.shape = (ny, nx)
        ctx.b = b
        return obs

    @staticmethod
    def backward(ctx, grad_obs):
        solver, dt, nsteps, every, K = ctx.solver, ctx.dt, ctx.nsteps, ctx.every, ctx.K
        gauges = ctx.gauges
        solver.set_bathymetry(ctx.b)
        ny, nx = ctx.shape
        dev = grad_obs.device
        qbar = torch.zeros((5, ny, nx), dtype=torch.float64, device=dev)
        bbar = torch.zeros((ny, nx), dtype=torch.float64, device=dev)
        grad_obs = grad_obs.to(torch.float64).contiguous()
        if K > 0:
            segments = [(s0, min(K, nsteps - s0)) for s0 in sorted(ctx.checkpoints)]
            if nsteps > 0:
                segments.append((ctx.last, nsteps - ctx.last))
        else:
            segments = [(0, nsteps)]
        order = list(reversed(segments))
        main = torch.cuda.current_stream(dev)
        if K > 0:
            # Segment k (last to first) is walked backwards on the current stream
            # while segment k + 1 is recomputed from its checkpoint on a second
            # stream into the other of two stash buffers (the recomputation uses
            # the context's RK registers, the adjoint its own scratch), so the
            # two overlap on the GPU.  Buffer k % 2 serves segment k; the last
            # segment's stages were kept by the forward pass in buffer 0.
            side = torch.cuda.Stream(dev)
            side.wait_stream(main)
            Kmax = max(L for _, L in order)
            taped = ctx.tapes is not None
            TP = 4 * sgn.TAPE_PLANES
            bufs = [ctx.stash, None]
            tbufs = [ctx.tapes, None]
            ready = [None] * len(order)             # recomputation of segment k done
            done = [None] * len(order)              # walk of segment k done

            def recompute(k):
                s0, L = order[k]
                slot = k % 2
                if bufs[slot] is None or bufs[slot].shape[0] < L:
                    bufs[slot] = torch.empty((Kmax, 20, ny, nx), dtype=torch.float64, device=dev)
                    if taped:
                        tbufs[slot] = torch.empty((Kmax, TP, ny, nx), dtype=torch.float64, device=dev)
                with torch.cuda.stream(side):
                    if k >= 2:
                        side.wait_event(done[k - 2])    # the walk that used this buffer
                    q = ctx.checkpoints[s0].clone()
                    solver.step_record(q, dt, L, bufs[slot], tbufs[slot] if taped else None)
                    ready[k] = torch.cuda.Event()
                    ready[k].record(side)

            if len(order) > 1:
                recompute(1)
            for k, (s0, L) in enumerate(order):
                if k > 0:
                    main.wait_event(ready[k])
                stash = bufs[k % 2]
                tp = tbufs[k % 2]
                for n in reversed(range(L)):
                    g = s0 + n + 1                  # this step produces q_g
                    if g % every == 0:
                        qbar[0].reshape(-1).index_add_(0, gauges, grad_obs[g // every - 1])
                    solver.step_vjp(stash[n], qbar, bbar, dt, tp[n] if taped else None)
                done[k] = torch.cuda.Event()
                done[k].record(main)
                if k + 2 < len(order):
                    recompute(k + 2)
            main.wait_stream(side)
        else:
            stash = ctx.stash
            for n in reversed(range(nsteps)):
                g = n + 1
                if g % every == 0:
                    qbar[0].reshape(-1).index_add_(0, gauges, grad_obs[g // every - 1])
                solver.step_vjp(stash[n], qbar, bbar, dt)
        ctx.stash = ctx.tapes = None
        h0bar = qbar[0] + qbar[4]
        return bbar, h0bar, None, None, None, None, None, None, None


def gauge_rollout(b, h0, solver, dt, nsteps, every, gauges, K=100, tape=None):
    return GaugeRollout.apply(b, h0, solver, dt, nsteps, every, gauges, K, tape)
