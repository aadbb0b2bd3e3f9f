"""torch.autograd front end of the step's adjoint.

``steps(grid, P0, kappa_scale, nsteps, checkpoint)`` advances a grid
``nsteps`` steps and returns the final primitives as a differentiable function
of the initial primitives ``P0`` and of the global opacity scale
``kappa_scale`` (a 0-d tensor equal to the grid's ``kappa_scale``).  The
backward pass uses the library's hand-written adjoint of one step
(``harmrad_step_adjoint``) with checkpointing: the forward keeps the state
every ``checkpoint`` steps; the backward re-runs each segment from its
checkpoint to recover the steps' inputs and sweeps the segment in reverse,
handing each step's input to the adjoint (which recomputes that step once
with recording on): per segment of n steps, n - 1 forward steps of replay
and the adjoints' n recomputations.
The time steps are those of the forward run (held fixed, not differentiated).
All arithmetic runs in the library's kernels; torch holds device memory.
"""
import torch

from . import harmrad as H


class _Steps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, P0, kappa_scale, grid, nsteps, checkpoint, dt):
        if abs(float(kappa_scale) - grid.params.kappa_scale) > 1e-15 * abs(grid.params.kappa_scale):
            raise H.HarmradError("kappa_scale differs from the grid's parameter")
        grid.adjoint_enable(True)
        grid.set_prims(P0.detach().contiguous())
        ckpts, dts = [], []
        for n in range(nsteps):
            if n % checkpoint == 0:
                ckpts.append(grid.get_prims(device=True))
            grid.step(dt)
            dts.append(grid.stats()["dt"])
        ctx.grid, ctx.nsteps, ctx.checkpoint = grid, nsteps, checkpoint
        ctx.ckpts, ctx.dts = ckpts, dts
        return grid.get_prims(device=True)

    @staticmethod
    def backward(ctx, gout):
        grid, nsteps, K = ctx.grid, ctx.nsteps, ctx.checkpoint
        g = gout.contiguous().to(torch.float64)
        gk = 0.0
        nseg = len(ctx.ckpts)
        for seg in reversed(range(nseg)):
            i0 = seg * K
            n = min(K, nsteps - i0)
            # inputs of the segment's steps, recomputed from its checkpoint
            grid.set_prims(ctx.ckpts[seg])
            inputs = []
            for j in range(n):
                inputs.append(grid.get_prims(device=True))
                if j < n - 1:
                    grid.step(ctx.dts[i0 + j])
            for j in reversed(range(n)):
                # the adjoint recomputes the step from its recorded input
                grid.adjoint_set_input(inputs[j], ctx.dts[i0 + j])
                g, gkj = grid.step_adjoint(g)
                gk += gkj
        return g, torch.tensor(gk, dtype=torch.float64), None, None, None, None


def steps(grid, P0, kappa_scale, nsteps, checkpoint=5, dt=0.0):
    """Differentiable ``nsteps`` steps of ``grid`` from ``P0`` ([12,n3,n2,n1]
    float64 CUDA tensor); ``kappa_scale`` a 0-d float64 tensor.  dt <= 0:
    each step takes its CFL time step (recorded and reused by the backward)."""
    return _Steps.apply(P0, kappa_scale, grid, int(nsteps), int(checkpoint), float(dt))
