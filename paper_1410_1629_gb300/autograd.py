"""Differentiable transport: a torch.autograd.Function over the C ABI.

forward(density) runs rt_launch_packets with the given cell densities and
returns the images and the absorption field; backward(adjoints) runs
rt_adjoint and returns d(loss)/d(density).  The derivative is the pathwise
one under common random numbers (directions and draws fixed); use bilinear
deposit and event-cap termination (weight_cut=False) so the tallies are
continuous in the density (Sect. 1 motivates this: fitting models to
observed images).

On cartesian grids with at most 256 events per packet the forward launch
records the adjoint tape, and a backward that follows with no other forward
on the same Simulation in between uses it instead of replaying the packets'
paths.  An adjoint of the absorption field always replays.
"""
from __future__ import annotations

import torch

from . import rt


class Transport(torch.autograd.Function):
    @staticmethod
    def forward(ctx, density, sim, n_per_lambda, first_id, seed, opts):
        ctx.set_materialize_grads(False)  # unused outputs give None, not zeros
        dens = density.detach().to(torch.float32).contiguous()
        stream = torch.cuda.current_stream()
        rt.rt_update_density(sim.ctx, dens.data_ptr(), 1, stream)
        sim.reset(stream=stream)
        launch_opts = dict(opts)
        max_events = launch_opts.get("max_events", sim.problem.run.max_events)
        if sim.problem.grid.kind == "cartesian" and max_events <= 256:
            launch_opts.setdefault("tape", 1)
        try:
            sim.launch(n_per_lambda, first_id, seed, stream=stream, **launch_opts)
        except rt.RTError as e:
            if e.status != rt.RT_ERR_OOM or not launch_opts.get("tape"):
                raise
            launch_opts["tape"] = 0  # no room for the tape: the backward replays
            sim.launch(n_per_lambda, first_id, seed, stream=stream, **launch_opts)
        sim.generation = getattr(sim, "generation", 0) + 1
        images = sim.images(stream=stream)
        absorption = sim.absorption(stream=stream)
        ctx.sim, ctx.n, ctx.first, ctx.seed, ctx.opts = sim, n_per_lambda, first_id, seed, launch_opts
        ctx.generation = sim.generation
        ctx.save_for_backward(dens)
        ctx.shape, ctx.dtype = density.shape, density.dtype
        return (*images, absorption)

    @staticmethod
    def backward(ctx, *grads):
        (dens,) = ctx.saved_tensors
        sim = ctx.sim
        stream = torch.cuda.current_stream()
        if getattr(sim, "generation", 0) != ctx.generation:
            # another forward ran since: restore this forward's density (the tape is then not used)
            rt.rt_update_density(sim.ctx, dens.data_ptr(), 1, stream)
        adj_imgs = [g.detach().to(torch.float64).contiguous() if g is not None else None for g in grads[:-1]]
        adj_abs = grads[-1].detach().to(torch.float64).contiguous() if grads[-1] is not None else None
        grad = torch.zeros(dens.numel(), dtype=torch.float64, device=dens.device)
        o = sim.opts(**{k: v for k, v in ctx.opts.items() if k != "tape"})
        rt.rt_adjoint(sim.ctx, [a.data_ptr() if a is not None else 0 for a in adj_imgs],
                      adj_abs.data_ptr() if adj_abs is not None else 0, grad.data_ptr(), ctx.n, ctx.first, ctx.seed,
                      o, stream)
        return grad.view(ctx.shape).to(ctx.dtype), None, None, None, None, None


def transport(density, sim, n_per_lambda=None, first_id=0, seed=None, **opts):
    """Images (list) and absorption field for `density`, differentiable in it."""
    n = sim.problem.run.n_per_lambda if n_per_lambda is None else n_per_lambda
    s = sim.problem.run.seed if seed is None else seed
    out = Transport.apply(density, sim, n, first_id, s, opts)
    return list(out[:-1]), out[-1]
