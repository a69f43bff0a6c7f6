"""Differentiable simulation: a torch.autograd.Function whose forward runs time steps through the C ABI and whose
backward runs the library's adjoint (sim_adjoint_step: one linear CG solve on the Hessian-vector kernel per step,
from checkpointed step states).  Gradients: the per-tet Young's modulus and the initial velocities."""
import dataclasses

import numpy as np
import torch

from . import binding as B


class Simulate(torch.autograd.Function):
    """x_T = Simulate.apply(youngs_per_tet [T], v0 [V, 3], scene, steps, precision, tol, max_iters, options).

    The forward creates a handle for `scene` with the given Young's moduli and initial velocities (float64 tensors;
    the scene's other data as given), advances `steps` time steps and keeps every step's positions (the checkpoints
    the reverse pass needs); `options` are the handle's keyword options (scatter, model, ...).  Each step is taken as the exact minimiser of its incremental potential, so the
    forward should be converged (enough iterations, or the eps rule) for the gradients to be those of the run."""

    @staticmethod
    def forward(ctx, youngs, v0, scene, steps, precision=B.SIM_FP64, tol=1e-10, max_iters=2000, options=None):
        sc = dataclasses.replace(scene, youngs=1.0, youngs_per_tet=youngs.detach().cpu().double().numpy().copy(),
                                 v0=v0.detach().cpu().double().numpy().copy())
        sim = B.Sim(sc, precision=precision, **(options or {}))
        xs = [np.ascontiguousarray(sc.x0, dtype=np.float64)]
        for t in range(steps):
            sim.step(1, sc.targets(t))
            xs.append(sim.state()[0])
        ctx.sim, ctx.xs = sim, xs
        ctx.tol, ctx.max_iters = tol, max_iters
        ctx.nt = sc.n_tets
        return torch.from_numpy(xs[-1].copy()).to(v0.device)

    @staticmethod
    def backward(ctx, grad_x):
        sim, xs = ctx.sim, ctx.xs
        ax = grad_x.detach().cpu().double().contiguous().numpy().copy()
        av = np.zeros_like(ax)
        dE = np.zeros(ctx.nt)
        ctx.cg = []
        for t in range(len(xs) - 1, 0, -1):
            ax, av, it, res = B.sim_adjoint_step(sim.h, xs[t], ax, av, dE=dE, tol=ctx.tol, max_iters=ctx.max_iters)
            ctx.cg.append((it, res))
        sim.close()
        dev = grad_x.device
        return (torch.from_numpy(dE).to(dev), torch.from_numpy(av).to(dev), None, None, None, None, None, None)


def simulate(youngs, v0, scene, steps, precision=B.SIM_FP64, tol=1e-10, max_iters=2000, options=None):
    return Simulate.apply(youngs, v0, scene, steps, precision, tol, max_iters, options)
