"""Differentiable rollouts of the implicit step (the differentiation form).

``rollout(system, E, x0, v0, n_steps)`` runs ``n_steps`` implicit steps
through the C ABI and returns the final (x, v) as tensors that autograd can
differentiate with respect to the per-tet Young's moduli ``E`` and the initial
state (x0, v0).  The backward pass walks the steps in reverse with
``yasps_adjoint_step`` (implicit-function theorem on each step's optimality
condition; one exact-Hessian PCG solve per step) -- no step is differentiated
through its Newton iterations.

Checkpointing: the forward pass keeps (x_t, v_t) and the fixed-vertex
positions of every ``checkpoint_every``-th step on the device; the backward
pass recomputes the states in between, one segment at a time, from its
checkpoint.  With ``checkpoint_every=1`` nothing is recomputed.
"""
import torch


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, system, n_steps, checkpoint_every, tol, E, x0, v0):
        system.set_tet_young(E)
        x = x0.detach().clone().contiguous()
        v = v0.detach().clone().contiguous()
        ckpt = {0: (x.clone(), v.clone(), system.get_fixed_positions())}
        for t in range(n_steps):
            system.step(x, v)
            if (t + 1) % checkpoint_every == 0 or t + 1 == n_steps:
                ckpt[t + 1] = (x.clone(), v.clone(), system.get_fixed_positions())
        ctx.system, ctx.n_steps, ctx.every, ctx.tol = system, n_steps, checkpoint_every, tol
        ctx.ckpt = ckpt
        ctx.E = E.detach().clone()
        return x.clone(), v.clone()

    @staticmethod
    def backward(ctx, gx, gv):
        S, n, every = ctx.system, ctx.n_steps, ctx.every
        S.set_tet_young(ctx.E)
        xbar = gx.contiguous() if gx is not None else S.zeros(S.n_nodes, 3)
        vbar = gv.contiguous() if gv is not None else S.zeros(S.n_nodes, 3)
        Ebar = S.zeros(ctx.E.numel())
        seg_end = n
        while seg_end > 0:
            seg_start = ((seg_end - 1) // every) * every
            # states of this segment: checkpoints where kept, else recomputed
            # from the segment's first checkpoint
            states = [ctx.ckpt[seg_start]]
            x = v = None
            for t in range(seg_start + 1, seg_end + 1):
                if t in ctx.ckpt:
                    states.append(ctx.ckpt[t])
                    continue
                if x is None:
                    x, v, fx = (a.clone() if torch.is_tensor(a) else a for a in states[-1])
                    S.set_fixed_positions(fx)
                S.step(x, v)
                states.append((x.clone(), v.clone(), S.get_fixed_positions()))
            for k in range(seg_end - seg_start - 1, -1, -1):
                xt, vt, _ = states[k]
                xn, _, fxn = states[k + 1]
                S.set_fixed_positions(fxn)
                xbar, vbar, _, _ = S.adjoint_step(xt, vt, xn, xbar, vbar, Ebar, tol=ctx.tol)
            seg_end = seg_start
        # leave the fixed vertices where the forward pass left them
        S.set_fixed_positions(ctx.ckpt[n][2])
        return None, None, None, None, Ebar, xbar, vbar


def rollout(system, E, x0, v0, n_steps, checkpoint_every=1, tol=1e-10):
    """Final (x, v) after ``n_steps`` implicit steps; differentiable in E, x0, v0."""
    return _Rollout.apply(system, int(n_steps), max(1, int(checkpoint_every)), float(tol), E, x0, v0)
