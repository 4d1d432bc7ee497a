"""torch.autograd.Function for the gasket diffusion with per-cell conductivity.

Forward: ``steps`` steps of the conductivity diffusion from u0, keeping the
state every ``every`` steps (checkpoints).  Backward: for each checkpoint
segment, from the last, the segment's states are recomputed forward from its
checkpoint, then the reverse step carries dJ/du back through the segment and
accumulates dJ/dkappa (in float64).  Memory: ceil(steps / every) + every
states instead of steps + 1.  Every step runs in the library's kernels; this
module only orders the calls and owns buffers.

``state="f64"`` (default) keeps the trajectory and the adjoint state in
float64 on the device: an FP32 trajectory rounds the state every step, and
over 200 steps those roundings alone move the gradients by a few 1e-4 of
their scale, beyond the 1e-4 agreement with an FP64 adjoint.  ``state="f32"``
runs the float32 kernels (half the memory traffic).  Inputs and outputs keep
the callers' dtypes.
"""
from __future__ import annotations

import torch

from . import (FRACTAL_F32, FRACTAL_LAMBDA, fractal_adjoint_diffusion_step, fractal_adjoint_diffusion_step_f64,
               fractal_map, fractal_map_write, fractal_step_diffusion_kappa, fractal_step_diffusion_kappa_f64)


def _member_mask(plan, like):
    """1.0 at the members, 0 elsewhere (the library's single-write kernel on zeros)."""
    m = torch.zeros(like.shape, dtype=torch.float32, device=like.device)
    fractal_map_write(plan, m, FRACTAL_F32, 1.0)
    return m


class GasketDiffusion(torch.autograd.Function):
    """u_T = GasketDiffusion.apply(u0, kappa, k, a, steps, every, mode, state).

    u0, kappa: flat float32 CUDA tensors of 4**k elements (the n x n arrays,
    row-major; non-member cells are ignored).  Returns u_T, 0 at every
    non-member cell.  Gradients: dJ/du0 and dJ/dkappa at member cells, 0
    elsewhere.
    """

    @staticmethod
    def forward(ctx, u0, kappa, k: int, a: float, steps: int, every: int = 20, mode: int = FRACTAL_LAMBDA,
                state: str = "f64"):
        if every < 1:
            raise ValueError("every >= 1")
        if state not in ("f32", "f64"):
            raise ValueError("state is 'f32' or 'f64'")
        dt = torch.float64 if state == "f64" else torch.float32
        step = fractal_step_diffusion_kappa_f64 if state == "f64" else fractal_step_diffusion_kappa
        plan = fractal_map(k, 8 if k >= 3 else 1 << k, mode)
        mask = _member_mask(plan, u0)
        kappa = kappa.detach().to(torch.float32).contiguous()
        # every buffer holds 0 at all non-member cells, so u_T does too
        u = (u0.detach().to(dt) * mask).contiguous()
        v = torch.zeros_like(u)
        ckpts = []
        t = 0
        while t < steps:
            ckpts.append(u.clone())
            ns = min(every, steps - t)
            out = step(plan, u, v, kappa, a, ns)
            if out is v:
                u, v = v, u
            t += ns
        ctx.save_for_backward(kappa, mask, *ckpts)
        ctx.plan, ctx.a, ctx.steps, ctx.every, ctx.state = plan, a, steps, every, state
        ctx.dtypes = (u0.dtype, kappa.dtype)
        return u.to(u0.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        kappa, mask, *ckpts = ctx.saved_tensors
        plan, a, steps, every, state = ctx.plan, ctx.a, ctx.steps, ctx.every, ctx.state
        f64 = state == "f64"
        step = fractal_step_diffusion_kappa_f64 if f64 else fractal_step_diffusion_kappa
        reverse = fractal_adjoint_diffusion_step_f64 if f64 else fractal_adjoint_diffusion_step
        dt = torch.float64 if f64 else torch.float32
        # u_T is 0 at non-members whatever u0 is: only member cells carry gradient
        p = (grad_out.detach().to(dt) * mask).contiguous()
        q = torch.zeros_like(p)
        gk = torch.zeros(kappa.shape, dtype=torch.float64, device=kappa.device)
        # the recomputed states of a segment, one pool for all segments: a
        # step writes every member tile of its output and the kernels read
        # member cells only, so the pool is neither cleared nor reallocated
        pool = [torch.empty_like(p) for _ in range(min(every, steps) - 1)]
        for seg in range(len(ckpts) - 1, -1, -1):
            t0 = seg * every
            ns = min(every, steps - t0)
            states = [ckpts[seg]]
            for i in range(ns - 1):
                # one step reads the first buffer and writes the second
                step(plan, states[-1], pool[i], kappa, a, 1)
                states.append(pool[i])
            for i in range(ns - 1, -1, -1):
                reverse(plan, states[i], p, q, kappa, gk, a)
                p, q = q, p
        du, dk = ctx.dtypes
        return p.to(du), gk.to(dk), None, None, None, None, None, None


def diffusion_kappa(u0, kappa, k: int, a: float, steps: int, every: int = 20, mode: int = FRACTAL_LAMBDA,
                    state: str = "f64"):
    """Functional form of :class:`GasketDiffusion`."""
    return GasketDiffusion.apply(u0, kappa, k, a, steps, every, mode, state)
