"""torch.autograd.Function for the gasket diffusion with per-cell conductivity.

Forward: ``steps`` steps of the conductivity diffusion from u0, keeping the
state every ``every`` steps (checkpoints).  Backward: for each checkpoint
segment, from the last, the segment's states are recomputed forward from its
checkpoint, then the reverse step carries dJ/du back through the segment and
accumulates dJ/dkappa (in float64).  Memory: ceil(steps / every) + every
states instead of steps + 1.  Every step runs in the library's kernels; this
module only orders the calls and owns buffers.

An FP32 trajectory rounds the state every step, and over 200 steps those
roundings alone move the gradients by a few 1e-4 of their scale, beyond the
1e-4 agreement with an FP64 adjoint, so the default state is wider:
``state="df"`` (default) keeps the trajectory, the adjoint state and dJ/dkappa
in double-float, (hi, lo) float pairs with about 48 significant bits,
computed on the FP32 pipes, and (k >= 4) runs temporally fused: the forward
steps several per launch, and per segment one recorded pass of u from its
checkpoint, one of p back (the reverse step is the same symmetric operator
applied to p) and one pass summing dJ/dkappa from the two records; ``state="f64"`` keeps them in float64 (the same
agreement, on this GPU's much slower FP64 units); ``state="f32"`` runs the
float32 kernels.  Inputs and outputs keep the callers' dtypes.
"""
from __future__ import annotations

import torch

from . import (FRACTAL_DF, FRACTAL_F32, FRACTAL_LAMBDA, FractalError, fractal_adjoint_diffusion_step,
               fractal_adjoint_diffusion_step_df, fractal_adjoint_diffusion_step_f64, fractal_kappa_fused_limits,
               fractal_kappa_gradient_df_io, fractal_kappa_trajectory_df_io, fractal_map, fractal_map_write,
               fractal_plan_set_kappa_fusion,
               fractal_step_diffusion_kappa, fractal_step_diffusion_kappa_df, fractal_step_diffusion_kappa_f64)

# per state: (step, reverse step, storage dtype, elements per cell)
_STATES = {
    "df": (fractal_step_diffusion_kappa_df, fractal_adjoint_diffusion_step_df, torch.float32, 2),
    "f64": (fractal_step_diffusion_kappa_f64, fractal_adjoint_diffusion_step_f64, torch.float64, 1),
    "f32": (fractal_step_diffusion_kappa, fractal_adjoint_diffusion_step, torch.float32, 1),
}


def _to_state(x, state):
    """A float field in the state's storage; double-float as (hi, lo) pairs
    (lo = 0 for float32 input, the float64 remainder otherwise)."""
    x = x.detach()
    if state == "df":
        if x.dtype == torch.float32:  # (x, 0) pairs in one pass: a complex with zero imaginary part
            return torch.view_as_real(x.to(torch.complex64)).reshape(-1)
        hi = x.to(torch.float32)
        lo = (x.double() - hi.double()).to(torch.float32)
        return torch.stack([hi, lo], dim=1).reshape(-1).contiguous()
    return x.to(_STATES[state][2]).contiguous()


def _from_state(y, state, dtype):
    """The state's values as `dtype` (double-float: hi + lo in float64 first)."""
    if state == "df":
        hl = y.view(-1, 2)
        if dtype == torch.float32:  # a float sum of the two parts rounds their exact sum correctly
            return hl[:, 0] + hl[:, 1]
        return (hl[:, 0].double() + hl[:, 1].double()).to(dtype)
    return y.to(dtype)


def _fused_limits(k, mode):
    """(floats per recorded state, steps per launch) of the fused double-float
    gradient path, or None where it does not apply (k < 4)."""
    try:
        return fractal_kappa_fused_limits(k, mode)
    except FractalError:
        return None


def _run_recorded(plan, src, dst, traj, rec_floats, kappa, a, steps, max_steps, temps, src_fmt=None, dst_fmt=None):
    """`steps` (>= 1) fused double-float steps from src: the state before each
    step into traj states 0 .. steps - 1 (traj may be None) and the result
    into dst (or, with dst None, into traj state `steps`), in launches of at
    most max_steps steps
    (temps: two spare double-float buffers for the chunks between launches).
    src_fmt / dst_fmt: FRACTAL_DF (default) or FRACTAL_F32 for src and dst."""
    src_fmt = FRACTAL_DF if src_fmt is None else src_fmt
    dst_fmt = FRACTAL_DF if dst_fmt is None else dst_fmt
    cur, fmt, s0, i = src, src_fmt, 0, 0
    while s0 < steps:
        n = min(max_steps, steps - s0)
        last = s0 + n == steps
        out, ofmt = (dst, dst_fmt) if last else (temps[i & 1], FRACTAL_DF)
        fractal_kappa_trajectory_df_io(plan, cur, fmt, out, ofmt, None if traj is None else traj[s0 * rec_floats:],
                                       kappa, a, n)
        cur, fmt, s0, i = out, FRACTAL_DF, s0 + n, i + 1


def _member_mask(plan, like):
    """1.0 at the members, 0 elsewhere (the library's single-write kernel on zeros)."""
    m = torch.zeros(like.shape, dtype=torch.float32, device=like.device)
    fractal_map_write(plan, m, FRACTAL_F32, 1.0)
    return m


class GasketDiffusion(torch.autograd.Function):
    """u_T = GasketDiffusion.apply(u0, kappa, k, a, steps, every, mode, state, fused).

    u0, kappa: flat float32 CUDA tensors of 4**k elements (the n x n arrays,
    row-major; non-member cells are ignored).  Returns u_T, 0 at every
    non-member cell.  Gradients: dJ/du0 and dJ/dkappa at member cells, 0
    elsewhere.
    """

    @staticmethod
    def forward(ctx, u0, kappa, k: int, a: float, steps: int, every: int = 20, mode: int = FRACTAL_LAMBDA,
                state: str = "df", fused: bool = True):
        if every < 1:
            raise ValueError("every >= 1")
        if state not in _STATES:
            raise ValueError("state is 'df', 'f64' or 'f32'")
        step = _STATES[state][0]
        plan = fractal_map(k, 8 if k >= 3 else 1 << k, mode)
        fractal_plan_set_kappa_fusion(plan, fused)
        kappa = kappa.detach().to(torch.float32).contiguous()
        lim = _fused_limits(k, mode) if state == "df" and fused else None
        ckpts = []
        t = 0
        ctx.f32_io = lim is not None and u0.dtype == torch.float32
        if lim is not None:
            # fused: each segment from its checkpoint into a new buffer (the
            # kernels read member cells only and write every cell of every
            # member block; the last buffer starts zeroed, so u_T is 0 at
            # every non-member cell).  A float32 u0 is read as it is and u_T
            # written as float32 by the kernels (no conversions around them).
            mask = None
            f32 = ctx.f32_io
            u, ufmt = (u0.detach().contiguous(), FRACTAL_F32) if f32 else (_to_state(u0.detach(), state), FRACTAL_DF)
            df_cells = 2 * u0.numel()
            temps = ([torch.empty(df_cells, dtype=torch.float32, device=u0.device) for _ in range(2)]
                     if min(every, steps) > lim[1] else [None, None])
            while t < steps:
                ns = min(every, steps - t)
                final = t + ns >= steps
                if final and f32:
                    v, vfmt = torch.zeros(u0.numel(), dtype=torch.float32, device=u0.device), FRACTAL_F32
                else:
                    v = (torch.zeros if final else torch.empty)(df_cells, dtype=torch.float32, device=u0.device)
                    vfmt = FRACTAL_DF
                _run_recorded(plan, u, v, None, 0, kappa, a, ns, lim[1], temps, ufmt, vfmt)
                ckpts.append(u)
                u, ufmt = v, vfmt
                t += ns
        else:
            mask = _member_mask(plan, u0)
            # every buffer holds 0 at all non-member cells, so u_T does too
            u = _to_state(u0.detach() * mask.to(u0.dtype), state)
            v = torch.zeros_like(u)
            while t < steps:
                ckpts.append(u.clone())
                ns = min(every, steps - t)
                out = step(plan, u, v, kappa, a, ns)
                if out is v:
                    u, v = v, u
                t += ns
        ctx.save_for_backward(kappa, *ckpts)
        ctx.mask = mask
        ctx.plan, ctx.a, ctx.steps, ctx.every, ctx.state = plan, a, steps, every, state
        ctx.fused = fused
        ctx.dtypes = (u0.dtype, kappa.dtype)
        return u if ctx.f32_io else _from_state(u, state, u0.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        kappa, *ckpts = ctx.saved_tensors
        plan, a, steps, every, state = ctx.plan, ctx.a, ctx.steps, ctx.every, ctx.state
        step, reverse = _STATES[state][0], _STATES[state][1]
        du, dk = ctx.dtypes
        lim = _fused_limits(plan.info()["k"], plan.info()["mode"]) if state == "df" and ctx.fused else None
        if lim is not None:
            # fused: per segment, u recorded forward from its checkpoint and p
            # carried back (the reverse step is A applied to p) in launches of
            # several steps, then dJ/dkappa of the segment from both records.
            # The kernels read member cells only, so a float32 dJ/du_T enters
            # as it is; dJ/du0 leaves as float32 into a zeroed buffer (0 at
            # non-members) when u0 was float32.
            rf, ms = lim
            cells = kappa.numel()
            dev = kappa.device
            if grad_out.dtype == torch.float32:
                p, pfmt = grad_out.detach().contiguous(), FRACTAL_F32
            else:
                p, pfmt = _to_state(grad_out.detach() * _member_mask(plan, grad_out).to(grad_out.dtype), state), \
                    FRACTAL_DF
            seg_max = min(every, steps)
            utraj = torch.empty(rf * (seg_max + 1), dtype=torch.float32, device=dev)
            ptraj = torch.empty(rf * seg_max, dtype=torch.float32, device=dev)
            df = lambda: torch.empty(2 * cells, dtype=torch.float32, device=dev)  # noqa: E731
            temps = [df(), df()] if seg_max > ms else [None, None]
            carry = [df(), df()] if len(ckpts) > 1 else []
            # dJ/dkappa: the first gradient pass starts the double-float sum
            # (no cleared buffer), the last writes it as float32 for a float32
            # kappa; a float64 kappa takes the sum from a zeroed buffer
            f32k = dk == torch.float32
            gk = ((df() if len(ckpts) > 1 else None) if f32k
                  else torch.zeros(2 * cells, dtype=torch.float32, device=dev))
            gk_out = torch.zeros(cells, dtype=torch.float32, device=dev) if f32k else None
            for i, seg in enumerate(range(len(ckpts) - 1, -1, -1)):
                t0 = seg * every
                ns = min(every, steps - t0)
                cfmt = FRACTAL_F32 if seg == 0 and ctx.f32_io else FRACTAL_DF
                # u_(t0) .. u_(t0 + ns - 1) (at least one step, so that the
                # segment's first state is recorded as well)
                _run_recorded(plan, ckpts[seg], None, utraj, rf, kappa, a, max(ns - 1, 1), ms, temps, cfmt)
                if seg > 0:
                    out, ofmt = carry[i & 1], FRACTAL_DF
                elif du == torch.float32:
                    out, ofmt = torch.zeros(cells, dtype=torch.float32, device=dev), FRACTAL_F32
                else:
                    out, ofmt = torch.zeros(2 * cells, dtype=torch.float32, device=dev), FRACTAL_DF
                _run_recorded(plan, p, out, ptraj, rf, kappa, a, ns, ms, temps, pfmt, ofmt)
                fractal_kappa_gradient_df_io(plan, utraj, ptraj, gk, i > 0, gk_out if seg == 0 else None, a, ns)
                p, pfmt = out, ofmt
            return (p if pfmt == FRACTAL_F32 else _from_state(p, state, du),
                    gk_out if f32k else _from_state(gk, "df", dk), None, None, None, None, None, None, None)
        # dJ/dkappa: double-float pairs for the "df" state, else float64
        gk = (torch.zeros(2 * kappa.numel(), dtype=torch.float32, device=kappa.device) if state == "df"
              else torch.zeros(kappa.shape, dtype=torch.float64, device=kappa.device))
        # u_T is 0 at non-members whatever u0 is: only member cells carry gradient
        p = _to_state(grad_out.detach() * ctx.mask.to(grad_out.dtype), state)
        q = torch.zeros_like(p)
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
        gk = _from_state(gk, "df", dk) if state == "df" else gk.to(dk)
        return _from_state(p, state, du), gk, None, None, None, None, None, None, None


def diffusion_kappa(u0, kappa, k: int, a: float, steps: int, every: int = 20, mode: int = FRACTAL_LAMBDA,
                    state: str = "df", fused: bool = True):
    """Functional form of :class:`GasketDiffusion` (fused=False: one launch
    per step, forward and backward, for comparison)."""
    return GasketDiffusion.apply(u0, kappa, k, a, steps, every, mode, state, fused)
