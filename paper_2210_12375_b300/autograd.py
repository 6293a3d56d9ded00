"""Differentiable solve: a torch.autograd.Function whose forward is
tode_solve (fused form, filling a checkpoint tape) and whose backward is the
hand-written discrete adjoint tode_adjoint (App. A: gradients by
backpropagation through the solver, on the forward's frozen mesh).

The tape is sized from the forward's accepted-step counts under an HBM
budget: one slot per accepted step when it fits, otherwise one slot every m
steps with the segments recomputed in the backward pass (gradients bitwise
equal to m = 1).  For the MLP field a slot every m steps holds the whole
solver state, and the backward re-solves one segment at a time into an
m-slot stage tape (tode_mlp_resolve) before reversing it.  Joint solves
(Sec. 4.1, ``joint=True``: one shared mesh, reversed per instance) keep
every step (m = 1).
"""
from __future__ import annotations

import math
from typing import Optional

import torch

from . import api

DEFAULT_BUDGET_BYTES = 40 << 30
# the most accepted steps the last solve of a problem shape needed
_LAST_N: dict = {}


def _tape_budget(dev, budget: Optional[int]) -> int:
    if budget is not None:
        return int(budget)
    free, _ = torch.cuda.mem_get_info(dev)
    return int(min(DEFAULT_BUDGET_BYTES, free // 2))


def _shape_key(field, y0, opt):
    return (type(field).__name__, tuple(y0.shape), y0.dtype, str(y0.device),
            bool(opt.get("joint")))


def _solve_with_tape(field, y0, t0, t1, t_eval, opt, budget, hint, want_yp=False):
    """(solution, tape or None, most accepted steps, MLP chunk size or 0)."""
    B, D = y0.shape
    dev, dtype = y0.device, y0.dtype
    mlp = isinstance(field, api.MLP)
    key = _shape_key(field, y0, opt)
    per_slot = api.TapeBuffers.bytes_per_slot(B, D, y0.element_size(), stages=mlp,
                                              minimal=True)
    max_slots = max(1, budget // max(per_slot, 1))
    if key in _LAST_N:
        hint = max(1, int(_LAST_N[key] * 1.25) + 1)
    slots = max(1, min(max_slots, hint))
    tape = api.TapeBuffers.allocate(B, D, dtype, slots, 1, dev, stages=mlp, minimal=True)
    sol = api.solve(field, y0, t0, t1, t_eval, tape=tape, form="fused", want_yp=want_yp, **opt)
    N = int(sol.n_acc.max().item()) if B > 0 else 0
    _LAST_N[key] = N
    chunk = 0
    if N > slots:
        full_slot = api.TapeBuffers.bytes_per_slot(B, D, y0.element_size(), stages=mlp)
        if N <= max_slots:
            stride = 1
        elif opt.get("joint"):
            raise RuntimeError(f"the adjoint of a joint solve keeps every accepted step: {N} "
                               f"slots of {per_slot} bytes exceed the tape budget of "
                               f"{budget} bytes")
        elif mlp and _mlp_segment_stride(B, D, N, budget) > 1:
            # checkpoints every m accepted steps; the backward re-solves one
            # segment at a time into an m-slot stage tape and reverses it
            stride = _mlp_segment_stride(B, D, N, budget)
        elif mlp:
            # not even that fits: the backward recomputes the batch chunk by
            # chunk (instances are independent); the forward needs no tape
            one = api.TapeBuffers.bytes_per_slot(1, D, y0.element_size(), stages=True,
                                                 minimal=True)
            chunk = int(budget // max(one * N, 1))
            if chunk < 1:
                raise RuntimeError(f"the MLP adjoint keeps every accepted step of an instance: "
                                   f"{N} steps of {one} bytes exceed the tape budget of "
                                   f"{budget} bytes")
            return sol, None, N, chunk
        else:  # strided segments are re-run: the tape keeps the whole state
            stride = math.ceil(N / max(1, budget // max(full_slot, 1)))
        slots = math.ceil(N / stride)
        tape = api.TapeBuffers.allocate(B, D, dtype, slots, stride, dev,
                                        stages=mlp and stride == 1, minimal=stride == 1)
        # the solve is deterministic: the re-run fills the tape on the same mesh
        sol = api.solve(field, y0, t0, t1, t_eval, tape=tape, form="fused", want_yp=want_yp,
                        **opt)
    return sol, tape, N, chunk


def _mlp_segment_stride(B, D, N, budget):
    """The largest m (2..N) whose checkpoint tape (ceil(N/m) slots of the
    whole solver state) plus one m-slot stage tape fits the budget; 0 if
    none does."""
    ck = api.TapeBuffers.bytes_per_slot(B, D, 4)
    st = api.TapeBuffers.bytes_per_slot(B, D, 4, stages=True, minimal=True)
    best = 0
    for m in range(2, max(N, 2) + 1):
        if math.ceil(N / m) * ck + m * st <= budget:
            best = m
    return best


def _mlp_adjoint_segments(field, t0, t1, t_eval, sol, ckpt, gye, gyf, opt, N, want_ts=False):
    """The MLP adjoint of a solve that recorded checkpoints every m accepted
    steps: segment by segment from the last, the segment is re-solved from
    its checkpoint into an m-slot stage tape (the same attempts, bit for bit)
    and reversed as a solve of its own -- from its end's cotangent, with the
    points inside it (the first segment also takes those at t0) -- and its
    start's cotangent carried to the segment before.  Weight gradients (and
    the time-translation sums) are summed over the segments."""
    B, D = sol.y_final.shape
    m = ckpt.stride
    dev = sol.y_final.device
    seg_tape = api.TapeBuffers.allocate(B, D, sol.y_final.dtype, m, 1, dev, stages=True,
                                        minimal=True)
    carry = gyf if gyf is not None else torch.zeros_like(sol.y_final)
    dirn = torch.where(t1 < t0, -1.0, 1.0).to(torch.float64)
    gW = gb = ts = None
    ws = None
    for j in reversed(range(math.ceil(N / m))):
        seg_n, s0, s1 = api.mlp_resolve(field, t0, t1, sol.n_acc, ckpt, j, seg_tape,
                                        workspace=ws, **opt)
        g_e = None
        if gye is not None and t_eval is not None:
            tq = dirn[:, None] * t_eval
            lo, hi = (dirn * s0)[:, None], (dirn * s1)[:, None]
            inside = (tq <= hi) & ((tq > lo) if j > 0 else (tq >= lo))
            g_e = (gye * inside[..., None].to(gye.dtype)).contiguous()
        seg = api.Solution(y_eval=sol.y_eval, y_final=sol.y_final, n_acc=seg_n,
                           n_rej=sol.n_rej, n_feval=sol.n_feval, status=sol.status)
        g0, gp, ovf = api.adjoint(field, s0, s1, t_eval, seg, seg_tape, g_e,
                                  carry.contiguous(), want_tshift=want_ts, **opt)
        if int(ovf.item()) != 0:
            raise RuntimeError("tode_adjoint: a segment overflowed its stage tape")
        carry = g0
        if gW is None:
            gW, gb = list(gp[0]), list(gp[1])
            ts = gp[2] if want_ts else None
        else:
            gW = [a + b for a, b in zip(gW, gp[0])]
            gb = [a + b for a, b in zip(gb, gp[1])]
            if want_ts:
                ts = ts + gp[2]
    return carry, (gW, gb) if not want_ts else (gW, gb, ts)


def _mlp_adjoint_chunked(field, y0, t0, t1, t_eval, sol, gye, gyf, opt, chunk, N):
    """The MLP adjoint of a solve whose tape did not fit: every chunk of
    `chunk` instances is re-solved with a stride-1 stage tape (its meshes and
    stage inputs are the forward's, bit for bit) and reversed; dL/dy0 per
    chunk, the weight gradients summed over the chunks in order."""
    B, D = y0.shape
    gy0 = torch.empty_like(y0)
    gW = gb = None
    for c0 in range(0, B, chunk):
        c1 = min(B, c0 + chunk)
        n_c = int(sol.n_acc[c0:c1].max().item())
        tape = api.TapeBuffers.allocate(c1 - c0, D, y0.dtype, max(1, n_c), 1, y0.device,
                                        stages=True, minimal=True)
        te = t_eval[c0:c1].contiguous() if t_eval is not None else None
        s = api.solve(field, y0[c0:c1].contiguous(), t0[c0:c1].contiguous(),
                      t1[c0:c1].contiguous(), te, tape=tape, form="fused", **opt)
        g_e = gye[c0:c1].contiguous() if gye is not None else None
        g_f = gyf[c0:c1].contiguous() if gyf is not None else None
        g0, (w_c, b_c), ovf = api.adjoint(field, t0[c0:c1].contiguous(), t1[c0:c1].contiguous(),
                                          te, s, tape, g_e, g_f, **opt)
        if int(ovf.item()) != 0:
            raise RuntimeError("tode_adjoint: the checkpoint tape overflowed")
        gy0[c0:c1] = g0
        if gW is None:
            gW, gb = list(w_c), list(b_c)
        else:
            gW = [a + b for a, b in zip(gW, w_c)]
            gb = [a + b for a, b in zip(gb, b_c)]
    return gy0, (gW, gb)


class _Odeint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, spec, y0, t0, t1, t_eval, *tensors):
        field = spec["field"].with_tensors(list(tensors))
        # dL/dt_eval = <dL/dy_eval, dy/dt> and dL/dt0 (which sums those):
        # the forward also writes dy/dt there
        want_t = ctx.needs_input_grad[2] or ctx.needs_input_grad[3]
        want_yp = t_eval is not None and (ctx.needs_input_grad[4] or ctx.needs_input_grad[2])
        if want_t and spec["opt"].get("joint"):
            raise RuntimeError("gradients with respect to t0 and t1 are built for independent "
                               "solves")
        sol, tape, N, chunk = _solve_with_tape(field, y0, t0, t1, t_eval, spec["opt"],
                                               spec["budget"], spec["hint"], want_yp)
        spec["last_n_acc_max"] = N
        spec["mlp_chunk"] = chunk
        ctx.field, ctx.sol, ctx.tape, ctx.opt = field, sol, tape, spec["opt"]
        ctx.chunk, ctx.N = chunk, N
        if want_t and (tape is None or tape.stride != 1):
            raise RuntimeError("gradients with respect to t0 and t1 need one tape slot per "
                               "accepted step: raise hbm_budget_bytes")
        ctx.want_t = want_t
        ctx.save_for_backward(y0, t0, t1, t_eval)
        ctx.mark_non_differentiable(sol.n_acc, sol.n_rej, sol.status)
        return sol.y_eval, sol.y_final, sol.n_acc, sol.n_rej, sol.status

    @staticmethod
    def backward(ctx, g_eval, g_final, *_):
        y0, t0, t1, t_eval = ctx.saved_tensors
        sol, field = ctx.sol, ctx.field
        dtype = sol.y_final.dtype
        gye = g_eval.to(dtype).contiguous() if g_eval is not None and t_eval is not None else None
        gyf = g_final.to(dtype).contiguous() if g_final is not None else None
        if ctx.chunk > 0:
            gy0, gp = _mlp_adjoint_chunked(field, y0.detach(), t0, t1, t_eval, sol, gye, gyf,
                                           ctx.opt, ctx.chunk, ctx.N)
        elif isinstance(field, api.MLP) and ctx.tape.stride > 1:
            gy0, gp = _mlp_adjoint_segments(field, t0, t1, t_eval, sol, ctx.tape, gye, gyf,
                                            ctx.opt, ctx.N)
        else:
            mlp_t = ctx.want_t and isinstance(field, api.MLP)
            gy0, gp, ovf = api.adjoint(field, t0, t1, t_eval, sol, ctx.tape, gye, gyf,
                                       want_tshift=mlp_t, **ctx.opt)
            if int(ovf.item()) != 0:
                raise RuntimeError("tode_adjoint: the checkpoint tape overflowed")
        tshift = None
        if isinstance(field, api.MLP):
            gW, gb = gp[0], gp[1]
            tshift = gp[2] if len(gp) > 2 else None
            grads = [g.to(w.dtype) for g, w in zip(gW + gb, field.W + field.b)]
        else:
            grads = [gp]
        g_te = None
        if sol.yp_eval is not None and gye is not None and ctx.needs_input_grad[4]:
            g_te = api.t_eval_grad(gye, sol.yp_eval).to(t_eval.dtype)
        g_t0 = g_t1 = None
        if ctx.want_t:
            g_t0, g_t1 = api.t_bounds_grad(field, t0, t1, t_eval, sol, ctx.tape, gye, gyf,
                                           want_t0=ctx.needs_input_grad[2], tshift=tshift,
                                           **ctx.opt)
            g_t0 = g_t0.to(t0.dtype) if g_t0 is not None and ctx.needs_input_grad[2] else None
            g_t1 = g_t1.to(t1.dtype) if ctx.needs_input_grad[3] else None
        return (None, gy0, g_t0, g_t1, g_te, *grads)


def odeint_adjoint(field, y0: torch.Tensor, t0: torch.Tensor, t1: torch.Tensor,
                   t_eval: Optional[torch.Tensor] = None, *,
                   hbm_budget_bytes: Optional[int] = None, slots_hint: int = 64, **opt_kw):
    """Solve every instance of the batch (Sec. 3) and make the result
    differentiable with respect to y0 and the field's tensors (mu for Van der
    Pol, A for linear, the weights and biases for the MLP) through the
    discrete adjoint of the fixed-mesh map (App. A).

    Returns (y_eval [B,K,D], y_final [B,D], n_acc, n_rej, status); the counters
    and the status carry no gradient.  A t_eval that requires grad receives
    dL/dt_eval through dy/dt of the dense output; t0 and t1 that require grad
    receive the gradients of the frozen map with respect to the integration
    bounds (every field, solved independently; one tape slot per accepted
    step).
    Keyword options as in ``make_options`` (the fused form is used).
    """
    opt = {k: v for k, v in opt_kw.items() if k != "form"}
    spec = {"field": field, "opt": opt, "budget": _tape_budget(y0.device, hbm_budget_bytes),
            "hint": int(slots_hint)}
    return _Odeint.apply(spec, y0, t0, t1, t_eval, *field.tensors())
