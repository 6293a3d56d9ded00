"""Differentiable solve: a torch.autograd.Function whose forward is
tode_solve (fused form, filling a checkpoint tape) and whose backward is the
hand-written discrete adjoint tode_adjoint (App. A: gradients by
backpropagation through the solver, on the forward's frozen mesh).

The tape is sized from the forward's accepted-step counts under an HBM
budget: one slot per accepted step when it fits, otherwise one slot every m
steps with the segments recomputed in the backward pass (gradients bitwise
equal to m = 1).  The MLP field and joint solves (Sec. 4.1, ``joint=True``:
one shared mesh, reversed per instance) keep every step (m = 1).
"""
from __future__ import annotations

import math
from typing import Optional

import torch

from . import api

DEFAULT_BUDGET_BYTES = 40 << 30


def _tape_budget(dev, budget: Optional[int]) -> int:
    if budget is not None:
        return int(budget)
    free, _ = torch.cuda.mem_get_info(dev)
    return int(min(DEFAULT_BUDGET_BYTES, free // 2))


def _solve_with_tape(field, y0, t0, t1, t_eval, opt, budget, hint, want_yp=False):
    B, D = y0.shape
    dev, dtype = y0.device, y0.dtype
    mlp = isinstance(field, api.MLP)
    per_slot = api.TapeBuffers.bytes_per_slot(B, D, y0.element_size(), stages=mlp,
                                              minimal=True)
    max_slots = max(1, budget // max(per_slot, 1))
    slots = max(1, min(max_slots, hint))
    tape = api.TapeBuffers.allocate(B, D, dtype, slots, 1, dev, stages=mlp, minimal=True)
    sol = api.solve(field, y0, t0, t1, t_eval, tape=tape, form="fused", want_yp=want_yp, **opt)
    N = int(sol.n_acc.max().item()) if B > 0 else 0
    if N > slots:
        full_slot = api.TapeBuffers.bytes_per_slot(B, D, y0.element_size(), stages=mlp)
        if N <= max_slots:
            stride = 1
        elif mlp or opt.get("joint"):
            what = "the MLP adjoint" if mlp else "the adjoint of a joint solve"
            raise RuntimeError(f"{what} keeps every accepted step: {N} slots of "
                               f"{per_slot} bytes exceed the tape budget of {budget} bytes")
        else:  # strided segments are re-run: the tape keeps the whole state
            stride = math.ceil(N / max(1, budget // max(full_slot, 1)))
        slots = math.ceil(N / stride)
        tape = api.TapeBuffers.allocate(B, D, dtype, slots, stride, dev, stages=mlp,
                                        minimal=stride == 1)
        # the solve is deterministic: the re-run fills the tape on the same mesh
        sol = api.solve(field, y0, t0, t1, t_eval, tape=tape, form="fused", want_yp=want_yp,
                        **opt)
    return sol, tape, N


class _Odeint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, spec, y0, t0, t1, t_eval, *tensors):
        field = spec["field"].with_tensors(list(tensors))
        # dL/dt_eval = <dL/dy_eval, dy/dt>: the forward also writes dy/dt there
        want_yp = t_eval is not None and ctx.needs_input_grad[4]
        sol, tape, N = _solve_with_tape(field, y0, t0, t1, t_eval, spec["opt"],
                                        spec["budget"], spec["hint"], want_yp)
        spec["last_n_acc_max"] = N
        ctx.field, ctx.sol, ctx.tape, ctx.opt = field, sol, tape, spec["opt"]
        ctx.save_for_backward(t0, t1, t_eval)
        ctx.mark_non_differentiable(sol.n_acc, sol.n_rej, sol.status)
        return sol.y_eval, sol.y_final, sol.n_acc, sol.n_rej, sol.status

    @staticmethod
    def backward(ctx, g_eval, g_final, *_):
        t0, t1, t_eval = ctx.saved_tensors
        sol, field = ctx.sol, ctx.field
        dtype = sol.y_final.dtype
        gye = g_eval.to(dtype).contiguous() if g_eval is not None and t_eval is not None else None
        gyf = g_final.to(dtype).contiguous() if g_final is not None else None
        gy0, gp, ovf = api.adjoint(field, t0, t1, t_eval, sol, ctx.tape, gye, gyf, **ctx.opt)
        if int(ovf.item()) != 0:
            raise RuntimeError("tode_adjoint: the checkpoint tape overflowed")
        if isinstance(field, api.MLP):
            gW, gb = gp
            grads = [g.to(w.dtype) for g, w in zip(gW + gb, field.W + field.b)]
        else:
            grads = [gp]
        g_te = None
        if sol.yp_eval is not None and gye is not None:
            g_te = api.t_eval_grad(gye, sol.yp_eval).to(t_eval.dtype)
        return (None, gy0, None, None, g_te, *grads)


def odeint_adjoint(field, y0: torch.Tensor, t0: torch.Tensor, t1: torch.Tensor,
                   t_eval: Optional[torch.Tensor] = None, *,
                   hbm_budget_bytes: Optional[int] = None, slots_hint: int = 64, **opt_kw):
    """Solve every instance of the batch (Sec. 3) and make the result
    differentiable with respect to y0 and the field's tensors (mu for Van der
    Pol, A for linear, the weights and biases for the MLP) through the
    discrete adjoint of the fixed-mesh map (App. A).

    Returns (y_eval [B,K,D], y_final [B,D], n_acc, n_rej, status); the counters
    and the status carry no gradient.  A t_eval that requires grad receives
    dL/dt_eval through dy/dt of the dense output (Van der Pol and linear).  Keyword options as in
    ``make_options`` (the fused form is used).
    """
    opt = {k: v for k, v in opt_kw.items() if k != "form"}
    spec = {"field": field, "opt": opt, "budget": _tape_budget(y0.device, hbm_budget_bytes),
            "hint": int(slots_hint)}
    return _Odeint.apply(spec, y0, t0, t1, t_eval, *field.tensors())
