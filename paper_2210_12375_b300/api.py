"""Python binding of the C ABI (include/tode.h) on torch CUDA tensors.

torch provides device memory and streams; every step of the solver runs in
libtode's kernels.  Names follow the paper: a batch of independent initial
value problems y' = f(t, y), one state, step size, accept/reject sequence and
set of evaluation points per instance (torchode, Sec. 3).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field as dc_field
from typing import Optional

import numpy as np
import torch

from . import _abi


# ------------------------------------------------------------------ fields
class VdP:
    """Van der Pol, Eq. 1 as a first-order system (D = 2); mu: [B]."""
    kind = _abi.TODE_VDP

    def __init__(self, mu: torch.Tensor):
        self.mu = mu

    def desc(self, B: int, D: int, keep: list) -> _abi.FieldDesc:
        f = _abi.FieldDesc()
        f.kind, f.B, f.D = self.kind, B, D
        f.mu = self.mu.data_ptr()
        return f

    def params(self):
        return self.mu

    def tensors(self):
        return [self.mu]

    def with_tensors(self, ts):
        return VdP(ts[0])


class Linear:
    """y' = A_i y; A: [B, D, D] row-major."""
    kind = _abi.TODE_LINEAR

    def __init__(self, A: torch.Tensor):
        self.A = A

    def desc(self, B: int, D: int, keep: list) -> _abi.FieldDesc:
        f = _abi.FieldDesc()
        f.kind, f.B, f.D = self.kind, B, D
        f.A = self.A.data_ptr()
        return f

    def params(self):
        return self.A

    def tensors(self):
        return [self.A]

    def with_tensors(self, ts):
        return Linear(ts[0])


class MLP:
    """f(t, y) = W_L tanh(... tanh(W_1 [y; t] + b_1) ...) + b_L with weights
    W_l [out, in] and float biases b_l [out].  The field computes with BF16
    weights: float weights are rounded to BF16 for each call (their gradients
    from the adjoint are then float, with respect to the rounded values)."""
    kind = _abi.TODE_MLP

    def __init__(self, weights, biases, split: bool = False):
        self.W = list(weights)
        self.b = list(biases)
        self.split = split

    @property
    def widths(self):
        return [self.W[0].shape[1]] + [w.shape[0] for w in self.W]

    def desc(self, B: int, D: int, keep: list) -> _abi.FieldDesc:
        f = _abi.FieldDesc()
        f.kind, f.B, f.D = self.kind, B, D
        wd = self.widths
        wa = (C.c_int * len(wd))(*wd)
        Wb = [w if w.dtype == torch.bfloat16 else w.detach().to(torch.bfloat16).contiguous()
              for w in self.W]
        keep += Wb
        Wp = (C.c_void_p * len(self.W))(*[w.data_ptr() for w in Wb])
        bp = (C.c_void_p * len(self.b))(*[b.data_ptr() for b in self.b])
        keep += [wa, Wp, bp]
        f.n_layers = len(self.W)
        f.widths = wa
        f.W = Wp
        f.b = bp
        return f

    def params(self):
        return None

    def tensors(self):
        return self.W + self.b

    def with_tensors(self, ts):
        n = len(self.W)
        return MLP(list(ts[:n]), list(ts[n:]), split=self.split)


# ------------------------------------------------------------------ options
def _prec_of(field, y0: torch.Tensor) -> int:
    if isinstance(field, MLP):
        return _abi.TODE_BF16W_SPLIT if field.split else _abi.TODE_BF16W
    if y0.dtype == torch.float64:
        return _abi.TODE_F64
    if y0.dtype == torch.float32:
        return _abi.TODE_F32
    raise TypeError(f"state dtype {y0.dtype} not supported")


def make_options(*, rtol=1e-6, atol=1e-6, rtol_b=None, atol_b=None, safety=0.9, fac_min=0.2,
                 fac_max=10.0, beta1=0.2, beta2=0.0, beta3=0.0, h0=0.0, max_steps=100000,
                 prec=_abi.TODE_F32, form="fused", group=0, block=0, ctas_per_sm=0,
                 poll_every=0, order=0, joint=False, method="dopri5") -> _abi.Options:
    """The C options struct.  ``method``: the Runge-Kutta pair, "dopri5"
    (Dormand & Prince) or "tsit5" (Tsitouras; App. A names both)."""
    o = _abi.Options()
    o.rtol, o.atol = float(rtol), float(atol)
    o.rtol_b = rtol_b.data_ptr() if rtol_b is not None else None
    o.atol_b = atol_b.data_ptr() if atol_b is not None else None
    o.safety, o.fac_min, o.fac_max = float(safety), float(fac_min), float(fac_max)
    o.beta1, o.beta2, o.h0 = float(beta1), float(beta2), float(h0)
    o.max_steps = int(max_steps)
    o.prec = int(prec)
    o.form = {"plain": _abi.TODE_PLAIN, "fused": _abi.TODE_FUSED}[form] \
        if isinstance(form, str) else int(form)
    o.group, o.block, o.ctas_per_sm, o.poll_every = int(group), int(block), int(ctas_per_sm), \
        int(poll_every)
    o.order = int(order)
    o.joint = int(bool(joint))
    o.beta3 = float(beta3)
    o.method = {"dopri5": _abi.TODE_DOPRI5, "tsit5": _abi.TODE_TSIT5}[method] \
        if isinstance(method, str) else int(method)
    return o


def _stream_handle(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ tape / trace
@dataclass
class TapeBuffers:
    """Checkpoint tape for the adjoint: slot j = solver state at the start of
    accepted step j*stride (state, FSAL stage, time, step, controller); with
    ``stages`` (required for the MLP field) also the stage inputs Y_2..Y_7 of
    every accepted step.  Instance-major: every array is [B, slots, ...], so
    an instance's slots are contiguous."""
    slots: int
    stride: int
    y: torch.Tensor
    y_lo: Optional[torch.Tensor]  # None: a minimal tape (below)
    k1: Optional[torch.Tensor]
    t: torch.Tensor
    h: Optional[torch.Tensor]
    err_prev: Optional[torch.Tensor]
    flags: Optional[torch.Tensor]
    h_acc: Optional[torch.Tensor]  # None: the adjoint re-runs each segment's attempts
    y_stage: Optional[torch.Tensor] = None  # [B, slots, 6, D]: Y_2..Y_7
    err_prev2: Optional[torch.Tensor] = None  # [B, slots]: the PID's second error entry

    @staticmethod
    def allocate(B, D, dtype, slots, stride, device, stages: bool = False,
                 minimal: bool = False):
        """``minimal`` (stride 1 only): just what the direct adjoint reads --
        y, t, the accepted step sizes and k1 (or, with ``stages``, the stage
        inputs instead); the forward then writes nothing else."""
        if minimal and stride != 1:
            raise ValueError("a minimal tape needs stride 1")

        def e(shape, dt=dtype, keep=True):
            return torch.empty(shape, dtype=dt, device=device) if keep else None
        full = not minimal
        comp = (B, slots, D) if dtype != torch.float64 else (1,)
        return TapeBuffers(slots, stride,
                           e((B, slots, D)),
                           e(comp, keep=full),
                           e((B, slots, D), keep=full or not stages),
                           e((B, slots), torch.float64),
                           e((B, slots), keep=full),
                           e((B, slots), keep=full),
                           e((B, slots), torch.int32, keep=full),
                           e((B, slots)),
                           e((B, slots, 6, D), keep=stages),
                           e((B, slots), keep=full))

    @staticmethod
    def bytes_per_slot(B, D, itemsize, stages: bool = False, minimal: bool = False):
        if minimal:  # y, k1 or the stage inputs, t, h_acc
            return B * (D * itemsize + (6 * D if stages else D) * itemsize + 8 + itemsize)
        comp = D * itemsize if itemsize == 4 else 0
        return B * (2 * D * itemsize + comp + 8 + 4 * itemsize + 4 +
                    (6 * D * itemsize if stages else 0))

    def c(self) -> _abi.Tape:
        def ptr(x):
            return x.data_ptr() if x is not None else None
        tp = _abi.Tape()
        tp.slots, tp.stride = self.slots, self.stride
        tp.y, tp.y_lo, tp.k1 = ptr(self.y), ptr(self.y_lo), ptr(self.k1)
        tp.t, tp.h = ptr(self.t), ptr(self.h)
        tp.err_prev, tp.flags = ptr(self.err_prev), ptr(self.flags)
        tp.h_acc, tp.y_stage = ptr(self.h_acc), ptr(self.y_stage)
        tp.err_prev2 = ptr(self.err_prev2)
        return tp


@dataclass
class Solution:
    y_eval: torch.Tensor
    y_final: torch.Tensor
    n_acc: torch.Tensor
    n_rej: torch.Tensor
    n_feval: torch.Tensor
    status: torch.Tensor
    trace: Optional[dict] = None
    extra: dict = dc_field(default_factory=dict)
    yp_eval: Optional[torch.Tensor] = None  # dy/dt at t_eval, when requested


def solve(field, y0: torch.Tensor, t0: torch.Tensor, t1: torch.Tensor,
          t_eval: Optional[torch.Tensor] = None, *, tape: Optional[TapeBuffers] = None,
          trace_cap: int = 0, stream: Optional[torch.cuda.Stream] = None,
          out: Optional[Solution] = None, workspace: Optional[torch.Tensor] = None,
          want_yp: bool = False, **opt_kw) -> Solution:
    """Solve every instance of the batch independently (Sec. 3), or, with
    ``joint=True``, the batch as one stacked problem (Sec. 4.1: one step size,
    error norm and accept decision; equal t0, t1 and t_eval rows required).

    y0 [B, D] (float64 or float32; MLP: float32), t0/t1 [B] float64,
    t_eval [B, K] float64.  Keyword options as in ``make_options``.  With
    ``want_yp`` the solution also carries yp_eval [B, K, D], dy/dt of the
    dense output at every evaluation point (every field, solved independently).
    """
    lib = _abi.load()
    B, D = y0.shape
    K = 0 if t_eval is None else t_eval.shape[1]
    dev = y0.device
    prec = _prec_of(field, y0)
    opts = make_options(prec=prec, **opt_kw)
    keep = []
    fd = field.desc(B, D, keep)
    if out is None:
        out = Solution(
            y_eval=torch.empty((B, K, D), dtype=y0.dtype, device=dev),
            y_final=torch.empty((B, D), dtype=y0.dtype, device=dev),
            n_acc=torch.empty(B, dtype=torch.int32, device=dev),
            n_rej=torch.empty(B, dtype=torch.int32, device=dev),
            n_feval=torch.empty(B, dtype=torch.int32, device=dev),
            status=torch.empty(B, dtype=torch.int32, device=dev))
    if want_yp and K > 0 and (out.yp_eval is None or out.yp_eval.shape != (B, K, D)):
        out.yp_eval = torch.empty((B, K, D), dtype=y0.dtype, device=dev)
    trace_c = None
    if trace_cap > 0:
        tr = dict(t=torch.zeros((B, trace_cap), dtype=torch.float64, device=dev),
                  h=torch.zeros((B, trace_cap), dtype=torch.float64, device=dev),
                  err=torch.zeros((B, trace_cap), dtype=torch.float64, device=dev),
                  accepted=torch.zeros((B, trace_cap), dtype=torch.int32, device=dev),
                  len=torch.zeros(B, dtype=torch.int32, device=dev))
        trace_c = _abi.Trace(trace_cap, tr["t"].data_ptr(), tr["h"].data_ptr(),
                             tr["err"].data_ptr(), tr["accepted"].data_ptr(),
                             tr["len"].data_ptr())
        out.trace = tr
    ws_bytes = lib.tode_workspace_size(C.byref(fd), C.byref(opts), int(K))
    if ws_bytes == 0 and B > 0:
        raise _abi.TodeError(_abi.TODE_EUNSUPPORTED, "tode_workspace_size")
    if workspace is None or workspace.numel() < ws_bytes:
        workspace = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=dev)
    tape_c = tape.c() if tape is not None else None
    code = lib.tode_solve(
        C.byref(fd), C.byref(opts), _ptr(y0), _ptr(t0), _ptr(t1),
        _ptr(t_eval) if K > 0 else None, int(K), _ptr(out.y_eval) if K > 0 else None,
        _ptr(out.yp_eval) if want_yp and K > 0 else None, _ptr(out.y_final), _ptr(out.n_acc), _ptr(out.n_rej), _ptr(out.n_feval), _ptr(out.status),
        C.byref(tape_c) if tape_c is not None else None,
        C.byref(trace_c) if trace_c is not None else None,
        _ptr(workspace), C.c_size_t(workspace.numel()), _stream_handle(stream))
    _abi.check(code, "tode_solve")
    out.extra["workspace"] = workspace
    return out


def mlp_resolve(field, t0, t1, n_acc: torch.Tensor, ckpt: TapeBuffers, seg: int,
                seg_tape: TapeBuffers, *, stream=None,
                workspace: Optional[torch.Tensor] = None, **opt_kw):
    """Re-run segment ``seg`` of an MLP-field solve that filled the
    checkpoint tape ``ckpt`` (stride m > 1): accepted steps seg*m .. of every
    instance, bit for bit, into the stride-1 stage tape ``seg_tape`` (m
    slots).  Returns (seg_n [B] int32, seg_t0 [B], seg_t1 [B] float64): the
    segment's accepted steps and its bounds in the caller's time, the
    arguments ``adjoint`` takes to reverse the segment.  ``n_acc``: the
    solve's accepted-step counts."""
    lib = _abi.load()
    B, D = ckpt.y.shape[0], ckpt.y.shape[2]
    dev = ckpt.y.device
    opts = make_options(prec=_abi.TODE_BF16W_SPLIT, **opt_kw)
    keep = []
    fd = field.desc(B, D, keep)
    ws_bytes = lib.tode_workspace_size(C.byref(fd), C.byref(opts), 0)
    if ws_bytes == 0 and B > 0:
        raise _abi.TodeError(_abi.TODE_EUNSUPPORTED, "tode_workspace_size")
    if workspace is None or workspace.numel() < ws_bytes:
        workspace = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=dev)
    seg_n = torch.empty(B, dtype=torch.int32, device=dev)
    seg_t0 = torch.empty(B, dtype=torch.float64, device=dev)
    seg_t1 = torch.empty(B, dtype=torch.float64, device=dev)
    ck_c, st_c = ckpt.c(), seg_tape.c()
    code = lib.tode_mlp_resolve(C.byref(fd), C.byref(opts), _ptr(t0), _ptr(t1), _ptr(n_acc),
                                C.byref(ck_c), int(seg), C.byref(st_c), _ptr(seg_n),
                                _ptr(seg_t0), _ptr(seg_t1), _ptr(workspace),
                                C.c_size_t(workspace.numel()), _stream_handle(stream))
    _abi.check(code, "tode_mlp_resolve")
    return seg_n, seg_t0, seg_t1


def t_eval_grad(gy_eval: torch.Tensor, yp_eval: torch.Tensor,
                stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """dL/dt_eval [B, K] (float64) = <dL/dy_eval, dy/dt> per evaluation point,
    from the yp_eval of a solve (``want_yp=True``)."""
    lib = _abi.load()
    B, K, D = yp_eval.shape
    prec = _abi.TODE_F64 if yp_eval.dtype == torch.float64 else _abi.TODE_F32
    gy = gy_eval.to(yp_eval.dtype).contiguous()
    g = torch.empty((B, K), dtype=torch.float64, device=yp_eval.device)
    _abi.check(lib.tode_t_eval_grad(B, K, D, prec, _ptr(gy), _ptr(yp_eval), _ptr(g),
                                    _stream_handle(stream)), "tode_t_eval_grad")
    return g


def adjoint(field, t0, t1, t_eval, sol: Solution, tape: TapeBuffers, gy_eval=None,
            gy_final=None, *, stream=None, scratch: Optional[torch.Tensor] = None,
            want_tshift: bool = False, **opt_kw):
    """Discrete adjoint of the forward solve that filled ``tape`` (App. A:
    backpropagation through the solver on the frozen mesh).  Returns
    (gy0, gparam, overflow); for the MLP field gparam is (gW, gb), and with
    ``want_tshift`` (gW, gb, tshift): tshift [B] float64, the derivative of L
    when every time of an instance (t0, t1, its evaluation points) moves
    together, which ``t_bounds_grad`` needs for dL/dt0 of this field."""
    lib = _abi.load()
    B, D = sol.y_final.shape
    K = 0 if t_eval is None else t_eval.shape[1]
    dev = sol.y_final.device
    dtype = sol.y_final.dtype
    prec = _prec_of(field, sol.y_final)
    opts = make_options(prec=prec, **opt_kw)
    keep = []
    fd = field.desc(B, D, keep)
    tape_c = tape.c()
    nb = lib.tode_adjoint_scratch_size(C.byref(fd), C.byref(opts), C.byref(tape_c))
    if nb == 0 and B > 0:
        raise _abi.TodeError(_abi.TODE_EUNSUPPORTED, "tode_adjoint_scratch_size")
    if scratch is None or scratch.numel() < nb:
        scratch = torch.empty(max(nb, 256), dtype=torch.uint8, device=dev)
    gy0 = torch.empty((B, D), dtype=dtype, device=dev)
    params = field.params()
    gparam = torch.empty_like(params) if params is not None else None
    gW_arr = gb_arr = None
    if isinstance(field, MLP):
        # float gradients of the weights and biases, summed over the batch
        gW = [torch.empty(w.shape, dtype=torch.float32, device=dev) for w in field.W]
        gb = [torch.empty(b.shape, dtype=torch.float32, device=dev) for b in field.b]
        gW_arr = (C.c_void_p * len(gW))(*[g.data_ptr() for g in gW])
        gb_arr = (C.c_void_p * len(gb))(*[g.data_ptr() for g in gb])
        gparam = (gW, gb)
    gp_ptr = _ptr(gparam) if params is not None else None
    if isinstance(field, MLP) and want_tshift:  # the MLP field's gparam: the time sums
        ts = torch.empty(B, dtype=torch.float64, device=dev)
        gparam = (gW, gb, ts)
        gp_ptr = _ptr(ts)
    overflow = torch.zeros(1, dtype=torch.int32, device=dev)
    code = lib.tode_adjoint(
        C.byref(fd), C.byref(opts), _ptr(t0), _ptr(t1), _ptr(t_eval) if K > 0 else None,
        int(K), _ptr(sol.n_acc), _ptr(sol.status), C.byref(tape_c), _ptr(gy_eval),
        _ptr(gy_final), _ptr(gy0), gp_ptr, gW_arr, gb_arr,
        _ptr(overflow), _ptr(scratch), C.c_size_t(scratch.numel()), _stream_handle(stream))
    _abi.check(code, "tode_adjoint")
    return gy0, gparam, overflow


def joint_adjoint_workspace(field, B: int, D: int, device="cuda", **opt_kw) -> torch.Tensor:
    """A device workspace large enough for joint_adjoint on B x D."""
    lib = _abi.load()
    opts = make_options(prec=_abi.TODE_BF16W_SPLIT if getattr(field, "split", False)
                        else _abi.TODE_BF16W, **opt_kw)
    keep = []
    fd = field.desc(B, D, keep)
    nb = lib.tode_joint_adjoint_workspace_size(C.byref(fd), C.byref(opts))
    if nb == 0 and B > 0:
        raise _abi.TodeError(_abi.TODE_EUNSUPPORTED, "tode_joint_adjoint_workspace_size")
    return torch.empty(max(nb, 256), dtype=torch.uint8, device=device)


def joint_adjoint(field, y1: torch.Tensor, t0: float, t1: float, t_eval=None, gy_eval=None,
                  gy_final=None, *, stream=None, workspace: Optional[torch.Tensor] = None,
                  **opt_kw):
    """Joint continuous adjoint (App. A, the CNF benchmark's "torchode-joint"
    backward pass): the adjoint equation of the whole batch -- the state
    integrated back from y1 = y(t1), its adjoint and the adjoint of the
    shared parameters -- solved backward from t1 to t0 as one problem with
    one step size and one error norm, stopping at every evaluation point for
    its cotangent.  ``field``: the MLP field (D = 32, H = 128, split);
    ``t0 < t1`` shared floats; ``t_eval`` a [K] sequence shared by the batch
    (host values); ``gy_eval`` [B, K, D], ``gy_final`` [B, D] float on the
    device.  Returns (gy0 [B, D], (gW, gb) lists, y0 [B, D] integrated back,
    stats dict with n_acc, n_rej, n_feval, status)."""
    lib = _abi.load()
    if not isinstance(field, MLP):
        raise _abi.TodeError(_abi.TODE_EUNSUPPORTED, "tode_joint_adjoint")
    B, D = y1.shape
    dev = y1.device
    te = np.ascontiguousarray(np.zeros(0) if t_eval is None else
                              (t_eval.detach().cpu().numpy() if torch.is_tensor(t_eval)
                               else np.asarray(t_eval)), dtype=np.float64).reshape(-1)
    K = te.shape[0]
    opts = make_options(prec=_prec_of(field, y1), **opt_kw)
    keep = []
    fd = field.desc(B, D, keep)
    nb = lib.tode_joint_adjoint_workspace_size(C.byref(fd), C.byref(opts))
    if nb == 0 and B > 0:
        raise _abi.TodeError(_abi.TODE_EUNSUPPORTED, "tode_joint_adjoint_workspace_size")
    if workspace is None or workspace.numel() < nb:
        workspace = torch.empty(max(nb, 256), dtype=torch.uint8, device=dev)
    gy0 = torch.empty((B, D), dtype=torch.float32, device=dev)
    y0 = torch.empty((B, D), dtype=torch.float32, device=dev)
    gW = [torch.empty(w.shape, dtype=torch.float32, device=dev) for w in field.W]
    gb = [torch.empty(b.shape, dtype=torch.float32, device=dev) for b in field.b]
    gW_arr = (C.c_void_p * len(gW))(*[g.data_ptr() for g in gW])
    gb_arr = (C.c_void_p * len(gb))(*[g.data_ptr() for g in gb])
    stats = (C.c_int32 * 4)()
    y1c = y1.contiguous()
    code = lib.tode_joint_adjoint(
        C.byref(fd), C.byref(opts), C.c_double(float(t0)), C.c_double(float(t1)),
        te.ctypes.data_as(C.POINTER(C.c_double)) if K > 0 else None, int(K), _ptr(y1c),
        _ptr(gy_eval), _ptr(gy_final), _ptr(gy0), gW_arr, gb_arr, _ptr(y0), stats,
        _ptr(workspace), C.c_size_t(workspace.numel()), _stream_handle(stream))
    _abi.check(code, "tode_joint_adjoint")
    return gy0, (gW, gb), y0, dict(n_acc=stats[0], n_rej=stats[1], n_feval=stats[2],
                                   status=stats[3])


def t_bounds_grad(field, t0, t1, t_eval, sol: Solution, tape: TapeBuffers, gy_eval=None,
                  gy_final=None, *, stream=None, want_t0: bool = True,
                  tshift: Optional[torch.Tensor] = None, **opt_kw):
    """(dL/dt0, dL/dt1) [B] float64 of the forward solve that filled
    ``tape`` (stride 1 with the accepted step sizes): the frozen map with
    every step size but the last held and the last ending at t1.  dL/dt0
    needs the solve's dy/dt at the points (``want_yp=True``) when gy_eval is
    given, and for the MLP field (time-dependent) the adjoint's ``tshift``
    (``adjoint(..., want_tshift=True)``) of the same cotangents."""
    lib = _abi.load()
    B, D = sol.y_final.shape
    K = 0 if t_eval is None else t_eval.shape[1]
    dev = sol.y_final.device
    opts = make_options(prec=_prec_of(field, sol.y_final), **opt_kw)
    keep = []
    fd = field.desc(B, D, keep)
    tape_c = tape.c()
    g1 = torch.empty(B, dtype=torch.float64, device=dev)
    g0 = None
    if want_t0:
        if isinstance(field, MLP):  # dL/dt0 starts from the translation sums
            if tshift is None:
                raise ValueError("dL/dt0 of the MLP field needs the adjoint's tshift")
            g0 = tshift.to(torch.float64).clone()
        else:
            g0 = torch.empty(B, dtype=torch.float64, device=dev)
    yp = sol.yp_eval if (want_t0 and K > 0 and gy_eval is not None) else None
    code = lib.tode_t_bounds_grad(
        C.byref(fd), C.byref(opts), _ptr(t0), _ptr(t1), _ptr(t_eval) if K > 0 else None,
        int(K), _ptr(sol.n_acc), _ptr(sol.status), C.byref(tape_c), _ptr(gy_eval),
        _ptr(gy_final), _ptr(yp), _ptr(g0), _ptr(g1), _stream_handle(stream))
    _abi.check(code, "tode_t_bounds_grad")
    return g0, g1
