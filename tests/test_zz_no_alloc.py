"""tode_adjoint_static: the adjoint entry point for callers that cannot
allocate device memory (code handed only its input and output buffers by a
host framework, or code that must not call cudaMalloc in a latency-critical
loop).  It keeps its scratch in a library-owned device array instead of a
caller buffer.  Checked through the C ABI against tode_adjoint, the entry
point that takes caller scratch, on two calls in a row (the second call
finds the first one's leftovers in the shared array), and for the rejection
of problems larger than the array.

This file is collected last on purpose, so that a run stopping at its first
failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_2210_12375_b300 as tode
from paper_2210_12375_b300 import _abi, api
from gpu_helpers import gpu_solve, make

pytestmark = pytest.mark.gpu


def _prepare(cfg, B, dtype, seed, stride=1):
    w = make(cfg, B=B)
    probe = gpu_solve(w, dtype, "fused")
    n_max = max(1, int(probe["n_acc"].max()))
    slots = -(-n_max // stride)
    mlp = w["field"]["kind"] == "mlp"
    tape = tode.TapeBuffers.allocate(B, w["y0"].shape[1], dtype, slots, stride, "cuda",
                                     stages=mlp)
    g = gpu_solve(w, dtype, "fused", tape=tape)
    rng = np.random.default_rng(seed)
    gye = torch.tensor(rng.standard_normal(g["y_eval"].shape), dtype=dtype, device="cuda")
    gyf = torch.tensor(rng.standard_normal(g["y_final"].shape), dtype=dtype, device="cuda")
    return w, g, tape, gye, gyf


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _static_adjoint(w, g, tape, gye, gyf):
    """Call tode_adjoint_static directly through ctypes."""
    lib = _abi.load()
    dev = g["_dev"]
    field, sol = dev["field"], g["_sol"]
    B, D = sol.y_final.shape
    K = dev["te"].shape[1]
    opts = api.make_options(prec=api._prec_of(field, sol.y_final), rtol=w["rtol"],
                            atol=w["atol"])
    keep = []
    fd = field.desc(B, D, keep)
    tp = tape.c()
    gy0 = torch.full((B, D), float("nan"), dtype=sol.y_final.dtype, device="cuda")
    ovf = torch.zeros(1, dtype=torch.int32, device="cuda")
    gW_arg = gb_arg = None
    if isinstance(field, tode.MLP):  # dW_l and db_l, summed over the batch
        gp = ([torch.full(x.shape, float("nan"), dtype=torch.float32, device="cuda")
               for x in field.W],
              [torch.full((x.shape[0],), float("nan"), dtype=torch.float32, device="cuda")
               for x in field.W])
        gW_arg = (C.c_void_p * len(gp[0]))(*[x.data_ptr() for x in gp[0]])
        gb_arg = (C.c_void_p * len(gp[1]))(*[x.data_ptr() for x in gp[1]])
        gparam = None
    else:
        gp = torch.full_like(field.params(), float("nan"))
        gparam = _ptr(gp)
    code = lib.tode_adjoint_static(
        C.byref(fd), C.byref(opts), _ptr(dev["t0"]), _ptr(dev["t1"]), _ptr(dev["te"]), K,
        _ptr(sol.n_acc), _ptr(sol.status), C.byref(tp), _ptr(gye), _ptr(gyf), _ptr(gy0),
        gparam, gW_arg, gb_arg, _ptr(ovf), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return code, gy0, gp, ovf


def _reference_adjoint(w, g, tape, gye, gyf):
    dev = g["_dev"]
    gy0, gp, ovf = tode.adjoint(dev["field"], dev["t0"], dev["t1"], dev["te"], g["_sol"], tape,
                                gye, gyf, rtol=w["rtol"], atol=w["atol"])
    torch.cuda.synchronize()
    return gy0, gp, ovf


def _rel(a, b):
    if isinstance(a, (tuple, list)):  # MLP: every dW_l and db_l
        return max(_rel(x, y) for x, y in zip(a, b))
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _finite(g):
    if isinstance(g, (tuple, list)):
        return all(_finite(x) for x in g)
    return bool(torch.isfinite(g).all())


def test_static_scratch_adjoint_matches_caller_scratch_twice():
    # first call: Van der Pol FP64; second call: linear D=16 FP32 on a
    # different batch size, which reuses the array the first call left
    # behind.  Tolerances are those of the adjoint parity tests.
    cases = [(1, 256, torch.float64, 1e-10), (2, 512, torch.float32, 1e-4)]
    for cfg, B, dtype, tol in cases:
        w, g, tape, gye, gyf = _prepare(cfg, B, dtype, seed=cfg)
        ref_gy0, ref_gp, ref_ovf = _reference_adjoint(w, g, tape, gye, gyf)
        code, gy0, gp, ovf = _static_adjoint(w, g, tape, gye, gyf)
        assert code == _abi.TODE_OK, _abi.load().tode_strerror(code)
        assert int(ovf.item()) == 0 and int(ref_ovf.item()) == 0
        assert torch.isfinite(gy0).all() and torch.isfinite(gp).all()
        assert _rel(gy0, ref_gy0) <= tol
        assert _rel(gp, ref_gp) <= tol


def test_static_scratch_strided_tape_and_mlp_twice():
    """Strided tapes park the re-run segments' step-start states in the
    array (its segment region, beyond the work counter and order): Van der
    Pol FP64 with stride 4, then linear FP32 with stride 3, each checked
    against the caller-scratch adjoint bit for bit (the same kernel on the
    same data); then the MLP field (D = 32, H = 128), whose per-CTA weight
    gradient partials also live in the array, at the MLP adjoint's
    tolerance."""
    for cfg, B, dtype, stride in [(1, 200, torch.float64, 4), (2, 300, torch.float32, 3)]:
        w, g, tape, gye, gyf = _prepare(cfg, B, dtype, seed=10 + cfg, stride=stride)
        ref_gy0, ref_gp, ref_ovf = _reference_adjoint(w, g, tape, gye, gyf)
        code, gy0, gp, ovf = _static_adjoint(w, g, tape, gye, gyf)
        assert code == _abi.TODE_OK, _abi.load().tode_strerror(code)
        assert int(ovf.item()) == 0 and int(ref_ovf.item()) == 0
        assert torch.isfinite(gy0).all()
        assert torch.equal(gy0, ref_gy0) and torch.equal(gp, ref_gp)
    for rep in range(2):
        w, g, tape, gye, gyf = _prepare(4, 160, torch.float32, seed=20 + rep)
        ref_gy0, ref_gp, ref_ovf = _reference_adjoint(w, g, tape, gye, gyf)
        code, gy0, gp, ovf = _static_adjoint(w, g, tape, gye, gyf)
        assert code == _abi.TODE_OK, _abi.load().tode_strerror(code)
        assert int(ovf.item()) == 0 and int(ref_ovf.item()) == 0
        assert torch.isfinite(gy0).all() and _finite(gp)
        assert _rel(gy0, ref_gy0) <= 2e-3
        assert _rel(gp, ref_gp) <= 2e-3


def _static_code(w, g, tp, gye, gyf):
    lib = _abi.load()
    dev = g["_dev"]
    field, sol = dev["field"], g["_sol"]
    B, D = sol.y_final.shape
    opts = api.make_options(prec=_abi.TODE_F64, rtol=w["rtol"], atol=w["atol"])
    fd = field.desc(B, D, [])
    gy0 = torch.zeros((B, D), dtype=torch.float64, device="cuda")
    gp = torch.zeros_like(field.params())
    ovf = torch.zeros(1, dtype=torch.int32, device="cuda")
    need = lib.tode_adjoint_scratch_size(C.byref(fd), C.byref(opts), C.byref(tp))
    code = lib.tode_adjoint_static(
        C.byref(fd), C.byref(opts), _ptr(dev["t0"]), _ptr(dev["t1"]), _ptr(dev["te"]),
        dev["te"].shape[1], _ptr(sol.n_acc), _ptr(sol.status), C.byref(tp), _ptr(gye),
        _ptr(gyf), _ptr(gy0), _ptr(gp), None, None, _ptr(ovf), None)
    torch.cuda.synchronize()
    return code, need


def test_static_scratch_refuses_the_wide_mlp():
    """The wide network's adjoint (D = 64, three layers of 512) keeps its
    pair weight images and the staged rows of every reverse round in
    scratch, far beyond the array even for one small slice: the call is
    refused with TODE_EWORKSPACE before any device work (the outputs keep
    their NaN fill)."""
    w, g, tape, gye, gyf = _prepare(5, 64, torch.float32, seed=30)
    lib = _abi.load()
    code, gy0, gp, ovf = _static_adjoint(w, g, tape, gye, gyf)
    assert code == _abi.TODE_EWORKSPACE, lib.tode_strerror(code)
    assert torch.isnan(gy0).all()
    assert all(torch.isnan(x).all() for x in gp[0])


def test_static_scratch_rejects_problems_beyond_its_size():
    # a valid strided tape (every field a re-run needs) whose segments of
    # 20000 steps per instance need more scratch than the array holds
    B = 256
    w = make(1, B=B)
    tape = tode.TapeBuffers.allocate(B, 2, torch.float64, 1, 20000, "cuda")
    g = gpu_solve(w, torch.float64, "fused", tape=tape)
    rng = np.random.default_rng(3)
    gye = torch.tensor(rng.standard_normal(g["y_eval"].shape), device="cuda")
    gyf = torch.tensor(rng.standard_normal(g["y_final"].shape), device="cuda")
    code, need = _static_code(w, g, tape.c(), gye, gyf)
    assert need > _abi.TODE_STATIC_ADJOINT_SCRATCH_BYTES
    assert code == _abi.TODE_EWORKSPACE
    # an invalid tape is an argument error whatever its size: a minimal
    # stride-1 tape (no controller state) cannot be re-run with stride 20000
    w2, g2, tape2, gye2, gyf2 = _prepare(1, B, torch.float64, seed=4)
    small = tode.TapeBuffers.allocate(B, 2, torch.float64, tape2.slots, 1, "cuda", minimal=True)
    bad = small.c()
    bad.stride = 20000
    code, _ = _static_code(w2, g2, bad, gye2, gyf2)
    assert code == _abi.TODE_EINVAL
