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


def _prepare(cfg, B, dtype, seed):
    w = make(cfg, B=B)
    probe = gpu_solve(w, dtype, "fused")
    slots = max(1, int(probe["n_acc"].max()))
    tape = tode.TapeBuffers.allocate(B, w["y0"].shape[1], dtype, slots, 1, "cuda")
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
    fd = field.desc(B, D, [])
    tp = tape.c()
    gy0 = torch.full((B, D), float("nan"), dtype=sol.y_final.dtype, device="cuda")
    gp = torch.full_like(field.params(), float("nan"))
    ovf = torch.zeros(1, dtype=torch.int32, device="cuda")
    code = lib.tode_adjoint_static(
        C.byref(fd), C.byref(opts), _ptr(dev["t0"]), _ptr(dev["t1"]), _ptr(dev["te"]), K,
        _ptr(sol.n_acc), _ptr(sol.status), C.byref(tp), _ptr(gye), _ptr(gyf), _ptr(gy0),
        _ptr(gp), None, None, _ptr(ovf), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return code, gy0, gp, ovf


def _reference_adjoint(w, g, tape, gye, gyf):
    dev = g["_dev"]
    gy0, gp, ovf = tode.adjoint(dev["field"], dev["t0"], dev["t1"], dev["te"], g["_sol"], tape,
                                gye, gyf, rtol=w["rtol"], atol=w["atol"])
    torch.cuda.synchronize()
    return gy0, gp, ovf


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


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


def test_static_scratch_rejects_problems_beyond_its_size():
    w, g, tape, gye, gyf = _prepare(1, 256, torch.float64, seed=3)
    lib = _abi.load()
    dev = g["_dev"]
    field, sol = dev["field"], g["_sol"]
    opts = api.make_options(prec=_abi.TODE_F64, rtol=w["rtol"], atol=w["atol"])
    fd = field.desc(256, 2, [])
    big = tape.c()
    big.stride = 20000  # segments of 20000 steps per instance exceed the array
    need = lib.tode_adjoint_scratch_size(C.byref(fd), C.byref(opts), C.byref(big))
    assert need > _abi.TODE_STATIC_ADJOINT_SCRATCH_BYTES
    gy0 = torch.zeros((256, 2), dtype=torch.float64, device="cuda")
    ovf = torch.zeros(1, dtype=torch.int32, device="cuda")
    code = lib.tode_adjoint_static(
        C.byref(fd), C.byref(opts), _ptr(dev["t0"]), _ptr(dev["t1"]), _ptr(dev["te"]),
        dev["te"].shape[1], _ptr(sol.n_acc), _ptr(sol.status), C.byref(big), _ptr(gye),
        _ptr(gyf), _ptr(gy0), None, None, None, _ptr(ovf), None)
    assert code == _abi.TODE_EWORKSPACE
