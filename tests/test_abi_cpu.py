"""The C-ABI library loads without a GPU, exports every entry point that
include/tode.h declares, and rejects bad arguments before touching a device."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2210_12375_b300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(tode_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = _abi.load()
    declared = _declared()
    assert declared, "no declarations found"
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (tode_[a-z0-9_]+)", out))
    missing = [n for n in declared if n not in exported]
    assert not missing, missing
    for n in declared:
        getattr(lib, n)
    assert set(_abi.EXPORTS) <= set(declared)
    assert lib.tode_version() == 1


def test_default_options_and_strerror():
    lib = _abi.load()
    o = _abi.Options()
    lib.tode_default_options(C.byref(o))
    assert (o.rtol, o.atol, o.safety, o.fac_min, o.fac_max, o.beta1, o.beta2) == \
        (1e-6, 1e-6, 0.9, 0.2, 10.0, 0.2, 0.0)
    assert o.max_steps == 100000 and o.form == _abi.TODE_FUSED and o.prec == _abi.TODE_F32
    for code in range(6):
        assert lib.tode_strerror(code)


def _desc(kind, B, D):
    f = _abi.FieldDesc()
    f.kind, f.B, f.D = kind, B, D
    f.mu = 0x1000
    f.A = 0x1000
    return f


def _opts(**kw):
    lib = _abi.load()
    o = _abi.Options()
    lib.tode_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def test_workspace_size_rules():
    lib = _abi.load()
    o = _opts(prec=_abi.TODE_F64, form=_abi.TODE_PLAIN)
    n = lib.tode_workspace_size(C.byref(_desc(_abi.TODE_VDP, 1000, 2)), C.byref(o), 16)
    assert n > 1000 * 2 * 8 * 3 and n % 256 == 0
    o2 = _opts(prec=_abi.TODE_F64, form=_abi.TODE_FUSED)
    # fused: the work counter and the work order (1000 int32, 256-byte padded)
    assert lib.tode_workspace_size(C.byref(_desc(_abi.TODE_VDP, 1000, 2)), C.byref(o2), 16) \
        == 256 + 4096
    assert lib.tode_workspace_size(C.byref(_desc(_abi.TODE_VDP, 1000, 2)),
                                   C.byref(_opts(prec=_abi.TODE_F64, order=2)), 16) == 0
    # unsupported or invalid combinations report 0
    assert lib.tode_workspace_size(C.byref(_desc(_abi.TODE_VDP, 10, 3)), C.byref(o), 1) == 0
    assert lib.tode_workspace_size(C.byref(_desc(_abi.TODE_LINEAR, 10, 5)), C.byref(o), 1) == 0
    bad = _opts(fac_min=2.0)
    assert lib.tode_workspace_size(C.byref(_desc(_abi.TODE_VDP, 10, 2)), C.byref(bad), 1) == 0
    # joint solving: the fused form's part, a 512-byte control block, three
    # partial sums per possible CTA and a double buffer of y, y_lo, k1
    oj = _opts(prec=_abi.TODE_F64, joint=1)
    B, D = 1000, 2
    bd = -(-B * D * 8 // 256) * 256
    assert lib.tode_workspace_size(C.byref(_desc(_abi.TODE_VDP, B, D)), C.byref(oj), 16) == \
        256 + 4096 + 512 + 24064 + 6 * bd
    assert lib.tode_workspace_size(C.byref(_desc(_abi.TODE_VDP, B, D)),
                                   C.byref(_opts(prec=_abi.TODE_F64, joint=2)), 16) == 0
    rb = np.ones(B)
    oj_b = _opts(prec=_abi.TODE_F64, joint=1, rtol_b=rb.ctypes.data)
    assert lib.tode_workspace_size(C.byref(_desc(_abi.TODE_VDP, B, D)), C.byref(oj_b), 16) == 0


def test_method_rules():
    """tsit5 (method 1) covers every field (the MLP field in its split
    form) and joint solving; an unknown method is invalid."""
    lib = _abi.load()
    assert _opts().method == _abi.TODE_DOPRI5
    vdp = C.byref(_desc(_abi.TODE_VDP, 100, 2))
    n_dp = lib.tode_workspace_size(vdp, C.byref(_opts(prec=_abi.TODE_F64)), 4)
    n_ts = lib.tode_workspace_size(vdp, C.byref(_opts(prec=_abi.TODE_F64, method=1)), 4)
    assert n_dp > 0 and n_ts == n_dp
    assert lib.tode_workspace_size(vdp, C.byref(_opts(prec=_abi.TODE_F64, method=2)), 4) == 0
    # joint solving takes either pair, with the same workspace
    n_jd = lib.tode_workspace_size(vdp, C.byref(_opts(prec=_abi.TODE_F64, joint=1)), 4)
    n_jt = lib.tode_workspace_size(vdp, C.byref(_opts(prec=_abi.TODE_F64, method=1, joint=1)), 4)
    assert n_jd > 0 and n_jt == n_jd
    f = _desc(_abi.TODE_VDP, 4, 2)
    p = C.c_void_p(0x1000)
    rc = lib.tode_solve(C.byref(f), C.byref(_opts(method=3)), p, p, p, p, 2, p, None,
                        p, p, p, p, p, None, None, p, C.c_size_t(1 << 20), None)
    assert rc == _abi.TODE_EINVAL


@pytest.mark.parametrize("mutate,code", [
    (dict(rtol=-1.0), _abi.TODE_EINVAL),
    (dict(max_steps=0), _abi.TODE_EINVAL),
    (dict(form=7), _abi.TODE_EINVAL),
    (dict(beta1=0.0), _abi.TODE_EINVAL),
    (dict(prec=_abi.TODE_BF16W), _abi.TODE_EUNSUPPORTED),
])
def test_solve_rejects_bad_options_before_launch(mutate, code):
    lib = _abi.load()
    o = _opts(**mutate)
    f = _desc(_abi.TODE_VDP, 4, 2)
    p = C.c_void_p(0x1000)
    rc = lib.tode_solve(C.byref(f), C.byref(o), p, p, p, p, 2, p, None,
                        p, p, p, p, p, None, None, p,
                        C.c_size_t(1 << 20), None)
    assert rc == code


def test_solve_rejects_null_pointers_and_small_workspace():
    lib = _abi.load()
    o = _opts(prec=_abi.TODE_F64)
    f = _desc(_abi.TODE_VDP, 4, 2)
    p = C.c_void_p(0x1000)
    # null y0
    assert lib.tode_solve(C.byref(f), C.byref(o), None, p, p, p, 2, p, None,
                          p, p, p, p, p, None, None,
                          p, C.c_size_t(1 << 20), None) == _abi.TODE_EINVAL
    # K > 0 without t_eval
    assert lib.tode_solve(C.byref(f), C.byref(o), p, p, p, None, 2, p, None,
                          p, p, p, p, p, None, None,
                          p, C.c_size_t(1 << 20), None) == _abi.TODE_EINVAL
    # workspace too small / misaligned
    assert lib.tode_solve(C.byref(f), C.byref(o), p, p, p, p, 2, p, None, p, p, p, p, p, None, None,
                          p, C.c_size_t(8), None) == _abi.TODE_EWORKSPACE
    assert lib.tode_solve(C.byref(f), C.byref(o), p, p, p, p, 2, p, None, p, p, p, p, p, None, None,
                          C.c_void_p(0x1008), C.c_size_t(1 << 20), None) == _abi.TODE_EWORKSPACE
    # empty batch is a no-op
    f0 = _desc(_abi.TODE_VDP, 0, 2)
    assert lib.tode_solve(C.byref(f0), C.byref(o), None, None, None, None, 0, None, None, None,
                          None, None, None, None, None, None, None, C.c_size_t(0),
                          None) == _abi.TODE_OK
    # bad tape: no slots, or an FP32 tape without its compensation buffer
    tp = _abi.Tape()
    tp.slots, tp.stride = 0, 1
    assert lib.tode_solve(C.byref(f), C.byref(o), p, p, p, p, 2, p, None,
                          p, p, p, p, p, C.byref(tp),
                          None, p, C.c_size_t(1 << 20), None) == _abi.TODE_EINVAL
    tp.slots = 2
    tp.y = tp.t = tp.h = tp.err_prev = tp.flags = tp.k1 = 0x1000
    o32 = _opts(prec=_abi.TODE_F32)
    assert lib.tode_solve(C.byref(f), C.byref(o32), p, p, p, p, 2, p, None,
                          p, p, p, p, p, C.byref(tp),
                          None, p, C.c_size_t(1 << 20), None) == _abi.TODE_EINVAL


def test_adjoint_rejects_bad_arguments():
    lib = _abi.load()
    o = _opts(prec=_abi.TODE_F64)
    f = _desc(_abi.TODE_VDP, 4, 2)
    p = C.c_void_p(0x1000)
    tp = _abi.Tape()
    tp.slots, tp.stride = 2, 1
    tp.y = tp.t = tp.h = tp.err_prev = tp.flags = tp.k1 = tp.y_lo = 0x1000
    need = lib.tode_adjoint_scratch_size(C.byref(f), C.byref(o), C.byref(tp))
    assert need > 0 and need % 256 == 0
    # null gy0
    assert lib.tode_adjoint(C.byref(f), C.byref(o), p, p, p, 2, p, p, C.byref(tp), p, p, None,
                            p, None, None, p, p, C.c_size_t(need), None) == _abi.TODE_EINVAL
    # scratch one byte short
    assert lib.tode_adjoint(C.byref(f), C.byref(o), p, p, p, 2, p, p, C.byref(tp), p, p, p,
                            p, None, None, p, p, C.c_size_t(need - 1), None) == \
        _abi.TODE_EWORKSPACE


def _tape(**kw):
    tp = _abi.Tape()
    tp.slots, tp.stride = 4, 1
    for k in ("y", "y_lo", "k1", "t", "h", "err_prev", "flags", "h_acc"):
        setattr(tp, k, 0x1000)
    tp.y_stage = None
    for k, v in kw.items():
        setattr(tp, k, v)
    return tp


@pytest.mark.parametrize("tape_kw,ok", [
    (dict(), True),
    (dict(y=0x1008), False),                                  # not 16-byte aligned
    (dict(y_lo=None, h=None, err_prev=None, flags=None), True),  # minimal direct tape
    (dict(y_lo=None, h=None, err_prev=None, flags=None, k1=None), False),  # no k1, no stages
    (dict(y_lo=None, h=None, err_prev=None, flags=None, k1=None, y_stage=0x2000), True),
    (dict(y_lo=None, h=None, err_prev=None, flags=None, stride=2), False),  # re-run needs all
    (dict(h_acc=None, h=None), False),                         # no step sizes: re-run
    (dict(t=None), False),
])
def test_tape_fields_checked_before_launch(tape_kw, ok):
    """Which tape arrays a solve needs: everything for strided (re-run)
    tapes; y, t, h_acc and k1 or y_stage for a stride-1 tape with step
    sizes; every array 16-byte aligned.  A rejected tape returns EINVAL
    before any device work; an accepted one passes on to the workspace
    check (here: too small)."""
    lib = _abi.load()
    o = _opts()
    f = _desc(_abi.TODE_VDP, 4, 2)
    p = C.c_void_p(0x1000)
    tp = _tape(**tape_kw)
    rc = lib.tode_solve(C.byref(f), C.byref(o), p, p, p, p, 2, p, None,
                        p, p, p, p, p, C.byref(tp), None,
                        p, C.c_size_t(0), None)
    assert rc == (_abi.TODE_EWORKSPACE if ok else _abi.TODE_EINVAL)


def test_derivative_output_and_t_eval_grad_checked_before_launch():
    """dy/dt at the points is for independent solving of the SIMT fields;
    tode_t_eval_grad validates its sizes, precision and pointers."""
    lib = _abi.load()
    f = _desc(_abi.TODE_VDP, 4, 2)
    p = C.c_void_p(0x1000)
    o = _opts(prec=_abi.TODE_F64, joint=1)
    # joint solving with yp_eval: refused before any pointer is touched
    assert lib.tode_solve(C.byref(f), C.byref(o), p, p, p, p, 2, p, p, p, p, p, p, p, None,
                          None, p, C.c_size_t(1 << 20), None) == _abi.TODE_EUNSUPPORTED
    g = lib.tode_t_eval_grad
    assert g(0, 5, 2, _abi.TODE_F64, None, None, None, None) == _abi.TODE_OK  # empty
    assert g(4, 5, 2, _abi.TODE_F64, None, p, p, None) == _abi.TODE_EINVAL
    assert g(4, 5, 0, _abi.TODE_F64, p, p, p, None) == _abi.TODE_EINVAL
    assert g(4, 5, 2, _abi.TODE_BF16W, p, p, p, None) == _abi.TODE_EUNSUPPORTED


def test_peak_kernel_rejects_bad_shapes_before_launch():
    """The micro-benchmark entry validates kind, grid, block and iters
    before any CUDA call (no GPU needed)."""
    lib = _abi.load()
    bad = [(99, 1, 32, 1), (_abi.TODE_PEAK_FMA32, 0, 32, 1), (_abi.TODE_PEAK_FMA32, 1, 0, 1),
           (_abi.TODE_PEAK_FMA32, 1, 2048, 1), (_abi.TODE_PEAK_FMA32, 1, 32, -1)]
    for kind, grid, block, iters in bad:
        assert lib.tode_peak_kernel(kind, grid, block, iters, None, None) == _abi.TODE_EINVAL
    # the arithmetic kernels need a sink
    assert lib.tode_peak_kernel(_abi.TODE_PEAK_EX2, 1, 32, 1, None, None) == _abi.TODE_EINVAL


def _mlp_desc(B, widths=(33, 128, 128, 32)):
    f = _abi.FieldDesc()
    f.kind, f.B, f.D = _abi.TODE_MLP, B, widths[-1]
    wa = (C.c_int * len(widths))(*widths)
    ptrs = (C.c_void_p * (len(widths) - 1))(*([0x1000] * (len(widths) - 1)))
    f.n_layers = len(widths) - 1
    f.widths = wa
    f.W = ptrs
    f.b = ptrs
    return f, (wa, ptrs)


def test_joint_adjoint_rules_before_launch():
    """The joint continuous adjoint covers the D = 32, H = 128 MLP field with
    split activations and scalar tolerances; its workspace grows with the
    batch; bad times, unordered points or other fields are refused before
    anything runs."""
    lib = _abi.load()
    split = _opts(prec=_abi.TODE_BF16W_SPLIT)
    f1, keep1 = _mlp_desc(128)
    f2, keep2 = _mlp_desc(1024)
    n1 = lib.tode_joint_adjoint_workspace_size(C.byref(f1), C.byref(split))
    n2 = lib.tode_joint_adjoint_workspace_size(C.byref(f2), C.byref(split))
    assert 0 < n1 < n2 and n1 % 256 == 0
    assert lib.tode_joint_adjoint_workspace_size(C.byref(f1), C.byref(_opts(prec=_abi.TODE_BF16W))) == 0
    wide, keep3 = _mlp_desc(128, (65, 512, 512, 512, 64))
    assert lib.tode_joint_adjoint_workspace_size(C.byref(wide), C.byref(split)) == 0
    assert lib.tode_joint_adjoint_workspace_size(C.byref(_desc(_abi.TODE_VDP, 10, 2)),
                                                 C.byref(_opts())) == 0
    stats = (C.c_int32 * 4)()
    p = C.c_void_p(0x1000)
    gw = (C.c_void_p * 3)(0x1000, 0x1000, 0x1000)
    te = (C.c_double * 3)(0.0, 0.7, 0.5)  # not ordered

    def call(f, o, t0, t1, tep, K):
        return lib.tode_joint_adjoint(C.byref(f), C.byref(o), t0, t1, tep, K, p, None, None, p,
                                      gw, None, None, stats, p, C.c_size_t(1 << 30), None)
    assert call(f1, split, 1.0, 0.0, None, 0) == _abi.TODE_EINVAL       # t1 <= t0
    assert call(f1, split, 0.0, 1.0, te, 3) == _abi.TODE_EINVAL         # unordered points
    assert call(f1, _opts(prec=_abi.TODE_BF16W), 0.0, 1.0, None, 0) == _abi.TODE_EUNSUPPORTED
    assert call(_desc(_abi.TODE_VDP, 4, 2), _opts(), 0.0, 1.0, None, 0) == _abi.TODE_EUNSUPPORTED
    # a misaligned workspace is reported before any launch
    rc = lib.tode_joint_adjoint(C.byref(f1), C.byref(split), 0.0, 1.0, None, 0, p, None, None, p,
                                gw, None, None, stats, C.c_void_p(0x1001), C.c_size_t(1 << 30),
                                None)
    assert rc == _abi.TODE_EWORKSPACE


def test_mlp_resolve_rules_before_launch():
    """tode_mlp_resolve (the MLP field's checkpointed segment re-solve)
    takes the split MLP field in the fused form, a checkpoint tape with
    stride > 1 that holds the whole solver state and a stride-1 stage tape
    with at least `stride` slots; anything else is refused before anything
    runs, and an empty batch is a no-op."""
    lib = _abi.load()
    split = _opts(prec=_abi.TODE_BF16W_SPLIT)
    f, keep = _mlp_desc(64)
    p = 0x1000  # 16-byte aligned stand-ins: nothing is dereferenced

    def tape(stride, slots, full=True, stages=False):
        t = _abi.Tape()
        t.slots, t.stride = slots, stride
        t.y = t.t = p
        if full:
            t.y_lo = t.k1 = t.h = t.err_prev = t.flags = p
        if stages:
            t.h_acc = t.y_stage = p
        return t
    ck, st = tape(4, 8), tape(1, 4, full=False, stages=True)
    out = C.c_void_p(p)

    def call(fd, o, ckt, seg, stt, ws_bytes=1 << 30):
        return lib.tode_mlp_resolve(C.byref(fd), C.byref(o), out, out, out, C.byref(ckt), seg,
                                    C.byref(stt), out, out, out, out, C.c_size_t(ws_bytes), None)
    assert call(f, split, ck, -1, st) == _abi.TODE_EINVAL                      # segment
    assert call(f, split, tape(1, 8, stages=True), 0, st) == _abi.TODE_EINVAL  # not strided
    assert call(f, split, tape(4, 8, full=False), 0, st) == _abi.TODE_EINVAL   # no state
    assert call(f, split, ck, 0, tape(1, 2, full=False, stages=True)) == _abi.TODE_EINVAL
    assert call(f, split, ck, 0, tape(2, 4, stages=True)) == _abi.TODE_EINVAL  # stage stride
    assert call(f, _opts(prec=_abi.TODE_BF16W), ck, 0, st) == _abi.TODE_EUNSUPPORTED
    assert call(f, _opts(prec=_abi.TODE_BF16W_SPLIT, form=_abi.TODE_PLAIN), ck, 0, st) == \
        _abi.TODE_EUNSUPPORTED
    assert call(_desc(_abi.TODE_VDP, 64, 2), _opts(prec=_abi.TODE_F32), ck, 0, st) == \
        _abi.TODE_EUNSUPPORTED
    assert call(f, split, ck, 0, st, ws_bytes=16) == _abi.TODE_EWORKSPACE
    f0, keep0 = _mlp_desc(0)
    assert call(f0, split, ck, 0, st) == _abi.TODE_OK
