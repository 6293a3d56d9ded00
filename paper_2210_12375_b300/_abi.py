"""ctypes mirror of ``include/tode.h`` and the loader of the in-tree
``libtode.so``.  Argument marshalling only: every step of the solver runs in
the library's CUDA kernels.  There is no fallback: a missing library raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtode.so")

# enums
TODE_OK, TODE_EINVAL, TODE_EWORKSPACE, TODE_ECUDA, TODE_EUNSUPPORTED, TODE_ETIMEOUT = range(6)
TODE_VDP, TODE_LINEAR, TODE_MLP = 1, 2, 3
TODE_F64, TODE_F32, TODE_BF16W, TODE_BF16W_SPLIT = 0, 1, 2, 3
TODE_PLAIN, TODE_FUSED = 0, 1
TODE_DOPRI5, TODE_TSIT5 = 0, 1
(TODE_PEAK_FMA32, TODE_PEAK_FFMA2, TODE_PEAK_FMA64, TODE_PEAK_EX2, TODE_PEAK_TANH,
 TODE_PEAK_EMPTY) = range(6)
STATUS = {"SUCCESS": 0, "MAX_STEPS": 1, "DT_UNDERFLOW": 2, "NONFINITE": 3, "INVALID_INPUT": 4}

# entry points include/tode.h declares
EXPORTS = ("tode_version", "tode_strerror", "tode_default_options", "tode_workspace_size",
           "tode_solve", "tode_adjoint_scratch_size", "tode_adjoint", "tode_adjoint_static",
           "tode_joint_adjoint_workspace_size", "tode_joint_adjoint",
           "tode_tc_gemm", "tode_t_eval_grad", "tode_peak_kernel",
           "tode_t_bounds_grad", "tode_mlp_resolve")
TODE_STATIC_ADJOINT_SCRATCH_BYTES = 32 << 20

_vp = C.c_void_p


class FieldDesc(C.Structure):
    _fields_ = [
        ("kind", C.c_int),
        ("B", C.c_int),
        ("D", C.c_int),
        ("mu", _vp),
        ("A", _vp),
        ("n_layers", C.c_int),
        ("widths", C.POINTER(C.c_int)),
        ("W", C.POINTER(_vp)),
        ("b", C.POINTER(_vp)),
    ]


class Options(C.Structure):
    _fields_ = [
        ("rtol", C.c_double),
        ("atol", C.c_double),
        ("rtol_b", _vp),
        ("atol_b", _vp),
        ("safety", C.c_double),
        ("fac_min", C.c_double),
        ("fac_max", C.c_double),
        ("beta1", C.c_double),
        ("beta2", C.c_double),
        ("h0", C.c_double),
        ("max_steps", C.c_int),
        ("prec", C.c_int),
        ("form", C.c_int),
        ("group", C.c_int),
        ("block", C.c_int),
        ("ctas_per_sm", C.c_int),
        ("poll_every", C.c_int),
        ("order", C.c_int),
        ("joint", C.c_int),
        ("beta3", C.c_double),
        ("method", C.c_int),
    ]


class Tape(C.Structure):
    _fields_ = [
        ("slots", C.c_int),
        ("stride", C.c_int),
        ("y", _vp),
        ("y_lo", _vp),
        ("k1", _vp),
        ("t", _vp),
        ("h", _vp),
        ("err_prev", _vp),
        ("flags", _vp),
        ("h_acc", _vp),
        ("y_stage", _vp),
        ("err_prev2", _vp),
    ]


class Trace(C.Structure):
    _fields_ = [
        ("cap", C.c_int),
        ("t", _vp),
        ("h", _vp),
        ("err", _vp),
        ("accepted", _vp),
        ("len", _vp),
    ]


_lib = None


class TodeError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = load().tode_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


def load(path: str = LIB_PATH):
    """Load libtode.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with `python -m paper_2210_12375_b300.build` "
            "(there is no CPU fallback)")
    lib = C.CDLL(path)
    lib.tode_version.restype = C.c_int
    lib.tode_strerror.restype = C.c_char_p
    lib.tode_strerror.argtypes = [C.c_int]
    lib.tode_default_options.argtypes = [C.POINTER(Options)]
    lib.tode_workspace_size.restype = C.c_size_t
    lib.tode_workspace_size.argtypes = [C.POINTER(FieldDesc), C.POINTER(Options), C.c_int]
    lib.tode_solve.restype = C.c_int
    lib.tode_solve.argtypes = [C.POINTER(FieldDesc), C.POINTER(Options), _vp, _vp, _vp, _vp,
                               C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.POINTER(Tape),
                               C.POINTER(Trace), _vp, C.c_size_t, _vp]
    lib.tode_t_eval_grad.restype = C.c_int
    lib.tode_t_eval_grad.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp, _vp]
    lib.tode_adjoint_scratch_size.restype = C.c_size_t
    lib.tode_adjoint_scratch_size.argtypes = [C.POINTER(FieldDesc), C.POINTER(Options),
                                              C.POINTER(Tape)]
    lib.tode_adjoint.restype = C.c_int
    lib.tode_adjoint.argtypes = [C.POINTER(FieldDesc), C.POINTER(Options), _vp, _vp, _vp, C.c_int,
                                 _vp, _vp, C.POINTER(Tape), _vp, _vp, _vp, _vp,
                                 C.POINTER(_vp), C.POINTER(_vp), _vp, _vp, C.c_size_t, _vp]
    lib.tode_joint_adjoint_workspace_size.restype = C.c_size_t
    lib.tode_joint_adjoint_workspace_size.argtypes = [C.POINTER(FieldDesc), C.POINTER(Options)]
    lib.tode_joint_adjoint.restype = C.c_int
    lib.tode_joint_adjoint.argtypes = [C.POINTER(FieldDesc), C.POINTER(Options), C.c_double,
                                       C.c_double, C.POINTER(C.c_double), C.c_int, _vp, _vp, _vp,
                                       _vp, _vp, _vp, _vp, C.POINTER(C.c_int32), _vp, C.c_size_t,
                                       _vp]
    lib.tode_adjoint_static.restype = C.c_int
    lib.tode_adjoint_static.argtypes = [C.POINTER(FieldDesc), C.POINTER(Options), _vp, _vp, _vp,
                                        C.c_int, _vp, _vp, C.POINTER(Tape), _vp, _vp, _vp, _vp,
                                        C.POINTER(_vp), C.POINTER(_vp), _vp, _vp]
    lib.tode_t_bounds_grad.restype = C.c_int
    lib.tode_t_bounds_grad.argtypes = [C.POINTER(FieldDesc), C.POINTER(Options), _vp, _vp, _vp,
                                       C.c_int, _vp, _vp, C.POINTER(Tape), _vp, _vp, _vp, _vp,
                                       _vp, _vp]
    lib.tode_mlp_resolve.restype = C.c_int
    lib.tode_mlp_resolve.argtypes = [C.POINTER(FieldDesc), C.POINTER(Options), _vp, _vp, _vp,
                                     C.POINTER(Tape), C.c_int, C.POINTER(Tape), _vp, _vp, _vp,
                                     _vp, C.c_size_t, _vp]
    lib.tode_peak_kernel.restype = C.c_int
    lib.tode_peak_kernel.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp]
    lib.tode_tc_gemm.restype = C.c_int
    lib.tode_tc_gemm.argtypes = [_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp]
    _lib = lib
    return lib


def check(code: int, where: str):
    if code != TODE_OK:
        raise TodeError(code, where)
