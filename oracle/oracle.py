"""ctypes front end of the FP64 CPU oracle (``tode_oracle.c``).

TEST INFRASTRUCTURE ONLY (tests, smoke check, bench CPU baseline).  It
shares no code with the CUDA path.  All arrays are numpy float64 / int32,
instance-major, on the host.

Parts follow the torchode paper (Sec. 3: independent per-instance solver
state, FSAL/SSAL, Horner dense output; App. A: dopri5 with an integral
controller; App. C: PI(D) controllers after Soderlind).  The starting-step
heuristic is HNW Sec. II.4's (the paper gives no rule), pinned by its closed
form on diagonal linear systems and an exact evaluation on Van der Pol.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tode_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {"SUCCESS": 0, "MAX_STEPS": 1, "DT_UNDERFLOW": 2, "NONFINITE": 3, "INVALID_INPUT": 4}
_KIND = {"vdp": 1, "linear": 2, "mlp": 3}
# the Runge-Kutta pair: dopri5 (Dormand & Prince 1980) or tsit5 (Tsitouras
# 2011), both named in App. A
METHODS = {"dopri5": 0, "tsit5": 1}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class _Field(C.Structure):
    _fields_ = [
        ("kind", C.c_int),
        ("D", C.c_int),
        ("mu", _dp),
        ("A", _dp),
        ("n_layers", C.c_int),
        ("widths", C.POINTER(C.c_int)),
        ("W", C.POINTER(_dp)),
        ("bias", C.POINTER(_dp)),
        ("inner", C.c_void_p),
        ("n_inner", C.c_int),
        ("scr", _dp),
    ]


class _Opts(C.Structure):
    _fields_ = [
        ("rtol", C.c_double),
        ("atol", C.c_double),
        ("rtol_b", _dp),
        ("atol_b", _dp),
        ("safety", C.c_double),
        ("fac_min", C.c_double),
        ("fac_max", C.c_double),
        ("beta1", C.c_double),
        ("beta2", C.c_double),
        ("h0", C.c_double),
        ("max_steps", C.c_int),
        ("beta3", C.c_double),
        ("method", C.c_int),
    ]


class _Trace(C.Structure):
    _fields_ = [
        ("cap", C.c_int),
        ("t", _dp),
        ("h", _dp),
        ("err", _dp),
        ("accepted", _ip),
        ("len", _ip),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, no fast-math)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC",
               "-shared", "-pthread", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        lib.orc_solve.restype = C.c_int
        lib.orc_solve_yp.restype = C.c_int
        lib.orc_replay.restype = C.c_int
        lib.orc_adjoint.restype = C.c_int
        lib.orc_adjoint_t.restype = C.c_int
        lib.orc_adjoint_tm.restype = C.c_int
        lib.orc_replay_m.restype = C.c_int
        lib.orc_replay_yp.restype = C.c_int
        lib.orc_joint_adjoint.restype = C.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _iptr(a):
    return a.ctypes.data_as(_ip) if a is not None else None


def default_opts(**kw) -> dict:
    """Integral controller defaults (App. A uses an I controller everywhere)."""
    o = dict(rtol=1e-6, atol=1e-6, rtol_b=None, atol_b=None, safety=0.9, fac_min=0.2,
             fac_max=10.0, beta1=0.2, beta2=0.0, beta3=0.0, h0=0.0, max_steps=100000,
             method="dopri5")
    o.update(kw)
    return o


class _FieldHolder:
    """Keeps every numpy buffer referenced by the C struct alive."""

    def __init__(self, field: dict, B: int):
        kind = field["kind"]
        self.keep = []
        f = _Field()
        f.kind = _KIND[kind]
        if kind == "vdp":
            mu = np.ascontiguousarray(field["mu"], dtype=np.float64).reshape(B)
            self.keep.append(mu)
            f.D = 2
            f.mu = _ptr(mu)
        elif kind == "linear":
            A = np.ascontiguousarray(field["A"], dtype=np.float64)
            assert A.shape[0] == B and A.shape[1] == A.shape[2]
            self.keep.append(A)
            f.D = A.shape[1]
            f.A = _ptr(A)
        elif kind == "mlp":
            Ws = [np.ascontiguousarray(w, dtype=np.float64) for w in field["W"]]
            bs = [np.ascontiguousarray(b, dtype=np.float64) for b in field["b"]]
            widths = [Ws[0].shape[1]] + [w.shape[0] for w in Ws]
            for l, w in enumerate(Ws):
                assert w.shape == (widths[l + 1], widths[l])
                assert bs[l].shape == (widths[l + 1],)
            f.D = widths[-1]
            assert widths[0] == f.D + 1, "MLP input is [y; t]"
            self.keep += Ws + bs
            wa = (C.c_int * len(widths))(*widths)
            Wp = (_dp * len(Ws))(*[_ptr(w) for w in Ws])
            bp = (_dp * len(bs))(*[_ptr(b) for b in bs])
            self.keep += [wa, Wp, bp]
            f.n_layers = len(Ws)
            f.widths = wa
            f.W = Wp
            f.bias = bp
        else:
            raise ValueError(kind)
        self.f = f
        self.D = f.D


def _opts_struct(opts: dict, B: int, keep: list):
    o = _Opts()
    for k in ("rtol", "atol", "safety", "fac_min", "fac_max", "beta1", "beta2", "beta3", "h0"):
        setattr(o, k, float(opts[k]))
    o.max_steps = int(opts["max_steps"])
    o.method = METHODS[opts.get("method", "dopri5")]
    for k in ("rtol_b", "atol_b"):
        v = opts.get(k)
        if v is not None:
            a = np.ascontiguousarray(v, dtype=np.float64).reshape(B)
            keep.append(a)
            setattr(o, k, _ptr(a))
    return o


def field_eval(field: dict, i: int, t: float, y, B: int | None = None) -> np.ndarray:
    """One evaluation f(t, y) of instance i's field."""
    lib = _load()
    if B is None:
        B = (len(field["mu"]) if field["kind"] == "vdp" else
             field["A"].shape[0] if field["kind"] == "linear" else 1)
    fh = _FieldHolder(field, B)
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(fh.D)
    out = np.zeros(fh.D)
    lib.orc_field_eval(C.byref(fh.f), C.c_int(i), C.c_double(t), _ptr(y), _ptr(out))
    return out


def dense_weights(theta: float) -> np.ndarray:
    lib = _load()
    out = np.zeros(7)
    lib.orc_dense_weights(C.c_double(theta), _ptr(out))
    return out


def tableau_m(method: str):
    """The pair's coefficients as the oracle uses them: (c [7], A [7,7],
    b [7], e = b - bhat [7], q [7,4] with b_i(theta) = theta*(q0 + theta*(q1 +
    theta*(q2 + theta*q3))))."""
    lib = _load()
    c, b, e = np.zeros(7), np.zeros(7), np.zeros(7)
    a, q = np.zeros((7, 7)), np.zeros((7, 4))
    lib.orc_tableau_m(C.c_int(METHODS[method]), _ptr(c), _ptr(a), _ptr(b), _ptr(e), _ptr(q))
    return c, a, b, e, q


def dense_weights_m(method: str, theta: float) -> np.ndarray:
    """b_i(theta) of the pair ``method``."""
    lib = _load()
    out = np.zeros(7)
    lib.orc_dense_weights_m(C.c_int(METHODS[method]), C.c_double(theta), _ptr(out))
    return out


def tableau_doubles():
    """(c, A, b, bhat, q) exactly as the oracle stores them."""
    lib = _load()
    c = np.zeros(7)
    a = np.zeros((7, 7))
    b = np.zeros(7)
    bh = np.zeros(7)
    q = np.zeros((7, 4))
    lib.orc_tableau(_ptr(c), _ptr(a), _ptr(b), _ptr(bh), _ptr(q))
    return c, a, b, bh, q


def _f64(a, shape):
    return np.ascontiguousarray(a, dtype=np.float64).reshape(shape)


def solve(field: dict, y0, t0, t1, t_eval=None, opts: dict | None = None,
          trace_cap: int = 0, nthreads: int = 0, want_yp: bool = False) -> dict:
    """Adaptive dopri5 over B independent instances (Sec. 3).

    Returns y_eval [B,K,D], y_final [B,D], n_acc, n_rej, n_feval, status [B]
    and, when trace_cap > 0, per-attempt traces t/h/err/accepted [B,cap] with
    their lengths.  ``threads`` is the number of host threads used.  With
    ``want_yp``, also yp_eval [B,K,D]: dy/dt of the dense output at every
    evaluation point (f(t0, y0) at points equal to t0).
    """
    lib = _load()
    opts = default_opts(**(opts or {}))
    y0 = np.asarray(y0, dtype=np.float64)
    B = y0.shape[0]
    fh = _FieldHolder(field, B)
    D = fh.D
    y0 = _f64(y0, (B, D))
    t0 = _f64(t0, (B,))
    t1 = _f64(t1, (B,))
    if t_eval is None:
        t_eval = np.zeros((B, 0))
    t_eval = np.ascontiguousarray(t_eval, dtype=np.float64)
    K = t_eval.shape[1]
    keep = []
    o = _opts_struct(opts, B, keep)
    y_eval = np.zeros((B, K, D))
    y_final = np.zeros((B, D))
    n_acc = np.zeros(B, np.int32)
    n_rej = np.zeros(B, np.int32)
    n_fe = np.zeros(B, np.int32)
    st = np.zeros(B, np.int32)
    tr = None
    out = {}
    if trace_cap > 0:
        tt = np.zeros((B, trace_cap))
        th = np.zeros((B, trace_cap))
        te = np.zeros((B, trace_cap))
        ta = np.zeros((B, trace_cap), np.int32)
        tl = np.zeros(B, np.int32)
        tr = _Trace(trace_cap, _ptr(tt), _ptr(th), _ptr(te), _iptr(ta), _iptr(tl))
        out.update(trace_t=tt, trace_h=th, trace_err=te, trace_accepted=ta, trace_len=tl)
    yp = np.zeros((B, K, D)) if want_yp else None
    used = lib.orc_solve_yp(C.byref(fh.f), C.byref(o), C.c_int(B), _ptr(y0), _ptr(t0),
                            _ptr(t1), _ptr(t_eval), C.c_int(K), _ptr(y_eval),
                            _ptr(yp) if yp is not None else None, _ptr(y_final),
                            _iptr(n_acc), _iptr(n_rej), _iptr(n_fe), _iptr(st),
                            C.byref(tr) if tr is not None else None, C.c_int(nthreads))
    out.update(y_eval=y_eval, y_final=y_final, n_acc=n_acc, n_rej=n_rej, n_feval=n_fe,
               status=st, threads=used)
    if yp is not None:
        out["yp_eval"] = yp
    return out


def solve_joint(field: dict, y0, t0: float, t1: float, t_eval=None, opts: dict | None = None,
                trace_cap: int = 0) -> dict:
    """Joint ("stacked") solving, Sec. 4.1: the B instances concatenated into
    one problem of size B*D -- one step size, one error norm over all B*D
    components, one accept/reject decision for the whole batch.

    The concatenation is a field of its own (block b of the state evolves by
    instance b's f) handed to the single-instance solver unchanged, so the
    norm, the starting step and the controller are those of one problem.
    y0 [B,D]; t0, t1 scalars; t_eval [K] shared.  Returns y_eval [B,K,D],
    y_final [B,D] and the one problem's n_acc, n_rej, n_feval, status (ints)
    and, when trace_cap > 0, its trace (1-D arrays).
    """
    lib = _load()
    opts = default_opts(**(opts or {}))
    assert opts.get("rtol_b") is None and opts.get("atol_b") is None, \
        "joint solving takes scalar tolerances"
    y0 = np.asarray(y0, dtype=np.float64)
    B = y0.shape[0]
    inner = _FieldHolder(field, B)
    D = inner.D
    f = _Field()
    f.kind = 4  # stacked
    f.D = B * D
    f.inner = C.cast(C.pointer(inner.f), C.c_void_p)
    f.n_inner = B
    y0 = _f64(y0, (1, B * D))
    te = np.zeros((1, 0)) if t_eval is None else _f64(t_eval, (1, -1))
    K = te.shape[1]
    keep = []
    o = _opts_struct(opts, 1, keep)
    y_eval = np.zeros((1, K, B * D))
    y_final = np.zeros((1, B * D))
    n_acc, n_rej, n_fe, st = (np.zeros(1, np.int32) for _ in range(4))
    tr = None
    out = {}
    if trace_cap > 0:
        tt, th, terr = (np.zeros((1, trace_cap)) for _ in range(3))
        ta = np.zeros((1, trace_cap), np.int32)
        tl = np.zeros(1, np.int32)
        tr = _Trace(trace_cap, _ptr(tt), _ptr(th), _ptr(terr), _iptr(ta), _iptr(tl))
    lib.orc_solve(C.byref(f), C.byref(o), C.c_int(1), _ptr(y0), _ptr(_f64([t0], (1,))),
                  _ptr(_f64([t1], (1,))), _ptr(te), C.c_int(K), _ptr(y_eval), _ptr(y_final),
                  _iptr(n_acc), _iptr(n_rej), _iptr(n_fe), _iptr(st),
                  C.byref(tr) if tr is not None else None, C.c_int(1))
    if tr is not None:
        n = int(tl[0])
        out.update(trace_t=tt[0, :n], trace_h=th[0, :n], trace_err=terr[0, :n],
                   trace_accepted=ta[0, :n], trace_len=n)
    out.update(y_eval=y_eval.reshape(K, B, D).transpose(1, 0, 2).copy(),
               y_final=y_final.reshape(B, D), n_acc=int(n_acc[0]), n_rej=int(n_rej[0]),
               n_feval=int(n_fe[0]), status=int(st[0]))
    return out


def replay(field: dict, y0, t0, t1, mesh_t, mesh_h, mesh_n, t_eval=None,
           nthreads: int = 0, method: str = "dopri5", want_yp: bool = False) -> dict:
    """Fixed-mesh steps of the pair ``method`` (no controller).  mesh_t/mesh_h
    [B,cap], mesh_n [B] accepted steps; the last step of instance i ends at
    t1[i].  With ``want_yp``, also yp_eval [B,K,D]: dy/dt of the dense output
    of the replayed steps at the points (f(t0, y0) at points equal to t0)."""
    lib = _load()
    y0 = np.asarray(y0, dtype=np.float64)
    B = y0.shape[0]
    fh = _FieldHolder(field, B)
    D = fh.D
    y0 = _f64(y0, (B, D))
    mesh_t = np.ascontiguousarray(mesh_t, dtype=np.float64)
    mesh_h = np.ascontiguousarray(mesh_h, dtype=np.float64)
    mesh_n = np.ascontiguousarray(mesh_n, dtype=np.int32)
    cap = mesh_t.shape[1]
    if t_eval is None:
        t_eval = np.zeros((B, 0))
    t_eval = np.ascontiguousarray(t_eval, dtype=np.float64)
    K = t_eval.shape[1]
    y_eval = np.zeros((B, K, D))
    y_final = np.zeros((B, D))
    yp = np.zeros((B, K, D)) if want_yp else None
    lib.orc_replay_yp(C.c_int(METHODS[method]), C.byref(fh.f), C.c_int(B), _ptr(y0),
                      _ptr(_f64(t0, (B,))), _ptr(_f64(t1, (B,))), _ptr(mesh_t), _ptr(mesh_h),
                      _iptr(mesh_n), C.c_int(cap), _ptr(t_eval), C.c_int(K), _ptr(y_eval),
                      _ptr(yp) if yp is not None else None, _ptr(y_final), C.c_int(nthreads))
    out = dict(y_eval=y_eval, y_final=y_final)
    if yp is not None:
        out["yp_eval"] = yp
    return out


def adjoint(field: dict, y0, t0, t1, mesh_t, mesh_h, mesh_n, t_eval=None, gy_eval=None,
            gy_final=None, nthreads: int = 0, want_t_bounds: bool = False,
            method: str = "dopri5") -> dict:
    """Discrete adjoint of the fixed-mesh map (App. A, backprop through the
    solver).  Returns gy0 [B,D] and the parameter cotangents: ``gmu`` [B]
    (VdP), ``gA`` [B,D,D] (linear) or ``gW``/``gb`` lists summed over the
    batch (MLP).  With ``want_t_bounds``, also ``gt0`` and ``gt1`` [B]: the
    gradients with respect to t0 and t1 of the same frozen map (every step
    size but the last and every evaluation point's step held, the last step
    ending at t1).  ``method`` is the pair the mesh was made with."""
    lib = _load()
    y0 = np.asarray(y0, dtype=np.float64)
    B = y0.shape[0]
    fh = _FieldHolder(field, B)
    D = fh.D
    y0 = _f64(y0, (B, D))
    mesh_t = np.ascontiguousarray(mesh_t, dtype=np.float64)
    mesh_h = np.ascontiguousarray(mesh_h, dtype=np.float64)
    mesh_n = np.ascontiguousarray(mesh_n, dtype=np.int32)
    cap = mesh_t.shape[1]
    if t_eval is None:
        t_eval = np.zeros((B, 0))
    t_eval = np.ascontiguousarray(t_eval, dtype=np.float64)
    K = t_eval.shape[1]
    gye = _f64(gy_eval, (B, K, D)) if gy_eval is not None else None
    gyf = _f64(gy_final, (B, D)) if gy_final is not None else None
    gy0 = np.zeros((B, D))
    kind = field["kind"]
    out = {}
    gparam = None
    gW_ptrs = gb_ptrs = None
    if kind == "vdp":
        gparam = np.zeros(B)
        out["gmu"] = gparam
    elif kind == "linear":
        gparam = np.zeros((B, D, D))
        out["gA"] = gparam
    else:
        gW = [np.zeros_like(np.asarray(w, dtype=np.float64)) for w in field["W"]]
        gb = [np.zeros_like(np.asarray(b, dtype=np.float64)) for b in field["b"]]
        gW_ptrs = (_dp * len(gW))(*[_ptr(w) for w in gW])
        gb_ptrs = (_dp * len(gb))(*[_ptr(b) for b in gb])
        out["gW"] = gW
        out["gb"] = gb
    gt0 = np.zeros(B) if want_t_bounds else None
    gt1 = np.zeros(B) if want_t_bounds else None
    lib.orc_adjoint_tm(C.c_int(METHODS[method]), C.byref(fh.f), C.c_int(B), _ptr(y0),
                       _ptr(_f64(t0, (B,))), _ptr(_f64(t1, (B,))), _ptr(mesh_t), _ptr(mesh_h),
                       _iptr(mesh_n), C.c_int(cap), _ptr(t_eval), C.c_int(K), _ptr(gye),
                       _ptr(gyf), _ptr(gy0), _ptr(gparam), gW_ptrs, gb_ptrs, _ptr(gt0),
                       _ptr(gt1), C.c_int(nthreads))
    if want_t_bounds:
        out["gt0"], out["gt1"] = gt0, gt1
    out["gy0"] = gy0
    return out


def joint_adjoint(field: dict, y1, t0: float, t1: float, t_eval=None, gy_eval=None,
                  gy_final=None, opts: dict | None = None) -> dict:
    """Joint continuous adjoint of B instances of an MLP field over a shared
    time axis (App. A, the CNF benchmark's "torchode-joint" backward pass):
    the augmented system [y; a; abar] of size 2BD + P solved backward from
    t1 to t0 as one problem, stopping at every evaluation point to add its
    cotangent.  y1 [B,D] = y(t1) of the forward solve; t_eval [K] shared;
    gy_eval [B,K,D], gy_final [B,D].  Returns gy0 [B,D], gW / gb (lists,
    like the MLP field's W / b), y0 [B,D] (the state integrated back to t0)
    and n_acc, n_rej, n_feval, status over all segments."""
    lib = _load()
    y1 = np.asarray(y1, dtype=np.float64)
    B, D = y1.shape
    fh = _FieldHolder(field, B)
    assert field["kind"] == "mlp" and fh.D == D
    keep = []
    o = _opts_struct(default_opts(**(opts or {})), B, keep)
    te = np.ascontiguousarray(np.zeros(0) if t_eval is None else t_eval, dtype=np.float64).reshape(-1)
    K = te.shape[0]
    gye = _f64(gy_eval, (B, K, D)) if gy_eval is not None else None
    gyf = _f64(gy_final, (B, D)) if gy_final is not None else None
    gy0 = np.zeros((B, D))
    y0 = np.zeros((B, D))
    gW = [np.zeros_like(np.asarray(w, dtype=np.float64)) for w in field["W"]]
    gb = [np.zeros_like(np.asarray(b, dtype=np.float64)) for b in field["b"]]
    gW_ptrs = (_dp * len(gW))(*[_ptr(w) for w in gW])
    gb_ptrs = (_dp * len(gb))(*[_ptr(b) for b in gb])
    stats = np.zeros(4, np.int32)
    rc = lib.orc_joint_adjoint(C.byref(fh.f), C.byref(o), C.c_int(B), _ptr(_f64(y1, (B, D))),
                               C.c_double(t0), C.c_double(t1), _ptr(te), C.c_int(K), _ptr(gye),
                               _ptr(gyf), _ptr(gy0), gW_ptrs, gb_ptrs, _ptr(y0), _iptr(stats))
    if rc != 0:
        raise ValueError("orc_joint_adjoint: invalid call")
    return dict(gy0=gy0, gW=gW, gb=gb, y0=y0, n_acc=int(stats[0]), n_rej=int(stats[1]),
                n_feval=int(stats[2]), status=int(stats[3]))


def mesh_from_trace(res: dict):
    """Accepted-step mesh (t_n, h_n, N) from a solve() trace."""
    B, cap = res["trace_t"].shape
    n = np.zeros(B, np.int32)
    mt = np.zeros((B, cap))
    mh = np.zeros((B, cap))
    for i in range(B):
        L = res["trace_len"][i]
        acc = res["trace_accepted"][i, :L].astype(bool)
        k = int(acc.sum())
        n[i] = k
        mt[i, :k] = res["trace_t"][i, :L][acc]
        mh[i, :k] = res["trace_h"][i, :L][acc]
    return mt, mh, n
