"""Seeded synthetic workloads shaped like the torchode paper's experiments.

This module only draws numbers: it holds none of the solver's arithmetic and
is the one piece shared by the CUDA path's tests/bench and the oracle.  Every
array is float64 numpy on the host (BF16 weights are float64 copies of values
that are exactly representable in BF16).

Workloads (seed = 20221022 + workload number, numpy PCG64):
  1 ``vdp_f64_b256``      Van der Pol (Sec. 4.1, Eq. 1), mu~U[0.5,3],
                          y0~U[-2,2]^2, t0=0, t1~U[5,15], 16 evenly spaced
                          t_eval, rtol=atol=1e-7, FP64.
  2 ``linear_d16_b8192``  y'=A_i y, A_i = Q_i diag(-lambda_i) Q_i^T, Q_i from
                          the QR of a N(0,1) 16x16 matrix (sign fixed so that
                          diag(R) > 0), lambda~U[0.1,10]^16, y0~N(0,1), t0=0,
                          t1 log-uniform in [0.1,10], 32 evenly spaced t_eval,
                          rtol=atol=1e-5, FP32 state.
  3 ``vdp_mix_b262144``   stiffness-mixed Van der Pol, mu log-uniform in
                          [0.1,20], y0~U[-2,2]^2, t1 log-uniform in [1,50],
                          8 evenly spaced t_eval, rtol=atol=1e-6, FP32 state.
  4 ``mlp_d32_h128``      MLP field W3 tanh(W2 tanh(W1[y;t]+b1)+b2)+b3, D=32,
                          hidden 128, W ~ N(0, 1/fan_in) rounded to BF16,
                          b = 0, B=16384, y0~N(0,1), t in [0,1], 8 t_eval,
                          rtol=atol=1e-4.
  5 ``mlp_d64_h512``      D=64, three tanh layers of 512, B=65536,
                          t1~U[0.5,2], 32 t_eval, rtol=atol=1e-5.
  0 ``vdp_paper_b256``    the paper's own VdP loop-time setup (App. A): B=256,
                          mu=2, y0=(2,0), rtol=atol=1e-5, 200 evenly spaced
                          t_eval over [0, 7.63] (about one cycle at mu=2).
"""
from __future__ import annotations

import numpy as np

NAMES = {
    0: "vdp_paper_b256",
    1: "vdp_f64_b256",
    2: "linear_d16_b8192",
    3: "vdp_mix_b262144",
    4: "mlp_d32_h128",
    5: "mlp_d64_h512",
}
FULL_B = {0: 256, 1: 256, 2: 8192, 3: 262144, 4: 16384, 5: 65536}


def _rng(cfg: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(20221022 + cfg))


def _log_uniform(rng, lo, hi, n):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n))


def _even(t0, t1, K):
    s = np.linspace(0.0, 1.0, K)
    te = t0[:, None] + (t1 - t0)[:, None] * s[None, :]
    te[:, -1] = t1  # the last point is exactly t1
    return np.ascontiguousarray(te)


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _mlp_weights(rng, widths):
    W, b = [], []
    for l in range(len(widths) - 1):
        fan_in = widths[l]
        w = rng.standard_normal((widths[l + 1], fan_in)) / np.sqrt(fan_in)
        W.append(round_bf16(w))
        b.append(np.zeros(widths[l + 1]))
    return W, b


def make(cfg: int, B: int | None = None) -> dict:
    """Workload ``cfg`` with its first ``B`` instances (default: all)."""
    rng = _rng(cfg)
    n = FULL_B[cfg]
    if cfg in (0, 1, 3):
        if cfg == 1:
            mu = rng.uniform(0.5, 3.0, n)
            y0 = rng.uniform(-2.0, 2.0, (n, 2))
            t1 = rng.uniform(5.0, 15.0, n)
            K, tol, prec = 16, 1e-7, "f64"
        elif cfg == 3:
            mu = _log_uniform(rng, 0.1, 20.0, n)
            y0 = rng.uniform(-2.0, 2.0, (n, 2))
            t1 = _log_uniform(rng, 1.0, 50.0, n)
            K, tol, prec = 8, 1e-6, "f32"
        else:
            mu = np.full(n, 2.0)
            y0 = np.tile(np.array([2.0, 0.0]), (n, 1))
            t1 = np.full(n, 7.63)
            K, tol, prec = 200, 1e-5, "f32"
        t0 = np.zeros(n)
        field = {"kind": "vdp", "mu": mu}
    elif cfg == 2:
        D = 16
        G = rng.standard_normal((n, D, D))
        Q, R = np.linalg.qr(G)
        s = np.sign(np.diagonal(R, axis1=1, axis2=2))
        s[s == 0] = 1.0
        Q = Q * s[:, None, :]
        lam = rng.uniform(0.1, 10.0, (n, D))
        A = np.einsum("bij,bj,bkj->bik", Q, -lam, Q)
        y0 = rng.standard_normal((n, D))
        t0 = np.zeros(n)
        t1 = _log_uniform(rng, 0.1, 10.0, n)
        K, tol, prec = 32, 1e-5, "f32"
        field = {"kind": "linear", "A": A, "Q": Q, "lam": lam}
    elif cfg in (4, 5):
        if cfg == 4:
            D, widths = 32, [33, 128, 128, 32]
            t1 = np.ones(n)
            K, tol = 8, 1e-4
        else:
            D, widths = 64, [65, 512, 512, 512, 64]
            K, tol = 32, 1e-5
            t1 = None
        W, b = _mlp_weights(rng, widths)
        y0 = rng.standard_normal((n, D))
        if t1 is None:
            t1 = rng.uniform(0.5, 2.0, n)
        t0 = np.zeros(n)
        prec = "bf16w"
        field = {"kind": "mlp", "W": W, "b": b}
    else:
        raise ValueError(cfg)
    t_eval = _even(t0, t1, K)
    if B is not None and B < n:
        y0, t0, t1, t_eval = y0[:B], t0[:B], t1[:B], t_eval[:B]
        field = dict(field)
        for k in ("mu", "A", "Q", "lam"):
            if k in field:
                field[k] = field[k][:B]
        n = B
    return dict(name=NAMES[cfg], cfg=cfg, B=n, field=field, y0=np.ascontiguousarray(y0),
                t0=t0, t1=t1, t_eval=t_eval, rtol=tol, atol=tol, prec=prec)
