"""Integration backward in time (t1 < t0) on the GPU against the oracle,
which runs the method with negative steps.  The kernels integrate in
tau = -t with the negated field; IEEE rounding is symmetric under negation,
so the FP64 meshes (t, signed h, err of every attempt) must be the oracle's
bit for bit.  FP32: the FP64 oracle within the band (the closed form
within three: the backward direction amplifies the method's own error).
The adjoint reverses such a mesh like any other."""
import numpy as np
import pytest
import torch

import oracle
import paper_2210_12375_b300 as tode
from gpu_helpers import gpu_solve, make, oracle_solve
from oracle.oracle import mesh_from_trace

pytestmark = pytest.mark.gpu


def _rel_close(a, b, tol):
    scale = np.maximum(np.abs(b).max(axis=-1, keepdims=True), 1.0)
    return np.abs(a - b) <= tol * scale


def _backward(cfg, B, span, mixed=False, seed=3, scale=None):
    """Workload cfg's fields and states, integrated from t0 = span_i down to
    0 (every other instance forward from 0 to span_i when mixed).  Van der
    Pol states are halved by default: backward in time the oscillator's
    solutions from |y1| > 1 escape to infinity within these spans."""
    w = make(cfg, B=B)
    if scale is None:
        scale = 0.5 if cfg == 1 else 1.0
    w = dict(w, y0=w["y0"] * scale)
    rng = np.random.default_rng(seed)
    T = rng.uniform(*span, B)
    K = w["t_eval"].shape[1]
    t0, t1 = T.copy(), np.zeros(B)
    if mixed:
        t0[1::2], t1[1::2] = 0.0, T[1::2]
    te = np.stack([np.linspace(a, b, K) for a, b in zip(t0, t1)])
    return dict(w, t0=t0, t1=t1, t_eval=te)


@pytest.mark.parametrize("form", ["plain", "fused"])
@pytest.mark.parametrize("mixed", [False, True])
def test_backward_f64_vdp_mesh_is_the_oracles(form, mixed):
    # short spans: Van der Pol's limit cycle repels backward in time
    w = _backward(1, 96, (0.5, 2.5), mixed)
    g = gpu_solve(w, torch.float64, form, trace_cap=4000)
    o = oracle_solve(w, trace_cap=4000)
    assert (g["status"] == 0).all() and np.array_equal(g["status"], o["status"])
    assert np.array_equal(g["n_acc"], o["n_acc"]) and np.array_equal(g["n_rej"], o["n_rej"])
    for k in ("trace_t", "trace_h", "trace_err"):
        assert np.array_equal(g[k], o[k]), k
    back = (np.arange(96) % 2 == 0) if mixed else np.ones(96, bool)
    assert (g["trace_h"][back, 0] < 0).all() and (g["trace_h"][~back, 0] > 0).all()
    assert _rel_close(g["y_eval"], o["y_eval"], 1e-12).all()
    assert _rel_close(g["y_final"], o["y_final"], 1e-12).all()


def test_backward_blowups_fail_like_the_oracle():
    """Unscaled states: some backward solutions escape to infinity; the GPU
    stops them with the oracle's statuses after the oracle's attempts."""
    w = _backward(1, 96, (0.5, 2.5), True, scale=1.0)
    g = gpu_solve(w, torch.float64, "fused", trace_cap=6000)
    o = oracle_solve(w, trace_cap=6000)
    assert np.array_equal(g["status"], o["status"]) and (o["status"] == 2).sum() >= 3
    for k in ("n_acc", "n_rej", "trace_t", "trace_h", "trace_err"):
        assert np.array_equal(g[k], o[k]), k
    nan_g, nan_o = np.isnan(g["y_eval"]), np.isnan(o["y_eval"])
    assert np.array_equal(nan_g, nan_o)
    assert _rel_close(np.where(nan_g, 0, g["y_eval"]), np.where(nan_o, 0, o["y_eval"]),
                      1e-12).all()


def test_backward_f64_linear_mixed_mesh_is_the_oracles():
    w = _backward(2, 64, (0.2, 1.0), mixed=True)
    w = dict(w, rtol=1e-9, atol=1e-9)
    g = gpu_solve(w, torch.float64, "fused", trace_cap=4000)
    o = oracle_solve(w, trace_cap=4000)
    assert (g["status"] == 0).all()
    for k in ("n_acc", "n_rej", "trace_t", "trace_h", "trace_err"):
        assert np.array_equal(g[k], o[k]), k
    assert _rel_close(g["y_eval"], o["y_eval"], 1e-12).all()


@pytest.mark.parametrize("form", ["plain", "fused"])
def test_backward_f32_linear_closed_form(form):
    w = _backward(2, 512, (0.1, 0.5))
    g = gpu_solve(w, torch.float32, form)
    assert (g["status"] == 0).all()
    Q, lam = w["field"]["Q"], w["field"]["lam"]
    c = np.einsum("bji,bj->bi", Q, w["y0"])
    # y(t) = Q exp(-Lambda (t - t0)) Q^T y0, here t <= t0
    dt = w["t_eval"] - w["t0"][:, None]
    exact = np.einsum("bij,bkj->bki", Q, np.exp(-lam[:, None, :] * dt[:, :, None]) * c[:, None, :])
    # backward, this decaying system grows (up to e^5 here) and amplifies
    # the method's own global error: the FP64 oracle at the same tolerance
    # reaches 1.97 of the band against the closed form.  The FP32 path must
    # stay within the band of that FP64 solution, and within 3 bands of the
    # closed form.
    o = oracle_solve(w)
    assert (np.abs(g["y_eval"] - o["y_eval"]) <=
            10 * (w["atol"] + w["rtol"] * np.abs(o["y_eval"]))).all()
    band = 10 * (w["atol"] + w["rtol"] * np.abs(exact))
    assert (np.abs(g["y_eval"] - exact) <= 3 * band).all()


@pytest.mark.parametrize("cfg", [1, 2])
def test_backward_adjoint_vs_oracle_and_rerun(cfg):
    w = _backward(cfg, 80, (0.5, 2.0) if cfg == 1 else (0.2, 1.0), mixed=True)
    dtype = torch.float64
    B, D = w["y0"].shape
    probe = gpu_solve(w, dtype, "fused", trace_cap=4000)
    N = int(probe["n_acc"].max())
    rng = np.random.default_rng(11)
    gye = rng.standard_normal(probe["y_eval"].shape)
    gyf = rng.standard_normal(probe["y_final"].shape)
    out = []
    for stride in (1, 4):
        tape = tode.TapeBuffers.allocate(B, D, dtype, -(-N // stride), stride, "cuda")
        g = gpu_solve(w, dtype, "fused", tape=tape)
        dev = g["_dev"]
        gy0, gp, ovf = tode.adjoint(dev["field"], dev["t0"], dev["t1"], dev["te"], g["_sol"],
                                    tape, torch.tensor(gye, dtype=dtype, device="cuda"),
                                    torch.tensor(gyf, dtype=dtype, device="cuda"),
                                    rtol=w["rtol"], atol=w["atol"])
        assert int(ovf.item()) == 0
        out.append((gy0.cpu().numpy(), gp.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    mt, mh, mn = mesh_from_trace(probe)
    ref = oracle.adjoint(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"],
                         gye, gyf)
    key = "gmu" if cfg == 1 else "gA"
    for a, b in ((out[0][0], ref["gy0"]), (out[0][1], ref[key])):
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)


def test_backward_joint_matches_oracle():
    w = make(1, B=40)
    te = np.linspace(2.0, 0.0, 6)
    w = dict(w, y0=0.5 * w["y0"], t0=np.full(40, 2.0), t1=np.zeros(40),
             t_eval=np.tile(te, (40, 1)))
    g = gpu_solve(w, torch.float64, "plain", joint=True, trace_cap=2000)
    o = oracle.solve_joint(w["field"], w["y0"], 2.0, 0.0, te,
                           dict(rtol=w["rtol"], atol=w["atol"]), trace_cap=2000)
    assert (g["status"] == 0).all() and o["status"] == 0
    assert (g["n_acc"] == o["n_acc"]).all() and (g["n_rej"] == o["n_rej"]).all()
    L = o["trace_len"]
    assert (g["trace_h"][0, :L] < 0).all()
    np.testing.assert_allclose(g["trace_h"][0, :L], o["trace_h"], rtol=1e-11, atol=1e-11)
    assert _rel_close(g["y_eval"], o["y_eval"], 1e-10).all()
