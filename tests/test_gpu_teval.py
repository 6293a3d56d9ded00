"""dy/dt at the evaluation points (the dense-output interpolant's
derivative) and the gradient with respect to t_eval built on it, against
the oracle: FP64 within 1e-12 of max(|dy/dt|, 1) per point (both forms,
both directions of integration), FP32 within 1e-5 relative of the FP64
oracle's derivative, and dL/dt_eval through autograd."""
import numpy as np
import pytest
import torch

import oracle
import paper_2210_12375_b300 as tode
from gpu_helpers import device_field, gpu_solve, make

pytestmark = pytest.mark.gpu


def _rel_close(a, b, tol):
    scale = np.maximum(np.abs(b).max(axis=-1, keepdims=True), 1.0)
    return np.abs(a - b) <= tol * scale


def _mixed(w, span=(0.5, 1.5), scale=0.5):
    """Every other instance integrated backward from t1 to t0."""
    B, K = w["t_eval"].shape
    t0, t1, te = w["t0"].copy(), w["t1"].copy(), w["t_eval"].copy()
    t0[::2], t1[::2] = w["t1"][::2], w["t0"][::2]
    te[::2] = te[::2, ::-1]
    return dict(w, y0=w["y0"] * scale, t0=t0, t1=t1, t_eval=te)


@pytest.mark.parametrize("form", ["plain", "fused"])
@pytest.mark.parametrize("mixed", [False, True])
def test_yp_eval_f64_vdp_matches_oracle(form, mixed):
    w = make(1, B=64)
    if mixed:
        w = _mixed(dict(w, t1=np.minimum(w["t1"], 2.0),
                        t_eval=np.stack([np.linspace(0, min(t, 2.0), w["t_eval"].shape[1])
                                         for t in w["t1"]])))
    g = gpu_solve(w, torch.float64, form, want_yp=True)
    o = oracle.solve(w["field"], w["y0"], w["t0"], w["t1"], w["t_eval"],
                     dict(rtol=w["rtol"], atol=w["atol"]), want_yp=True)
    assert (g["status"] == 0).all() and np.array_equal(g["n_acc"], o["n_acc"])
    assert np.isfinite(g["yp_eval"]).all()
    assert _rel_close(g["yp_eval"], o["yp_eval"], 1e-12).all()


def test_yp_eval_f32_linear_matches_oracle():
    w = make(2, B=512)
    g = gpu_solve(w, torch.float32, "fused", want_yp=True)
    o = oracle.solve(w["field"], w["y0"], w["t0"], w["t1"], w["t_eval"],
                     dict(rtol=w["rtol"], atol=w["atol"]), want_yp=True)
    scale = np.maximum(np.abs(o["yp_eval"]).max(axis=-1, keepdims=True), 1.0)
    # the FP32 mesh differs from the FP64 one in the last bits: the derivative
    # of the interpolant agrees to the method's accuracy, not to rounding
    assert (np.abs(g["yp_eval"] - o["yp_eval"]) <= 1e-3 * scale).mean() > 0.999


def test_yp_eval_failed_points_nan_and_refusals():
    w = make(1, B=16)
    g = gpu_solve(w, torch.float64, "fused", want_yp=True, max_steps=6)
    assert np.array_equal(np.isnan(g["yp_eval"]), np.isnan(g["y_eval"]))
    assert np.isnan(g["yp_eval"]).any()
    te = np.tile(np.linspace(0.0, 2.0, 4), (16, 1))
    wj = dict(w, t0=np.zeros(16), t1=np.full(16, 2.0), t_eval=te)
    with pytest.raises(tode._abi.TodeError):
        gpu_solve(wj, torch.float64, "plain", joint=True, want_yp=True)
    m = dict(make(4, B=8), split=True)
    with pytest.raises(tode._abi.TodeError):
        gpu_solve(m, torch.float32, "fused", want_yp=True)


def test_t_eval_gradient_through_autograd():
    """L = sum y(t_eval)^2: dL/dt_q = 2 <y(t_q), dy/dt(t_q)>, with the
    oracle's y and dy/dt on the same (bit-identical FP64) mesh."""
    w = make(1, B=48)
    dev = "cuda"
    field = device_field(w, torch.float64)
    y0 = torch.tensor(w["y0"], dtype=torch.float64, device=dev)
    t0 = torch.tensor(w["t0"], dtype=torch.float64, device=dev)
    t1 = torch.tensor(w["t1"], dtype=torch.float64, device=dev)
    te = torch.tensor(w["t_eval"], dtype=torch.float64, device=dev, requires_grad=True)
    ye, yf, n_acc, _, status = tode.odeint_adjoint(field, y0, t0, t1, te, rtol=w["rtol"],
                                                   atol=w["atol"])
    (g_te,) = torch.autograd.grad((ye ** 2).sum(), [te])
    o = oracle.solve(w["field"], w["y0"], w["t0"], w["t1"], w["t_eval"],
                     dict(rtol=w["rtol"], atol=w["atol"]), want_yp=True)
    ref = 2.0 * np.einsum("bkd,bkd->bk", o["y_eval"], o["yp_eval"])
    got = g_te.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max())
    # the direct helper gives the same numbers
    sol = tode.solve(field, y0, t0, t1, te.detach(), rtol=w["rtol"], atol=w["atol"],
                     want_yp=True)
    g2 = tode.t_eval_grad(2.0 * sol.y_eval, sol.yp_eval).cpu().numpy()
    assert np.array_equal(g2, got)
