"""dy/dt at the evaluation points (the dense-output interpolant's
derivative) and the gradient with respect to t_eval built on it, against
the oracle: FP64 within 1e-12 of max(|dy/dt|, 1) per point (both forms,
both directions of integration), FP32 within 1e-5 relative of the FP64
oracle's derivative, the MLP field (tensor-core stages, both networks, both
forms, both directions) within 1e-4 of the oracle's derivative replayed on
the GPU's mesh, and dL/dt_eval through autograd."""
import numpy as np
import pytest
import torch

import oracle
import paper_2210_12375_b300 as tode
from oracle.oracle import mesh_from_trace
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
    m = dict(make(4, B=160), split=True)
    g = gpu_solve(m, torch.float32, "fused", want_yp=True, max_steps=2)
    assert np.array_equal(np.isnan(g["yp_eval"]), np.isnan(g["y_eval"]))
    assert np.isnan(g["yp_eval"]).any()


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


def _mlp_mixed(w):
    """Every other instance integrated backward over the same interval."""
    return _mixed(w, scale=1.0)


@pytest.mark.parametrize("cfg,B,form,mixed", [(4, 300, "fused", False), (4, 300, "plain", True),
                                              (4, 300, "fused", True), (5, 96, "fused", True)])
def test_yp_eval_mlp_matches_oracle(cfg, B, form, mixed):
    """dy/dt of the MLP field's dense output against the FP64 oracle's (same
    BF16 weights) replayed on the GPU's own mesh: the two then differ only
    by the field's split BF16 evaluation (~16 significant bits of the
    activations) carried along the trajectory -- within 1e-4 max(|dy/dt|, 1)
    (measured ~1e-5).  (At the workload tolerance the oracle's own mesh
    differs: the BF16 field noise puts a floor under the GPU's error
    estimate, so its steps grow more slowly.)  Points at t0 carry f(t0, y0);
    an instance with t1 = t0 gets f(t0, y0) at its points and zero
    counters."""
    w = dict(make(cfg, B=B), split=True)
    if mixed:
        w = _mlp_mixed(w)
    t0, t1, te = w["t0"].copy(), w["t1"].copy(), w["t_eval"].copy()
    te[1, :2] = t0[1]           # two points at t0
    t1[2] = t0[2]               # an empty interval with points
    te[2] = t0[2]
    w = dict(w, t1=t1, t_eval=te)
    g = gpu_solve(w, torch.float32, form, want_yp=True, trace_cap=64)
    assert (g["status"] == 0).all()
    assert g["n_acc"][2] == 0 and g["n_feval"][2] == 0
    assert np.isfinite(g["yp_eval"]).all()
    mt, mh, mn = mesh_from_trace(g)
    assert np.array_equal(mn, g["n_acc"])
    o = oracle.replay(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"],
                      want_yp=True)
    assert _rel_close(g["yp_eval"], o["yp_eval"], 1e-4).all()
    for i in (1, 2):  # f(t0, y0) at the points of t0 and of the empty interval
        n0 = int((te[i] == t0[i]).sum())
        f0 = oracle.field_eval(w["field"], i, t0[i], w["y0"][i], B)
        assert _rel_close(g["yp_eval"][i, :n0], np.tile(f0, (n0, 1)), 1e-4).all()
    # the derivative output changes no other result
    g0 = gpu_solve(w, torch.float32, form)
    for k in ("y_eval", "y_final", "n_acc", "n_rej", "status"):
        assert np.array_equal(g0[k], g[k]), k


def test_t_eval_gradient_mlp_through_autograd():
    """L = sum y(t_eval)^2 with the MLP field: dL/dt_q = 2 <y(t_q), dy/dt(t_q)>
    against the oracle's y and dy/dt replayed on the GPU's mesh,
    and bit for bit the GPU's own y and dy/dt through tode.t_eval_grad."""
    w = dict(make(4, B=256), split=True)
    dev = "cuda"
    field = device_field(w, torch.float32)
    y0 = torch.tensor(w["y0"], dtype=torch.float32, device=dev)
    t0 = torch.tensor(w["t0"], dtype=torch.float64, device=dev)
    t1 = torch.tensor(w["t1"], dtype=torch.float64, device=dev)
    te = torch.tensor(w["t_eval"], dtype=torch.float64, device=dev, requires_grad=True)
    ye, yf, n_acc, _, status = tode.odeint_adjoint(field, y0, t0, t1, te, rtol=w["rtol"],
                                                   atol=w["atol"])
    (g_te,) = torch.autograd.grad((ye.double() ** 2).sum(), [te])
    tr = gpu_solve(w, torch.float32, "fused", trace_cap=64)
    assert np.array_equal(tr["n_acc"], n_acc.cpu().numpy())
    mt, mh, mn = mesh_from_trace(tr)
    o = oracle.replay(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"],
                      want_yp=True)
    ref = 2.0 * np.einsum("bkd,bkd->bk", o["y_eval"], o["yp_eval"])
    got = g_te.cpu().numpy()
    scale = np.maximum(np.abs(ref).max(axis=-1, keepdims=True), 1.0)
    assert (np.abs(got - ref) <= 1e-4 * scale).all()
    sol = tode.solve(field, y0, t0, t1, te.detach(), rtol=w["rtol"], atol=w["atol"],
                     want_yp=True)
    g2 = tode.t_eval_grad(2.0 * sol.y_eval, sol.yp_eval).cpu().numpy()
    assert np.allclose(g2, got, rtol=1e-6, atol=1e-6)
