"""Pins of the oracle's joint continuous adjoint (App. A, CNF benchmark: the
"torchode-joint" backward pass solving one adjoint equation of size bf + p
for the whole batch): against central differences of a tight FP64 forward
solve (dL/dy0 of every instance, sampled weights and biases of every layer),
against the discrete adjoint on that solve's mesh (both tend to the exact
gradient), the backward-integrated state against y0, and the jumps of
evaluation points at t0, inside and at t1."""
import numpy as np
import pytest

import oracle
from oracle.oracle import mesh_from_trace
from paper_2210_12375_b300 import workloads

T0, T1 = 0.0, 1.0
TIGHT = dict(rtol=1e-12, atol=1e-12)


def _setup(B=3, seed=0, te=None):
    w = workloads.make(4, B=B)
    te = w["t_eval"][0] if te is None else np.asarray(te, dtype=np.float64)
    rng = np.random.default_rng(seed)
    r = oracle.solve(w["field"], w["y0"], np.full(B, T0), np.full(B, T1), np.tile(te, (B, 1)),
                     TIGHT, trace_cap=20000)
    gye = rng.standard_normal(r["y_eval"].shape)
    gyf = rng.standard_normal(r["y_final"].shape)
    return w, te, r, gye, gyf


def _loss(w, te, gye, gyf, y0=None, W=None, b=None):
    B = w["y0"].shape[0]
    f = dict(w["field"], W=W if W is not None else w["field"]["W"],
             b=b if b is not None else w["field"]["b"])
    rr = oracle.solve(f, w["y0"] if y0 is None else y0, np.full(B, T0), np.full(B, T1),
                      np.tile(te, (B, 1)), TIGHT)
    return float((rr["y_eval"] * gye).sum() + (rr["y_final"] * gyf).sum())


def test_joint_adjoint_dy0_vs_central_differences():
    w, te, r, gye, gyf = _setup()
    ja = oracle.joint_adjoint(w["field"], r["y_final"], T0, T1, te, gye, gyf,
                              dict(rtol=1e-10, atol=1e-10))
    assert ja["status"] == 0 and ja["n_acc"] > 0
    B, D = w["y0"].shape
    num = np.zeros((B, D))
    for i in range(B):
        for j in range(0, D, 3):
            eps = 1e-6
            yp, ym = w["y0"].copy(), w["y0"].copy()
            yp[i, j] += eps
            ym[i, j] -= eps
            num[i, j] = (_loss(w, te, gye, gyf, y0=yp) - _loss(w, te, gye, gyf, y0=ym)) / (2 * eps)
    m = np.zeros((B, D), bool)
    m[:, ::3] = True
    assert np.abs(ja["gy0"][m] - num[m]).max() <= 1e-6 * np.abs(num[m]).max()
    # the state integrated back from y(t1) returns to y0
    assert np.abs(ja["y0"] - w["y0"]).max() <= 1e-8


@pytest.mark.parametrize("layer", [0, 1, 2])
def test_joint_adjoint_weights_vs_central_differences(layer):
    w, te, r, gye, gyf = _setup(seed=layer + 1)
    ja = oracle.joint_adjoint(w["field"], r["y_final"], T0, T1, te, gye, gyf,
                              dict(rtol=1e-10, atol=1e-10))
    W, b = w["field"]["W"], w["field"]["b"]
    rng = np.random.default_rng(10 + layer)
    scale = max(np.abs(ja["gW"][layer]).max(), 1e-3)
    for _ in range(4):
        rr, cc = rng.integers(W[layer].shape[0]), rng.integers(W[layer].shape[1])
        eps = 1e-6
        Wp = [x.copy() for x in W]
        Wm = [x.copy() for x in W]
        Wp[layer][rr, cc] += eps
        Wm[layer][rr, cc] -= eps
        d = (_loss(w, te, gye, gyf, W=Wp) - _loss(w, te, gye, gyf, W=Wm)) / (2 * eps)
        assert abs(ja["gW"][layer][rr, cc] - d) <= 1e-6 * scale, (rr, cc)
    rb = rng.integers(b[layer].shape[0])
    bp = [x.copy() for x in b]
    bm = [x.copy() for x in b]
    bp[layer][rb] += 1e-6
    bm[layer][rb] -= 1e-6
    d = (_loss(w, te, gye, gyf, b=bp) - _loss(w, te, gye, gyf, b=bm)) / 2e-6
    assert abs(ja["gb"][layer][rb] - d) <= 1e-6 * max(np.abs(ja["gb"][layer]).max(), 1e-3)


def test_joint_adjoint_matches_the_discrete_adjoint_at_tight_tolerance():
    """Both the continuous and the discrete adjoint tend to the exact
    gradient: at tight tolerances they agree to ~1e-8."""
    w, te, r, gye, gyf = _setup(B=4, seed=7)
    mt, mh, mn = mesh_from_trace(r)
    B = w["y0"].shape[0]
    da = oracle.adjoint(w["field"], w["y0"], np.full(B, T0), np.full(B, T1), mt, mh, mn,
                        np.tile(te, (B, 1)), gye, gyf)
    ja = oracle.joint_adjoint(w["field"], r["y_final"], T0, T1, te, gye, gyf,
                              dict(rtol=1e-11, atol=1e-11))

    def rel(x, y):
        return np.linalg.norm(x - y) / np.linalg.norm(y)
    assert rel(ja["gy0"], da["gy0"]) <= 1e-7
    for l in range(3):
        assert rel(ja["gW"][l], da["gW"][l]) <= 1e-7
        assert rel(ja["gb"][l], da["gb"][l]) <= 1e-7


def test_joint_adjoint_jumps_and_segments():
    """Cotangents of points at t1 start the adjoint, points inside stop the
    integration and jump, points at t0 add at the end: moving a point's
    cotangent between two equal times changes nothing, and a loss on y(t0)
    alone gives dL/dy0 = its cotangent exactly."""
    w = workloads.make(4, B=2)
    B, D = w["y0"].shape
    rng = np.random.default_rng(3)
    te = np.array([0.0, 0.5, 1.0])
    r = oracle.solve(w["field"], w["y0"], np.full(B, T0), np.full(B, T1), np.tile(te, (B, 1)), TIGHT)
    g0 = np.zeros((B, 3, D))
    g0[:, 0] = rng.standard_normal((B, D))
    ja = oracle.joint_adjoint(w["field"], r["y_final"], T0, T1, te, g0, None)
    assert np.array_equal(ja["gy0"], g0[:, 0])
    assert all(np.abs(x).max() == 0.0 for x in ja["gW"])
    # a cotangent on the point at t1 equals the same cotangent on y_final
    g1 = np.zeros((B, 3, D))
    g1[:, 2] = rng.standard_normal((B, D))
    a = oracle.joint_adjoint(w["field"], r["y_final"], T0, T1, te, g1, None)
    b = oracle.joint_adjoint(w["field"], r["y_final"], T0, T1, te, None, g1[:, 2])
    assert np.array_equal(a["gy0"], b["gy0"])
    # an interior point splits the integration: more steps than without it
    gm = np.zeros((B, 3, D))
    gm[:, 1] = rng.standard_normal((B, D))
    m = oracle.joint_adjoint(w["field"], r["y_final"], T0, T1, te, gm, None)
    n = oracle.joint_adjoint(w["field"], r["y_final"], T0, T1, np.array([0.0, 1.0]), None,
                             None)
    assert m["n_acc"] >= n["n_acc"] and m["status"] == 0


def test_joint_adjoint_rejects_invalid_calls():
    w = workloads.make(4, B=2)
    y1 = w["y0"]
    with pytest.raises(ValueError):
        oracle.joint_adjoint(w["field"], y1, 1.0, 0.0)  # t1 <= t0
    with pytest.raises(ValueError):
        oracle.joint_adjoint(w["field"], y1, 0.0, 1.0, np.array([0.5, 0.2]))  # unordered
