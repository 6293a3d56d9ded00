"""Discrete adjoint of the MLP field on the tensor cores (App. A:
backpropagation through the solver on the frozen mesh) against the FP64
oracle adjoint run on the GPU's own mesh with the same BF16 weights.

Bar: relative l2 error <= 2e-3 for gy0 and for every weight and bias
gradient (summed over the batch).  The GPU recomputes the stages with the
forward's BF16 arithmetic (weights exact, inputs and activations as two BF16
terms, FP32 accumulation) and feeds the backward GEMMs split operands too, so
its error is dominated by the forward field's ~1e-5 relative error."""
import numpy as np
import pytest
import torch

import oracle
import paper_2210_12375_b300 as tode
from gpu_helpers import gpu_solve, make, subset
from oracle.oracle import mesh_from_trace

pytestmark = pytest.mark.gpu

TOL = 2e-3


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _run(w, slots=None, mask=None, seed=1, repeat=1):
    B, D = w["y0"].shape
    probe = gpu_solve(w, torch.float32, "fused", trace_cap=256)
    assert (probe["n_acc"] + probe["n_rej"] <= 256).all()
    N = int(probe["n_acc"].max())
    tape = tode.TapeBuffers.allocate(B, D, torch.float32, slots or max(N, 1), 1, "cuda",
                                     stages=True)
    g = gpu_solve(w, torch.float32, "fused", tape=tape)
    for k in ("y_eval", "n_acc", "status"):
        assert np.array_equal(g[k], probe[k], equal_nan=True), k  # the tape changes nothing
    rng = np.random.default_rng(seed)
    gye = rng.standard_normal(g["y_eval"].shape)
    gyf = rng.standard_normal(g["y_final"].shape)
    if mask is not None:
        gye[~mask] = 0.0
        gyf[~mask] = 0.0
    dev = g["_dev"]
    outs = []
    for _ in range(repeat):
        gy0, (gW, gb), ovf = tode.adjoint(
            dev["field"], dev["t0"], dev["t1"], dev["te"], g["_sol"], tape,
            torch.tensor(gye, dtype=torch.float32, device="cuda"),
            torch.tensor(gyf, dtype=torch.float32, device="cuda"), rtol=w["rtol"], atol=w["atol"])
        torch.cuda.synchronize()
        outs.append(dict(gy0=gy0.double().cpu().numpy(),
                         gW=[x.double().cpu().numpy() for x in gW],
                         gb=[x.double().cpu().numpy() for x in gb], ovf=int(ovf.item())))
    return dict(probe=probe, fwd=g, gye=gye, gyf=gyf, out=outs)


def _oracle_adj(w, probe, gye, gyf, idx=None):
    mt, mh, mn = mesh_from_trace(probe)
    if idx is not None:
        w = subset(w, idx)
        mt, mh, mn, gye, gyf = mt[idx], mh[idx], mn[idx], gye[idx], gyf[idx]
    return oracle.adjoint(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"], gye,
                          gyf)


def _check_params(o, ref):
    for l in range(3):
        assert _rel(o["gW"][l], ref["gW"][l]) <= TOL, ("W", l, _rel(o["gW"][l], ref["gW"][l]))
        assert _rel(o["gb"][l], ref["gb"][l]) <= TOL, ("b", l, _rel(o["gb"][l], ref["gb"][l]))


def test_mlp_adjoint_vs_oracle_adjoint():
    """Three 128-row tiles, the last ragged (44 rows)."""
    w = dict(make(4, B=300), split=True)
    r = _run(w)
    o = r["out"][0]
    assert o["ovf"] == 0
    ref = _oracle_adj(w, r["probe"], r["gye"], r["gyf"])
    assert _rel(o["gy0"], ref["gy0"]) <= TOL
    worst = max(_rel(o["gy0"][i], ref["gy0"][i]) for i in range(w["B"]))
    assert worst <= 5 * TOL, worst
    _check_params(o, ref)


def test_mlp_adjoint_rows_serving_several_instances():
    """More instances than one per row of a full grid (148 SMs x 128 rows):
    rows reverse a second instance after the first.  Cotangents are nonzero
    on a sample only, so the batch-summed weight gradients equal the
    oracle's over that sample, and every other instance's gy0 is exactly 0."""
    B = 148 * 128 + 256
    base = make(4)  # 16384 instances, repeated to B
    w = dict(subset(base, np.arange(B) % base["B"]), split=True)
    idx = np.unique(np.concatenate([np.arange(0, B, 151), np.arange(B - 256, B, 9), [B - 1]]))
    mask = np.zeros(B, bool)
    mask[idx] = True
    r = _run(w, mask=mask)
    o = r["out"][0]
    assert o["ovf"] == 0
    ref = _oracle_adj(w, r["probe"], r["gye"], r["gyf"], idx)
    assert _rel(o["gy0"][idx], ref["gy0"]) <= TOL
    assert (o["gy0"][~mask] == 0.0).all()
    _check_params(o, ref)


def test_mlp_adjoint_is_deterministic():
    """Static row assignment and an ordered sum over CTAs: repeated calls
    give the same bits."""
    w = dict(make(4, B=1000), split=True)
    r = _run(w, repeat=2)
    a, b = r["out"]
    assert np.array_equal(a["gy0"], b["gy0"])
    for l in range(3):
        assert np.array_equal(a["gW"][l], b["gW"][l]) and np.array_equal(a["gb"][l], b["gb"][l])


def test_mlp_adjoint_overflow_and_failed_instances():
    w = dict(make(4, B=260), split=True)
    t1, te = w["t1"].copy(), w["t_eval"].copy()
    short_iv = np.arange(20, 260, 3)  # shorter intervals: fewer steps
    t1[short_iv] = 0.4
    te[short_iv] = np.linspace(0.0, 0.4, te.shape[1])[None, :]
    t1[5] = -1.0  # invalid interval: NaN gradient, no contribution
    w = dict(w, t1=t1, t_eval=te)
    full = _run(w)
    n_acc = full["probe"]["n_acc"]
    slots = int(n_acc[short_iv].max())
    short = _run(w, slots=slots)
    o, f = short["out"][0], full["out"][0]
    assert o["ovf"] == 1 and f["ovf"] == 0
    over = n_acc > slots
    assert over.any() and (~over).any()
    assert np.isnan(o["gy0"][over]).all() and np.isnan(o["gy0"][5]).all()
    assert np.isnan(f["gy0"][5]).all()
    ok = ~over
    ok[5] = False
    # the instances that fit reverse exactly as with a full tape
    assert np.array_equal(o["gy0"][ok], f["gy0"][ok])
    # the parameter gradients cover exactly the instances that fit
    ref = _oracle_adj(w, full["probe"], full["gye"], full["gyf"], np.nonzero(ok)[0])
    _check_params(o, ref)


def test_mlp_adjoint_zero_length_interval():
    """t1 == t0: no steps; gy0 = gy_final + the cotangents of all t_eval
    points (which all sit at t0)."""
    w = dict(make(4, B=130), split=True)
    t1, te = w["t1"].copy(), w["t_eval"].copy()
    t1[[0, 129]] = w["t0"][[0, 129]]
    te[[0, 129]] = w["t0"][[0, 129], None]
    w = dict(w, t1=t1, t_eval=te)
    r = _run(w)
    o = r["out"][0]
    for i in (0, 129):
        exp = (r["gyf"][i] + r["gye"][i].sum(axis=0)).astype(np.float32).astype(np.float64)
        assert np.allclose(o["gy0"][i], exp, rtol=1e-6, atol=1e-6)
    ref = _oracle_adj(w, r["probe"], r["gye"], r["gyf"])
    assert _rel(o["gy0"], ref["gy0"]) <= TOL
    _check_params(o, ref)


def test_mlp_adjoint_needs_split_precision():
    w = dict(make(4, B=64), split=False)
    B, D = w["y0"].shape
    tape = tode.TapeBuffers.allocate(B, D, torch.float32, 64, 1, "cuda", stages=True)
    g = gpu_solve(w, torch.float32, "fused", tape=tape)
    dev = g["_dev"]
    with pytest.raises(tode._abi.TodeError):
        tode.adjoint(dev["field"], dev["t0"], dev["t1"], dev["te"], g["_sol"], tape,
                     None, torch.ones((B, D), device="cuda"), rtol=w["rtol"], atol=w["atol"])
