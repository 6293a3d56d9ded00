"""Discrete adjoint of the wide MLP field (D = 64, three tanh layers of 512;
App. A) against the FP64 oracle adjoint on the GPU's own mesh with the same
BF16 weights: gy0 and every weight and bias gradient within 2e-3 relative
l2.  The weight gradients come from the staged rows of every reverse round
through the library's own tensor-core products over the split operands
(hi*hi + lo*hi + hi*lo)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2210_12375_b300 as tode
from gpu_helpers import gpu_solve, make, oracle_solve, subset
from oracle.oracle import mesh_from_trace

pytestmark = pytest.mark.gpu

TOL = 2e-3


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _run(w, mask=None, seed=1, repeat=1):
    B, D = w["y0"].shape
    probe = gpu_solve(w, torch.float32, "fused", trace_cap=128)
    assert (probe["n_acc"] + probe["n_rej"] <= 128).all()
    tape = tode.TapeBuffers.allocate(B, D, torch.float32, int(probe["n_acc"].max()), 1, "cuda",
                                     stages=True)
    g = gpu_solve(w, torch.float32, "fused", tape=tape)
    assert np.array_equal(g["y_eval"], probe["y_eval"], equal_nan=True)
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
        outs.append(dict(gy0=gy0.double().cpu().numpy(), gW=[x.double().cpu().numpy() for x in gW],
                         gb=[x.double().cpu().numpy() for x in gb], ovf=int(ovf.item())))
    return dict(probe=probe, gye=gye, gyf=gyf, out=outs)


def _oracle_adj(w, probe, gye, gyf, idx=None):
    mt, mh, mn = mesh_from_trace(probe)
    if idx is not None:
        w = subset(w, idx)
        mt, mh, mn, gye, gyf = mt[idx], mh[idx], mn[idx], gye[idx], gyf[idx]
    return oracle.adjoint(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"], gye,
                          gyf)


def _check(o, ref, idx=None):
    gy0 = o["gy0"] if idx is None else o["gy0"][idx]
    assert _rel(gy0, ref["gy0"]) <= TOL, _rel(gy0, ref["gy0"])
    for l in range(4):
        assert _rel(o["gW"][l], ref["gW"][l]) <= TOL, ("W", l, _rel(o["gW"][l], ref["gW"][l]))
        assert _rel(o["gb"][l], ref["gb"][l]) <= TOL, ("b", l, _rel(o["gb"][l], ref["gb"][l]))


def test_wide_mlp_adjoint_vs_oracle_adjoint():
    """Four 64-row tiles, the last ragged (8 rows); one slice."""
    w = dict(make(5, B=200), split=True)
    r = _run(w)
    o = r["out"][0]
    assert o["ovf"] == 0
    _check(o, _oracle_adj(w, r["probe"], r["gye"], r["gyf"]))


def test_wide_mlp_adjoint_several_slices_and_deterministic():
    """More instances than one per row of a full grid (148 x 64): the staged
    adjoint runs in two slices whose GEMMs accumulate; cotangents only on a
    sample, so the summed gradients equal the oracle's over that sample.
    Two calls give the same bits."""
    B = 148 * 64 + 200
    base = make(5, B=4096)
    w = dict(subset(base, np.arange(B) % base["B"]), split=True)
    idx = np.unique(np.concatenate([np.arange(0, B, 331), np.arange(B - 200, B, 17), [B - 1]]))
    mask = np.zeros(B, bool)
    mask[idx] = True
    r = _run(w, mask=mask, repeat=2)
    a, b = r["out"]
    assert a["ovf"] == 0
    assert (a["gy0"][~mask] == 0.0).all()
    _check(a, _oracle_adj(w, r["probe"], r["gye"], r["gyf"], idx), idx)
    assert np.array_equal(a["gy0"], b["gy0"])
    for l in range(4):
        assert np.array_equal(a["gW"][l], b["gW"][l]) and np.array_equal(a["gb"][l], b["gb"][l])


def test_wide_mlp_adjoint_odd_tile_count():
    """Three 64-row tiles (the last ragged): the reverse chain runs on CTA
    pairs, so the second pair's CTA 1 holds no instance and runs the pair's
    rounds on zeros; its staged rows add nothing to the weight gradients."""
    w = dict(make(5, B=130), split=True)
    r = _run(w, seed=3)
    o = r["out"][0]
    assert o["ovf"] == 0
    _check(o, _oracle_adj(w, r["probe"], r["gye"], r["gyf"]))


def test_wide_mlp_full_size_sampled():
    """The bench's workload at full size (65,536 instances: 1024 tiles, the
    reverse chain on 74 CTA pairs in several slices): the forward on a
    stratified sample within the FP32 band of a 1e-12 oracle solution, and
    the adjoint with cotangents only on that sample, whose summed gradients
    equal the oracle's over it."""
    w = dict(make(5), split=True)
    B = w["B"]
    assert B == 65536
    idx = np.unique(np.concatenate([np.arange(0, B, 2731), np.arange(B - 64, B, 21), [B - 1]]))
    mask = np.zeros(B, bool)
    mask[idx] = True
    r = _run(w, mask=mask, seed=5)
    o = r["out"][0]
    assert o["ovf"] == 0
    assert (r["probe"]["status"] == 0).all()
    ws = subset(w, idx)
    ref = oracle_solve(ws, rtol=1e-12, atol=1e-12)
    band = 10 * (w["atol"] + w["rtol"] * np.abs(ref["y_eval"]))
    ratio = np.abs(r["probe"]["y_eval"][idx] - ref["y_eval"]) / band
    assert np.isfinite(ratio).all() and ratio.max() <= 1.0, ratio.max()
    assert (o["gy0"][~mask] == 0.0).all()
    _check(o, _oracle_adj(w, r["probe"], r["gye"], r["gyf"], idx), idx)
