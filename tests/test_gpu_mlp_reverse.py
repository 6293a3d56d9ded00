"""Backward integration (t1 < t0) of the MLP field on the tensor cores (the
same method with negative steps; the network sees the caller's time): the
GPU's backward solve equals its forward solve of the negated network in
s = -t bit for bit, a mixed-direction batch stays within the FP32 band of a
1e-12 FP64 oracle solution and is the same in both forms, and the discrete
adjoints of both networks (D = 32, H = 128 and the wide D = 64, three
layers of 512) match the oracle's on the GPU's mesh within the BF16-weight
tolerance (2e-3 relative l2)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2210_12375_b300 as tode
from gpu_helpers import gpu_solve, make, oracle_solve, subset
from oracle.oracle import mesh_from_trace

pytestmark = pytest.mark.gpu


def _reverse(w, which):
    """The instances in `which` run from their t1 back to their t0, their
    points in reverse order."""
    t0, t1, te = w["t0"].copy(), w["t1"].copy(), w["t_eval"].copy()
    t0[which], t1[which] = w["t1"][which], w["t0"][which]
    te[which] = w["t_eval"][which][:, ::-1]
    return dict(w, t0=t0, t1=t1, t_eval=np.ascontiguousarray(te))


def _negated(w):
    W = [x.copy() for x in w["field"]["W"]]
    b = [x.copy() for x in w["field"]["b"]]
    D = W[-1].shape[0]
    W[0][:, D] = -W[0][:, D]
    W[-1] = -W[-1]
    b[-1] = -b[-1]
    return dict(w, field=dict(w["field"], W=W, b=b))


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("cfg,B", [(4, 300), (5, 160)])
def test_mlp_backward_is_the_negated_network_forward_bitwise(cfg, B):
    w = dict(make(cfg, B=B), split=True)
    bw = _reverse(w, np.arange(B))
    g = gpu_solve(bw, torch.float32, "fused", trace_cap=64)
    nf = _negated(w)
    nf = dict(nf, t0=-bw["t0"], t1=-bw["t1"], t_eval=np.ascontiguousarray(-bw["t_eval"]))
    f = gpu_solve(nf, torch.float32, "fused", trace_cap=64)
    assert (g["status"] == 0).all()
    for k in ("y_eval", "y_final", "n_acc", "n_rej", "n_feval"):
        assert np.array_equal(g[k], f[k]), k
    L = g["trace_len"]
    for i in range(0, B, 17):
        assert np.array_equal(g["trace_h"][i, :L[i]], -f["trace_h"][i, :L[i]])


@pytest.mark.parametrize("cfg", [4, 5])
def test_mlp_mixed_directions_within_band_and_forms_agree(cfg):
    B = 256 if cfg == 4 else 128
    w = _reverse(dict(make(cfg, B=B), split=True), np.arange(0, B, 2))
    g = gpu_solve(w, torch.float32, "fused")
    p = gpu_solve(w, torch.float32, "plain")
    assert (g["status"] == 0).all()
    for k in ("y_eval", "y_final", "n_acc", "n_rej", "status"):
        assert np.array_equal(g[k], p[k]), k
    idx = np.arange(0, B, 5 if cfg == 4 else 9)
    ws = subset(w, idx)
    ref = oracle_solve(ws, rtol=1e-12, atol=1e-12)
    band = 10 * (w["atol"] + w["rtol"] * np.abs(ref["y_eval"]))
    assert (np.abs(g["y_eval"][idx] - ref["y_eval"]) <= band).all()


@pytest.mark.parametrize("cfg", [4, 5])
def test_mlp_backward_adjoint_vs_oracle(cfg):
    B = 256 if cfg == 4 else 96
    w = _reverse(dict(make(cfg, B=B), split=True), np.arange(1, B, 2))
    D = w["y0"].shape[1]
    probe = gpu_solve(w, torch.float32, "fused", trace_cap=128)
    tape = tode.TapeBuffers.allocate(B, D, torch.float32, int(probe["n_acc"].max()), 1, "cuda",
                                     stages=True)
    g = gpu_solve(w, torch.float32, "fused", tape=tape)
    rng = np.random.default_rng(8)
    gye = rng.standard_normal(g["y_eval"].shape)
    gyf = rng.standard_normal(g["y_final"].shape)
    dev = g["_dev"]
    gy0, (gW, gb), ovf = tode.adjoint(
        dev["field"], dev["t0"], dev["t1"], dev["te"], g["_sol"], tape,
        torch.tensor(gye, dtype=torch.float32, device="cuda"),
        torch.tensor(gyf, dtype=torch.float32, device="cuda"), rtol=w["rtol"], atol=w["atol"])
    torch.cuda.synchronize()
    assert int(ovf.item()) == 0
    mt, mh, mn = mesh_from_trace(probe)
    ref = oracle.adjoint(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"], gye, gyf)
    assert _rel(gy0.double().cpu().numpy(), ref["gy0"]) <= 2e-3
    for l in range(len(gW)):
        assert _rel(gW[l].double().cpu().numpy(), ref["gW"][l]) <= 2e-3, l
        assert _rel(gb[l].double().cpu().numpy(), ref["gb"][l]) <= 2e-3, l
