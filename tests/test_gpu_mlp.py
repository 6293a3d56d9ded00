"""The MLP field on the tensor cores (tcgen05, BF16 weights, FP32
accumulation; input [y; t] as two BF16 terms) against the FP64 oracle run
with the same BF16 weights.  Tolerance: 10 (atol + rtol |y|) of a
1e-12-tolerance oracle solution."""
import numpy as np
import pytest
import torch

from gpu_helpers import gpu_solve, make, oracle_solve, subset  # noqa: F401

pytestmark = pytest.mark.gpu


def _band_ratio(g, ref, w):
    band = 10 * (w["atol"] + w["rtol"] * np.abs(ref["y_eval"]))
    return np.abs(g["y_eval"] - ref["y_eval"]) / band


def test_mlp_split_matches_oracle_full_size_sampled():
    w = dict(make(4), split=True)
    g = gpu_solve(w, torch.float32, "fused")
    assert (g["status"] == 0).all()
    assert (g["n_feval"] == 2 + 6 * (g["n_acc"] + g["n_rej"])).all()
    idx = np.arange(0, w["B"], 61)
    ws = subset(w, idx)
    ref = oracle_solve(ws, rtol=1e-12, atol=1e-12)
    r = _band_ratio({"y_eval": g["y_eval"][idx]}, ref, w)
    assert np.isfinite(r).all() and r.max() <= 1.0, r.max()
    # matched steps: the same accepted-step counts as the FP64 oracle at the
    # workload tolerance on nearly every instance
    cfg = oracle_solve(ws)
    assert (g["n_acc"][idx] == cfg["n_acc"]).mean() > 0.95


def test_mlp_bf16_activations_error_is_reported():
    """Hidden activations rounded to BF16: f carries ~1e-3 relative noise;
    the solution stays within a few bands (reported, not the default)."""
    w = dict(make(4, B=2048), split=False)
    g = gpu_solve(w, torch.float32, "fused")
    assert (g["status"] == 0).all()
    ref = oracle_solve(subset(w, np.arange(256)), rtol=1e-12, atol=1e-12)
    r = _band_ratio({"y_eval": g["y_eval"][:256]}, ref, w)
    assert r.max() <= 3.0 and (r <= 1.0).mean() > 0.99


def test_mlp_batch_invariance_bitwise():
    w = dict(make(4, B=700), split=True)
    full = gpu_solve(w, torch.float32, "fused")
    perm = np.random.default_rng(9).permutation(w["B"])
    sh = gpu_solve(subset(w, perm), torch.float32, "fused")
    for k in ("y_eval", "y_final", "n_acc", "n_rej", "status"):
        assert np.array_equal(full[k][perm], sh[k]), k
    one = gpu_solve(subset(w, [123]), torch.float32, "fused")
    assert np.array_equal(one["y_eval"][0], full["y_eval"][123])


def test_mlp_edge_cases():
    w = dict(make(4, B=200), split=True)
    y0, t0, t1, te = w["y0"].copy(), w["t0"].copy(), w["t1"].copy(), w["t_eval"].copy()
    te[1, 3], te[1, 4] = te[1, 4], te[1, 3]
    t1[2] = -1.0
    t1[3] = t0[3]
    te[3] = t0[3]
    y0[4, 7] = np.nan
    w2 = dict(w, y0=y0, t1=t1, t_eval=te)
    g = gpu_solve(w2, torch.float32, "fused")
    o = oracle_solve(w2)
    assert list(g["status"][[1, 2]]) == [4, 4]
    assert g["status"][3] == 0 and g["n_acc"][3] == 0
    assert np.array_equal(g["y_eval"][3], np.repeat(y0[3:4].astype(np.float32), 8, 0))
    assert g["status"][4] == 3 and o["status"][4] == 3
    assert np.array_equal(np.isnan(g["y_eval"][4]), np.isnan(o["y_eval"][4]))
    assert (g["status"][5:] == 0).all()
    # the healthy rows of the same tiles are unaffected
    ref = gpu_solve(subset(w, np.arange(5, 200)), torch.float32, "fused")
    assert np.array_equal(ref["y_eval"], g["y_eval"][5:])


@pytest.mark.parametrize("form", ["plain", "fused"])
def test_mlp_max_steps_leaves_unreached_points_nan(form):
    w = dict(make(4, B=300), split=True)
    g = gpu_solve(w, torch.float32, form, max_steps=2)
    assert (g["status"] == 1).all() and ((g["n_acc"] + g["n_rej"]) == 2).all()
    nan = np.isnan(g["y_eval"])
    rows = nan.any(axis=2)
    assert np.array_equal(nan.all(axis=2), rows)           # whole points
    assert (np.diff(rows.astype(int), axis=1) >= 0).all()  # from some point to the end
    assert rows[:, -1].all() and not rows[:, 0].any()


def test_mlp_unsupported_requests_fail_loudly():
    """The MLP adjoint reverses recorded stage inputs: a checkpoint tape
    (stride 2) is accepted by the solve, which records checkpoints there,
    but refused by the adjoint (it is the re-solve's input), and a stride-2
    tape without the solver state is refused by the solve."""
    import paper_2210_12375_b300 as tode
    w = dict(make(4, B=64), split=True)
    tape = tode.TapeBuffers.allocate(64, 32, torch.float32, 8, 2, "cuda")
    g = gpu_solve(w, torch.float32, "fused", tape=tape)
    dev = g["_dev"]
    with pytest.raises(tode._abi.TodeError):
        tode.adjoint(dev["field"], dev["t0"], dev["t1"], dev["te"], g["_sol"], tape,
                     torch.ones_like(g["_sol"].y_eval), None, rtol=w["rtol"], atol=w["atol"])
    bare = tode.TapeBuffers.allocate(64, 32, torch.float32, 8, 1, "cuda", stages=True,
                                     minimal=True)
    bare.stride = 2
    with pytest.raises(tode._abi.TodeError):
        gpu_solve(w, torch.float32, "fused", tape=bare)


@pytest.mark.parametrize("B", [300, 148 * 128 + 256])
def test_mlp_plain_form_equals_fused_bitwise(B):
    """Plain form (one launch per attempt over the masked batch, state parked
    in the workspace; several tiles per CTA at the larger size) and fused
    form give the same bits, including the checkpoint tape and the trace."""
    import paper_2210_12375_b300 as tode
    base = make(4)
    w = dict(subset(base, np.arange(B) % base["B"]), split=True)
    out = {}
    for form in ("fused", "plain"):
        tape = tode.TapeBuffers.allocate(B, 32, torch.float32, 16, 1, "cuda", stages=True)
        for t in (tape.y, tape.k1, tape.t, tape.h_acc, tape.y_stage):
            t.zero_()  # slots past an instance's last step stay zero
        g = gpu_solve(w, torch.float32, form, tape=tape, trace_cap=32)
        out[form] = (g, tape)
    (gf, tf), (gp, tp) = out["fused"], out["plain"]
    assert (gf["status"] == 0).all()
    for k in ("y_eval", "y_final", "n_acc", "n_rej", "n_feval", "status", "trace_t", "trace_h",
              "trace_err", "trace_accepted", "trace_len"):
        assert np.array_equal(gf[k], gp[k]), k
    N = int(gf["n_acc"].max())
    for name in ("y", "k1", "t", "h_acc", "y_stage"):
        assert torch.equal(getattr(tf, name)[:, :N], getattr(tp, name)[:, :N]), name
