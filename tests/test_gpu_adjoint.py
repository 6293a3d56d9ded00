"""GPU discrete adjoint (App. A: backpropagation through the solver on the
frozen mesh) against the FP64 oracle adjoint on the GPU's own mesh, against
central finite differences, and checkpoint-stride invariance."""
import numpy as np
import pytest
import torch

import oracle
import paper_2210_12375_b300 as tode
from gpu_helpers import gpu_solve, make
from oracle.oracle import mesh_from_trace

pytestmark = pytest.mark.gpu


def _run(w, dtype, form, stride, slots=None, gy_seed=1, **kw):
    B, D = w["y0"].shape
    probe = gpu_solve(w, dtype, form, trace_cap=20000, **kw)
    N = int(probe["n_acc"].max())
    if slots is None:
        slots = max(1, -(-N // stride))
    tape = tode.TapeBuffers.allocate(B, D, dtype, slots, stride, "cuda")
    g = gpu_solve(w, dtype, form, tape=tape, **kw)
    rng = np.random.default_rng(gy_seed)
    gye = rng.standard_normal(g["y_eval"].shape)
    gyf = rng.standard_normal(g["y_final"].shape)
    dev = g["_dev"]
    gy0, gp, ovf = tode.adjoint(dev["field"], dev["t0"], dev["t1"], dev["te"], g["_sol"], tape,
                                torch.tensor(gye, dtype=dtype, device="cuda"),
                                torch.tensor(gyf, dtype=dtype, device="cuda"),
                                rtol=kw.get("rtol", w["rtol"]), atol=kw.get("atol", w["atol"]),
                                **{k: v for k, v in kw.items() if k not in ("rtol", "atol")})
    torch.cuda.synchronize()
    return dict(probe=probe, fwd=g, gy0=gy0.double().cpu().numpy(),
                gp=gp.double().cpu().numpy(), ovf=int(ovf.item()), gye=gye, gyf=gyf)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("cfg", [1, 2])
@pytest.mark.parametrize("form", ["plain", "fused"])
def test_adjoint_f64_vs_oracle_adjoint(cfg, form):
    w = make(cfg, B=64 if cfg == 2 else 256)
    r = _run(w, torch.float64, form, stride=1)
    assert r["ovf"] == 0
    mt, mh, mn = mesh_from_trace(r["probe"])
    ref = oracle.adjoint(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"],
                         r["gye"], r["gyf"])
    assert _rel(r["gy0"], ref["gy0"]) <= 1e-10
    key = "gmu" if cfg == 1 else "gA"
    assert _rel(r["gp"], ref[key]) <= 1e-10
    for i in range(0, w["B"], 7):
        assert _rel(r["gy0"][i], ref["gy0"][i]) <= 1e-10


@pytest.mark.parametrize("cfg", [1, 2])
def test_adjoint_recompute_stride_is_bitwise(cfg):
    """A small checkpoint budget (one slot every m accepted steps, segments
    recomputed) gives gradients bitwise equal to full storage."""
    w = make(cfg, B=200)
    dtype = torch.float64 if cfg == 1 else torch.float32
    a = _run(w, dtype, "fused", stride=1)
    for m in (3, 8):
        b = _run(w, dtype, "fused", stride=m)
        assert np.array_equal(a["gy0"], b["gy0"])
        assert np.array_equal(a["gp"], b["gp"])


def test_adjoint_overflow_is_reported():
    w = make(1, B=32)
    r = _run(w, torch.float64, "fused", stride=1, slots=3)
    assert r["ovf"] == 1
    assert np.isnan(r["gy0"]).all()


def test_adjoint_f64_vs_central_fd():
    w = make(1, B=4)
    r = _run(w, torch.float64, "fused", stride=1)
    mt, mh, mn = mesh_from_trace(r["probe"])

    def loss(y0):
        rr = oracle.replay(w["field"], y0, w["t0"], w["t1"], mt, mh, mn, w["t_eval"])
        return float((r["gye"] * rr["y_eval"]).sum() + (r["gyf"] * rr["y_final"]).sum())

    num = np.zeros_like(w["y0"])
    for i in range(4):
        for j in range(2):
            eps = 1e-6 * max(1.0, abs(w["y0"][i, j]))
            yp = w["y0"].copy()
            yp[i, j] += eps
            ym = w["y0"].copy()
            ym[i, j] -= eps
            num[i, j] = (loss(yp) - loss(ym)) / (2 * eps)
    assert _rel(r["gy0"], num) <= 1e-6


def test_adjoint_f32_linear_vs_oracle():
    w = make(2, B=512)
    r = _run(w, torch.float32, "fused", stride=1)
    mt, mh, mn = mesh_from_trace(r["probe"])
    ref = oracle.adjoint(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"],
                         r["gye"], r["gyf"])
    assert _rel(r["gy0"], ref["gy0"]) <= 1e-4
    assert _rel(r["gp"], ref["gA"]) <= 1e-4


@pytest.mark.parametrize("group", [4, 8, 16])
def test_adjoint_recompute_matches_forward_mesh_for_every_group(group):
    """The adjoint re-runs the forward's attempts from the checkpoints with
    the forward's lane grouping, so a recomputing budget (stride 5) and full
    storage (stride 1) give the same bits for every group size, and both
    agree with the oracle adjoint on the GPU's mesh."""
    w = make(2, B=300)
    a = _run(w, torch.float32, "fused", stride=1, group=group)
    b = _run(w, torch.float32, "fused", stride=5, group=group)
    assert np.array_equal(a["gy0"], b["gy0"]) and np.array_equal(a["gp"], b["gp"])
    mt, mh, mn = mesh_from_trace(a["probe"])
    ref = oracle.adjoint(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"],
                         a["gye"], a["gyf"])
    assert _rel(a["gy0"], ref["gy0"]) <= 1e-4


@pytest.mark.parametrize("cfg", [1, 2])
def test_adjoint_direct_from_tape_equals_rerun(cfg):
    """With one slot per accepted step the adjoint reverses straight from the
    tape (accepted step sizes recorded); without the recorded sizes it
    re-runs each step's attempts from its slot.  Same bits."""
    import dataclasses
    w = make(cfg, B=300)
    dtype = torch.float64 if cfg == 1 else torch.float32
    B, D = w["y0"].shape
    probe = gpu_solve(w, dtype, "fused")
    tape = tode.TapeBuffers.allocate(B, D, dtype, int(probe["n_acc"].max()), 1, "cuda")
    g = gpu_solve(w, dtype, "fused", tape=tape)
    dev = g["_dev"]
    rng = np.random.default_rng(3)
    gye = torch.tensor(rng.standard_normal(g["y_eval"].shape), dtype=dtype, device="cuda")
    gyf = torch.tensor(rng.standard_normal(g["y_final"].shape), dtype=dtype, device="cuda")
    outs = []
    for tp in (tape, dataclasses.replace(tape, h_acc=None)):
        gy0, gp, ovf = tode.adjoint(dev["field"], dev["t0"], dev["t1"], dev["te"], g["_sol"], tp,
                                    gye, gyf, rtol=w["rtol"], atol=w["atol"])
        torch.cuda.synchronize()
        assert int(ovf.item()) == 0
        outs.append((gy0.cpu().numpy(), gp.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("cfg", [1, 2])
def test_adjoint_recorded_stage_inputs_equal_recomputed(cfg):
    """A tape that also records each accepted step's stage inputs Y_2..Y_7
    lets the adjoint skip the stage re-evaluations; the reverse sweep gives
    the same bits as recomputing them."""
    w = make(cfg, B=300)
    dtype = torch.float64 if cfg == 1 else torch.float32
    B, D = w["y0"].shape
    probe = gpu_solve(w, dtype, "fused")
    N = int(probe["n_acc"].max())
    outs = []
    for stages in (False, True):
        tape = tode.TapeBuffers.allocate(B, D, dtype, N, 1, "cuda", stages=stages)
        g = gpu_solve(w, dtype, "fused", tape=tape)
        dev = g["_dev"]
        rng = np.random.default_rng(4)
        gye = torch.tensor(rng.standard_normal(g["y_eval"].shape), dtype=dtype, device="cuda")
        gyf = torch.tensor(rng.standard_normal(g["y_final"].shape), dtype=dtype, device="cuda")
        gy0, gp, ovf = tode.adjoint(dev["field"], dev["t0"], dev["t1"], dev["te"], g["_sol"], tape,
                                    gye, gyf, rtol=w["rtol"], atol=w["atol"])
        torch.cuda.synchronize()
        assert int(ovf.item()) == 0
        outs.append((gy0.cpu().numpy(), gp.cpu().numpy(), g["y_eval"]))
    assert np.array_equal(outs[0][2], outs[1][2])  # recording changes nothing in the solve
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("form", ["fused", "plain"])
@pytest.mark.parametrize("cfg,stages", [(2, True), (2, False), (3, False), (1, False)])
def test_minimal_tape_reverses_like_the_full_tape(cfg, stages, form):
    """A stride-1 tape that keeps only y, t, the accepted step sizes and k1
    (or the stage inputs) gives the adjoint the same bits as the full tape,
    and the forward's outputs are unchanged."""
    w = make(cfg, B=700 if cfg != 1 else 128)
    dtype = torch.float64 if cfg == 1 else torch.float32
    B, D = w["y0"].shape
    probe = gpu_solve(w, dtype, "fused")
    slots = max(1, int(probe["n_acc"].max()))
    res = []
    for minimal in (False, True):
        tape = tode.TapeBuffers.allocate(B, D, dtype, slots, 1, "cuda", stages=stages,
                                         minimal=minimal)
        if minimal:
            assert tape.y_lo is None and tape.h is None and tape.flags is None
            assert (tape.k1 is None) == stages
        g = gpu_solve(w, dtype, form, tape=tape)
        dev = g["_dev"]
        rng = np.random.default_rng(4)
        gye = torch.tensor(rng.standard_normal(g["y_eval"].shape), dtype=dtype, device="cuda")
        gyf = torch.tensor(rng.standard_normal((B, D)), dtype=dtype, device="cuda")
        gy0, gp, ovf = tode.adjoint(dev["field"], dev["t0"], dev["t1"], dev["te"], g["_sol"],
                                    tape, gye, gyf, rtol=w["rtol"], atol=w["atol"])
        torch.cuda.synchronize()
        res.append((g, gy0.cpu().numpy(), gp.cpu().numpy(), int(ovf.item())))
    (g0, a0, p0, o0), (g1, a1, p1, o1) = res
    assert o0 == o1 == 0
    for k in ("y_eval", "y_final", "n_acc", "n_rej", "status"):
        assert np.array_equal(g0[k], g1[k], equal_nan=True), k
    assert np.array_equal(a0, a1, equal_nan=True)
    assert np.array_equal(p0, p1, equal_nan=True)


def test_minimal_tape_needs_stride_one():
    with pytest.raises(ValueError):
        tode.TapeBuffers.allocate(8, 16, torch.float32, 4, 2, "cuda", minimal=True)
