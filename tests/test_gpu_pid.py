"""The PID controller (App. C: the step-size decision uses the last three
error estimates, factor safety*err^-b1*err_prev^b2*err_prev2^-b3) on the
GPU against the oracle: FP64 meshes bit-identical, FP32 and MLP forms
bit-identical to each other and within the FP32 band of the oracle, the
joint solve with the oracle's stacked solve, and a re-run (strided) adjoint
tape that carries the controller's second error entry."""
import numpy as np
import pytest
import torch

import paper_2210_12375_b300 as tode
from gpu_helpers import gpu_solve, make, oracle_solve

pytestmark = pytest.mark.gpu

PID = dict(beta1=(0.3 + 0.3 + 0.1) / 5, beta2=(0.3 + 2 * 0.1) / 5, beta3=0.1 / 5)


def _rel_close(a, b, tol):
    scale = np.maximum(np.abs(b).max(axis=-1, keepdims=True), 1.0)
    return np.abs(a - b) <= tol * scale


@pytest.mark.parametrize("form", ["plain", "fused"])
def test_pid_f64_mesh_is_the_oracles(form):
    w = make(1, B=96)
    g = gpu_solve(w, torch.float64, form, trace_cap=4000, **PID)
    o = oracle_solve(w, trace_cap=4000, **PID)
    assert np.array_equal(g["status"], o["status"]) and (g["status"] == 0).all()
    assert np.array_equal(g["n_acc"], o["n_acc"]) and np.array_equal(g["n_rej"], o["n_rej"])
    for k in ("trace_t", "trace_h", "trace_err"):
        assert np.array_equal(g[k], o[k]), k
    assert _rel_close(g["y_eval"], o["y_eval"], 1e-12).all()
    # the derivative term changes the mesh: not the PI controller's
    pi = oracle_solve(w, beta1=PID["beta1"], beta2=PID["beta2"])
    assert not np.array_equal(pi["n_acc"], o["n_acc"])


def test_pid_f32_linear_forms_agree_and_match_oracle():
    w = make(2, B=512)
    f = gpu_solve(w, torch.float32, "fused", **PID)
    p = gpu_solve(w, torch.float32, "plain", **PID)
    for k in ("y_eval", "y_final", "n_acc", "n_rej", "status"):
        assert np.array_equal(f[k], p[k]), k
    ref = oracle_solve(w, rtol=1e-12, atol=1e-12)
    band = 10 * (w["atol"] + w["rtol"] * np.abs(ref["y_eval"]))
    assert (np.abs(f["y_eval"] - ref["y_eval"]) <= band).all()
    # matched steps: FP32 state and FP64 oracle take the same accepted-step
    # counts on nearly every instance (the controller's history lets an
    # early rounding difference change a later decision, so not on all)
    o = oracle_solve(w, **PID)
    d = np.abs(f["n_acc"].astype(int) - o["n_acc"])
    assert (d == 0).mean() > 0.9 and d.max() <= 5, np.bincount(d)


def test_pid_mlp_forms_agree_and_match_oracle():
    w = dict(make(4, B=600), split=True)
    f = gpu_solve(w, torch.float32, "fused", **PID)
    p = gpu_solve(w, torch.float32, "plain", **PID)
    for k in ("y_eval", "y_final", "n_acc", "n_rej", "status"):
        assert np.array_equal(f[k], p[k]), k
    idx = np.arange(0, 600, 7)
    from gpu_helpers import subset
    ref = oracle_solve(subset(w, idx), rtol=1e-12, atol=1e-12)
    band = 10 * (w["atol"] + w["rtol"] * np.abs(ref["y_eval"]))
    assert (np.abs(f["y_eval"][idx] - ref["y_eval"]) <= band).all()


def test_pid_joint_matches_oracle():
    import oracle
    w = make(1, B=48)
    T = 8.0
    te = np.linspace(0.0, T, 6)
    w = dict(w, t0=np.zeros(48), t1=np.full(48, T), t_eval=np.tile(te, (48, 1)))
    g = gpu_solve(w, torch.float64, "plain", joint=True, **PID)
    o = oracle.solve_joint(w["field"], w["y0"], 0.0, T, te,
                           dict(rtol=w["rtol"], atol=w["atol"], **PID))
    assert (g["n_acc"] == o["n_acc"]).all() and (g["n_rej"] == o["n_rej"]).all()
    assert _rel_close(g["y_eval"], o["y_eval"], 1e-10).all()


@pytest.mark.parametrize("cfg", [1, 2])
def test_pid_strided_tape_rerun_is_bitwise(cfg):
    """The adjoint re-runs each tape segment with the controller state of
    its slot, the derivative term's err_prev2 included: gradients with a
    small checkpoint budget equal those of full storage bit for bit."""
    w = make(cfg, B=150)
    dtype = torch.float64 if cfg == 1 else torch.float32
    B, D = w["y0"].shape
    probe = gpu_solve(w, dtype, "fused", **PID)
    N = int(probe["n_acc"].max())
    rng = np.random.default_rng(5)
    gye = torch.tensor(rng.standard_normal(probe["y_eval"].shape), dtype=dtype, device="cuda")
    gyf = torch.tensor(rng.standard_normal(probe["y_final"].shape), dtype=dtype, device="cuda")
    out = []
    for stride in (1, 5):
        tape = tode.TapeBuffers.allocate(B, D, dtype, -(-N // stride), stride, "cuda")
        g = gpu_solve(w, dtype, "fused", tape=tape, **PID)
        dev = g["_dev"]
        gy0, gp, ovf = tode.adjoint(dev["field"], dev["t0"], dev["t1"], dev["te"], g["_sol"],
                                    tape, gye, gyf, rtol=w["rtol"], atol=w["atol"], **PID)
        assert int(ovf.item()) == 0
        out.append((gy0.cpu().numpy(), gp.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    # without the second error entry a re-run tape cannot reproduce the mesh
    tape = tode.TapeBuffers.allocate(B, D, dtype, -(-N // 5), 5, "cuda")
    tape.err_prev2 = None
    with pytest.raises(tode._abi.TodeError):
        gpu_solve(w, dtype, "fused", tape=tape, **PID)


def test_pid_vs_integral_on_the_gpu_over_one_vdp_cycle():
    """App. C's comparison, on the GPU path (FP64, the oracle's meshes):
    PID costs attempts at mu = 5 and saves them at mu = 50."""
    import math
    counts = {}
    for mu in (5.0, 50.0):
        T = (3 - 2 * math.log(2)) * mu + 2 * math.pi / (1 + mu) + 4.676 * mu ** (-1 / 3)
        w = dict(field=dict(kind="vdp", mu=np.array([mu])), y0=np.array([[2.0, 0.0]]),
                 t0=np.zeros(1), t1=np.array([T]), t_eval=np.zeros((1, 0)), rtol=1e-6,
                 atol=1e-6, B=1)
        for name, kw in (("I", dict(beta1=0.2)), ("PID", PID)):
            g = gpu_solve(w, torch.float64, "fused", **kw)
            o = oracle_solve(w, **kw)
            assert np.array_equal(g["n_acc"], o["n_acc"]) and np.array_equal(g["n_rej"], o["n_rej"])
            counts[mu, name] = int(g["n_acc"][0] + g["n_rej"][0])
    assert counts[5.0, "PID"] > counts[5.0, "I"]
    assert counts[50.0, "PID"] < 0.97 * counts[50.0, "I"]
