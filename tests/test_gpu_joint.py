"""Joint ("stacked") solving on the GPU (Sec. 4.1: the batch as one problem
of size B*D with one step size, one error norm and one accept decision)
against the oracle's stacked solve, and its batching interaction against
the independent solver.

Tolerances: the GPU sums the squared scaled errors per instance and then
over CTAs, the oracle left to right over all B*D components, so the error
norms differ in the last bits.  FP64: identical accept/reject sequences,
mesh times and step sizes within 1e-11 relative (the last, clipped step
within 1e-12 t1 absolute), outputs within 1e-10 of max(|y|, 1).  FP32 state: accepted-step counts within one of the FP64
oracle and outputs within 10 (atol + rtol |y|) of it."""
import numpy as np
import pytest
import torch

import oracle
import paper_2210_12375_b300 as tode
from gpu_helpers import gpu_solve, make
from oracle.oracle import mesh_from_trace

pytestmark = pytest.mark.gpu


def _joint(cfg, B, T, K):
    """Workload cfg's fields and initial states on one shared time axis."""
    w = make(cfg, B=B)
    te = np.linspace(0.0, T, K)
    return dict(w, t0=np.zeros(B), t1=np.full(B, T), t_eval=np.tile(te, (B, 1)))


def _oracle_joint(w, trace_cap=0, **kw):
    o = dict(rtol=w["rtol"], atol=w["atol"])
    o.update(kw)
    return oracle.solve_joint(w["field"], w["y0"], float(w["t0"][0]), float(w["t1"][0]),
                              w["t_eval"][0], o, trace_cap=trace_cap)


def _rel_close(a, b, tol):
    scale = np.maximum(np.abs(b).max(axis=-1, keepdims=True), 1.0)
    return np.abs(a - b) <= tol * scale


def test_joint_f64_vdp_matches_oracle():
    w = _joint(1, 64, 10.0, 16)
    g = gpu_solve(w, torch.float64, "plain", trace_cap=4000, joint=True)
    o = _oracle_joint(w, trace_cap=4000)
    assert o["status"] == 0 and (g["status"] == 0).all()
    assert (g["n_acc"] == o["n_acc"]).all() and (g["n_rej"] == o["n_rej"]).all()
    assert (g["n_feval"] == o["n_feval"]).all()
    L = o["trace_len"]
    assert (g["trace_len"] == L).all()
    for i in (0, 17, 63):  # every instance carries the problem's trace
        assert np.array_equal(g["trace_accepted"][i, :L], o["trace_accepted"])
        np.testing.assert_allclose(g["trace_t"][i, :L], o["trace_t"], rtol=1e-11, atol=0)
        # the last step is t1 - t: t's rounding difference, absolute
        np.testing.assert_allclose(g["trace_h"][i, :L], o["trace_h"], rtol=1e-11, atol=1e-12 * 10)
    assert _rel_close(g["y_eval"], o["y_eval"], 1e-10).all()
    assert _rel_close(g["y_final"], o["y_final"], 1e-10).all()


@pytest.mark.parametrize("launch", [dict(block=32), dict(block=256),
                                    dict(block=32, ctas_per_sm=1, group=16)])
def test_joint_f32_linear_matches_oracle(launch):
    # the last launch shape: 16-lane groups, 148 one-warp CTAs, so some
    # threads take a second instance in the grid-stride loop
    w = _joint(2, 300, 1.5, 32)
    g = gpu_solve(w, torch.float32, "plain", joint=True, **launch)
    o = _oracle_joint(w)
    assert (g["status"] == 0).all() and o["status"] == 0
    assert (g["n_acc"] == g["n_acc"][0]).all()
    assert abs(int(g["n_acc"][0]) - o["n_acc"]) <= 1
    band = 10 * (w["atol"] + w["rtol"] * np.abs(o["y_eval"]))
    assert (np.abs(g["y_eval"] - o["y_eval"]) <= band).all()


@pytest.mark.parametrize("B", [1, 33, 1000, 20000])
@pytest.mark.parametrize("launch", [dict(block=64), dict(block=32, ctas_per_sm=1)])
def test_joint_ragged_and_multi_cta_batches(B, launch):
    # the second launch shape runs 148 CTAs of one warp: each thread takes
    # several instances in turn on the larger batches
    w = _joint(1, B, 6.0, 5)
    g = gpu_solve(w, torch.float64, "plain", joint=True, **launch)
    o = _oracle_joint(w)
    assert (g["status"] == o["status"]).all()
    assert (g["n_acc"] == o["n_acc"]).all() and (g["n_rej"] == o["n_rej"]).all()
    assert _rel_close(g["y_eval"], o["y_eval"], 1e-10).all()


def test_joint_reproduces_the_batching_interaction():
    """Sec. 4.1: stacked strongly damped oscillators take several times the
    steps of the same oscillators solved independently."""
    B, mu = 16, 10.0
    rng = np.random.default_rng(4)
    y0 = rng.uniform(-2.0, 2.0, (B, 2))
    T = 40.0
    te = np.linspace(0.0, T, 9)
    w = dict(field=dict(kind="vdp", mu=np.full(B, mu)), y0=y0, t0=np.zeros(B),
             t1=np.full(B, T), t_eval=np.tile(te, (B, 1)), rtol=1e-6, atol=1e-6, B=B)
    ind = gpu_solve(w, torch.float64, "fused")
    j = gpu_solve(w, torch.float64, "plain", joint=True)
    o = _oracle_joint(w)
    assert (j["n_acc"] == o["n_acc"]).all()
    assert j["n_acc"][0] >= ind["n_acc"].max()
    assert j["n_acc"][0] / ind["n_acc"].mean() > 2.5


def test_joint_of_identical_copies_steps_like_one_instance():
    w1 = _joint(1, 1, 12.0, 7)
    n = 24
    wn = dict(w1, field=dict(kind="vdp", mu=np.repeat(w1["field"]["mu"], n)),
              y0=np.repeat(w1["y0"], n, 0), t0=np.zeros(n), t1=np.full(n, 12.0),
              t_eval=np.repeat(w1["t_eval"], n, 0), B=n)
    one = gpu_solve(w1, torch.float64, "fused")
    j = gpu_solve(wn, torch.float64, "plain", joint=True)
    assert (j["n_acc"] == one["n_acc"][0]).all() and (j["n_rej"] == one["n_rej"][0]).all()
    assert _rel_close(j["y_eval"], np.repeat(one["y_eval"], n, 0), 1e-10).all()


def test_joint_edge_cases():
    w = _joint(1, 40, 5.0, 6)
    # an instance on another time axis: the batch is not one problem
    bad = dict(w, t1=w["t1"].copy())
    bad["t1"][7] = 5.5
    g = gpu_solve(bad, torch.float64, "plain", joint=True)
    assert (g["status"] == 4).all() and (g["n_acc"] == 0).all() and (g["n_feval"] == 0).all()
    assert np.isnan(g["y_eval"]).all() and np.isnan(g["y_final"]).all()
    bad = dict(w, t_eval=w["t_eval"].copy())
    bad["t_eval"][3, 2] += 1e-3
    assert (gpu_solve(bad, torch.float64, "plain", joint=True)["status"] == 4).all()
    # an empty range
    e = dict(w, t1=np.zeros(40), t_eval=np.zeros((40, 3)))
    g = gpu_solve(e, torch.float64, "plain", joint=True)
    assert (g["status"] == 0).all() and (g["n_acc"] == 0).all() and (g["n_feval"] == 0).all()
    assert np.array_equal(g["y_eval"], np.repeat(w["y0"][:, None, :], 3, 1))
    # the attempt limit: the unreached points are NaN as in the oracle
    g = gpu_solve(w, torch.float64, "plain", joint=True, max_steps=5)
    o = _oracle_joint(w, max_steps=5)
    assert (g["status"] == 1).all() and o["status"] == 1
    assert ((g["n_acc"] + g["n_rej"]) == 5).all()
    assert np.array_equal(np.isnan(g["y_eval"]), np.isnan(o["y_eval"]))
    # a given first step
    g = gpu_solve(w, torch.float64, "plain", joint=True, h0=1e-3)
    o = _oracle_joint(w, h0=1e-3)
    assert (g["n_acc"] == o["n_acc"]).all() and (g["n_feval"] == o["n_feval"]).all()
    assert _rel_close(g["y_eval"], o["y_eval"], 1e-10).all()


def test_joint_refuses_what_it_cannot_mean():
    w = _joint(1, 8, 2.0, 3)
    # per-instance tolerances: one problem has one norm
    with pytest.raises(tode._abi.TodeError):
        gpu_solve(w, torch.float64, "plain", joint=True,
                  rtol_b=torch.full((8,), 1e-6, dtype=torch.float64, device="cuda"))
    tape = tode.TapeBuffers.allocate(8, 2, torch.float64, 50, 4, "cuda")
    with pytest.raises(tode._abi.TodeError):  # a strided tape would re-run per instance
        gpu_solve(w, torch.float64, "plain", joint=True, tape=tape)
    m = dict(make(4, B=8), split=True)
    with pytest.raises(tode._abi.TodeError):
        gpu_solve(m, torch.float32, "fused", joint=True)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_joint_adjoint_on_the_shared_mesh(dtype):
    """The gradient of a joint solve is each instance's discrete adjoint on
    the shared frozen mesh (the controller is not differentiated)."""
    w = _joint(1, 32, 6.0, 8)
    probe = gpu_solve(w, dtype, "plain", joint=True, trace_cap=4000)
    N = int(probe["n_acc"].max())
    tape = tode.TapeBuffers.allocate(32, 2, dtype, N, 1, "cuda")
    g = gpu_solve(w, dtype, "plain", joint=True, tape=tape)
    assert np.array_equal(g["y_eval"], probe["y_eval"])
    rng = np.random.default_rng(3)
    gye = rng.standard_normal(g["y_eval"].shape)
    gyf = rng.standard_normal(g["y_final"].shape)
    dev = g["_dev"]
    gy0, gmu, ovf = tode.adjoint(dev["field"], dev["t0"], dev["t1"], dev["te"], g["_sol"], tape,
                                 torch.tensor(gye, dtype=dtype, device="cuda"),
                                 torch.tensor(gyf, dtype=dtype, device="cuda"),
                                 rtol=w["rtol"], atol=w["atol"])
    assert int(ovf.item()) == 0
    mt, mh, mn = mesh_from_trace(probe)
    ref = oracle.adjoint(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"],
                         gye, gyf)
    tol = 1e-10 if dtype == torch.float64 else 1e-4
    for a, b in ((gy0, ref["gy0"]), (gmu, ref["gmu"])):
        a = a.double().cpu().numpy()
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b)
