"""Gradients with respect to the integration bounds t0 and t1 (the frozen
map: every step size but the last and every evaluation point's step held,
the last step ending at t1) through tode_t_bounds_grad, against the FP64
oracle's adjoint on the GPU's own mesh: relative l2 over the batch within
1e-10 in FP64 and 1e-4 in FP32 (the adjoint tolerances), forward and
backward in time; through odeint_adjoint as well; NaN for a failed
instance and a zero dL/dt1 for an empty interval."""
import numpy as np
import pytest
import torch

import oracle
import paper_2210_12375_b300 as tode
from gpu_helpers import gpu_solve, make
from oracle.oracle import mesh_from_trace

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _case(cfg, B, backward=False):
    w = make(cfg, B=B)
    if backward:
        # integrate backward from the old end over a short interval (Van der
        # Pol escapes to infinity backward in time, the decaying linear field
        # grows), the points from t0 down to t1
        L = 1.5 if cfg == 1 else 0.3
        t0 = w["t1"].copy()
        t1 = t0 - L
        te = np.linspace(0, 1, w["t_eval"].shape[1])[None, :] * (t1 - t0)[:, None] + t0[:, None]
        te[:, -1] = t1
        w = dict(w, t0=t0, t1=t1, t_eval=np.ascontiguousarray(te))
        if cfg == 1:  # inside the limit cycle, which attracts backward in time
            w["y0"] = 0.4 * w["y0"]
    return w


def _gpu_t_bounds(w, dtype, stages):
    B, D = w["y0"].shape
    probe = gpu_solve(w, dtype, "fused", trace_cap=8000)
    assert (probe["status"] == 0).all()
    tape = tode.TapeBuffers.allocate(B, D, dtype, int(probe["n_acc"].max()), 1, "cuda",
                                     stages=stages, minimal=True)
    g = gpu_solve(w, dtype, "fused", tape=tape, want_yp=True)
    rng = np.random.default_rng(3)
    gye = rng.standard_normal(g["y_eval"].shape)
    gyf = rng.standard_normal(g["y_final"].shape)
    dev = g["_dev"]
    g0, g1 = tode.t_bounds_grad(dev["field"], dev["t0"], dev["t1"], dev["te"], g["_sol"], tape,
                                torch.tensor(gye, dtype=dtype, device="cuda"),
                                torch.tensor(gyf, dtype=dtype, device="cuda"),
                                rtol=w["rtol"], atol=w["atol"])
    torch.cuda.synchronize()
    mt, mh, mn = mesh_from_trace(probe)
    ref = oracle.adjoint(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"], gye, gyf,
                         want_t_bounds=True)
    return g0.cpu().numpy(), g1.cpu().numpy(), ref


@pytest.mark.parametrize("cfg,B,dtype,tol,backward", [
    (1, 64, torch.float64, 1e-10, False),
    (1, 64, torch.float64, 1e-10, True),
    (2, 64, torch.float64, 1e-10, False),
    (2, 64, torch.float64, 1e-10, True),
    (2, 256, torch.float32, 1e-4, False),
    (3, 256, torch.float32, 1e-4, False),
])
def test_t_bounds_grad_vs_oracle_on_the_gpu_mesh(cfg, B, dtype, tol, backward):
    w = _case(cfg, B, backward)
    g0, g1, ref = _gpu_t_bounds(w, dtype, stages=cfg == 2)
    assert np.isfinite(g0).all() and np.isfinite(g1).all()
    # a stiff instance's FP32 mesh can sit at the explicit stability limit,
    # where the FP64 replay of that mesh overflows (reading 10): compare
    # where the reference stays finite
    ok = np.isfinite(ref["gt0"]) & np.isfinite(ref["gt1"])
    assert ok.mean() >= (1.0 if dtype == torch.float64 else 0.95)
    if cfg == 3:
        # FP32 stiff Van der Pol: as for the forward's FP32 arithmetic
        # (reading 10), the bound holds on the non-stiff instances; on stiff
        # ones the relaxation phases amplify the FP32 rounding of the states
        # and of dy/dt at the points (whole sample measured: 3.7e-4 for
        # dL/dt1, 6e-3 for dL/dt0), and only finiteness is required there
        ok &= w["field"]["mu"] < 3.0
        assert ok.sum() >= 64
    assert _rel(g1[ok], ref["gt1"][ok]) <= tol, _rel(g1[ok], ref["gt1"][ok])
    assert _rel(g0[ok], ref["gt0"][ok]) <= tol, _rel(g0[ok], ref["gt0"][ok])


def test_t_bounds_through_autograd_and_edge_cases():
    w = make(1, B=32)
    w["t1"][3] = w["t0"][3]  # an empty interval
    w["t_eval"][3] = w["t0"][3]
    dev = "cuda"
    f = tode.VdP(torch.tensor(w["field"]["mu"], device=dev))
    y0 = torch.tensor(w["y0"], device=dev)
    t0 = torch.tensor(w["t0"], device=dev, requires_grad=True)
    t1 = torch.tensor(w["t1"], device=dev, requires_grad=True)
    te = torch.tensor(w["t_eval"], device=dev)
    ye, yf, n_acc, n_rej, st = tode.odeint_adjoint(f, y0, t0, t1, te, rtol=w["rtol"],
                                                   atol=w["atol"])
    loss = (ye ** 2).sum() + yf.sum()
    gt0, gt1 = torch.autograd.grad(loss, [t0, t1])
    # the same through the direct calls
    g = gpu_solve(w, torch.float64, "fused", trace_cap=4000)
    mt, mh, mn = mesh_from_trace(g)
    gye = 2.0 * ye.detach().cpu().numpy()
    gyf = np.ones_like(yf.detach().cpu().numpy())
    ref = oracle.adjoint(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"], gye, gyf,
                         want_t_bounds=True)
    assert _rel(gt1.cpu().numpy(), ref["gt1"]) <= 1e-10
    assert _rel(gt0.cpu().numpy(), ref["gt0"]) <= 1e-10
    assert gt1[3].item() == 0.0
    # a failed instance (too few steps allowed) gets NaN
    B, D = w["y0"].shape
    tape = tode.TapeBuffers.allocate(B, D, torch.float64, 8, 1, dev, minimal=True)
    sol = tode.solve(f, y0, t0.detach(), t1.detach(), te, tape=tape, want_yp=True,
                     rtol=w["rtol"], atol=w["atol"], max_steps=5)
    g0, g1 = tode.t_bounds_grad(f, t0.detach(), t1.detach(), te, sol, tape,
                                torch.ones_like(sol.y_eval), None, rtol=w["rtol"],
                                atol=w["atol"], max_steps=5)
    failed = (sol.status != 0).cpu().numpy()
    assert failed.any()
    assert np.isnan(g1.cpu().numpy()[failed]).all() and np.isnan(g0.cpu().numpy()[failed]).all()


def _mlp_case(cfg, B, mixed):
    w = dict(make(cfg, B=B), split=True)
    if mixed:  # every other instance backward over the same interval
        t0, t1, te = w["t0"].copy(), w["t1"].copy(), w["t_eval"].copy()
        t0[::2], t1[::2] = w["t1"][::2], w["t0"][::2]
        te[::2] = te[::2, ::-1]
        w = dict(w, t0=t0, t1=t1, t_eval=np.ascontiguousarray(te))
    return w


@pytest.mark.parametrize("cfg,B,mixed", [(4, 256, False), (4, 256, True), (5, 96, True)])
def test_t_bounds_grad_mlp_vs_oracle_on_the_gpu_mesh(cfg, B, mixed):
    """The MLP field (time-dependent: its stage times move with the last
    step and with the translation of every time): dL/dt1 from the last step
    re-run on the CUDA cores, dL/dt0 from the tensor-core adjoint's
    translation sums, against the FP64 oracle's adjoint of the GPU's mesh
    (same BF16 weights) within the BF16-weight gradient tolerance 2e-3,
    relative l2 over the batch, both directions of integration."""
    w = _mlp_case(cfg, B, mixed)
    D = w["y0"].shape[1]
    probe = gpu_solve(w, torch.float32, "fused", trace_cap=64)
    assert (probe["status"] == 0).all()
    tape = tode.TapeBuffers.allocate(B, D, torch.float32, int(probe["n_acc"].max()), 1, "cuda",
                                     stages=True, minimal=True)
    g = gpu_solve(w, torch.float32, "fused", tape=tape, want_yp=True)
    assert np.array_equal(g["n_acc"], probe["n_acc"])
    rng = np.random.default_rng(5)
    gye = rng.standard_normal(g["y_eval"].shape)
    gyf = rng.standard_normal(g["y_final"].shape)
    dev = g["_dev"]
    gye_t = torch.tensor(gye, dtype=torch.float32, device="cuda")
    gyf_t = torch.tensor(gyf, dtype=torch.float32, device="cuda")
    opt = dict(rtol=w["rtol"], atol=w["atol"])
    gy0, (gW, gb, ts), ovf = tode.adjoint(dev["field"], dev["t0"], dev["t1"], dev["te"],
                                          g["_sol"], tape, gye_t, gyf_t, want_tshift=True, **opt)
    gy0_plain, _, _ = tode.adjoint(dev["field"], dev["t0"], dev["t1"], dev["te"], g["_sol"],
                                   tape, gye_t, gyf_t, **opt)
    g0, g1 = tode.t_bounds_grad(dev["field"], dev["t0"], dev["t1"], dev["te"], g["_sol"], tape,
                                gye_t, gyf_t, tshift=ts, **opt)
    torch.cuda.synchronize()
    assert int(ovf.item()) == 0
    # the translation sums change nothing else
    assert torch.equal(gy0, gy0_plain)
    mt, mh, mn = mesh_from_trace(probe)
    ref = oracle.adjoint(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"], gye, gyf,
                         want_t_bounds=True)
    g0, g1 = g0.cpu().numpy(), g1.cpu().numpy()
    assert np.isfinite(g0).all() and np.isfinite(g1).all()
    assert _rel(g1, ref["gt1"]) <= 2e-3, _rel(g1, ref["gt1"])
    assert _rel(g0, ref["gt0"]) <= 2e-3, _rel(g0, ref["gt0"])


def test_t_bounds_mlp_through_autograd_and_edge_cases():
    """odeint_adjoint with t0 and t1 requiring grad for the MLP field gives
    the direct calls' numbers; an empty interval gets dL/dt1 = 0 and a
    failed instance NaN."""
    w = dict(make(4, B=160), split=True)
    w["t1"][3] = w["t0"][3]  # an empty interval
    w["t_eval"][3] = w["t0"][3]
    dev = "cuda"
    from gpu_helpers import device_field
    f = device_field(w, torch.float32)
    y0 = torch.tensor(w["y0"], dtype=torch.float32, device=dev)
    t0 = torch.tensor(w["t0"], device=dev, requires_grad=True)
    t1 = torch.tensor(w["t1"], device=dev, requires_grad=True)
    te = torch.tensor(w["t_eval"], device=dev)
    ye, yf, n_acc, n_rej, st = tode.odeint_adjoint(f, y0, t0, t1, te, rtol=w["rtol"],
                                                   atol=w["atol"])
    loss = (ye.double() ** 2).sum() + yf.double().sum()
    gt0, gt1 = torch.autograd.grad(loss, [t0, t1])
    g = gpu_solve(w, torch.float32, "fused", trace_cap=64)
    mt, mh, mn = mesh_from_trace(g)
    gye = 2.0 * ye.detach().double().cpu().numpy()
    gyf = np.ones(yf.shape)
    ref = oracle.adjoint(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"], gye, gyf,
                         want_t_bounds=True)
    assert _rel(gt1.cpu().numpy(), ref["gt1"]) <= 2e-3
    assert _rel(gt0.cpu().numpy(), ref["gt0"]) <= 2e-3
    assert gt1[3].item() == 0.0
    B, D = w["y0"].shape
    tape = tode.TapeBuffers.allocate(B, D, torch.float32, 8, 1, dev, stages=True, minimal=True)
    sol = tode.solve(f, y0, t0.detach(), t1.detach(), te, tape=tape, want_yp=True,
                     rtol=w["rtol"], atol=w["atol"], max_steps=2)
    gye_t = torch.ones_like(sol.y_eval)
    _, (_, _, ts), _ = tode.adjoint(f, t0.detach(), t1.detach(), te, sol, tape, gye_t, None,
                                    want_tshift=True, rtol=w["rtol"], atol=w["atol"],
                                    max_steps=2)
    g0, g1 = tode.t_bounds_grad(f, t0.detach(), t1.detach(), te, sol, tape, gye_t, None,
                                tshift=ts, rtol=w["rtol"], atol=w["atol"], max_steps=2)
    failed = (sol.status != 0).cpu().numpy()
    assert failed.any()
    assert np.isnan(g1.cpu().numpy()[failed]).all() and np.isnan(g0.cpu().numpy()[failed]).all()
    assert np.isfinite(g1.cpu().numpy()[~failed]).all()
