"""odeint_adjoint: the torch.autograd.Function around the fused solve and
the discrete adjoint (App. A).  Gradients of L = sum y(t_eval)^2 + <d, y(t1)>
against the FP64 oracle adjoint on the GPU's mesh, the checkpoint budget
(recomputed segments give the same bits), and the MLP's weight gradients."""
import numpy as np
import pytest
import torch

import oracle
import paper_2210_12375_b300 as tode
from gpu_helpers import device_field, gpu_solve, make
from oracle.oracle import mesh_from_trace

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _inputs(w, dtype):
    dev = "cuda"
    y0 = torch.tensor(w["y0"], dtype=dtype, device=dev, requires_grad=True)
    t0 = torch.tensor(w["t0"], dtype=torch.float64, device=dev)
    t1 = torch.tensor(w["t1"], dtype=torch.float64, device=dev)
    te = torch.tensor(w["t_eval"], dtype=torch.float64, device=dev)
    return y0, t0, t1, te


def _loss_and_grads(w, dtype, field, **kw):
    y0, t0, t1, te = _inputs(w, dtype)
    ts = [t.requires_grad_(True) for t in field.tensors()]
    ye, yf, n_acc, n_rej, status = tode.odeint_adjoint(field, y0, t0, t1, te, rtol=w["rtol"],
                                                       atol=w["atol"], **kw)
    d = torch.linspace(-1.0, 1.0, yf.shape[1], dtype=yf.dtype, device=yf.device)
    loss = (ye ** 2).sum() + (yf * d).sum()
    grads = torch.autograd.grad(loss, [y0] + ts)
    return ye.detach(), yf.detach(), n_acc, [g.double().cpu().numpy() for g in grads]


def test_autograd_vdp_f64_vs_oracle_adjoint():
    w = make(1, B=96)
    field = device_field(w, torch.float64)
    ye, yf, n_acc, (gy0, gmu) = _loss_and_grads(w, torch.float64, field)
    probe = gpu_solve(w, torch.float64, "fused", trace_cap=4000)
    assert np.array_equal(probe["n_acc"], n_acc.cpu().numpy())
    mt, mh, mn = mesh_from_trace(probe)
    D = w["y0"].shape[1]
    gye = 2.0 * ye.cpu().numpy()
    gyf = np.tile(np.linspace(-1.0, 1.0, D), (w["B"], 1))
    ref = oracle.adjoint(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"], gye, gyf)
    assert _rel(gy0, ref["gy0"]) <= 1e-10
    assert _rel(gmu, ref["gmu"]) <= 1e-10


def test_autograd_budget_recompute_is_bitwise():
    """A tape budget below one slot per step (segments recomputed) gives the
    same gradients as a full tape."""
    w = make(2, B=512)
    field = device_field(w, torch.float32)
    full = _loss_and_grads(w, torch.float32, field)
    per_slot = tode.TapeBuffers.bytes_per_slot(512, 16, 4)
    small = _loss_and_grads(w, torch.float32, field, hbm_budget_bytes=per_slot * 5, slots_hint=2)
    for a, b in zip(full[3], small[3]):
        assert np.array_equal(a, b)


def test_autograd_mlp_matches_direct_adjoint_call():
    """Float master weights: the autograd path returns exactly the direct
    adjoint's float gradients (taken at the BF16-rounded weights)."""
    w = dict(make(4, B=300), split=True)
    f = w["field"]
    W32 = [torch.tensor(x, dtype=torch.float32, device="cuda") for x in f["W"]]
    b32 = [torch.tensor(x, dtype=torch.float32, device="cuda") for x in f["b"]]
    field = tode.MLP(W32, b32, split=True)
    ye, yf, n_acc, grads = _loss_and_grads(w, torch.float32, field)
    # the same through solve + adjoint
    g = gpu_solve(w, torch.float32, "fused")
    B, D = w["y0"].shape
    tape = tode.TapeBuffers.allocate(B, D, torch.float32, int(g["n_acc"].max()), 1, "cuda",
                                     stages=True)
    y0, t0, t1, te = _inputs(w, torch.float32)
    sol = tode.solve(field, y0.detach(), t0, t1, te, tape=tape, rtol=w["rtol"], atol=w["atol"])
    assert torch.equal(sol.y_eval, ye)
    d = torch.linspace(-1.0, 1.0, D, dtype=torch.float32, device="cuda")
    gy0, (gW, gb), ovf = tode.adjoint(field, t0, t1, te, sol, tape, 2.0 * sol.y_eval,
                                      d.expand(B, D).contiguous(), rtol=w["rtol"],
                                      atol=w["atol"])
    ref = [gy0] + gW + gb
    for a, b in zip(grads, ref):
        assert np.array_equal(a, b.double().cpu().numpy())


@pytest.mark.parametrize("cfg,B", [(4, 300), (5, 150)])
def test_autograd_mlp_budget_recomputes_chunks(cfg, B):
    """A tape budget below the batch's stage tape: the backward re-solves
    the batch chunk by chunk with tapes that fit and reverses each chunk.
    dL/dy0 equals the full tape's bit for bit (an instance's solve and
    reversal do not depend on its batch); the weight and bias gradients are
    the same per-row products summed chunk by chunk, so they differ only by
    FP32 summation order: measured 3.3e-5 relative on the D = 32 field,
    where the per-CTA partials of a few hundred instances cancel heavily
    (a dropped or doubled chunk would differ at O(1)); a budget below one
    instance's tape is refused."""
    w = dict(make(cfg, B=B), split=True)
    field = device_field(w, torch.float32)
    full = _loss_and_grads(w, torch.float32, field)
    n_max = int(full[2].max())
    D = w["y0"].shape[1]
    one = tode.TapeBuffers.bytes_per_slot(1, D, 4, stages=True, minimal=True)
    budget = one * n_max * (B // 3 + 1)  # three or four chunks
    small = _loss_and_grads(w, torch.float32, field, hbm_budget_bytes=budget)
    assert np.array_equal(full[0].cpu().numpy(), small[0].cpu().numpy())
    assert np.array_equal(full[3][0], small[3][0])  # dL/dy0
    for a, b in zip(full[3][1:], small[3][1:]):
        assert np.linalg.norm(a - b) <= 2e-4 * max(np.linalg.norm(a), 1e-30)
    with pytest.raises(RuntimeError):
        _loss_and_grads(w, torch.float32, field, hbm_budget_bytes=one)


def test_autograd_joint_solve_vs_oracle_adjoint_on_the_shared_mesh():
    """Sec. 4.1's joint solve under autograd: the gradient is each
    instance's discrete adjoint on the one shared mesh; a budget too small
    for one slot per step is refused (a joint mesh is never re-run)."""
    w = make(1, B=40)
    T = 6.0
    te_row = np.linspace(0.0, T, 7)
    w = dict(w, t0=np.zeros(40), t1=np.full(40, T), t_eval=np.tile(te_row, (40, 1)))
    field = device_field(w, torch.float64)
    ye, yf, n_acc, (gy0, gmu) = _loss_and_grads(w, torch.float64, field, joint=True)
    probe = gpu_solve(w, torch.float64, "plain", joint=True, trace_cap=4000)
    assert np.array_equal(probe["n_acc"], n_acc.cpu().numpy())
    assert (probe["n_acc"] == probe["n_acc"][0]).all()
    mt, mh, mn = mesh_from_trace(probe)
    D = w["y0"].shape[1]
    gye = 2.0 * ye.cpu().numpy()
    gyf = np.tile(np.linspace(-1.0, 1.0, D), (w["B"], 1))
    ref = oracle.adjoint(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"], gye, gyf)
    assert _rel(gy0, ref["gy0"]) <= 1e-10
    assert _rel(gmu, ref["gmu"]) <= 1e-10
    with pytest.raises(RuntimeError):
        _loss_and_grads(w, torch.float64, field, joint=True, hbm_budget_bytes=40 * 40,
                        slots_hint=1)


@pytest.mark.parametrize("cfg,B", [(4, 300), (5, 150)])
def test_mlp_resolve_reproduces_the_stage_tape_bitwise(cfg, B):
    """A solve with a checkpoint tape (every m-th accepted step) and
    tode_mlp_resolve of each segment give, slot for slot, the stage inputs,
    times and step sizes a stride-1 tape records in one solve -- the same
    attempts from the same states -- and the segment counts and bounds."""
    w = dict(make(cfg, B=B), split=True)
    field = device_field(w, torch.float32)
    y0, t0, t1, te = _inputs(w, torch.float32)
    y0 = y0.detach()
    opt = dict(rtol=w["rtol"], atol=w["atol"])
    probe = tode.solve(field, y0, t0, t1, te, **opt)
    N = int(probe.n_acc.max().item())
    D = w["y0"].shape[1]
    full = tode.TapeBuffers.allocate(B, D, torch.float32, N, 1, "cuda", stages=True, minimal=True)
    ref = tode.solve(field, y0, t0, t1, te, tape=full, **opt)
    m = 2
    ck = tode.TapeBuffers.allocate(B, D, torch.float32, -(-N // m), m, "cuda")
    sol = tode.solve(field, y0, t0, t1, te, tape=ck, **opt)
    for k in ("y_eval", "y_final", "n_acc", "n_rej", "status"):
        assert torch.equal(getattr(sol, k), getattr(ref, k)), k
    seg_tape = tode.TapeBuffers.allocate(B, D, torch.float32, m, 1, "cuda", stages=True,
                                         minimal=True)
    n_acc = sol.n_acc.cpu().numpy()
    for j in range(-(-N // m)):
        seg_n, s0, s1 = tode.mlp_resolve(field, t0, t1, sol.n_acc, ck, j, seg_tape, **opt)
        torch.cuda.synchronize()
        want = np.clip(n_acc - j * m, 0, m)
        assert np.array_equal(seg_n.cpu().numpy(), want)
        for i in range(B):
            n = int(want[i])
            if n == 0:
                assert s0[i].item() == s1[i].item() == w["t1"][i]
                continue
            sl = slice(j * m, j * m + n)
            assert torch.equal(seg_tape.y_stage[i, :n], full.y_stage[i, sl]), (j, i)
            assert torch.equal(seg_tape.y[i, :n], full.y[i, sl]), (j, i)
            assert torch.equal(seg_tape.t[i, :n], full.t[i, sl]), (j, i)
            assert torch.equal(seg_tape.h_acc[i, :n], full.h_acc[i, sl]), (j, i)
            assert s0[i].item() == full.t[i, j * m].item()
            end = w["t1"][i] if j * m + n == n_acc[i] else full.t[i, j * m + n].item()
            assert s1[i].item() == end


@pytest.mark.parametrize("cfg,B", [(4, 300), (5, 150)])
def test_autograd_mlp_budget_checkpoints_segments(cfg, B, monkeypatch):
    """A tape budget just below the stride-1 stage tape: the forward keeps
    the solver state every m accepted steps, the backward re-solves each
    segment into an m-slot stage tape and reverses it from the cotangent the
    later segment handed over.  dL/dy0 equals the full tape's bit for bit
    (the same stage inputs, the same per-row reversal); the weight and bias
    gradients are summed segment by segment (FP32 summation order, as for
    chunks)."""
    w = dict(make(cfg, B=B), split=True)
    field = device_field(w, torch.float32)
    full = _loss_and_grads(w, torch.float32, field)
    n_max = int(full[2].max())
    D = w["y0"].shape[1]
    st = tode.TapeBuffers.bytes_per_slot(B, D, 4, stages=True, minimal=True)
    calls = []
    real = tode.api.mlp_resolve

    def counting(*a, **k):
        calls.append(a[5])
        return real(*a, **k)
    monkeypatch.setattr(tode.api, "mlp_resolve", counting)
    small = _loss_and_grads(w, torch.float32, field, hbm_budget_bytes=n_max * st - 1)
    assert len(calls) >= 2 and calls == sorted(calls, reverse=True)
    assert np.array_equal(full[0].cpu().numpy(), small[0].cpu().numpy())
    assert np.array_equal(full[3][0], small[3][0])  # dL/dy0
    for a, b in zip(full[3][1:], small[3][1:]):
        assert np.linalg.norm(a - b) <= 2e-4 * max(np.linalg.norm(a), 1e-30)


def test_autograd_mlp_budget_segments_pid_mixed_directions_tsit5(monkeypatch):
    """The checkpoints carry the whole controller state: with the PID
    controller (beta2, beta3 != 0, so err_prev and err_prev2 steer the
    steps), every other instance integrated backward, and the tsit5 pair,
    the budgeted backward's dL/dy0 still equals the full tape's bit for
    bit, and the (BF16) weight gradients agree to the BF16 unit roundoff."""
    B = 300
    w = dict(make(4, B=B), split=True)
    t0, t1, te = w["t0"].copy(), w["t1"].copy(), w["t_eval"].copy()
    t0[::2], t1[::2] = w["t1"][::2], w["t0"][::2]
    te[::2] = te[::2, ::-1]
    w = dict(w, t0=t0, t1=t1, t_eval=np.ascontiguousarray(te), rtol=1e-6, atol=1e-6)
    field = device_field(w, torch.float32)
    opt = dict(beta1=0.7 / 5, beta2=0.5 / 5, beta3=0.1 / 5, method="tsit5")
    full = _loss_and_grads(w, torch.float32, field, **opt)
    n_max = int(full[2].max())
    assert n_max >= 4
    D = w["y0"].shape[1]
    st = tode.TapeBuffers.bytes_per_slot(B, D, 4, stages=True, minimal=True)
    calls = []
    real = tode.api.mlp_resolve

    def counting(*a, **k):
        calls.append(a[5])
        return real(*a, **k)
    monkeypatch.setattr(tode.api, "mlp_resolve", counting)
    small = _loss_and_grads(w, torch.float32, field, hbm_budget_bytes=n_max * st - 1, **opt)
    assert len(calls) >= 2
    assert np.array_equal(full[0].cpu().numpy(), small[0].cpu().numpy())
    assert np.array_equal(full[3][0], small[3][0])  # dL/dy0
    # the weight gradients come back in the weights' BF16: sums that differ
    # in FP32 summation order round to the same BF16 value or to a
    # neighbour, so the tensors agree to the BF16 unit roundoff (2^-8)
    for a, b in zip(full[3][1:], small[3][1:]):
        assert np.linalg.norm(a - b) <= 2.0 ** -8 * max(np.linalg.norm(a), 1e-30)
