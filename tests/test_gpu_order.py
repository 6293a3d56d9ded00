"""The work order of the Van der Pol and linear solvers (longest interval
first, or index order) decides only which instances share a warp and which
start first: every output of both forms and of the adjoint is the same bits
either way, including instances that are invalid or finish at t0.  Batches
above 2048 instances take the multi-CTA sort, the 256-instance one the
one-CTA sort."""
import numpy as np
import pytest
import torch

import paper_2210_12375_b300 as tode
from gpu_helpers import gpu_solve, make, subset

pytestmark = pytest.mark.gpu

KEYS = ("y_eval", "y_final", "n_acc", "n_rej", "n_feval", "status")


def _workload(cfg, B):
    w = make(cfg)
    w = subset(w, np.random.default_rng(3).permutation(w["B"])[:B])
    t1, te = w["t1"].copy(), w["t_eval"].copy()
    t1[1] = w["t0"][1]                      # empty interval: finishes at t0
    te[1] = w["t0"][1]
    t1[2] = w["t0"][2] - 1.0                # invalid interval
    return dict(w, t1=t1, t_eval=te)


@pytest.mark.parametrize("cfg,B", [(2, 1500), (2, 2049), (3, 3000), (1, 256), (3, 40000)])
@pytest.mark.parametrize("form", ["fused", "plain"])
def test_order_changes_no_bit(cfg, B, form):
    w = _workload(cfg, B)
    dtype = torch.float64 if cfg == 1 else torch.float32
    res = [gpu_solve(w, dtype, form, order=o) for o in (0, 1)]
    for k in KEYS:
        assert np.array_equal(res[0][k], res[1][k], equal_nan=True), k
    assert res[0]["status"][2] == tode._abi.STATUS["INVALID_INPUT"]
    assert res[0]["status"][1] == tode._abi.STATUS["SUCCESS"] and res[0]["n_acc"][1] == 0


@pytest.mark.parametrize("cfg,B", [(2, 1500), (3, 3000), (3, 40000)])
def test_adjoint_order_changes_no_bit(cfg, B):
    """The forward's order (either) feeds a tape; the adjoint reverses it
    longest first: gradients equal those of the index-order forward."""
    w = _workload(cfg, B)
    probe = gpu_solve(w, torch.float32, "fused")
    slots = max(1, int(probe["n_acc"].max()))
    outs = []
    for o in (0, 1):
        tape = tode.TapeBuffers.allocate(B, w["y0"].shape[1], torch.float32, slots, 1, "cuda")
        g = gpu_solve(w, torch.float32, "fused", tape=tape, order=o)
        dev = g["_dev"]
        gyf = torch.ones((B, w["y0"].shape[1]), dtype=torch.float32, device="cuda")
        gy0, gp, ovf = tode.adjoint(dev["field"], dev["t0"], dev["t1"], dev["te"], g["_sol"],
                                    tape, None, gyf, rtol=w["rtol"], atol=w["atol"])
        torch.cuda.synchronize()
        outs.append((gy0.cpu().numpy(), gp.cpu().numpy(), int(ovf.item())))
    assert outs[0][2] == outs[1][2] == 0
    assert np.array_equal(outs[0][0], outs[1][0], equal_nan=True)
    assert np.array_equal(outs[0][1], outs[1][1], equal_nan=True)


def test_order_sort_grid_stride_batch():
    """More instances than the multi-CTA sort has threads (1024 CTAs x 1024):
    its CTAs walk the batch in more than one stride, and the forward (no
    tape, Van der Pol, durations cut short) gives the same bits either way."""
    base = make(3)
    B = 1024 * 1024 + 4099
    w = subset(base, np.arange(B) % base["B"])
    w = dict(w, t1=np.minimum(w["t1"], w["t0"] + 0.5))
    w = dict(w, t_eval=np.linspace(0.0, 1.0, 3)[None, :] * (w["t1"] - w["t0"])[:, None]
             + w["t0"][:, None])
    res = [gpu_solve(w, torch.float32, "fused", order=o) for o in (0, 1)]
    for k in KEYS:
        assert np.array_equal(res[0][k], res[1][k], equal_nan=True), k
    assert (res[0]["status"] == 0).all()
