"""The fused forward and the adjoint under CUDA-graph capture: one captured
step (solve with checkpoint tape + discrete adjoint) replays bit for bit
like the eager calls, also after new inputs are copied into the captured
buffers."""
import numpy as np
import pytest
import torch

import paper_2210_12375_b300 as tode
from gpu_helpers import device_field, make, subset

pytestmark = pytest.mark.gpu


def _bufs(w, dtype):
    dev = "cuda"
    return dict(y0=torch.tensor(w["y0"], dtype=dtype, device=dev),
                t0=torch.tensor(w["t0"], dtype=torch.float64, device=dev),
                t1=torch.tensor(w["t1"], dtype=torch.float64, device=dev),
                te=torch.tensor(w["t_eval"], dtype=torch.float64, device=dev))


def _step(field, x, tape, opt, sol=None, ws=None, scratch=None):
    s = tode.solve(field, x["y0"], x["t0"], x["t1"], x["te"], form="fused", tape=tape, out=sol,
                   workspace=ws, **opt)
    gye = 2.0 * s.y_eval
    gy0, gp, ovf = tode.adjoint(field, x["t0"], x["t1"], x["te"], s, tape, gye, None,
                                scratch=scratch, **opt)
    return s, gy0, gp, ovf


def _flat(s, gy0, gp):
    out = [s.y_eval, s.y_final, s.n_acc, s.status, gy0]
    if isinstance(gp, tuple):
        out += list(gp[0]) + list(gp[1])
    else:
        out.append(gp)
    return [t.clone() for t in out]


@pytest.mark.parametrize("cfg", [1, 2, 4])
def test_fused_step_replays_under_cuda_graph(cfg):
    w = dict(make(cfg, B=512 if cfg != 1 else 128), split=True)
    dtype = torch.float64 if cfg == 1 else torch.float32
    field = device_field(w, dtype)
    opt = dict(rtol=w["rtol"], atol=w["atol"])
    B, D = w["y0"].shape
    x = _bufs(w, dtype)
    probe = tode.solve(field, x["y0"], x["t0"], x["t1"], x["te"], form="fused", **opt)
    torch.cuda.synchronize()
    slots = int(probe.n_acc.max().item()) + 8
    tape = tode.TapeBuffers.allocate(B, D, dtype, slots, 1, "cuda", stages=cfg == 4)
    # eager reference for the original inputs and for a second input set
    ref1 = _flat(*_step(field, x, tape, opt)[:3])
    w2 = subset(w, np.random.default_rng(5).permutation(B))
    x2 = _bufs(w2, dtype)
    if cfg != 4:
        field2 = device_field(w2, dtype)  # per-instance parameters move with the instances
    else:
        field2 = field
    ref2 = _flat(*_step(field2, x2, tape, opt)[:3])
    torch.cuda.synchronize()

    # capture: static inputs, outputs, workspace and scratch
    xs = {k: v.clone() for k, v in x.items()}
    fs = device_field(w, dtype)
    sol = tode.solve(fs, xs["y0"], xs["t0"], xs["t1"], xs["te"], form="fused", tape=tape, **opt)
    ws = sol.extra["workspace"]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        _step(fs, xs, tape, opt, sol, ws)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        s, gy0, gp, ovf = _step(fs, xs, tape, opt, sol, ws)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(_flat(s, gy0, gp), ref1):
        assert torch.equal(a, b)
    # new inputs into the captured buffers (and the per-instance parameters)
    for k in xs:
        xs[k].copy_(x2[k])
    for dst, src in zip(fs.tensors(), field2.tensors()):
        dst.copy_(src)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(_flat(s, gy0, gp), ref2):
        assert torch.equal(a, b)
    assert int(ovf.item()) == 0
