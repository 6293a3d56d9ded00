"""Shared helpers of the GPU parity tests: move a seeded workload to the
device, run the CUDA path through the C ABI, run the oracle on the same
inputs."""
from __future__ import annotations

import numpy as np
import torch

import oracle
import paper_2210_12375_b300 as tode
from paper_2210_12375_b300 import workloads


def device_field(w, dtype, dev="cuda"):
    f = w["field"]
    if f["kind"] == "vdp":
        return tode.VdP(torch.tensor(f["mu"], dtype=dtype, device=dev))
    if f["kind"] == "linear":
        return tode.Linear(torch.tensor(f["A"], dtype=dtype, device=dev).contiguous())
    if f["kind"] == "mlp":  # BF16 weights (exactly the oracle's values), float biases
        W = [torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(dev).contiguous()
             for x in f["W"]]
        b = [torch.tensor(x, dtype=torch.float32, device=dev) for x in f["b"]]
        return tode.MLP(W, b, split=w.get("split", True))
    raise ValueError(f["kind"])


def gpu_solve(w, dtype, form, rtol=None, atol=None, trace_cap=0, tape=None, **kw):
    dev = "cuda"
    field = device_field(w, dtype)
    y0 = torch.tensor(w["y0"], dtype=dtype, device=dev)
    t0 = torch.tensor(w["t0"], dtype=torch.float64, device=dev)
    t1 = torch.tensor(w["t1"], dtype=torch.float64, device=dev)
    te = torch.tensor(w["t_eval"], dtype=torch.float64, device=dev) \
        if w["t_eval"] is not None and w["t_eval"].shape[1] > 0 else None
    sol = tode.solve(field, y0, t0, t1, te, rtol=w["rtol"] if rtol is None else rtol,
                     atol=w["atol"] if atol is None else atol, form=form,
                     trace_cap=trace_cap, tape=tape, **kw)
    torch.cuda.synchronize()
    out = {k: getattr(sol, k).cpu().numpy() for k in
           ("y_eval", "y_final", "n_acc", "n_rej", "n_feval", "status")}
    out["y_eval"] = out["y_eval"].astype(np.float64)
    out["y_final"] = out["y_final"].astype(np.float64)
    if sol.trace is not None:
        for k, v in sol.trace.items():
            out["trace_" + k] = v.cpu().numpy()
    if sol.yp_eval is not None:
        out["yp_eval"] = sol.yp_eval.cpu().numpy().astype(np.float64)
    out["_sol"] = sol
    out["_dev"] = dict(field=field, y0=y0, t0=t0, t1=t1, te=te)
    return out


def oracle_solve(w, rtol=None, atol=None, trace_cap=0, **kw):
    return oracle.solve(w["field"], w["y0"], w["t0"], w["t1"], w["t_eval"],
                        dict(rtol=w["rtol"] if rtol is None else rtol,
                             atol=w["atol"] if atol is None else atol, **kw),
                        trace_cap=trace_cap)


def subset(w, idx):
    """Instances idx of workload w (a new workload dict)."""
    idx = np.asarray(idx)
    f = dict(w["field"])
    for k in ("mu", "A", "Q", "lam"):
        if k in f:
            f[k] = f[k][idx]
    return dict(w, field=f, y0=w["y0"][idx], t0=w["t0"][idx], t1=w["t1"][idx],
                t_eval=w["t_eval"][idx], B=len(idx))


def make(cfg, B=None):
    return workloads.make(cfg, B)
