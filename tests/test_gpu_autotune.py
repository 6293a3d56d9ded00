"""The launch-shape autotuner on the GPU: it times the candidate shapes on
the caller's batch, the choice runs and stays within the workload band of
the closed form, and the cache answers the next call."""
import numpy as np
import pytest
import torch

import paper_2210_12375_b300 as tode
from paper_2210_12375_b300 import tuning as at
from gpu_helpers import device_field, make

pytestmark = pytest.mark.gpu


def test_autotune_linear_fwd_adj(tmp_path):
    at.set_cache_path(str(tmp_path / "tune.json"))
    at._mem.clear()
    try:
        w = make(2, B=2048)
        field = device_field(w, torch.float32)
        dev = "cuda"
        y0 = torch.tensor(w["y0"], dtype=torch.float32, device=dev)
        t0 = torch.tensor(w["t0"], device=dev)
        t1 = torch.tensor(w["t1"], device=dev)
        te = torch.tensor(w["t_eval"], device=dev)
        opt = dict(rtol=w["rtol"], atol=w["atol"])
        best = tode.autotune(field, y0, t0, t1, te, with_adjoint=True, reps=2, **opt)
        assert best in at.candidates("linear", 16, "fused")
        entry = next(iter(at._mem.values()))
        assert len(entry["tried"]) == len(at.candidates("linear", 16, "fused"))
        sol = tode.solve(field, y0, t0, t1, te, **opt, **best)
        torch.cuda.synchronize()
        Q, lam = w["field"]["Q"], w["field"]["lam"]
        c = np.einsum("bji,bj->bi", Q, w["y0"])
        ex = np.exp(-lam[:, None, :] * w["t_eval"][:, :, None])
        exact = np.einsum("bij,bkj->bki", Q, ex * c[:, None, :])
        ye = sol.y_eval.double().cpu().numpy()
        assert (np.abs(ye - exact) <= 10 * (w["atol"] + w["rtol"] * np.abs(exact))).mean() > 0.99

        def boom(o):
            raise AssertionError("cached")
        at._mem.clear()
        assert tode.autotune(field, y0, t0, t1, te, with_adjoint=True, timer=boom, **opt) == best
    finally:
        at.set_cache_path(None)
        at._mem.clear()
