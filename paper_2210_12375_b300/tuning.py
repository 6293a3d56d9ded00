"""Launch-shape autotuner for the solver kernels.

The fused persistent kernel and its adjoint take three launch knobs
(``tode_options``): ``group`` (lanes per instance of the linear field),
``block`` (threads per CTA) and ``ctas_per_sm`` (resident CTAs per SM of the
persistent grid); the plain form also takes ``poll_every``, and both forms
take ``order`` (index order, or longest integration interval first).
``autotune`` times the candidates on the caller's own batch (solve, or
solve + adjoint) with CUDA events -- the fused form replayed from a CUDA
graph, so that host launch costs stay off the device timeline -- and
returns the fastest, and caches the choice in a JSON
file keyed by field kind, state size, precision, form, batch size (rounded
to a power of two) and GPU name.  The cache file is ``$TODE_AUTOTUNE_CACHE``
or the path given to ``set_cache_path``; without either, choices live in
memory only.

Different ``group`` values change the FP32 summation order of the error
norm, so results of different candidates agree to rounding, not bit for bit;
the adjoint must run with the forward's options (it re-runs the forward's
attempts when the tape is strided).  The MLP field's tiles are fixed by its
network shape (tensor-memory lanes, shared memory); its knobs are the work
order of the persistent grid and, for the wide network's adjoint, the size
of the slices the adjoint stages (``ctas_per_sm``: 1 or 2 CTAs' worth of
instances per SM); its results do not depend on either.
"""
from __future__ import annotations

import json
import math
import os
import threading
from typing import Callable, Dict, List, Optional

import torch

from . import api

_lock = threading.Lock()
_mem: Dict[str, dict] = {}
_path: Optional[str] = None


def set_cache_path(path: Optional[str]) -> None:
    """Cache file for autotuning choices (None: memory only, unless
    $TODE_AUTOTUNE_CACHE is set)."""
    global _path
    _path = path


def _cache_file() -> Optional[str]:
    return _path or os.environ.get("TODE_AUTOTUNE_CACHE")


def _load() -> Dict[str, dict]:
    f = _cache_file()
    if f and os.path.exists(f):
        with open(f) as fh:
            return json.load(fh)
    return {}


def _store(key: str, choice: dict) -> None:
    _mem[key] = choice
    f = _cache_file()
    if not f:
        return
    data = _load()
    data[key] = choice
    d = os.path.dirname(os.path.abspath(f))
    os.makedirs(d, exist_ok=True)
    tmp = f + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, f)


def cache_key(kind: str, D: int, B: int, prec: str, form: str, with_adjoint: bool,
              device_name: str) -> str:
    b2 = 1 << max(0, math.ceil(math.log2(max(B, 1))))
    return f"{device_name}|{kind}|D{D}|B{b2}|{prec}|{form}|{'adj' if with_adjoint else 'fwd'}"


def candidates(kind: str, D: int, form: str, with_adjoint: bool = False) -> List[dict]:
    """The launch shapes tried for a field (each a dict of tode_options keys)."""
    if kind == "mlp":
        # the MLP tiles are fixed by the network (tensor-memory lanes, shared
        # memory); what varies is the instances' order on the persistent
        # grid and, for the wide network's adjoint, the size of its slices
        out = [{"order": o} for o in (0, 1)]
        if with_adjoint and D == 64:
            out = [dict(x, ctas_per_sm=m) for x in out for m in (1, 2)]
        return out
    groups = [0]
    if kind == "linear":
        groups = {16: [4, 8, 16], 32: [16]}.get(D, [D])
    blocks = [32, 64, 128, 256]
    out = []
    for g in groups:
        for b in blocks:
            for order in (0, 1):
                if form == "plain":
                    for p in (8, 16, 32):
                        out.append({"group": g, "block": b, "poll_every": p, "order": order})
                else:
                    for c in (0, 1, 2, 4):
                        out.append({"group": g, "block": b, "ctas_per_sm": c, "order": order})
    return out


def _kind(field) -> str:
    return {api.VdP: "vdp", api.Linear: "linear", api.MLP: "mlp"}[type(field)]


def _time_candidate(run: Callable[[], None], reps: int, graph: bool = False) -> float:
    run()  # warm-up (and first-call set-up outside any capture)
    torch.cuda.synchronize()
    if graph:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            run()
        run = g.replay
        run()
        torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        run()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    times.sort()
    return times[len(times) // 2]


def autotune(field, y0: torch.Tensor, t0: torch.Tensor, t1: torch.Tensor,
             t_eval: Optional[torch.Tensor] = None, *, form: str = "fused",
             with_adjoint: bool = False, reps: int = 5, timer: Optional[Callable] = None,
             refresh: bool = False, **opt_kw) -> dict:
    """Fastest launch options for this batch, from the cache when present.

    ``timer(options) -> ms`` replaces the CUDA-event timing (tests).  Returns
    the chosen options (a dict to pass on to ``solve`` / ``adjoint``)."""
    kind = _kind(field)
    B, D = y0.shape
    prec = str(y0.dtype).replace("torch.", "")
    dev_name = torch.cuda.get_device_name(y0.device) if y0.is_cuda else "cpu"
    key = cache_key(kind, D, B, prec, form, with_adjoint, dev_name)
    with _lock:
        if not refresh:
            if key in _mem:
                return dict(_mem[key]["options"])
            disk = _load()
            if key in disk:
                _mem[key] = disk[key]
                return dict(disk[key]["options"])
        cands = candidates(kind, D, form, with_adjoint)
        if timer is None:
            tape = None
            if with_adjoint:
                probe = api.solve(field, y0, t0, t1, t_eval, form="fused", **opt_kw)
                torch.cuda.synchronize()
                slots = max(1, int(probe.n_acc.max().item()))
                tape = api.TapeBuffers.allocate(B, D, y0.dtype, slots, 1, y0.device,
                                                stages=kind in ("mlp", "linear"), minimal=True)

            def timer(o):
                def run():
                    kw = dict(opt_kw, **o)  # the candidate's knobs override the caller's
                    s = api.solve(field, y0, t0, t1, t_eval, form=form, tape=tape, **kw)
                    if with_adjoint:
                        gy = torch.ones_like(s.y_final)
                        api.adjoint(field, t0, t1, t_eval, s, tape, None, gy, **kw)
                return _time_candidate(run, reps, graph=form == "fused")
        results = []
        for o in cands:
            try:
                results.append((float(timer(o)), o))
            except api._abi.TodeError:
                continue  # a shape the library refuses for this problem
        if not results:
            raise RuntimeError("autotune: no candidate launch shape ran")
        best_ms, best = min(results, key=lambda r: r[0])
        _store(key, {"options": best, "ms": best_ms,
                     "tried": [{"options": o, "ms": ms} for ms, o in results]})
        return dict(best)
