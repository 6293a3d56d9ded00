"""Benchmark: batched adaptive dopri5 instance-steps/s, forward + discrete
adjoint, fused persistent form vs plain per-step form, on one B300.

Default workload: linear y' = A_i y, D = 16, FP32 state / FP64 time,
B = 8192, 32 t_eval, rtol = atol = 1e-5 (A_i = Q diag(-lambda) Q^T).  One
"step" is one pass of the whole solver path over the batch: the fused
forward solve (stages, error norm, PI control, dense output, checkpoint
tape) followed by the discrete adjoint of L = <c, y(t_eval)> + <d, y(t1)>
for fixed seeded cotangents c, d.  An instance-step is one attempted step
of a live instance.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       [--workload 2|3|1|4]
Under torchrun (N > 1) every rank solves its own copy of the batch (weak
scaling, no data-path collective) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2210_12375_b300 import workloads  # noqa: E402
from paper_2210_12375_b300.dist import max_over_ranks  # noqa: E402

METRIC = "instance-steps/s, dopri5 fwd and fwd+adjoint, fused vs plain form at matched error"
L2_FLUSH_BYTES = 256 << 20


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=400)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="tode", choices=["tode", "reference"])
    p.add_argument("--workload", type=int, default=2)
    p.add_argument("--plain-steps", type=int, default=30)
    p.add_argument("--batch", type=int, default=0, help="instances (default: the workload's)")
    p.add_argument("--kernel-reps", type=int, default=20)
    p.add_argument("--fwd-only", action="store_true", help="time the forward solve alone")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--order", type=int, default=0, choices=[0, 1],
                   help="work order of the SIMT solvers: 0 index, 1 longest interval first")
    p.add_argument("--no-graph", action="store_true",
                   help="issue the fused step eagerly instead of replaying a CUDA graph")
    p.add_argument("--no-autotune", action="store_true",
                   help="library default launch shapes instead of the autotuner's choice")
    p.add_argument("--joint", action="store_true",
                   help="the batching experiment of Sec. 4.1: one batch of strongly damped "
                        "oscillators solved jointly (one stacked problem) and independently")
    return p.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers
# DRAM bytes (read + write) of one launch of a kernel on a workload, from
# one ncu capture of that kernel as it stands (summaries under profiles/);
# kernels without a capture of their current code report null.
TRAFFIC = {
    ("linear_d16_b8192", "k_fused<LinearField<float,2,8>>"): 28.52e6,
    ("linear_d16_b8192", "k_fused<LinearField<float,1,16>>"): 27.59e6,
    ("linear_d16_b8192", "k_adjoint_steps<LinearAdj<float,1,16>>"): 86.14e6,
    ("mlp_d32_h128", "k_mlp_adjoint"): 67.41e6,
    # captured on the first 32,768 instances, x8 (the tape grows with the steps)
    ("vdp_mix_b262144", "k_fused<VdpField<float>>"): 8 * 91.71e6,
    ("vdp_mix_b262144", "k_adjoint_steps<VdpAdj<float>>"): 8 * 124.07e6,
    ("mlp_d32_h128", "k_mlp_fused"): 12.68e6,
    ("vdp_joint_mu10_b2097152", "k_joint_step<VdpField<float>>"): 69.53e6,
}


def _traffic(workload: str, kernel: str):
    for (wl, prefix), v in TRAFFIC.items():
        if wl == workload and kernel.startswith(prefix):
            return v
    return None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
            "sm_max_mhz": 2032.0}, "fallback"


def flops_per_attempt(kind: str, D: int) -> float:
    """Algorithmic FLOPs of one attempted dopri5 step (FMA = 2 FLOPs): six
    field evaluations, the 20 stage-combination terms plus 6 state updates per
    component, the 6-term error estimate and its weighted norm."""
    f_eval = 2 * D * D if kind == "linear" else 6
    comb = 2 * (20 + 6 + 7) * D + 6 * D
    return 6 * f_eval + comb


def adjoint_flops_per_step(kind: str, D: int, recorded: bool) -> float:
    """Algorithmic FLOPs of reversing one accepted step: the stage
    re-evaluations (none when the tape recorded the stage inputs), 6
    transposed-Jacobian products with their parameter outer products, and the
    stage-cotangent combinations."""
    if kind == "linear":
        f_eval, vjp = 2 * D * D, 4 * D * D
    else:
        f_eval, vjp = 6, 12
    return (0 if recorded else 7 * f_eval) + 6 * vjp + 2 * (26 + 21) * D


def _events(torch, n):
    return [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(n)]


# ------------------------------------------------------------------ joint solving
# Bytes one k_joint_step launch moves per instance and component while the
# problem runs: it reads the state y, y_lo, k1 from one half of the double
# buffer and writes the candidate to the other (6 values); the dense output
# (K points over the whole solve) is left out.
JOINT_VALUES_PER_COMPONENT = 6


def run_joint(args):
    """Sec. 4.1 / Fig. 1 on the B300: B Van der Pol oscillators with strong
    damping (mu = 10) and varying initial states, on one shared time axis,
    solved jointly (one stacked problem: one step size, norm and decision)
    and independently (the fused solver).  The line's value is the joint
    solve's instance-attempts per second; "batching" holds both step counts
    and both times."""
    import torch

    import paper_2210_12375_b300 as tode

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    B = args.batch or (1 << 21)
    mu, T, K, tol = 10.0, 40.0, 16, 1e-6
    rng = np.random.default_rng(20221023)
    y0 = torch.tensor(rng.uniform(-2.0, 2.0, (B, 2)), dtype=torch.float32, device=dev)
    field = tode.VdP(torch.full((B,), mu, dtype=torch.float32, device=dev))
    t0 = torch.zeros(B, dtype=torch.float64, device=dev)
    t1 = torch.full((B,), T, dtype=torch.float64, device=dev)
    te = torch.linspace(0.0, T, K, dtype=torch.float64, device=dev).expand(B, K).contiguous()
    opt = dict(rtol=tol, atol=tol)
    poll = 64
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    ind = tode.solve(field, y0, t0, t1, te, form="fused", **opt)
    jnt = tode.solve(field, y0, t0, t1, te, joint=True, poll_every=poll, **opt)
    torch.cuda.synchronize()
    assert int((ind.status != 0).sum()) == 0 and int((jnt.status != 0).sum()) == 0
    j_acc, j_rej = int(jnt.n_acc[0]), int(jnt.n_rej[0])
    i_acc = ind.n_acc.double()
    i_att = int((ind.n_acc.long() + ind.n_rej.long()).sum())

    def timed(fn, n):
        for _ in range(max(args.warmup, 1)):
            fn()
        torch.cuda.synchronize()
        ev = _events(torch, n)
        for k in range(n):
            flush.zero_()
            ev[k][0].record(stream)
            fn()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    sol_i, sol_j = ind, jnt
    ws_i, ws_j = ind.extra["workspace"], jnt.extra["workspace"]
    n = max(3, min(args.steps, 10))
    with ClockSampler(0) as clk:
        ms_j = timed(lambda: tode.solve(field, y0, t0, t1, te, joint=True, poll_every=poll,
                                        out=sol_j, workspace=ws_j, **opt), n)
        ms_i = timed(lambda: tode.solve(field, y0, t0, t1, te, form="fused", out=sol_i,
                                        workspace=ws_i, **opt), n)
    clocks = clk.summary()
    # launches: init, first step, then attempts + the final commit, issued in
    # groups of `poll` (the group that finishes the solve ends in no-ops)
    step_launches = -(-(j_acc + j_rej + 1) // poll) * poll
    launches = 2 + step_launches
    per_launch_ms = ms_j / launches  # an upper bound: host polls and no-op launches included
    by = B * 2 * (JOINT_VALUES_PER_COMPONENT * 4) + B * 4  # + mu
    peaks, src = _peaks()
    achieved = by / (per_launch_ms * 1e-3) / 1e9
    value = B * (j_acc + j_rej) / (ms_j * 1e-3)
    print(json.dumps({
        "metric": "instance-steps/s, joint (stacked) dopri5 solve, Sec. 4.1 batching experiment",
        "value": value, "unit": "instance-steps/s", "n_gpus": 1, "steps": n,
        "warmup": max(args.warmup, 1), "ms_per_step": ms_j, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded Van der Pol oscillators, mu = 10, y0 ~ U[-2,2]^2)",
        "config": {"workload": f"vdp_joint_mu10_b{B}", "B": B, "t": [0.0, T], "t_eval": K,
                   "rtol": tol, "atol": tol, "pass": "fwd", "l2": "flushed between passes",
                   "poll_every": poll},
        "batching": {"joint_n_acc": j_acc, "joint_n_rej": j_rej,
                     "independent_n_acc_mean": float(i_acc.mean()),
                     "independent_n_acc_max": int(i_acc.max()),
                     "steps_ratio_vs_mean": j_acc / float(i_acc.mean()),
                     "joint_ms": ms_j, "independent_ms": ms_i, "time_ratio": ms_j / ms_i,
                     "independent_instance_steps_per_s": i_att / (ms_i * 1e-3)},
        "roofline": {"bound": "hbm", "kernel": "k_joint_step<VdpField<float>>",
                     "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "peak_source": src,
                     "traffic": _traffic(f"vdp_joint_mu10_b{B}", "k_joint_step<VdpField<float>>"),
                     "kernel_ms": per_launch_ms,
                     "bytes_per_launch": by},
        "clocks": clocks,
        "gpu_launches": launches,
    }), flush=True)


# ------------------------------------------------------------------ GPU arm
def run_tode(args):
    import torch
    import torch.distributed as dist

    import paper_2210_12375_b300 as tode

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    w = workloads.make(args.workload, args.batch or None)
    kind = w["field"]["kind"]
    dtype = torch.float64 if w["prec"] == "f64" else torch.float32
    B, D = w["y0"].shape
    K = w["t_eval"].shape[1]
    mlp = kind == "mlp"
    if kind == "linear":
        field = tode.Linear(torch.tensor(w["field"]["A"], dtype=dtype, device=dev).contiguous())
    elif mlp:
        field = tode.MLP([torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(dev)
                          .contiguous() for x in w["field"]["W"]],
                         [torch.tensor(x, dtype=torch.float32, device=dev)
                          for x in w["field"]["b"]], split=True)
    else:
        field = tode.VdP(torch.tensor(w["field"]["mu"], dtype=dtype, device=dev))
    y0 = torch.tensor(w["y0"], dtype=dtype, device=dev)
    t0 = torch.tensor(w["t0"], dtype=torch.float64, device=dev)
    t1 = torch.tensor(w["t1"], dtype=torch.float64, device=dev)
    te = torch.tensor(w["t_eval"], dtype=torch.float64, device=dev)
    rng = np.random.default_rng(20221022)
    gye = torch.tensor(rng.standard_normal((B, K, D)), dtype=dtype, device=dev)
    gyf = torch.tensor(rng.standard_normal((B, D)), dtype=dtype, device=dev)
    opt = dict(rtol=w["rtol"], atol=w["atol"])
    if not mlp:
        opt["order"] = args.order
    tuned = tuned_plain = None
    opt_plain = dict(opt)
    if not args.no_autotune and not mlp:
        # the launch shape (lanes per instance, CTA size, resident CTAs, work
        # order; for the plain form its poll interval) the autotuner picks for
        # this batch, timed on it (fwd + adjoint), for each form
        tuned = tode.autotune(field, y0, t0, t1, te, with_adjoint=True, reps=7, **opt)
        tuned_plain = tode.autotune(field, y0, t0, t1, te, form="plain", with_adjoint=True,
                                    reps=2, **opt)
        opt.update(tuned)
        opt_plain.update(tuned_plain)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # probe: step counts (identical every pass) and the tape size
    probe = tode.solve(field, y0, t0, t1, te, form="fused", **opt)
    torch.cuda.synchronize()
    assert int((probe.status != 0).sum().item()) == 0, "benchmark workload must solve cleanly"
    n_att = int((probe.n_acc.long() + probe.n_rej.long()).sum().item())
    n_acc_total = int(probe.n_acc.long().sum().item())
    n_acc_max = int(probe.n_acc.max().item())
    # every field has both forms and the adjoint (--fwd-only drops the latter)
    with_adjoint = not args.fwd_only
    tape = tode.TapeBuffers.allocate(B, D, dtype, max(1, n_acc_max), 1, dev,
                                     stages=mlp or kind == "linear", minimal=True)

    def fwd(form, sol=None, ws=None):
        return tode.solve(field, y0, t0, t1, te, form=form, tape=tape, out=sol, workspace=ws,
                          **(opt if form == "fused" else opt_plain))

    def step(form, sol=None, ws=None, scratch=None):
        s = fwd(form, sol, ws)
        return s, tode.adjoint(field, t0, t1, te, s, tape, gye, gyf, scratch=scratch,
                               **(opt if form == "fused" else opt_plain))

    # matched error: both forms against the exact solution of the same batch
    sol_f = fwd("fused")
    sol_p = fwd("plain")
    torch.cuda.synchronize()
    same = bool(torch.equal(sol_f.y_eval, sol_p.y_eval)) if sol_p is not None else None
    err = None
    if kind == "linear":
        Q, lam = w["field"]["Q"], w["field"]["lam"]
        c = np.einsum("bji,bj->bi", Q, w["y0"])
        ex = np.exp(-lam[:, None, :] * w["t_eval"][:, :, None])
        exact = np.einsum("bij,bkj->bki", Q, ex * c[:, None, :])
        ye = sol_f.y_eval.double().cpu().numpy()
        err = float(np.max(np.abs(ye - exact) / (w["atol"] + w["rtol"] * np.abs(exact))))

    def capture(fn):
        """A CUDA graph of the work fn enqueues (fn runs once outside the
        capture first); None when the calls cannot be captured."""
        if args.no_graph:
            return None
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            fn()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        try:
            with torch.cuda.graph(g):
                fn()
        except RuntimeError as e:  # report it in the JSON line and time eagerly
            graph_notes.append(str(e).splitlines()[0][:160])
            torch.cuda.synchronize()
            return None
        return g

    graph_notes = []

    def runner(form, with_adj, sol, ws):
        """One pass as the timed loop issues it: the fused form as a CUDA
        graph replay (host launch cost off the device timeline), the plain
        form eagerly (its host loop polls the device for completion)."""
        def eager():
            return step(form, sol, ws) if with_adj else fwd(form, sol, ws)
        g = capture(eager) if form == "fused" else None
        return (g.replay, True) if g is not None else (eager, False)

    def timed(form, nsteps, with_adj=True):
        sol = fwd(form)
        ws = sol.extra["workspace"]
        run, graphed = runner(form, with_adj, sol, ws)
        for _ in range(args.warmup):
            run()
        torch.cuda.synchronize()
        ev = _events(torch, nsteps)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        for k in range(nsteps):
            flush.zero_()  # L2 flush, outside the timed events
            ev[k][0].record(stream)
            run()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_wall
        ms = float(sum(a.elapsed_time(b) for a, b in ev))
        if world > 1:  # the slowest rank's time (instances are independent: no other exchange)
            ms = max_over_ranks(ms, dev)
            dist.barrier()
        return ms, wall, graphed

    def kernel_ms(nrep, adjoint_only):
        """Device time of the fused forward alone, or of the adjoint alone
        (its work-order kernel included), replayed from a CUDA graph."""
        sol = fwd("fused")
        ws = sol.extra["workspace"]
        torch.cuda.synchronize()
        if adjoint_only:
            def eager():
                return tode.adjoint(field, t0, t1, te, sol, tape, gye, gyf, **opt)
        else:
            def eager():
                return fwd("fused", sol, ws)
        g = capture(eager)
        run = g.replay if g is not None else eager
        run()
        torch.cuda.synchronize()
        ev = _events(torch, nrep)
        for k in range(nrep):
            flush.zero_()
            ev[k][0].record(stream)
            run()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    nk = max(1, args.kernel_reps)
    with ClockSampler(local) as clk:
        ms_fused, wall_fused, graphed = timed("fused", args.steps, with_adjoint)
        k_fwd_ms = kernel_ms(nk, False)
        k_adj_ms = kernel_ms(nk, True) if with_adjoint else None
    clocks = clk.summary()
    ms_fused_fwd, _, _ = timed("fused", nk, False)
    ms_plain, _, _ = timed("plain", args.plain_steps, with_adjoint)
    ms_plain_fwd, _, _ = timed("plain", args.plain_steps, False)

    per_step = ms_fused / args.steps
    value = world * n_att / (per_step * 1e-3)

    # end to end through the public API with pinned host buffers: every step
    # copies its inputs host -> device, solves + reverses, and copies its
    # results back; two buffer sets let step k+1's input copy and step k-1's
    # output copy overlap step k's kernels (three streams)
    e2e = None
    if not args.no_e2e:
        src = dict(y0=y0, t0=t0, t1=t1, te=te)
        src.update(gye=gye, gyf=gyf)
        if mlp:
            src.update({f"W{l}": x for l, x in enumerate(field.W)})
        else:
            src.update(P=field.params())
        host = {k: v.cpu().pin_memory() for k, v in src.items()}
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        NBUF = 2
        bufs = []
        for _ in range(NBUF):
            d_in = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
            if kind == "linear":
                f_b = tode.Linear(d_in["P"])
            elif mlp:
                f_b = tode.MLP([d_in[f"W{l}"] for l in range(len(field.W))], field.b, split=True)
            else:
                f_b = tode.VdP(d_in["P"])
            bufs.append(dict(d_in=d_in, field=f_b, sol=None, out_h={},
                             ev_in=torch.cuda.Event(), ev_done=torch.cuda.Event(),
                             ev_out=torch.cuda.Event()))
        ws_e2e = [None]

        def issue(k):
            bb = bufs[k % NBUF]
            with torch.cuda.stream(s_in):
                s_in.wait_event(bb["ev_done"])  # step k-NBUF no longer reads the inputs
                for name, v in host.items():
                    bb["d_in"][name].copy_(v, non_blocking=True)
                bb["ev_in"].record(s_in)
            with torch.cuda.stream(s_cmp):
                s_cmp.wait_event(bb["ev_in"])
                s_cmp.wait_event(bb["ev_out"])  # step k-NBUF's results are copied out
                d = bb["d_in"]
                sl = tode.solve(bb["field"], d["y0"], d["t0"], d["t1"], d["te"], form="fused",
                                tape=tape, out=bb["sol"], workspace=ws_e2e[0], stream=s_cmp,
                                **opt)
                bb["sol"] = sl
                ws_e2e[0] = sl.extra["workspace"]
                res = dict(y_eval=sl.y_eval, y_final=sl.y_final, n_acc=sl.n_acc,
                           n_rej=sl.n_rej, n_feval=sl.n_feval, status=sl.status)
                if with_adjoint:
                    g0, gp, _ = tode.adjoint(bb["field"], d["t0"], d["t1"], d["te"], sl, tape,
                                             d["gye"], d["gyf"], stream=s_cmp, **opt)
                    res["gy0"] = g0
                    if mlp:  # (gW, gb) lists of the MLP field
                        res.update({f"gW{l}": x for l, x in enumerate(gp[0])})
                        res.update({f"gb{l}": x for l, x in enumerate(gp[1])})
                    else:
                        res["gp"] = gp
                bb["ev_done"].record(s_cmp)
            with torch.cuda.stream(s_out):
                s_out.wait_event(bb["ev_done"])
                for name, v in res.items():
                    if name not in bb["out_h"]:
                        bb["out_h"][name] = torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
                    bb["out_h"][name].copy_(v, non_blocking=True)
                    v.record_stream(s_out)
                bb["ev_out"].record(s_out)

        for bb in bufs:  # events start out complete
            for e in ("ev_done", "ev_out"):
                bb[e].record(torch.cuda.current_stream())
        for k in range(max(args.warmup, NBUF)):
            issue(k)
        torch.cuda.synchronize()
        d2h = sum(v.numel() * v.element_size() for v in bufs[0]["out_h"].values())
        e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_start.record(s_in)
        for k in range(nk):
            issue(k)
        s_in.wait_stream(s_out)
        e_end.record(s_in)
        torch.cuda.synchronize()
        ms_e2e = e_start.elapsed_time(e_end) / nk
        if world > 1:
            ms_e2e = max_over_ranks(ms_e2e, dev)
        e2e = {"value": world * n_att / (ms_e2e * 1e-3), "unit": "instance-steps/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": ms_e2e,
               "pipelining": f"{NBUF} buffer sets, copies on their own streams"}

    peaks, src = _peaks()
    clk_mhz = peaks.get("sm_max_mhz", 2032.0)
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = n_sms * 128 * 2 * clk_mhz * 1e6 / 1e12  # TFLOP/s, FMA = 2 FLOPs
    if mlp:
        # tensor-bound: algorithmic FLOPs of the field and of its VJP
        wd = [x.shape[1] for x in w["field"]["W"]] + [w["field"]["W"][-1].shape[0]]
        S = sum(wd[l] * wd[l + 1] for l in range(len(wd) - 1))  # MACs of one evaluation
        peak = peaks["bf16_tflops"]
        net = f"D={D},H={wd[1]},{len(wd) - 2} hidden layers,split"
        kf = {"achieved": 6 * 2 * S * n_att / (k_fwd_ms * 1e-3) / 1e12,
              "kernel": f"k_mlp_fused<{net}> (fused forward)", "kernel_ms": k_fwd_ms}
        # per accepted step, at each of the 7 recorded stage inputs: the
        # hidden activations (2 S_hid) and the transposed products dX + dW
        # (2 x 2S); the output layer is not re-evaluated
        S_hid = sum(wd[l] * wd[l + 1] for l in range(len(wd) - 2))
        ka = {"achieved": 7 * (2 * S_hid + 4 * S) * n_acc_total / (k_adj_ms * 1e-3) / 1e12,
              "kernel": f"k_mlp_adjoint<{net}>", "kernel_ms": k_adj_ms} if with_adjoint else None
        for r in (kf, ka) if with_adjoint else (kf,):
            r.update(bound="tensor", peak=peak, unit="TFLOP/s", frac=r["achieved"] / peak,
                     traffic=_traffic(w["name"], r["kernel"]),
                     peak_source=f"bf16 burst, {src} (MEASURED_PEAKS.json)")
    else:
        psrc = f"derived: {n_sms} SMs x 128 FP32 lanes x 2 x {clk_mhz:.0f} MHz"
        tn = "double" if dtype == torch.float64 else "float"
        if kind == "linear":  # lanes per instance: the launch's group (default 8 for D = 16,
            # D for D <= 8, 16 for D = 32); the stride-1 adjoint of D = 16 takes 16
            g = int(opt.get("group") or 0) or {16: 8, 32: 16}.get(D, D)
            ga = 16 if D == 16 else g
            fld = f"LinearField<{tn},{D // g},{g}>"
            adj = f"LinearAdj<{tn},{D // ga},{ga}>"
        else:
            fld, adj = f"VdpField<{tn}>", f"VdpAdj<{tn}>"
        kf = {"achieved": flops_per_attempt(kind, D) * n_att / (k_fwd_ms * 1e-3) / 1e12,
              "kernel": f"k_fused<{fld}> (fused forward)", "kernel_ms": k_fwd_ms}
        ka = {"achieved": adjoint_flops_per_step(kind, D, kind == "linear") * n_acc_total
              / (k_adj_ms * 1e-3)
              / 1e12, "kernel": f"k_adjoint_steps<{adj}> (stride-1 tape)", "kernel_ms": k_adj_ms}
        for r in (kf, ka):
            r.update(bound="alu", peak=fp32_peak, unit="TFLOP/s",
                     frac=r["achieved"] / fp32_peak, traffic=_traffic(w["name"], r["kernel"]),
                     peak_source=psrc)
    # the dominant kernel of the timed step (forward + adjoint) is the roofline line
    if with_adjoint:
        roofline, other = (ka, kf) if k_adj_ms >= k_fwd_ms else (kf, ka)
    else:
        roofline, other = kf, None
    breakdown = {
        "fused_fwd": world * n_att / (ms_fused_fwd / nk * 1e-3),
        "max_err_over_tol_vs_closed_form": err,
        "fused_equals_plain_bitwise": same,
        "instance_steps_per_pass": n_att,
        "other_kernel_roofline": other,
    }
    if with_adjoint:
        breakdown.update({
            "fused_fwd_adj": value,
            "adjoint_kernel_ms": k_adj_ms,
            "accepted_steps_per_pass": n_acc_total,
        })
    breakdown.update({
        "plain_fwd_adj": world * n_att / (ms_plain / args.plain_steps * 1e-3),
        "plain_fwd": world * n_att / (ms_plain_fwd / args.plain_steps * 1e-3),
        "fused_over_plain_fwd_adj": (ms_plain / args.plain_steps) / per_step,
        "fused_over_plain_fwd": (ms_plain_fwd / args.plain_steps) / (ms_fused_fwd / nk),
    })
    # our kernels per timed step: the fused forward (+ one weight-image build
    # for the MLP; for the SIMT fields the work-order sort when the launch
    # orders longest first) and the adjoint (SIMT fields: the longest-first
    # sort and the reverse sweep; MLP D=32: image, adjoint, ordered dW
    # reduction; wide MLP: two images, the stable work order, per batch slice
    # the reverse sweep and the weight-gradient products, and their ordered
    # reduction).  The sort is one launch up to 2048 instances, three above.
    if mlp:
        adj = (4 + 2 * -(-B // (148 * 64))) if D == 64 else 3
        gpu_launches = 2 + (adj if with_adjoint else 0)
    else:
        sort = 1 if B <= 2048 else 3
        fwd_sort = sort if int(opt.get("order") or 0) == 1 else 0
        gpu_launches = 1 + fwd_sort + ((1 + sort) if with_adjoint else 0)
    result = {
        "metric": METRIC, "value": value, "unit": "instance-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 (field, split activations) / f32 state" if mlp else "f32",
        "data": "synthetic (seeded, shaped like the paper's workloads)",
        "config": {"workload": w["name"], "B": B, "D": D, "K": K, "rtol": w["rtol"],
                   "atol": w["atol"], "form": "fused",
                   "pass": "fwd+adjoint" if with_adjoint else "fwd",
                   "state": "f32 (compensated), time f64", "controller": "I (beta1=0.2)",
                   "l2": "flushed between timed steps (256 MiB write outside the events)",
                   "parallelism": f"dp{world} (independent replicas of the batch)",
                   "launch": tuned if tuned is not None else "defaults",
                   "launch_plain": tuned_plain if tuned_plain is not None else "defaults",
                   "issue": ("fused step replayed as one CUDA graph (forward + adjoint), "
                             "plain form from its host loop" if graphed else
                             "eager calls (graph capture off or unavailable)")
                   + ("; capture: " + "; ".join(graph_notes) if graph_notes else "")},
        "gpu_launches": gpu_launches * args.steps,
        "clocks": clocks, "e2e": e2e, "roofline": roofline, "breakdown": breakdown,
        "wall_s_timed_region": wall_fused,
    }
    if rank == 0 and not args.no_cpu and world == 1:
        result["cpu_baseline"] = cpu_baseline(w, budget_s=12.0, with_adjoint=with_adjoint)
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


# ------------------------------------------------------------------ CPU oracle
_PREFIX = {}


def cpu_baseline(w, budget_s=12.0, nthreads=0, with_adjoint=True, n_fixed=None):
    """The FP64 oracle as it stands (forward, + adjoint when the GPU pass has
    one) on a seeded prefix of the same workload, sized to take roughly
    `budget_s` seconds (or on the first `n_fixed` instances, once)."""
    import oracle
    from oracle.oracle import mesh_from_trace

    def run(n):
        key = (w["cfg"], n)
        if key not in _PREFIX:  # generated once, outside the timing
            _PREFIX[key] = workloads.make(w["cfg"], n)
        ws = _PREFIX[key]
        t = time.perf_counter()
        r = oracle.solve(ws["field"], ws["y0"], ws["t0"], ws["t1"], ws["t_eval"],
                         dict(rtol=ws["rtol"], atol=ws["atol"]), trace_cap=8192,
                         nthreads=nthreads)
        if with_adjoint:
            mt, mh, mn = mesh_from_trace(r)
            K, D = ws["t_eval"].shape[1], ws["y0"].shape[1]
            rng = np.random.default_rng(1)
            oracle.adjoint(ws["field"], ws["y0"], ws["t0"], ws["t1"], mt, mh, mn, ws["t_eval"],
                           rng.standard_normal((n, K, D)), rng.standard_normal((n, D)),
                           nthreads=nthreads)
        dt = time.perf_counter() - t
        return int((r["n_acc"] + r["n_rej"]).sum()), dt, r["threads"]

    if n_fixed is not None:
        n = n_fixed
        att, dt, thr = run(n)
        return {"value": att / dt, "unit": "instance-steps/s", "cores": thr, "kind": "oracle",
                "n": n, "sample": f"first {n} of {w['B']} instances of {w['name']}, "
                                  f"{'fwd+adjoint' if with_adjoint else 'fwd'}, {dt:.2f} s"}
    n = 64
    att, dt, thr = run(n)
    while dt < budget_s / 4 and n < w["B"]:
        n = min(w["B"], int(n * max(2.0, budget_s / max(dt, 1e-3) * 0.8)))
        att, dt, thr = run(n)
    passes = 1
    while dt < budget_s / 2:  # the whole workload is quick: repeat it
        a2, d2, thr = run(n)
        att, dt, passes = att + a2, dt + d2, passes + 1
    return {"value": att / dt, "unit": "instance-steps/s", "cores": thr, "kind": "oracle",
            "n": n, "sample": f"first {n} of {w['B']} instances of {w['name']}"
                      f"{f' x {passes} passes' if passes > 1 else ''}, "
                      f"{'fwd+adjoint' if with_adjoint else 'fwd'}, {dt:.1f} s"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on the host cores."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    w = workloads.make(args.workload)
    # one step: the oracle on a fixed prefix of the workload, sized once so
    # that the whole run stays near 90 s of oracle time
    n = cpu_baseline(w, budget_s=min(2.0, 90.0 / max(args.steps, 1)))["n"]
    for _ in range(args.warmup):
        cpu_baseline(w, n_fixed=n)
    vals = []
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(w, n_fixed=n)
        vals.append(last["value"])
    wall = time.perf_counter() - t0
    v = float(np.mean(vals))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "instance-steps/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": wall / max(args.steps, 1) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded, shaped like the paper's workloads)",
        "config": {"workload": w["name"], "B": w["B"], "pass": "fwd+adjoint",
                   "form": "oracle (scalar C, one thread per core)"},
        "cpu_baseline": {"value": v, "unit": "instance-steps/s", "cores": last["cores"],
                         "kind": "oracle", "sample": last["sample"]},
        "e2e": {"value": v, "unit": "instance-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


if __name__ == "__main__":
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    elif a.joint:
        run_joint(a)
    else:
        run_tode(a)
