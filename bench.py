"""Benchmark: batched adaptive dopri5 instance-steps/s, forward + discrete
adjoint, fused persistent form vs plain per-step form, on one B300.

Default line: the wide MLP neural ODE (D = 64, three tanh layers of 512,
BF16 weights with split activations, FP32 state / FP64 time, B = 65,536,
32 t_eval, rtol = atol = 1e-5) -- the largest single-GPU configuration.  One
"step" is one pass of the whole solver path over the batch: the fused
forward solve (stages, error norm, PI control, dense output, checkpoint
tape) followed by the discrete adjoint of L = <c, y(t_eval)> + <d, y(t1)>
for fixed seeded cotangents c, d (dL/dy0 and every weight and bias
gradient).  An instance-step is one attempted step of a live instance.

The line also carries:
  configs  every workload (FP64 Van der Pol, linear D=16, stiffness-mixed
           Van der Pol, MLP D=32, the wide MLP, and the paper's own Van der
           Pol setup as context): fused and plain form, forward and forward
           + adjoint, their ratio, the dominant kernel's roofline, and both
           forms' error against an FP64 reference (closed form for the
           linear field, the FP64 oracle at 1e-12 on a stated sample
           elsewhere; the oracle runs in the CPU leg only)
  peaks    the FP32, FP32x2, FP64 and MUFU (ex2, tanh) rates and the
           empty-kernel launch and graph-replay rates, measured here by the
           library's micro-benchmark kernels, with the SM clock seen

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       [--workload 0..5 (one workload's line)] [--joint]
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
HEADLINE = 5          # the wide MLP: the largest configuration that fits one GPU
CONFIG_ORDER = (1, 2, 3, 4, 5, 0)
# the paper's own number for the Van der Pol loop-time setup (App. A, Table 3:
# torchode-JIT 1.629 ms per step for 256 instances on a GTX 1080 Ti), as
# instance-steps/s -- context for that config only, another machine
PAPER_VDP_JIT = {"instance_steps_per_s": 256 / 1.629e-3, "hardware": "GTX 1080 Ti",
                 "source": "App. A, Table 3 (torchode-JIT loop time)"}
FP64_FLOP_PER_ATTEMPT_VDP = 200  # the FP64 Van der Pol attempt (stages, norm, controller)


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="tode", choices=["tode", "reference"])
    p.add_argument("--workload", type=int, default=-1,
                   help="one workload's line (0..5); default: the headline with every config")
    p.add_argument("--config-steps", type=int, default=0,
                   help="timed passes per config entry (default min(steps, 10))")
    p.add_argument("--plain-steps", type=int, default=0,
                   help="timed plain-form passes (default: the config steps)")
    p.add_argument("--batch", type=int, default=0, help="instances (default: the workload's)")
    p.add_argument("--kernel-reps", type=int, default=10)
    p.add_argument("--fwd-only", action="store_true", help="time the forward solve alone")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true", help="no CPU leg (baseline, FP64 errors)")
    p.add_argument("--no-peaks", action="store_true")
    p.add_argument("--order", type=int, default=0, choices=[0, 1],
                   help="work order of the SIMT solvers: 0 index, 1 longest interval first")
    p.add_argument("--no-graph", action="store_true",
                   help="issue the fused step eagerly instead of replaying a CUDA graph")
    p.add_argument("--no-autotune", action="store_true",
                   help="library default launch shapes instead of the autotuner's choice")
    p.add_argument("--launch", default="",
                   help="explicit launch options of the fused form, e.g. group=16,block=256")
    p.add_argument("--joint", action="store_true",
                   help="the batching experiment of Sec. 4.1: one batch of strongly damped "
                        "oscillators solved jointly (one stacked problem) and independently")
    a = p.parse_args()
    a.config_steps = a.config_steps or min(a.steps, 10)
    a.plain_steps = a.plain_steps or a.config_steps
    return a


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
    # dram__bytes_read.sum + dram__bytes_write.sum per launch, from the
    # captures summarised under profiles/ (launch shapes as given there)
    ("vdp_f64_b256", "k_fused<VdpField<double>>"): 0.141e6,
    ("linear_d16_b8192", "k_fused<LinearField<float,1,16>>"): 28.11e6,
    ("linear_d16_b8192", "k_adjoint_steps<LinearAdj<float,1,16>>"): 86.32e6,
    # captured on the first 32,768 instances, x8 (the tape grows with the steps)
    ("vdp_mix_b262144", "k_fused<VdpField<float>>"): 8 * 93.10e6,
    ("vdp_mix_b262144", "k_adjoint_steps<VdpAdj<float>>"): 8 * 123.80e6,
    ("mlp_d32_h128", "k_mlp_fused"): 11.17e6,
    ("mlp_d32_h128", "k_mlp_adjoint"): 48.45e6,
    # full size (B = 65,536), one pass per launch: the forward launch, and the
    # sum over the 16 launches of one adjoint call (the call is the entry)
    ("mlp_d64_h512", "k_mlp_fused"): 1066.11e6,
    ("mlp_d64_h512", "k_mlp_adjoint"): 53.981e9,
    ("vdp_joint_mu10_b2097152", "k_joint_step<VdpField<float>>"): 69.76e6,
}


def _traffic(workload: str, kernel: str):
    for (wl, prefix), v in TRAFFIC.items():
        if wl == workload and kernel.startswith(prefix):
            return v
    return None


def _peaks_file():
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


def _launch_opts(s: str) -> dict:
    out = {}
    for kv in filter(None, s.split(",")):
        k, v = kv.split("=")
        out[k.strip()] = int(v)
    return out


# ------------------------------------------------------------------ peaks (K7)
def measure_peaks(torch, dev, local):
    """The rooflines' denominators on this GPU, from the library's
    micro-benchmark kernels: FP32 / FP32x2 / FP64 FMA rates, MUFU ex2 and
    tanh rates (8 independent chains per thread, 4 CTAs of 256 threads per
    SM), the rate of eager empty-kernel launches and of empty kernels
    replayed from a CUDA graph; CUDA events on the launching stream, the SM
    clock sampled meanwhile."""
    import ctypes as C
    from paper_2210_12375_b300 import _abi
    lib = _abi.load()
    stream = torch.cuda.current_stream()
    sh = C.c_void_p(stream.cuda_stream)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.zeros(1024, dtype=torch.float32, device=dev)
    grid, block = 4 * sms, 256

    def run(kind, iters, reps=5):
        def launch():
            _abi.check(lib.tode_peak_kernel(kind, grid, block, iters,
                                            C.c_void_p(sink.data_ptr()), sh), "peak")
        for _ in range(2):
            launch()
        torch.cuda.synchronize()
        ev = _events(torch, reps)
        for a, b in ev:
            a.record(stream)
            launch()
            b.record(stream)
        torch.cuda.synchronize()
        ms = min(a.elapsed_time(b) for a, b in ev)
        return grid * block * iters * 8 / (ms * 1e-3)  # operations per second

    out = {}
    n = 2000
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        out["fp32_tflops"] = 2 * run(_abi.TODE_PEAK_FMA32, 16384) / 1e12
        out["ffma2_tflops"] = 4 * run(_abi.TODE_PEAK_FFMA2, 8192) / 1e12
        out["fp64_tflops"] = 2 * run(_abi.TODE_PEAK_FMA64, 1024) / 1e12
        out["mufu_ex2_gops"] = run(_abi.TODE_PEAK_EX2, 4096) / 1e9
        out["mufu_tanh_gops"] = run(_abi.TODE_PEAK_TANH, 4096) / 1e9

        def empties(st):
            for _ in range(n):
                lib.tode_peak_kernel(_abi.TODE_PEAK_EMPTY, 1, 32, 0, None, st)
        empties(sh)
        torch.cuda.synchronize()
        a, b = _events(torch, 1)[0]
        a.record(stream)
        empties(sh)
        b.record(stream)
        torch.cuda.synchronize()
        out["launch_per_s"] = n / (a.elapsed_time(b) * 1e-3)
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(g):
                empties(C.c_void_p(torch.cuda.current_stream().cuda_stream))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        a, b = _events(torch, 1)[0]
        a.record(stream)
        g.replay()
        b.record(stream)
        torch.cuda.synchronize()
        out["graph_node_per_s"] = n / (a.elapsed_time(b) * 1e-3)
        out["wall_s"] = time.perf_counter() - t0
    out["clocks"] = clk.summary()
    mhz = out["clocks"]["sm_mhz"]
    if mhz:
        # the per-SM, per-clock rates these imply (time x MHz)
        out["fp32_flop_per_clk_per_sm"] = out["fp32_tflops"] * 1e12 / (sms * mhz * 1e6)
        out["fp64_flop_per_clk_per_sm"] = out["fp64_tflops"] * 1e12 / (sms * mhz * 1e6)
        out["mufu_ex2_per_clk_per_sm"] = out["mufu_ex2_gops"] * 1e9 / (sms * mhz * 1e6)
        out["mufu_tanh_per_clk_per_sm"] = out["mufu_tanh_gops"] * 1e9 / (sms * mhz * 1e6)
    out["how"] = (f"{grid} CTAs x {block} threads, 8 independent chains per thread, best of 5 "
                  f"launches; {n} empty kernels issued eagerly and replayed from one CUDA graph")
    return out


# ------------------------------------------------------------------ one workload on the GPU
class Workload:
    """One workload resident on the device: field, inputs, seeded cotangents,
    launch options (autotuned per form for the SIMT fields), its step counts
    and a stride-1 checkpoint tape."""

    def __init__(self, cfg, args, dev, batch=None):
        import torch
        import paper_2210_12375_b300 as tode
        self.torch, self.tode, self.dev, self.args = torch, tode, dev, args
        w = workloads.make(cfg, batch or None)
        self.w = w
        kind = w["field"]["kind"]
        self.kind = kind
        self.dtype = torch.float64 if w["prec"] == "f64" else torch.float32
        B, D = w["y0"].shape
        self.B, self.D, self.K = B, D, w["t_eval"].shape[1]
        self.mlp = kind == "mlp"
        if kind == "linear":
            self.field = tode.Linear(torch.tensor(w["field"]["A"], dtype=self.dtype,
                                                  device=dev).contiguous())
        elif self.mlp:
            self.field = tode.MLP([torch.tensor(x, dtype=torch.float32).to(torch.bfloat16)
                                   .to(dev).contiguous() for x in w["field"]["W"]],
                                  [torch.tensor(x, dtype=torch.float32, device=dev)
                                   for x in w["field"]["b"]], split=True)
        else:
            self.field = tode.VdP(torch.tensor(w["field"]["mu"], dtype=self.dtype, device=dev))
        self.y0 = torch.tensor(w["y0"], dtype=self.dtype, device=dev)
        self.t0 = torch.tensor(w["t0"], dtype=torch.float64, device=dev)
        self.t1 = torch.tensor(w["t1"], dtype=torch.float64, device=dev)
        self.te = torch.tensor(w["t_eval"], dtype=torch.float64, device=dev)
        rng = np.random.default_rng(20221022)
        self.gye = torch.tensor(rng.standard_normal((B, self.K, D)), dtype=self.dtype, device=dev)
        self.gyf = torch.tensor(rng.standard_normal((B, D)), dtype=self.dtype, device=dev)
        opt = dict(rtol=w["rtol"], atol=w["atol"])
        if not self.mlp:
            opt["order"] = args.order
        self.opt, self.opt_plain = dict(opt), dict(opt)
        self.tuned = self.tuned_plain = None
        if args.launch:
            self.tuned = _launch_opts(args.launch)
            self.opt.update(self.tuned)
        elif not args.no_autotune:
            # the launch shape (lanes per instance, CTA size, resident CTAs,
            # work order; for the plain form its poll interval) the
            # autotuner picks for this batch, timed on it (fwd + adjoint)
            self.tuned = tode.autotune(self.field, self.y0, self.t0, self.t1, self.te,
                                       with_adjoint=True, reps=5, **opt)
            self.tuned_plain = tode.autotune(self.field, self.y0, self.t0, self.t1, self.te,
                                             form="plain", with_adjoint=True, reps=2, **opt)
            self.opt.update(self.tuned)
            self.opt_plain.update(self.tuned_plain)
        probe = tode.solve(self.field, self.y0, self.t0, self.t1, self.te, form="fused",
                           **self.opt)
        torch.cuda.synchronize()
        assert int((probe.status != 0).sum().item()) == 0, "workload must solve cleanly"
        att = probe.n_acc.long() + probe.n_rej.long()
        self.n_att = int(att.sum().item())
        self.max_att = int(att.max().item())
        self.n_acc_total = int(probe.n_acc.long().sum().item())
        n_acc_max = int(probe.n_acc.max().item())
        self.tape = tode.TapeBuffers.allocate(B, D, self.dtype, max(1, n_acc_max), 1, dev,
                                              stages=self.mlp or kind == "linear", minimal=True)
        self.flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        self.graph_notes = []

    def fwd(self, form, sol=None, ws=None):
        return self.tode.solve(self.field, self.y0, self.t0, self.t1, self.te, form=form,
                               tape=self.tape, out=sol, workspace=ws,
                               **(self.opt if form == "fused" else self.opt_plain))

    def step(self, form, sol=None, ws=None):
        s = self.fwd(form, sol, ws)
        return s, self.tode.adjoint(self.field, self.t0, self.t1, self.te, s, self.tape,
                                    self.gye, self.gyf,
                                    **(self.opt if form == "fused" else self.opt_plain))

    def capture(self, fn):
        """A CUDA graph of the work fn enqueues (fn runs once outside the
        capture first); None when the calls cannot be captured."""
        torch = self.torch
        if self.args.no_graph:
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
        except RuntimeError as e:  # reported in the JSON line; timed eagerly
            self.graph_notes.append(str(e).splitlines()[0][:160])
            torch.cuda.synchronize()
            return None
        return g

    def timed(self, form, nsteps, with_adj, world=1):
        """ms of nsteps passes, each bracketed by CUDA events on the stream
        with an L2 flush outside: the fused form replayed as one CUDA graph
        (host launch cost off the device timeline), the plain form from its
        host loop (it polls the device for completion)."""
        torch = self.torch
        import torch.distributed as dist
        stream = torch.cuda.current_stream()
        sol = self.fwd(form)
        ws = sol.extra["workspace"]

        def eager():
            return self.step(form, sol, ws) if with_adj else self.fwd(form, sol, ws)
        g = self.capture(eager) if form == "fused" else None
        run = g.replay if g is not None else eager
        for _ in range(self.args.warmup):
            run()
        torch.cuda.synchronize()
        ev = _events(torch, nsteps)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        for k in range(nsteps):
            self.flush.zero_()  # L2 flush, outside the timed events
            ev[k][0].record(stream)
            run()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_wall
        ms = float(sum(a.elapsed_time(b) for a, b in ev))
        if world > 1:  # the slowest rank's time (instances are independent)
            ms = max_over_ranks(ms, self.dev)
            dist.barrier()
        return ms, wall, g is not None, sol

    def kernel_ms(self, nrep, adjoint_only):
        """Device time of the fused forward call alone, or of the adjoint call
        alone, replayed from a CUDA graph (mean over nrep, L2 flushed)."""
        torch = self.torch
        stream = torch.cuda.current_stream()
        sol = self.fwd("fused")
        ws = sol.extra["workspace"]
        torch.cuda.synchronize()
        if adjoint_only:
            def eager():
                return self.tode.adjoint(self.field, self.t0, self.t1, self.te, sol, self.tape,
                                         self.gye, self.gyf, **self.opt)
        else:
            def eager():
                return self.fwd("fused", sol, ws)
        g = self.capture(eager)
        run = g.replay if g is not None else eager
        run()
        torch.cuda.synchronize()
        ev = _events(torch, nrep)
        for k in range(nrep):
            self.flush.zero_()
            ev[k][0].record(stream)
            run()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    def rooflines(self, k_fwd_ms, k_adj_ms, fp32_peak, fp32_src, fp64=None):
        """The forward's and the adjoint's rooflines: tensor (BF16) for the
        MLP field, the FP32 pipe (measured here) for the SIMT fields."""
        w, D = self.w, self.D
        peaks, src = _peaks_file()
        if self.mlp:
            wd = [x.shape[1] for x in w["field"]["W"]] + [w["field"]["W"][-1].shape[0]]
            S = sum(wd[l] * wd[l + 1] for l in range(len(wd) - 1))  # MACs of one evaluation
            S_hid = sum(wd[l] * wd[l + 1] for l in range(len(wd) - 2))
            net = f"D={D},H={wd[1]},{len(wd) - 2} hidden layers,split"
            wide = D == 64
            kf = {"achieved": 6 * 2 * S * self.n_att / (k_fwd_ms * 1e-3) / 1e12,
                  "kernel": f"k_mlp_fused<{net}> (fused forward call)", "kernel_ms": k_fwd_ms}
            # per accepted step, at each of the 7 recorded stage inputs: the
            # hidden activations (2 S_hid) and the transposed products dX + dW
            # (2 x 2S); the output layer is not re-evaluated
            ka = None
            if k_adj_ms is not None:
                ka = {"achieved": 7 * (2 * S_hid + 4 * S) * self.n_acc_total
                      / (k_adj_ms * 1e-3) / 1e12,
                      "kernel": (f"k_mlp_adjoint<{net}> call: " + (
                          "k_order_steps_stable, per batch slice k_mlp_adjoint_wide + k_mlp_dw, "
                          "k_mlp_dw_reduce" if wide else "k_mlp_adjoint + k_mlp_grad_reduce")),
                      "kernel_ms": k_adj_ms}
            for r in (kf, ka):
                if r is None:
                    continue
                r.update(bound="tensor", peak=peaks["bf16_tflops"], unit="TFLOP/s",
                         frac=r["achieved"] / peaks["bf16_tflops"],
                         traffic=_traffic(w["name"], r["kernel"]),
                         peak_source=f"bf16 burst, MEASURED_PEAKS.json; of {src}")
        else:
            tn = "double" if self.dtype == self.torch.float64 else "float"
            if self.kind == "linear":
                g = int(self.opt.get("group") or 0) or {16: 8, 32: 16}.get(D, D)
                ga = 16 if D == 16 else g
                fld, adj = f"LinearField<{tn},{D // g},{g}>", f"LinearAdj<{tn},{D // ga},{ga}>"
            else:
                fld, adj = f"VdpField<{tn}>", f"VdpAdj<{tn}>"
            kf = {"achieved": flops_per_attempt(self.kind, D) * self.n_att / (k_fwd_ms * 1e-3)
                  / 1e12, "kernel": f"k_fused<{fld}> (fused forward)", "kernel_ms": k_fwd_ms}
            ka = None
            if k_adj_ms is not None:
                ka = {"achieved": adjoint_flops_per_step(self.kind, D, self.kind == "linear")
                      * self.n_acc_total / (k_adj_ms * 1e-3) / 1e12,
                      "kernel": f"k_adjoint_steps<{adj}> (stride-1 tape)", "kernel_ms": k_adj_ms}
            # FP64 state: the FP64 pipe's measured peak (when measured), else FP32's
            pk, src_ = fp64 if (tn == "double" and fp64) else (fp32_peak, fp32_src)
            for r in (kf, ka):
                if r is None:
                    continue
                r.update(bound="alu", peak=pk, unit="TFLOP/s", frac=r["achieved"] / pk,
                         traffic=_traffic(w["name"], r["kernel"]), peak_source=src_)
        return kf, ka


def measure(cfg, args, dev, fp32_peak, fp32_src, world=1, headline=False, peaks=None):
    """Fused and plain form, forward and forward + adjoint, on one workload;
    the outputs of both forms on the error sample are kept for the CPU leg."""
    torch = __import__("torch")
    wl = Workload(cfg, args, dev, args.batch if headline else None)
    steps = args.steps if headline else args.config_steps
    with_adj = not args.fwd_only
    clocks = None
    if headline:
        with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
            ms_f, wall_f, graphed, sol_f = wl.timed("fused", steps, with_adj, world)
        clocks = clk.summary()
    else:
        ms_f, wall_f, graphed, sol_f = wl.timed("fused", steps, with_adj, world)
    k_fwd = wl.kernel_ms(args.kernel_reps, False)
    k_adj = wl.kernel_ms(args.kernel_reps, True) if with_adj else None
    if with_adj:
        ms_ff = wl.timed("fused", steps, False, world)[0]
    else:
        ms_ff = ms_f
    ms_p, _, _, sol_p = wl.timed("plain", args.plain_steps, with_adj, world)
    ms_pf = wl.timed("plain", args.plain_steps, False, world)[0] if with_adj else ms_p
    fp64 = ((peaks["fp64_tflops"], "measured here: FP64 FMA micro-benchmark (tode_peak_kernel)")
            if peaks else None)
    kf, ka = wl.rooflines(k_fwd, k_adj, fp32_peak, fp32_src, fp64=fp64)
    dom, other = ((ka, kf) if (ka is not None and k_adj >= k_fwd) else (kf, ka))
    per = ms_f / steps
    n = world * wl.n_att
    entry = {
        "B": wl.B, "D": wl.D, "K": wl.K, "rtol": wl.w["rtol"],
        "state": {"f64": "f64", "f32": "f32 (compensated), time f64",
                  "bf16w": "bf16 field (split activations), f32 state, time f64"}[wl.w["prec"]],
        "instance_steps_per_pass": wl.n_att, "accepted_steps_per_pass": wl.n_acc_total,
        "max_attempts": wl.max_att,
        ("fused_fwd_adj" if with_adj else "fused_fwd"): n / (per * 1e-3),
        "fused_fwd": n / (ms_ff / steps * 1e-3),
        ("plain_fwd_adj" if with_adj else "plain_fwd"): n / (ms_p / args.plain_steps * 1e-3),
        "plain_fwd": n / (ms_pf / args.plain_steps * 1e-3),
        "fused_over_plain_fwd_adj": (ms_p / args.plain_steps) / per if with_adj else None,
        "fused_over_plain_fwd": (ms_pf / args.plain_steps) / (ms_ff / steps),
        "ms_per_pass_fused": per, "ms_per_pass_plain": ms_p / args.plain_steps,
        "fused_equals_plain_bitwise": bool(torch.equal(sol_f.y_eval, sol_p.y_eval)),
        "roofline": dom, "other_kernel_roofline": other,
        "launch": wl.tuned if wl.tuned is not None else "defaults",
        "launch_plain": wl.tuned_plain if wl.tuned_plain is not None else "defaults",
    }
    if peaks and wl.dtype == torch.float64 and wl.kind == "vdp":
        # FP64 Van der Pol: the fused forward against the measured FP64 pipe,
        # the plain form (one launch per attempt of the slowest instance, the
        # host polling every poll_every launches) against the eager launch rate
        poll = int(wl.opt_plain.get("poll_every") or 16)
        plain_launches = 1 + -(-(wl.max_att + 1) // poll) * poll
        fwd_plain_ms = ms_pf / args.plain_steps
        entry["fp64_roofline"] = {
            "bound": "fp64", "kernel": kf["kernel"], "kernel_ms": k_fwd,
            "achieved": FP64_FLOP_PER_ATTEMPT_VDP * wl.n_att / (k_fwd * 1e-3) / 1e12,
            "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
            "frac": FP64_FLOP_PER_ATTEMPT_VDP * wl.n_att / (k_fwd * 1e-3) / 1e12
            / peaks["fp64_tflops"], "peak_source": "measured here (tode_peak_kernel FP64 FMA)"}
        entry["plain_launch_bound"] = {
            "launches_per_pass": plain_launches,
            "achieved_launch_per_s": plain_launches / (fwd_plain_ms * 1e-3),
            "peak_launch_per_s": peaks["launch_per_s"],
            "frac": plain_launches / (fwd_plain_ms * 1e-3) / peaks["launch_per_s"]}
    idx = error_sample(wl.w)
    it = torch.tensor(idx, device=dev)
    keep = dict(idx=idx, fused=sol_f.y_eval[it].double().cpu().numpy(),
                plain=sol_p.y_eval[it].double().cpu().numpy())
    return dict(wl=wl, entry=entry, keep=keep, ms=ms_f, wall=wall_f, graphed=graphed,
                clocks=clocks, steps=steps, with_adj=with_adj)


# ------------------------------------------------------------------ joint continuous adjoint
JADJ_FLOP_PER_ROW_EVAL = 3 * 2 * (33 * 128 + 128 * 128 + 128 * 32)  # fwd, VJP, parameter products


def measure_joint_adjoint(args, dev, peaks, do_cpu):
    """The joint continuous adjoint (App. A, the CNF benchmark's
    "torchode-joint" backward pass) on the D = 32, H = 128 MLP workload: one
    adjoint equation of size 2BD + P for the whole batch, from the fused
    forward's y(t1), timed (CUDA events, L2 flushed outside) beside the
    per-instance discrete adjoint of the same gradient."""
    torch = __import__("torch")
    import paper_2210_12375_b300 as tode
    wl = Workload(4, args, dev)
    w = wl.w
    te = w["t_eval"][0]
    assert (w["t_eval"] == te).all() and (w["t0"] == w["t0"][0]).all() and \
        (w["t1"] == w["t1"][0]).all(), "a shared time axis"
    t0, t1 = float(w["t0"][0]), float(w["t1"][0])
    opt = dict(rtol=w["rtol"], atol=w["atol"])
    sol = wl.fwd("fused")
    torch.cuda.synchronize()
    y1 = sol.y_final.clone()
    ws = tode.joint_adjoint_workspace(wl.field, wl.B, wl.D, dev, **opt)

    def once():
        return tode.joint_adjoint(wl.field, y1, t0, t1, te, wl.gye, wl.gyf, workspace=ws, **opt)
    for _ in range(max(args.warmup, 1)):
        out = once()
    torch.cuda.synchronize()
    n = max(1, min(args.config_steps, 5))
    stream = torch.cuda.current_stream()
    ev = _events(torch, n)
    for k in range(n):
        wl.flush.zero_()
        ev[k][0].record(stream)
        out = once()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    st = out[3]
    ms_disc = wl.kernel_ms(args.kernel_reps, True)
    flop = st["n_feval"] * wl.B * JADJ_FLOP_PER_ROW_EVAL
    pk, src = _peaks_file()
    P = 128 * 33 + 128 + 128 * 128 + 128 + 32 * 128 + 32
    entry = {
        "B": wl.B, "D": wl.D, "K": wl.K, "rtol": w["rtol"], "t0": t0, "t1": t1,
        "augmented_size": 2 * wl.B * wl.D + P,
        "accepted": st["n_acc"], "rejected": st["n_rej"], "augmented_evaluations": st["n_feval"],
        "segments": int(((te > t0) & (te < t1)).sum()) + 1,
        "ms_joint_backward": ms, "ms_discrete_adjoint": ms_disc,
        "discrete_over_joint": ms_disc / ms,
        "roofline": {"bound": "tensor", "kernel": "k_mlp_jadj + k_mlp_jadj_decide (per attempt)",
                     "achieved": flop / (ms * 1e-3) / 1e12, "peak": pk["bf16_tflops"],
                     "unit": "TFLOP/s", "frac": flop / (ms * 1e-3) / 1e12 / pk["bf16_tflops"],
                     "flop_per_row_evaluation": JADJ_FLOP_PER_ROW_EVAL, "traffic": None,
                     "peak_source": f"bf16 burst, MEASURED_PEAKS.json; of {src}"},
        "issue": "host-synchronous: the decision read every 4 attempts, one launch pair per "
                 "attempt, restarted at every evaluation point",
    }
    if do_cpu:
        # FP64 oracle of the same joint problem on a 256-instance prefix
        import oracle
        ws_ = workloads.make(4, 256)
        r = oracle.solve(ws_["field"], ws_["y0"], ws_["t0"], ws_["t1"], ws_["t_eval"],
                         dict(rtol=1e-10, atol=1e-10))
        y1s = r["y_final"].astype(np.float32).astype(np.float64)
        gye = wl.gye[:256].double().cpu().numpy()
        gyf = wl.gyf[:256].double().cpu().numpy()
        tt = time.perf_counter()
        ref = oracle.joint_adjoint(ws_["field"], y1s, t0, t1, te, gye, gyf, opt)
        cpu_s = time.perf_counter() - tt
        f32 = lambda x: torch.tensor(x, dtype=torch.float32, device=dev)
        g = tode.joint_adjoint(wl.field, f32(y1s), t0, t1, te, wl.gye[:256].contiguous(),
                               wl.gyf[:256].contiguous(), **opt)
        rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        entry["error_vs_fp64"] = {
            "reference": "FP64 oracle joint adjoint, same y(t1), on a 256-instance prefix",
            "gy0_rel_l2": rel(g[0].double().cpu().numpy(), ref["gy0"]),
            "gW_rel_l2": [rel(x.double().cpu().numpy(), y) for x, y in zip(g[1][0], ref["gW"])],
            "accepted_gpu_vs_oracle": [g[3]["n_acc"], ref["n_acc"]], "cpu_s": cpu_s}
    return entry


# ------------------------------------------------------------------ CPU leg
def error_sample(w):
    """Instances on which the FP64 reference is computed: all of the small
    batches, a stratified (mu, t1) sample of the stiffness-mixed Van der Pol,
    evenly spaced ones of the MLP batches."""
    B = w["B"]
    if w["cfg"] == 0:
        return np.array([0])  # every instance of the paper's setup is the same
    if w["cfg"] == 3:
        order = np.lexsort((w["t1"], w["field"]["mu"]))
        return np.unique(order[np.linspace(0, len(order) - 1, min(B, 256)).astype(int)])
    if w["cfg"] == 4:
        return np.arange(0, B, max(1, B // 64))
    if w["cfg"] == 5:
        return np.arange(0, B, max(1, B // 16))
    return np.arange(B)


def _sub(w, idx):
    f = dict(w["field"])
    for k in ("mu", "A", "Q", "lam"):
        if k in f:
            f[k] = f[k][idx]
    return dict(w, field=f, y0=w["y0"][idx], t0=w["t0"][idx], t1=w["t1"][idx],
                t_eval=w["t_eval"][idx], B=len(idx))


def fp64_errors(w, keep):
    """Both forms' error against FP64, over the sample's points, of
    |y - y_ref| / (atol + rtol |y_ref|): the closed form for the linear
    field, else the FP64 oracle at rtol = atol = 1e-12.  The FP64 oracle at
    the workload's own tolerance on the same sample gives the method's error
    at that tolerance (the matched-error yardstick)."""
    import oracle
    idx = keep["idx"]
    ws = _sub(w, idx)
    t = time.perf_counter()
    if w["field"]["kind"] == "linear":
        Q, lam = ws["field"]["Q"], ws["field"]["lam"]
        c = np.einsum("bji,bj->bi", Q, ws["y0"])
        ex = np.exp(-lam[:, None, :] * ws["t_eval"][:, :, None])
        ref = np.einsum("bij,bkj->bki", Q, ex * c[:, None, :])
        what = f"closed form Q diag(exp(-lambda t)) Q^T y0, all {len(idx)} instances"
    else:
        r = oracle.solve(ws["field"], ws["y0"], ws["t0"], ws["t1"], ws["t_eval"],
                         dict(rtol=1e-12, atol=1e-12, max_steps=5_000_000))
        ref = r["y_eval"]
        what = f"FP64 oracle at 1e-12 on {len(idx)} of {w['B']} instances"
    own = oracle.solve(ws["field"], ws["y0"], ws["t0"], ws["t1"], ws["t_eval"],
                       dict(rtol=w["rtol"], atol=w["atol"]))["y_eval"]
    scale = w["atol"] + w["rtol"] * np.abs(ref)

    def stats(y):
        e = np.abs(y - ref) / scale
        return {"max": float(e.max()), "p99": float(np.quantile(e, 0.99)),
                "within_10": float((e <= 10).mean())}
    return {"reference": what, "fused": stats(keep["fused"]), "plain": stats(keep["plain"]),
            "fp64_oracle_at_tol": stats(own), "unit": "|y - y_ref| / (atol + rtol |y_ref|)",
            "cpu_s": time.perf_counter() - t}


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
    n = 16
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
                      f"{'fwd+adjoint' if with_adjoint else 'fwd'}, {dt:.1f} s "
                      f"(instances are independent: the rate extrapolates per instance)"}


# ------------------------------------------------------------------ e2e
def measure_e2e(wl, nk, world):
    """End to end through the public API with pinned host buffers: every step
    copies its inputs host -> device, solves + reverses, and copies its
    results back; two buffer sets let step k+1's input copy and step k-1's
    output copy overlap step k's kernels (three streams)."""
    torch, tode = wl.torch, wl.tode
    dev = wl.dev
    src = dict(y0=wl.y0, t0=wl.t0, t1=wl.t1, te=wl.te, gye=wl.gye, gyf=wl.gyf)
    if wl.mlp:
        src.update({f"W{l}": x for l, x in enumerate(wl.field.W)})
    else:
        src.update(P=wl.field.params())
    host = {k: v.cpu().pin_memory() for k, v in src.items()}
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    NBUF = 2
    bufs = []
    for _ in range(NBUF):
        d_in = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
        if wl.kind == "linear":
            f_b = tode.Linear(d_in["P"])
        elif wl.mlp:
            f_b = tode.MLP([d_in[f"W{l}"] for l in range(len(wl.field.W))], wl.field.b,
                           split=True)
        else:
            f_b = tode.VdP(d_in["P"])
        bufs.append(dict(d_in=d_in, field=f_b, sol=None, out_h={},
                         ev_in=torch.cuda.Event(), ev_done=torch.cuda.Event(),
                         ev_out=torch.cuda.Event()))
    ws_e2e = [None]
    with_adj = not wl.args.fwd_only

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
                            tape=wl.tape, out=bb["sol"], workspace=ws_e2e[0], stream=s_cmp,
                            **wl.opt)
            bb["sol"] = sl
            ws_e2e[0] = sl.extra["workspace"]
            res = dict(y_eval=sl.y_eval, y_final=sl.y_final, n_acc=sl.n_acc,
                       n_rej=sl.n_rej, n_feval=sl.n_feval, status=sl.status)
            if with_adj:
                g0, gp, _ = tode.adjoint(bb["field"], d["t0"], d["t1"], d["te"], sl, wl.tape,
                                         d["gye"], d["gyf"], stream=s_cmp, **wl.opt)
                res["gy0"] = g0
                if wl.mlp:  # (gW, gb) lists of the MLP field
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
    for k in range(max(wl.args.warmup, NBUF)):
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
    return {"value": world * wl.n_att / (ms_e2e * 1e-3), "unit": "instance-steps/s",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": ms_e2e,
            "pipelining": f"{NBUF} buffer sets, copies on their own streams"}


def launches_per_step(wl):
    """Kernels of the library per timed step: the fused forward (+ one
    weight-image build for the MLP; for the SIMT fields the work-order sort
    when the launch orders longest first) and the adjoint (SIMT fields: the
    longest-first sort and the reverse sweep; MLP D=32: image, adjoint,
    ordered dW reduction; wide MLP: two images, the stable work order, per
    batch slice the reverse sweep and the weight-gradient products, and
    their ordered reduction).  The sort is one launch up to 2048 instances,
    three above."""
    B, D = wl.B, wl.D
    with_adj = not wl.args.fwd_only
    if wl.mlp:
        adj = (4 + 2 * -(-B // (148 * 64))) if D == 64 else 3
        return 2 + (adj if with_adj else 0)
    sort = 1 if B <= 2048 else 3
    fwd_sort = sort if int(wl.opt.get("order") or 0) == 1 else 0
    return 1 + fwd_sort + ((1 + sort) if with_adj else 0)


# ------------------------------------------------------------------ GPU arm
def run_tode(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = None
    if not args.no_peaks:
        peaks = measure_peaks(torch, dev, local)
        fp32_peak = peaks["fp32_tflops"]
        fp32_src = (f"measured here: FP32 FMA micro-benchmark (tode_peak_kernel) at "
                    f"{peaks['clocks']['sm_mhz']} MHz median SM clock")
    else:
        clk = _peaks_file()[0].get("sm_max_mhz", 2032.0)
        fp32_peak = n_sms * 128 * 2 * clk * 1e6 / 1e12
        fp32_src = f"derived: {n_sms} SMs x 128 FP32 lanes x 2 x {clk:.0f} MHz"

    head_cfg = args.workload if args.workload >= 0 else HEADLINE
    head = measure(head_cfg, args, dev, fp32_peak, fp32_src, world, headline=True, peaks=peaks)
    wl = head["wl"]
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(wl, max(1, min(args.steps, 10)), world)
    configs = {wl.w["name"]: head["entry"]}
    kept = {wl.w["name"]: (wl.w, head["keep"])}
    if args.workload < 0:
        for cfg in CONFIG_ORDER:
            if cfg == head_cfg:
                continue
            m = measure(cfg, args, dev, fp32_peak, fp32_src, world, peaks=peaks)
            if cfg == 0:
                m["entry"]["paper"] = PAPER_VDP_JIT
            configs[m["wl"].w["name"]] = m["entry"]
            kept[m["wl"].w["name"]] = (m["wl"].w, m["keep"])
            del m
            torch.cuda.empty_cache()
    if args.workload < 0:
        configs["mlp_d32_h128_joint_adjoint"] = measure_joint_adjoint(
            args, dev, peaks, rank == 0 and not args.no_cpu and world == 1)
        torch.cuda.empty_cache()
    steps = head["steps"]
    per_step = head["ms"] / steps
    value = world * wl.n_att / (per_step * 1e-3)
    entry = head["entry"]
    result = {
        "metric": METRIC, "value": value, "unit": "instance-steps/s", "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f64": "f64", "f32": "f32",
                  "bf16w": "bf16 (field, split activations) / f32 state"}[wl.w["prec"]],
        "data": "synthetic (seeded, shaped like the paper's workloads)",
        "config": {"workload": wl.w["name"], "B": wl.B, "D": wl.D, "K": wl.K,
                   "rtol": wl.w["rtol"], "atol": wl.w["atol"], "form": "fused",
                   "pass": "fwd+adjoint" if head["with_adj"] else "fwd",
                   "state": entry["state"], "controller": "I (beta1=0.2)",
                   "l2": "flushed between timed steps (256 MiB write outside the events)",
                   "parallelism": f"dp{world} (independent replicas of the batch)",
                   "launch": entry["launch"], "launch_plain": entry["launch_plain"],
                   "issue": ("fused step replayed as one CUDA graph (forward + adjoint), "
                             "plain form from its host loop" if head["graphed"] else
                             "eager calls (graph capture off or unavailable)")
                   + ("; capture: " + "; ".join(wl.graph_notes) if wl.graph_notes else "")},
        "gpu_launches": launches_per_step(wl) * steps,
        "clocks": head["clocks"], "e2e": e2e, "roofline": entry["roofline"],
        "breakdown": {k: v for k, v in entry.items() if k != "roofline"},
        "configs": configs, "peaks": peaks, "wall_s_timed_region": head["wall"],
    }
    if rank == 0 and not args.no_cpu and world == 1:
        for name, (w, keep) in kept.items():
            configs[name]["error_vs_fp64"] = fp64_errors(w, keep)
        result["cpu_baseline"] = cpu_baseline(wl.w, budget_s=12.0,
                                              with_adjoint=head["with_adj"])
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


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
    peaks, src = _peaks_file()
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
                     "frac": achieved / peaks["hbm_gbs"], "peak_source": f"of {src}",
                     "traffic": _traffic(f"vdp_joint_mu10_b{B}", "k_joint_step<VdpField<float>>"),
                     "kernel_ms": per_launch_ms,
                     "bytes_per_launch": by},
        "clocks": clocks,
        "gpu_launches": launches,
    }), flush=True)


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on the host cores, on
    the same workload as the default line (bounded samples of it)."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    w = workloads.make(args.workload if args.workload >= 0 else HEADLINE)
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
