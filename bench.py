"""Benchmark of the explicit-implicit r-z heat-conduction step on GB300.

Workload: the 5-layer 512 x 4096 production cylinder (properties jittered
+/-10 %, seed 0), FP64 path, tau = 0.4 ns (axial stability bound).  One bench
step = one cc_step_n call advancing the field by --inner time steps (all of
the time step: properties, explicit axial stencil, source, tridiagonal line
solves, boundary rows, surface trace and energy sums).  Metric: node-updates/s
(nr * nz per time step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--inner n] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the reference arm of this build)
on the same workload, on the host cores.  With N > 1 (torchrun) every rank
runs an independent replica (the path has no exchange between problems), rank
0 prints the JSON line with the total over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "node-updates/s at 512x4096 r-z, FP64 path"
UNIT = "node-updates/s"
BYTES_PER_NODE_FP64 = 16      # read T^n + write T^{n+1}
BYTES_PER_NODE_MIXED = 8
FLOPS_PER_NODE_FP64 = 150     # FP64 operations per node-update (2 power laws ~ 2x(log+exp), 1 div, 1 rcp, ~30 fma/add/mul)

# DRAM bytes (read + write) of one step_fp64_pipe_kernel launch (launch mode 4, 128 threads)
# on the 512x4096 workload, from the ncu capture summarised in
# profiles/step_fp64_pipe_kernel_512x4096.md (cache flushed before the launch).  Valid only for
# the kernel as captured there: reset to None when the kernel changes.
STEP_FP64_TRAFFIC_512x4096 = 17.355e6
FP64_PEAK_NOMINAL_TFLOPS = 152 * 4 * 0.5 * 2 * 2.07e9 / 1e12   # SMs x SMSPs x DFMA lanes/clk x 2 x max clock
# Per launch mode of the FP64 headline: the dominant kernel, the FP64-pipe thread-instructions it
# executes per node-update on the 512x4096 workload (ncu sm__thread_inst_executed_pipe_fp64_pred_on
# of one launch / nodes) and the summary that holds the capture; None once the kernel changes until
# it is captured again.
EXECUTED_FP64 = {
    0: ("step_fp64_kernel", None, None),
    1: ("steps_fp64_persistent_kernel", None, None),
    2: ("step_fp64_lines_kernel", None, None),
    3: ("steps_fp64_resident_kernel", None, None),
    4: ("step_fp64_pipe_kernel", 57.6, "profiles/step_fp64_pipe_kernel_512x4096.md"),
}
L2_FLUSH_BYTES = 256 << 20


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6800.0, "source": "fallback"}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_ours(args, world, rank, local):
    import torch
    import torch.distributed as dist

    from paper_1408_5853_gb300 import ccell, inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = inputs.production_case()
    nodes = cfg["nr"] * cfg["nz"]
    n_in = args.inner
    T0 = inputs.initial_field(cfg, "smooth", seed=0)
    t0 = 0.0

    def make(precision):
        sol = ccell.Solver(cfg, precision=precision)
        dt = torch.float64 if precision == ccell.FP64 else torch.float32
        T = torch.tensor(T0.ravel(), dtype=dt, device=dev)
        if precision == ccell.MIXED and args.mixed_launch:
            sol.set_launch(*_launch_arg(args.mixed_launch))
        elif args.launch:
            sol.set_launch(*_launch_arg(args.launch))
        elif precision == ccell.MIXED:
            # the library's autotuner picks the mixed path's launch shape (field
            # restored); the FP64 headline keeps the library's default shape
            # (pipelined tiles, 128 threads)
            sol.autotune(T, n_trial=args.tune_steps)
        trace = torch.zeros(2 * n_in, dtype=torch.float64, device=dev)
        energy = torch.zeros(5, dtype=torch.float64, device=dev)
        return sol, T, trace, energy

    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    # the FP64-pipe roofline denominator, measured on this GPU by the library
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    rate_buf = torch.empty(1024 * sms, dtype=torch.float64, device=dev)
    fma_rate = max(ccell.cc_measure_fp64_rate(rate_buf.data_ptr(), rate_buf.numel(), 20000,
                                              stream.cuda_stream)[0] for _ in range(3))
    fp64_peak_tflops = 2.0 * fma_rate / 1e12
    del rate_buf

    def timed_steps(sol, T, trace, energy, k_steps, warm):
        for w in range(warm):
            sol.step(T, n_in, t0 + w * n_in * cfg["dt"], 0.0, trace, energy)
        sol.sync()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        times = []
        launches0 = ccell.cc_kernel_launches()
        for k in range(k_steps):
            flush.fill_(float(k))                       # L2 flush outside the timed events
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sol.step(T, n_in, t0 + (warm + k) * n_in * cfg["dt"], 0.0, trace, energy)
            e1.record(stream)
            times.append((e0, e1))
        torch.cuda.synchronize()
        launches = ccell.cc_kernel_launches() - launches0
        sol.sync()
        ms = sum(a.elapsed_time(b) for a, b in times)
        if world > 1:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, launches

    # ---- FP64 path (headline)
    clocks = Clocks(local)
    sol, T, trace, energy = make(ccell.FP64)
    clocks.start()
    ms, launches = timed_steps(sol, T, trace, energy, args.steps, args.warmup)
    clk = clocks.stop()
    launch_shape = sol.get_launch()
    total_nodes = nodes * n_in * args.steps * world
    value = total_nodes / (ms / 1e3)
    per_launch_ms = ms / (args.steps * n_in)
    e = energy.cpu().numpy()
    ident = abs(e[0] - e[1:].sum()) / max(abs(e[0]), abs(e[1]), 1e-300)

    # ---- end to end through the C ABI with pinned host buffers
    hT = torch.tensor(T0.ravel(), dtype=torch.float64).pin_memory()
    hOut = torch.empty_like(hT).pin_memory()
    hTr = torch.empty(2 * n_in, dtype=torch.float64).pin_memory()
    T.copy_(hT)
    sol.step(T, n_in, 0.0, 0.0, trace, energy)
    torch.cuda.synchronize()
    e2e_times = []
    for k in range(max(1, args.steps)):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t_a = time.perf_counter()
        T.copy_(hT, non_blocking=True)
        sol.step(T, n_in, 0.0, 0.0, trace, energy)
        hOut.copy_(T, non_blocking=True)
        hTr.copy_(trace, non_blocking=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t_a)
    e2e_s = sum(e2e_times)
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_val = nodes * n_in * len(e2e_times) * world / e2e_s

    # ---- time steps per cc_step_n call: the rate with every call's launch and host
    # overhead included (device time from the first call's start to the last one's end)
    nsweep = None
    if "nsweep" in args.parts:
        nsweep = {"unit": UNIT}
        for n_call in (1, 10, 100, 1000):
            calls = max(3, 4000 // n_call)
            tr_n = torch.zeros(2 * n_call, dtype=torch.float64, device=dev)
            sol.step(T, n_call, 0.0, 0.0, tr_n, energy)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for c in range(calls):
                sol.step(T, n_call, c * n_call * cfg["dt"], 0.0, tr_n, energy)
            e1.record(stream)
            torch.cuda.synchronize()
            nsweep[str(n_call)] = nodes * n_call * calls / (e0.elapsed_time(e1) / 1e3)
        sol.sync()
    sol.close()

    # ---- mixed-precision path on the same workload
    mixed = None
    base = None
    if "mixed" not in args.parts:
        mixed = {"skipped": True}
    else:
      try:
        solm, Tm, trm, enm = make(ccell.MIXED)
        msm, _ = timed_steps(solm, Tm, trm, enm, args.steps, args.warmup)
        mixed = {"value": nodes * n_in * args.steps * world / (msm / 1e3),
                 "ms_per_step": msm / args.steps,
                 "launch": dict(zip(("mode", "threads", "rows_per_lane"), solm.get_launch())),
                 "speedup_vs_fp64": (nodes * n_in * args.steps * world / (msm / 1e3)) / value,
                 "hbm_frac_effective": BYTES_PER_NODE_MIXED * nodes * n_in * args.steps * world
                 / (msm / 1e3) / (_peaks()["hbm_gbs"] * 1e9)}
        solm.close()
        if args.acc_steps > 0:
            mixed.update(mixed_accuracy(cfg, T0, args.acc_steps, dev))
        if world == 1 and not args.no_cpu_baseline:
            # the oracle sample of cpu_baseline (below) doubles as the parity
            # reference of both paths at its horizon
            base, T_or = cpu_baseline(args.cpu_sample_steps, _f32(T0))
            mixed.update(vs_oracle(cfg, _f32(T0), args.cpu_sample_steps, T_or, dev))
      except ccell.CCError as err:
        mixed = {"unavailable": str(err)}
    batched = run_batched(args, dev) if "batched" in args.parts else {"skipped": True}
    adjoint = run_adjoint(args, dev) if "adjoint" in args.parts else {"skipped": True}
    paper = run_paper(args, dev) if "paper" in args.parts else {"skipped": True}
    adi = (run_adi(args, dev, ms / (args.steps * n_in)) if "adi" in args.parts
           else {"skipped": True})

    if rank != 0:
        return None
    peaks = _peaks()
    hbm_peak = peaks["hbm_gbs"]
    kname, executed_ops, executed_src = EXECUTED_FP64.get(
        tuple(launch_shape)[0], ("step_fp64_kernel", None, None))
    achieved_tflops = FLOPS_PER_NODE_FP64 * nodes / (per_launch_ms / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": headline_config(cfg, n_in, world, launch_shape),
        "roofline": {"bound": "alu", "kernel": kname,
                     "achieved": achieved_tflops, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved_tflops / fp64_peak_tflops,
                     "traffic": (STEP_FP64_TRAFFIC_512x4096
                                 if (cfg["nr"], cfg["nz"]) == (512, 4096)
                                 and tuple(launch_shape) == (4, 128, 16) else None),
                     "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, "
                                     "cold L2 (the output rows stay in L2)",
                     "peak_source": "measured on this GPU: cc_measure_fp64_rate, 8 independent "
                                    "DFMA chains per thread, 4 x 256 threads per SM, x 2 flops "
                                    "(profiles/fp64_rate_gb300.md)",
                     "peak_nominal": FP64_PEAK_NOMINAL_TFLOPS,
                     "peak_nominal_source": "FP64 unit counts x max SM clock "
                                            "(152 x 4 x 0.5 DFMA/clk x 2 x 2.07 GHz)",
                     "per_unit": f"{FLOPS_PER_NODE_FP64} FP64 ops per node-update "
                                 "(algorithmic count: two power laws as log + exp, 1 divide, "
                                 "1 reciprocal, ~30 FMA/add/mul)",
                     "executed": (None if executed_ops is None else {
                         "fp64_pipe_ops_per_node_update": executed_ops,
                         "achieved": executed_ops * nodes / (per_launch_ms / 1e3) / 1e12,
                         "peak": fma_rate / 1e12,
                         "frac": executed_ops * nodes / (per_launch_ms / 1e3) / fma_rate,
                         "unit": "T thread-instructions/s",
                         "source": executed_src})},
        "hbm_roofline": {"bound": "hbm", "achieved": BYTES_PER_NODE_FP64 * value / world / 1e9,
                         "peak": hbm_peak, "unit": "GB/s",
                         "frac": BYTES_PER_NODE_FP64 * value / world / 1e9 / hbm_peak,
                         "per_unit": "16 B per node-update (read T^n, write T^n+1)",
                         "note": "effective: the field stays L2-resident during a call"},
        "energy_identity_rel": ident,
        "mixed": mixed,
        "steps_per_call_sweep": nsweep if nsweep is not None else {"skipped": True},
        "batched": batched,
        "adjoint": adjoint,
        "paper_cell": paper,
        "adi": adi,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(hT.numel() * 8),
                "d2h_bytes_per_step": int(hOut.numel() * 8 + hTr.numel() * 8)},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        if base is None:
            base, _ = cpu_baseline(args.cpu_sample_steps, _f32(T0))
        line["cpu_baseline"] = base
    return line


def run_batched(args, dev) -> dict:
    """Design sweep: 256 ragged 5-layer instances (seed 1) in one context,
    mixed precision, per-instance dt = 0.9 x the axial stability bound, the
    launch shape chosen by the autotuner; one cc_step_n call of --batch-inner
    time steps (2000 by default) captured in a CUDA graph, one warm-up replay,
    then --batch-replays timed replays."""
    import torch

    from paper_1408_5853_gb300 import ccell, inputs, shard
    world, rank, _ = _dist()
    all_cfgs = inputs.batched_cases(seed=1, n=args.batch_instances)
    mine = shard.balanced_shards([c["nr"] * c["nz"] for c in all_cfgs], world)[rank]
    cfgs = [all_cfgs[k] for k in mine]   # independent instances: no exchange between ranks
    total_all = sum(c["nr"] * c["nz"] for c in all_cfgs)
    sol = ccell.Solver(cfgs, precision=ccell.MIXED)
    for k in range(len(cfgs)):
        ccell.cc_set_dt(sol.ctx, k, 0.9 * sol.tau_stab(k))
    total = sol.total
    T0 = np.concatenate([inputs.initial_field(c, "uniform").ravel() for c in cfgs])
    T = torch.tensor(T0, dtype=torch.float32, device=dev)
    if args.batch_launch:
        sol.set_launch(*[int(v) for v in args.batch_launch.split(",")])
        tune_ms = None
    else:
        tune_ms = sol.autotune(T, n_trial=2)
    n_in = args.batch_inner
    trace = torch.zeros(len(cfgs) * n_in * 2, dtype=torch.float64, device=dev)
    energy = torch.zeros(len(cfgs) * 5, dtype=torch.float64, device=dev)
    sol.step(T, n_in, 0.0, 0.0, trace, energy)      # warm-up sizes the buffers
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        sol.step(T, n_in, 0.0, 0.0, trace, energy)
    graph.replay()                                  # warm-up replay
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.batch_replays):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    sol.sync()
    ms = shard.max_over_ranks(e0.elapsed_time(e1), dev)
    mode, threads, rows = sol.get_launch()
    sol.close()
    return {"instances": len(all_cfgs), "nodes": int(total_all), "time_steps_per_replay": n_in,
            "ranks": world, "scaling": "strong (instances sharded over ranks)",
            "precision": "mixed", "value": total_all * n_in * args.batch_replays / (ms / 1e3),
            "unit": "node-updates/s", "replays": args.batch_replays,
            "ms_per_replay": ms / args.batch_replays,
            "launch": {"mode": mode, "threads": threads,
                       "rows_per_lane": rows, "autotune_ms_per_step": tune_ms},
            "graph": "each replay is one captured cc_step_n call"}


def run_adjoint(args, dev) -> dict:
    """Gradient of the surface-waveform loss on the 5-layer 256 x 1024 case
    (tanh pulse edges, 28/42 K target), checkpoint every 256 steps; then a
    batch of 64 such gradients in one context."""
    import torch

    from paper_1408_5853_gb300 import ccell, inputs
    out = {}
    # checkpoints every 256 steps (the workload's setting); then every state of
    # the single run kept in HBM (about 84 GB at 40 000 steps), which removes
    # the recompute
    # the library's default launch, then (every state kept) the launch the
    # autotuner picks for this grid's forward step
    runs = [("single", 1, args.adj_steps, 256, False),
            ("batch64", 64, args.adj_batch_steps, 256, False)]
    if args.adj_keep_all:
        runs += [("single_all_states", 1, args.adj_steps, args.adj_steps, False),
                 ("single_all_states_autotuned", 1, args.adj_steps, args.adj_steps, True)]
    for label, n_inst, n, ckpt, tune in runs:
        cfg = inputs.adjoint_case()
        cfgs = [cfg] * n_inst
        sol = ccell.Solver(cfgs)
        T0 = torch.tensor(np.tile(inputs.initial_field(cfg, "uniform").ravel(), n_inst),
                          dtype=torch.float64, device=dev)
        if tune:
            sol.autotune(T0.clone(), n_trial=args.tune_steps)
        t = cfg["dt"] * np.arange(1, n + 1)
        tgt = torch.tensor(np.tile(inputs.target_waveform(cfg, t), n_inst), dtype=torch.float64,
                           device=dev)
        n_w = min(n, 256)                                     # warm-up on the first steps
        sol.adjoint(T0, n_w, 0.0, 0.0, tgt.view(n_inst, n)[:, :n_w].contiguous().view(-1),
                    ckpt_every=256)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        loss, grad, _ = sol.adjoint(T0, n, 0.0, 0.0, tgt, ckpt_every=ckpt)
        e1.record()
        torch.cuda.synchronize()
        sol.sync()
        ms = e0.elapsed_time(e1)
        nodes = cfg["nr"] * cfg["nz"] * n_inst
        # one forward step of the same context, for the reverse step's cost in forward steps
        T1 = T0.clone()
        sol.step(T1, 64, 0.0, 0.0, None, None)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        sol.step(T1, 256, 0.0, 0.0, None, None)
        f1.record()
        torch.cuda.synchronize()
        fwd_ms = f0.elapsed_time(f1) / 256
        out[label] = {"instances": n_inst, "grid": f"{cfg['nr']}x{cfg['nz']}", "steps": n,
                      "ckpt_every": ckpt, "ms_per_reverse_step": ms / n,
                      "forward_steps_per_reverse_step": (ms / n) / fwd_ms,
                      "ms_per_gradient": ms / n_inst, "ms_total": ms,
                      "forward_equivalent_node_updates_per_s": nodes * n / (ms / 1e3),
                      "launch": dict(zip(("mode", "threads", "rows_per_lane"), sol.get_launch())),
                      "ms_per_forward_step": fwd_ms,
                      # the configured horizon, 20 ms = 3.2e6 steps of 6.25 ns, at this run's
                      # cost per reverse step (with checkpoints: every state would need 6.7 TB)
                      "projected_full_20ms_s": ((20e-3 / cfg["dt"]) * (ms / n) / 1e3
                                                if ckpt < n and n_inst == 1 else None),
                      "loss": float(loss[0].item()), "grad_norm": float(grad.norm().item())}
        sol.close()
    return out


def run_paper(args, dev) -> dict:
    """The paper's cryogenic cell (Section 5 fits, resistive source, transient
    turn-on with tau* = tau/100 sub-steps, outer layers on z <= z_0 = 4 cm and
    the copper core alone up to z_max = 5 cm) on a Table calc_table-like grid:
    nr = 512 (the paper used N = 631) x nz = 1201, tau = 2.5e-7 s, FP64.  The
    paper's K40 OpenCL run of 631 x 1201 for 25 ms (1e5 steps) took 12.9 min
    (9.8e7 node-updates/s); this times the first args.paper_ms of that window
    (the printed graphite c_V fit turns negative above ~22 K, which the heater
    reaches after ~0.1 ms at this resolution) and projects the 25 ms run."""
    import torch

    from paper_1408_5853_gb300 import ccell, inputs, schedule
    cfg = inputs.paper_case(nr=512, nz=1201, stepped=True)
    cfg["dt"] = 2.5e-7
    cfg["source"]["edge_w"] = cfg["dt"]       # tau of the transient model = the time step
    cfg["t_guard"] = (4.2, 20.0)              # graphite c_V fit positive below ~22 K
    sol = ccell.Solver(cfg)
    nodes = cfg["nr"] * cfg["nz"]
    T = torch.full((nodes,), 4.2, dtype=torch.float64, device=dev)
    sol.autotune(T, n_trial=8)                # launch shape for the stepped outline (T restored)
    chunks = schedule.transient_schedule(cfg["source"]["t_period"], cfg["dt"],
                                         args.paper_ms * 1e-3)
    steps = sum(n for _, _, n in chunks)
    sol.step(T.clone(), 100, 0.0, cfg["dt"] / 100, None, None)   # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for t0, dt, n in chunks:
        sol.step(T, n, t0, dt, None, None)
    e1.record()
    torch.cuda.synchronize()
    sol.sync()
    ms = e0.elapsed_time(e1)
    rate = nodes * steps / (ms / 1e3)
    tmax = float(T.max().item())
    launch = dict(zip(("mode", "threads", "rows_per_lane"), sol.get_launch()))
    sol.close()
    paper_rate = 631 * 1201 * 1e5 / (12.9 * 60)
    return {"grid": f"{cfg['nr']}x{cfg['nz']}", "outline": "stepped at z_0 = 4 cm (core only beyond)",
            "simulated_ms": args.paper_ms, "steps": steps,
            "value": rate, "unit": "node-updates/s", "precision": "fp64",
            "max_T_K": tmax, "launch": launch,
            "paper_k40_opencl_631x1201": {"value": paper_rate, "unit": "node-updates/s",
                                          "source": "Table calc_table (12.9 min for 1e5 steps)"},
            "projected_25ms_run_s": nodes * 1e5 / rate}


def run_adi(args, dev, main_ms_per_time_step: float) -> dict:
    """ADI variant (Peaceman-Rachford, implicit in r and z) on the 512x4096
    workload at dt = 0.25 us, the time step that workload is configured with
    (625 x the explicit bound of the paper's scheme): time per step, and the
    simulated time per wall second against the paper's scheme at its stable
    0.4 ns.  Accuracy cost: both from the same field over args.adi_check_us
    microseconds across the end of a heater pulse, max |dT| between them."""
    import torch

    from paper_1408_5853_gb300 import ccell, inputs
    cfg = inputs.production_case()
    nodes = cfg["nr"] * cfg["nz"]
    T0 = inputs.initial_field(cfg, "smooth", seed=0)
    dt = 2.5e-7
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sol = ccell.Solver(cfg)
    T = torch.tensor(T0.ravel(), dtype=torch.float64, device=dev)
    tr = torch.zeros(2 * args.adi_steps, dtype=torch.float64, device=dev)
    sol.step_adi(T, 5, 0.0, dt)  # warm-up, sizes the scratch
    sol.sync()
    flush.fill_(1.0)
    l0 = ccell.cc_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    sol.step_adi(T, args.adi_steps, 5 * dt, dt, tr)
    e1.record()
    torch.cuda.synchronize()
    launches = ccell.cc_kernel_launches() - l0
    sol.sync()
    ms = e0.elapsed_time(e1) / args.adi_steps
    # accuracy against the paper's scheme over the same simulated interval
    t_span = args.adi_check_us * 1e-6
    t0 = 1.0e-3 - 0.5 * t_span
    Ta = torch.tensor(T0.ravel(), dtype=torch.float64, device=dev)
    Tm = Ta.clone()
    sol.step_adi(Ta, int(round(t_span / dt)), t0, dt)
    solm = ccell.Solver(cfg)
    solm.step(Tm, int(round(t_span / cfg["dt"])), t0, cfg["dt"], None, None)
    solm.sync()
    sol.sync()
    err = float((Ta - Tm).abs().max().item())
    solm.close()
    sol.close()
    return {"dt_s": dt, "value": nodes / (ms / 1e3), "unit": "node-updates/s",
            "ms_per_step": ms, "launches_per_step": launches / args.adi_steps,
            "simulated_s_per_wall_s": dt / (ms / 1e3),
            "paper_scheme_simulated_s_per_wall_s": cfg["dt"] / (main_ms_per_time_step / 1e3),
            "check": {"simulated_us": args.adi_check_us,
                      "max_dT_vs_paper_scheme_K": err,
                      "paper_scheme_dt_s": cfg["dt"]}}


def _f32(T):
    return np.asarray(T, dtype=np.float32).astype(np.float64)


def vs_oracle(cfg, T0, n, T_oracle, dev) -> dict:
    """Both paths from the FP32-rounded field over the n steps of the oracle
    sample that cpu_baseline timed: max |dT| over the field against the oracle."""
    import torch

    from paper_1408_5853_gb300 import ccell
    out = {}
    for prec, dt, key in ((ccell.FP64, torch.float64, "fp64"), (ccell.MIXED, torch.float32, "mixed")):
        sol = ccell.Solver(cfg, precision=prec)
        T = torch.tensor(T0.ravel(), dtype=dt, device=dev)
        sol.step(T, n, 0.0, 0.0, None, None)
        sol.sync()
        out[key] = float(np.max(np.abs(T.double().cpu().numpy().reshape(T_oracle.shape) - T_oracle)))
        sol.close()
    return {"oracle_steps": n, "max_dT_vs_oracle_K": out["mixed"],
            "fp64_max_dT_vs_oracle_K": out["fp64"]}


def mixed_accuracy(cfg, T0, n, dev) -> dict:
    """Mixed path against the FP64 path (itself parity-checked against the
    oracle to 1e-9 K) from the same FP32-rounded field, n steps from t = 0
    (heater on): max |dT| over the field, surface-trace peak error, and the
    energy-identity residuals of both."""
    import numpy as np
    import torch

    from paper_1408_5853_gb300 import ccell
    T0 = np.asarray(T0, dtype=np.float32).astype(np.float64).ravel()
    out = {}
    for prec, dt in ((ccell.FP64, torch.float64), (ccell.MIXED, torch.float32)):
        sol = ccell.Solver(cfg, precision=prec)
        T = torch.tensor(T0, dtype=dt, device=dev)
        tr = torch.zeros(2 * n, dtype=torch.float64, device=dev)
        en = torch.zeros(5, dtype=torch.float64, device=dev)
        sol.step(T, n, 0.0, 0.0, tr, en)
        sol.sync()
        out[prec] = (T.double(), tr.view(n, 2), en.cpu().numpy())
        sol.close()
    (Td, trd, ed), (Tm, trm, em) = out[ccell.FP64], out[ccell.MIXED]
    ident = lambda e: float(abs(e[0] - e[1:].sum()) / max(abs(e[0]), abs(e[1])))
    return {"acc_steps": n,
            "max_dT_vs_fp64_K": float((Tm - Td).abs().max().item()),
            "surface_peak_err_K": float(abs(trm[:, 1].max().item() - trd[:, 1].max().item())),
            "surface_trace_max_err_K": float((trm - trd).abs().max().item()),
            "energy_identity_rel": ident(em), "energy_identity_rel_fp64": ident(ed)}


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline(sample_steps: int, T0) -> tuple:
    """The FP64 oracle, as it stands, on the host cores for a bounded sample
    (sample_steps time steps of the workload from T0 at t = 0); also one thread
    on a sample 1/16 of the size.  Returns the line's entry and the oracle's
    field after the sample."""
    from oracle import oracle
    from paper_1408_5853_gb300 import inputs
    cfg = inputs.production_case()
    nodes = cfg["nr"] * cfg["nz"]
    cores = oracle.num_threads()
    t = time.perf_counter()
    T_out, _, _ = oracle.step_n(cfg, T0, sample_steps, 0.0, cfg["dt"])
    s = time.perf_counter() - t
    one_steps = max(1, sample_steps // 16)
    oracle.set_threads(1)
    try:
        t = time.perf_counter()
        oracle.step_n(cfg, T0, one_steps, 0.0, cfg["dt"])
        s1 = time.perf_counter() - t
    finally:
        oracle.set_threads(cores)
    return ({"value": nodes * sample_steps / s, "unit": UNIT, "cores": cores, "kind": "oracle",
             "sample": f"{sample_steps} time steps of the 512x4096 workload ({s:.1f} s)",
             "single_thread": {"value": nodes * one_steps / s1, "unit": UNIT, "cores": 1,
                               "sample": f"{one_steps} time steps ({s1:.1f} s)"},
             "cpu_model": _cpu_model(), "nproc": os.cpu_count()}, T_out)


# The library's default launch shape of an FP64 context (cc_set_launch).
DEFAULT_FP64_LAUNCH = (4, 128, 16)


def _launch_arg(text):
    return tuple(int(v) for v in text.split(",")) if text else None


def headline_config(cfg, n_in, world, launch_shape) -> dict:
    """The headline workload, as both arms name it."""
    return {"workload": f"5-layer r-z cylinder {cfg['nr']}x{cfg['nz']}, jittered seed 0, "
                        f"tau {cfg['dt']:.2e} s, {n_in} time steps per bench step",
            "nr": cfg["nr"], "nz": cfg["nz"], "time_steps_per_step": n_in,
            "precision": "fp64",
            "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MB write)",
            "parallelism": f"replicas x{world}",
            "launch": dict(zip(("mode", "threads", "rows_per_lane"), launch_shape))}


def run_reference(args, world, rank):
    """Reference arm: the FP64 CPU oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return None
    from oracle import oracle
    from paper_1408_5853_gb300 import inputs
    cfg = inputs.production_case()
    nodes = cfg["nr"] * cfg["nz"]
    n_in = args.ref_inner
    T = inputs.initial_field(cfg, "smooth", seed=0)
    for w in range(args.warmup):
        T, _, _ = oracle.step_n(cfg, T, n_in, w * n_in * cfg["dt"], cfg["dt"])
    times = []
    for k in range(args.steps):
        t = time.perf_counter()
        T, _, _ = oracle.step_n(cfg, T, n_in, (args.warmup + k) * n_in * cfg["dt"], cfg["dt"])
        times.append(time.perf_counter() - t)
    s = sum(times)
    value = nodes * n_in * args.steps / s
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": headline_config(cfg, args.inner, world, _launch_arg(args.launch)
                                  or DEFAULT_FP64_LAUNCH),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": f"{n_in} time steps of the 512x4096 workload per bench step "
                                   f"(the GPU arm's bench step is {args.inner})",
                         "cpu_model": _cpu_model(), "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--inner", type=int, default=1000, help="time steps per bench step")
    ap.add_argument("--ref-inner", type=int, default=60, help="time steps per reference step")
    ap.add_argument("--cpu-sample-steps", type=int, default=1000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--adi-steps", type=int, default=200, help="timed ADI steps")
    ap.add_argument("--adi-check-us", type=float, default=10.0,
                    help="simulated microseconds of the ADI accuracy check")
    ap.add_argument("--parts", default="fp64,nsweep,mixed,batched,adjoint,paper,adi",
                    help="comma list of extra parts to run besides the FP64 headline")
    ap.add_argument("--batch-instances", type=int, default=256)
    ap.add_argument("--batch-inner", type=int, default=2000,
                    help="time steps per batched replay (one captured cc_step_n call)")
    ap.add_argument("--batch-replays", type=int, default=2, help="timed replays of the sweep")
    ap.add_argument("--adj-steps", type=int, default=40000)
    ap.add_argument("--adj-batch-steps", type=int, default=512)
    ap.add_argument("--no-adj-keep-all", dest="adj_keep_all", action="store_false",
                    help="skip the adjoint run that keeps every state (no recompute)")
    ap.add_argument("--paper-ms", type=float, default=0.08,
                    help="simulated ms of the paper-cell run; with the printed graphite c_V fit "
                         "(negative above ~22 K) the heater stays below 20 K up to ~0.1 ms")
    ap.add_argument("--acc-steps", type=int, default=20000,
                    help="steps of the mixed-vs-FP64 accuracy check (0: skip)")
    ap.add_argument("--launch", default="",
                    help="mode,threads,rows_per_lane of the 512x4096 runs (default: library "
                         "default for FP64, autotuned for the mixed path)")
    ap.add_argument("--mixed-launch", default="",
                    help="mode,threads,rows_per_lane of the mixed 512x4096 runs (overrides --launch)")
    ap.add_argument("--batch-launch", default="",
                    help="mode,threads,rows_per_lane of the batched sweep (default: autotuned)")
    ap.add_argument("--tune-steps", type=int, default=30,
                    help="time steps per candidate launch shape of the autotuner")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    args = ap.parse_args()
    args.parts = set(args.parts.split(","))
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        if args.impl == "ours":
            import torch
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    if args.impl == "reference":
        line = run_reference(args, world, rank)
    else:
        line = run_ours(args, world, rank, local)
    if line is not None:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
