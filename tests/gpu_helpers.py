"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs."""
from __future__ import annotations

import copy

import numpy as np


def run_gpu(cfgs, T0_list, n_steps, t0=0.0, dt=0.0, precision=0, want_trace=True,
            want_energy=True, chunks=None, launch=None):
    """Run n_steps on the GPU for the instances `cfgs` from fields `T0_list`
    (launch: (mode, threads, rows_per_lane), "autotune" for the shape the
    library's autotuner picks on the initial field, or None for the default).

    Returns (list of fields, trace[n_inst, n_steps, 2], energy[n_inst, 5])."""
    import torch
    from paper_1408_5853_gb300 import ccell
    if isinstance(cfgs, dict):
        cfgs, T0_list = [cfgs], [T0_list]
    sol = ccell.Solver(cfgs, precision=precision)
    dtype = torch.float64 if precision == ccell.FP64 else torch.float32
    flat = np.concatenate([np.asarray(T, dtype=np.float64).ravel() for T in T0_list])
    T = torch.tensor(flat, dtype=dtype, device="cuda")
    if launch == "autotune":
        sol.autotune(T, n_trial=2)          # restores T
    elif launch is not None:
        sol.set_launch(*launch)
    n_inst = len(cfgs)
    trace = torch.zeros(n_inst * n_steps * 2, dtype=torch.float64, device="cuda") if want_trace else None
    energy = torch.zeros(n_inst * 5, dtype=torch.float64, device="cuda") if want_energy else None
    if chunks is None:
        sol.step(T, n_steps, t0, dt, trace, energy)
    else:  # several calls: trace is per call, energy accumulates
        done = 0
        traces = []
        for c in chunks:
            tr = torch.zeros(n_inst * c * 2, dtype=torch.float64, device="cuda") if want_trace else None
            step_dt = dt if dt > 0 else cfgs[0]["dt"]
            sol.step(T, c, t0 + done * step_dt, dt, tr, energy)
            if want_trace:
                traces.append(tr.view(n_inst, c, 2))
            done += c
        if want_trace:
            trace = torch.cat(traces, dim=1)
    sol.sync()
    torch.cuda.synchronize()
    out = T.double().cpu().numpy()
    fields, ofs = [], 0
    for c in cfgs:
        n = c["nr"] * c["nz"]
        fields.append(out[ofs:ofs + n].reshape(c["nz"], c["nr"]))
        ofs += n
    tr = trace.view(n_inst, n_steps, 2).cpu().numpy() if want_trace else None
    en = energy.view(n_inst, 5).cpu().numpy() if want_energy else None
    shape = sol.get_launch()
    sol.close()
    run_gpu.last_launch = shape
    return fields, tr, en


def oracle_cone(cfg, T0, j, n_steps, t0, dt):
    """Oracle value of line j after n_steps, computed on the slab of lines that
    can influence it (the axial coupling is explicit: one line per step)."""
    from oracle import oracle
    M = cfg["nz"] - 1
    lo, hi = max(0, j - n_steps - 1), min(M, j + n_steps + 1)
    sub = copy.deepcopy(cfg)
    eta = cfg["length"] / M
    sub["nz"] = hi - lo + 1
    sub["length"] = (hi - lo) * eta
    if lo > 0:
        sub["bc_z0"] = 0
    if hi < M:
        sub["bc_zmax"] = 0
    T, _, _ = oracle.step_n(sub, T0[lo:hi + 1], n_steps, t0, dt, want_trace=False,
                            want_energy=False)
    return T[j - lo]
