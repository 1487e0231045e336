"""GPU reverse-time adjoint against the FP64 oracle adjoint and finite differences.

Loss: J = sum_n dt (Sbar_n - target_n)^2 with Sbar_n the z-mean surface
temperature after step n and the 28 K / 42 K target waveform; parameters
(q0, t_on, lam_scale[L], cap_scale[L]); smoothed (tanh) pulse edges.
Bars: gradients and dJ/dT0 equal the oracle adjoint's to 1e-8 relative, and
the gradient matches central finite differences of the GPU loss
(h = 1e-6 relative) to 1e-5 relative.
"""
import copy

import numpy as np
import pytest

from oracle import oracle
from paper_1408_5853_gb300 import inputs

pytestmark = pytest.mark.gpu


def _case(nr=32, nz=48, layers=5):
    cfg = inputs.adjoint_case(nr=nr, nz=nz)
    cfg["layers"] = cfg["layers"][:layers]
    cfg["dt"] = 0.5 * oracle.tau_stab(cfg, 20.0, 100.0)
    return cfg


def _gpu_adjoint(cfgs, T0s, n, t0, targets, ckpt, want_dT0=True):
    import torch
    from paper_1408_5853_gb300 import ccell
    sol = ccell.Solver(cfgs)
    T0 = torch.tensor(np.concatenate([t.ravel() for t in T0s]), dtype=torch.float64, device="cuda")
    tgt = torch.tensor(np.concatenate(targets), dtype=torch.float64, device="cuda")
    loss, grad, dT0 = sol.adjoint(T0, n, t0, 0.0, tgt, ckpt_every=ckpt, want_dT0=want_dT0)
    sol.sync()
    out = (loss.cpu().numpy(), grad.cpu().numpy(), dT0.cpu().numpy() if want_dT0 else None)
    sol.close()
    return out


def _gpu_loss(cfg, T0, n, t0, target):
    from gpu_helpers import run_gpu
    _, tr, _ = run_gpu(cfg, T0, n, t0=t0, want_energy=False)
    return float(np.sum(cfg["dt"] * (tr[0, :, 1] - target) ** 2))


def test_gpu_adjoint_matches_oracle_adjoint():
    cfg = _case()
    n = 300
    t0 = 1.0e-3 - 150 * cfg["dt"]
    T0 = inputs.initial_field(cfg, "smooth", seed=2)
    target = inputs.target_waveform(cfg, t0 + cfg["dt"] * np.arange(1, n + 1))
    lo, go, do = oracle.adjoint(cfg, T0, n, t0, cfg["dt"], target, ckpt=64)
    lg, gg, dg = _gpu_adjoint([cfg], [T0], n, t0, [target], ckpt=37)
    assert abs(lg[0] - lo) <= 1e-10 * lo
    assert np.max(np.abs(gg - go)) <= 1e-8 * np.max(np.abs(go)), (gg, go)
    assert np.max(np.abs(dg.reshape(T0.shape) - do)) <= 1e-8 * np.max(np.abs(do))


@pytest.mark.parametrize("variant", ["interface_rule_1", "face_rule_1", "rmax_dirichlet_g_model"])
def test_gpu_adjoint_variants(variant):
    cfg = _case(nr=24, nz=20, layers=4)
    if variant == "interface_rule_1":
        cfg["interface_rule"] = 1
    elif variant == "face_rule_1":
        cfg["face_rule"] = 1
    else:
        cfg["bc_rmax"] = 1
        cfg["source"].update(g_model=1, g_ref=4.0)
    n = 120
    t0 = 1.0e-3 - 60 * cfg["dt"]
    T0 = inputs.initial_field(cfg, "smooth", seed=4)
    target = inputs.target_waveform(cfg, t0 + cfg["dt"] * np.arange(1, n + 1))
    lo, go, do = oracle.adjoint(cfg, T0, n, t0, cfg["dt"], target, ckpt=16)
    lg, gg, dg = _gpu_adjoint([cfg], [T0], n, t0, [target], ckpt=50)
    assert np.max(np.abs(gg - go)) <= 1e-8 * np.max(np.abs(go))
    assert np.max(np.abs(dg.reshape(T0.shape) - do)) <= 1e-8 * np.max(np.abs(do))


def test_gpu_adjoint_central_differences():
    cfg = _case(nr=32, nz=40)
    n = 200
    t0 = 1.0e-3 - 100 * cfg["dt"]
    T0 = inputs.initial_field(cfg, "smooth", seed=6)
    target = inputs.target_waveform(cfg, t0 + cfg["dt"] * np.arange(1, n + 1))
    _, gg, _ = _gpu_adjoint([cfg], [T0], n, t0, [target], ckpt=64, want_dT0=False)
    L = len(cfg["layers"])
    for k in range(2 + 2 * L):
        h = 1e-6
        vals = []
        for sgn in (+1, -1):
            c = copy.deepcopy(cfg)
            if k == 0:
                base = c["source"]["q0"]
                c["source"]["q0"] = base * (1 + sgn * h)
            elif k == 1:
                base = c["source"]["t_on"]
                c["source"]["t_on"] = base * (1 + sgn * h)
            else:
                key = "lam_scale" if k < 2 + L else "cap_scale"
                m = (k - 2) % L
                base = c["layers"][m].get(key, 1.0)
                c["layers"][m][key] = base * (1 + sgn * h)
            vals.append(_gpu_loss(c, T0, n, t0, target))
        fd = (vals[0] - vals[1]) / (2 * h * base)
        assert abs(fd - gg[k]) <= 1e-5 * abs(fd) + 1e-9 * max(abs(gg).max(), 1e-300), (k, fd, gg[k])


def test_gpu_adjoint_batched_ragged():
    cfgs, T0s, targets = [], [], []
    n = 60
    for k, (nr, nz) in enumerate([(20, 30), (33, 17), (64, 24), (17, 50)]):
        c = _case(nr=nr, nz=nz, layers=5 if nr >= 20 else 3)
        cfgs.append(c)
        T0s.append(inputs.initial_field(c, "smooth", seed=k))
    dt = min(c["dt"] for c in cfgs)
    for c in cfgs:
        c["dt"] = dt
    t0 = 1.0e-3 - 30 * dt
    for c in cfgs:
        targets.append(inputs.target_waveform(c, t0 + dt * np.arange(1, n + 1)))
    lg, gg, dg = _gpu_adjoint(cfgs, T0s, n, t0, targets, ckpt=16)
    gofs, nofs = 0, 0
    for k, c in enumerate(cfgs):
        lo, go, do = oracle.adjoint(c, T0s[k], n, t0, dt, targets[k], ckpt=16)
        npar = 2 + 2 * len(c["layers"])
        nn = c["nr"] * c["nz"]
        assert abs(lg[k] - lo) <= 1e-10 * lo
        assert np.max(np.abs(gg[gofs:gofs + npar] - go)) <= 1e-8 * np.max(np.abs(go)), k
        assert np.max(np.abs(dg[nofs:nofs + nn].reshape(T0s[k].shape) - do)) <= 1e-8 * np.max(np.abs(do))
        gofs += npar
        nofs += nn


def test_autograd_surface_trace():
    import torch
    from paper_1408_5853_gb300 import ccell
    cfg = _case(nr=24, nz=30)
    n = 80
    t0 = 1.0e-3 - 40 * cfg["dt"]
    T0n = inputs.initial_field(cfg, "smooth", seed=9)
    target = inputs.target_waveform(cfg, t0 + cfg["dt"] * np.arange(1, n + 1))
    sol = ccell.Solver(cfg)
    theta = torch.tensor([sol.get_params(0)], dtype=torch.float64, requires_grad=True)
    T0 = torch.tensor(T0n.ravel(), dtype=torch.float64, device="cuda", requires_grad=True)
    sbar = ccell.surface_trace(theta, T0, sol, n, t0, 0.0, ckpt=32)
    tgt = torch.tensor(target, device="cuda")
    loss = (cfg["dt"] * (sbar[0] - tgt) ** 2).sum()
    loss.backward()
    lo, go, do = oracle.adjoint(cfg, T0n, n, t0, cfg["dt"], target, ckpt=32)
    assert abs(loss.item() - lo) <= 1e-10 * lo
    assert np.max(np.abs(theta.grad[0].numpy() - go)) <= 1e-8 * np.max(np.abs(go))
    assert np.max(np.abs(T0.grad.cpu().numpy().reshape(T0n.shape) - do)) <= 1e-8 * np.max(np.abs(do))
    sol.close()


def test_gpu_adjoint_256x1024_short_horizon():
    """The gradient workload's grid (5 layers, 256 x 1024), 300 steps across a
    smoothed pulse edge, against the oracle adjoint."""
    cfg = inputs.adjoint_case()
    n = 300
    t0 = 1.0e-3 - 150 * cfg["dt"]
    T0 = inputs.initial_field(cfg, "smooth", seed=1)
    target = inputs.target_waveform(cfg, t0 + cfg["dt"] * np.arange(1, n + 1))
    lo, go, do = oracle.adjoint(cfg, T0, n, t0, cfg["dt"], target, ckpt=100)
    lg, gg, dg = _gpu_adjoint([cfg], [T0], n, t0, [target], ckpt=256)
    assert abs(lg[0] - lo) <= 1e-10 * lo
    assert np.max(np.abs(gg - go)) <= 1e-8 * np.max(np.abs(go)), (gg, go)
    assert np.max(np.abs(dg.reshape(T0.shape) - do)) <= 1e-8 * np.max(np.abs(do))


@pytest.mark.parametrize("ckpt", [1, 7, 37, 59, 60, 1000])
def test_gpu_adjoint_checkpoint_invariance(ckpt):
    """The gradient does not depend on the checkpoint interval: many segments,
    a last segment starting at an odd step (37, 59), one segment (60, 1000)."""
    cfg = _case()
    n = 60
    t0 = 1.0e-3 - 30 * cfg["dt"]
    T0 = inputs.initial_field(cfg, "smooth", seed=6)
    target = inputs.target_waveform(cfg, t0 + cfg["dt"] * np.arange(1, n + 1))
    lo, go, do = oracle.adjoint(cfg, T0, n, t0, cfg["dt"], target, ckpt=16)
    lg, gg, dg = _gpu_adjoint([cfg], [T0], n, t0, [target], ckpt=ckpt)
    assert abs(lg[0] - lo) <= 1e-10 * lo
    assert np.max(np.abs(gg - go)) <= 1e-8 * np.max(np.abs(go)), (gg, go)
    assert np.max(np.abs(dg.reshape(T0.shape) - do)) <= 1e-8 * np.max(np.abs(do))


def test_gpu_adjoint_central_differences_256x1024():
    """Central differences of the GPU loss on the gradient workload's own grid
    (5 layers, 256 x 1024, tanh pulse edges), 400 steps across the pulse's
    switch-off, for the three parameters the loss depends on most over that
    horizon (in 2.5 us the heater's effect has not reached the surface, so the
    heater amplitude and pulse length move the loss by less than its FP64
    summation error; they are checked on the smaller grid above and against
    the oracle adjoint at this size).  h = 1e-4 relative keeps both the
    cancellation in the differences and their O(h^2) truncation well below the
    1e-5 bar."""
    cfg = inputs.adjoint_case()
    n = 400
    t0 = cfg["source"]["t_on"] - 200 * cfg["dt"]   # the smoothed falling edge mid-run
    T0 = inputs.initial_field(cfg, "smooth", seed=3)
    target = inputs.target_waveform(cfg, t0 + cfg["dt"] * np.arange(1, n + 1))
    _, gg, _ = _gpu_adjoint([cfg], [T0], n, t0, [target], ckpt=128, want_dT0=False)
    L = len(cfg["layers"])
    loss0 = _gpu_loss(cfg, T0, n, t0, target)
    for k in np.argsort(-np.abs(gg[2:]))[:3] + 2:   # layer scales by |dJ/dtheta|
        k = int(k)
        assert abs(gg[k]) > 1e-8 * loss0, (k, gg)      # sensitive enough for differences
        h = 1e-4
        key = "lam_scale" if k < 2 + L else "cap_scale"
        m = (k - 2) % L
        vals = []
        for sgn in (+1, -1):
            c = copy.deepcopy(cfg)
            base = c["layers"][m].get(key, 1.0)
            c["layers"][m][key] = base * (1 + sgn * h)
            vals.append(_gpu_loss(c, T0, n, t0, target))
        fd = (vals[0] - vals[1]) / (2 * h * base)
        assert abs(fd - gg[k]) <= 1e-5 * abs(fd), (k, fd, gg[k])


def test_gpu_adjoint_64x128_full_20ms():
    """The gradient workload's source and materials on the 64 x 128 grid over
    the full 20 ms (40 000 steps of 0.5 us, two smoothed pulses) from the
    configured 20 K start, checkpoints every 256 steps, against the oracle
    adjoint: loss, every parameter and dJ/dT0."""
    cfg = inputs.adjoint_case(nr=64, nz=128)
    cfg["dt"] = 5.0e-7                               # 0.92 x the stability bound
    assert cfg["dt"] <= oracle.tau_stab(cfg, 20.0, 100.0)
    n = int(round(20e-3 / cfg["dt"]))
    T0 = inputs.initial_field(cfg, "uniform")
    target = inputs.target_waveform(cfg, cfg["dt"] * np.arange(1, n + 1))
    lo, go, do = oracle.adjoint(cfg, T0, n, 0.0, cfg["dt"], target, ckpt=256)
    lg, gg, dg = _gpu_adjoint([cfg], [T0], n, 0.0, [target], ckpt=256)
    assert abs(lg[0] - lo) <= 1e-10 * lo
    assert np.max(np.abs(gg - go)) <= 1e-8 * np.max(np.abs(go)), (gg, go)
    assert np.max(np.abs(dg.reshape(T0.shape) - do)) <= 1e-8 * np.max(np.abs(do))
