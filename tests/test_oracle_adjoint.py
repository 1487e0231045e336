"""Pins of the oracle's discrete adjoint (reverse-time VJP of the scheme).

The adjoint is pinned to the forward oracle, which is itself pinned: its
vector-Jacobian products must agree with central finite differences of the
forward step (dot-product tests in state and parameter directions), and the
gradient of the surface-waveform loss must agree with central finite
differences of the loss (h = 1e-6 relative) to 1e-5 relative.
"""
import copy

import numpy as np
import pytest

from oracle import oracle
from paper_1408_5853_gb300 import inputs


def _case(nr=14, nz=9, rule=0, face=0, g_model=0, bc_rmax=0, bc_z=(0, 1)):
    cfg = inputs.adjoint_case(nr=nr, nz=nz)
    cfg["layers"] = cfg["layers"][:3]
    cfg["source"].update(layer=2, g_model=g_model, g_ref=4.0, edge_w=20e-6)
    cfg.update(interface_rule=rule, face_rule=face, bc_rmax=bc_rmax, bc_z0=bc_z[0],
               bc_zmax=bc_z[1])
    cfg["dt"] = 0.5 * oracle.tau_stab(cfg, 20.0, 100.0)
    return cfg


def _params(cfg):
    L = len(cfg["layers"])
    return ([("q0", None)] + [("t_on", None)] + [("lam_scale", m) for m in range(L)]
            + [("cap_scale", m) for m in range(L)])


def _perturb(cfg, k, h):
    c = copy.deepcopy(cfg)
    name, m = _params(cfg)[k]
    if name == "q0":
        c["source"]["q0"] += h * cfg["source"]["q0"]
        return c, h * cfg["source"]["q0"]
    if name == "t_on":
        c["source"]["t_on"] += h * cfg["source"]["t_on"]
        return c, h * cfg["source"]["t_on"]
    base = c["layers"][m].get(name, 1.0)
    c["layers"][m][name] = base + h * base
    return c, h * base


@pytest.mark.parametrize("rule,face,g_model,bc_rmax,bc_z", [
    (0, 0, 0, 0, (0, 1)), (1, 0, 1, 0, (0, 1)), (0, 1, 0, 1, (0, 1)),
    (0, 0, 0, 0, (1, 0)),     # Dirichlet z = 0, Neumann z = z_max
])
def test_step_vjp_dot_product(rule, face, g_model, bc_rmax, bc_z):
    cfg = _case(rule=rule, face=face, g_model=g_model, bc_rmax=bc_rmax, bc_z=bc_z)
    rng = np.random.default_rng(11)
    x = inputs.initial_field(cfg, "smooth", seed=4) + 0.3 * rng.random((cfg["nz"], cfg["nr"]))
    tn = 1.0e-3 - 5e-6        # on the falling tanh edge: d s / d t_on != 0
    dt = cfg["dt"]
    y, _, _ = oracle.step_n(cfg, x, 1, tn, dt)
    mu = rng.standard_normal(x.shape)
    xbar, gbar = oracle.step_vjp(cfg, x, y, mu, tn, dt)
    # state directions
    for trial in range(3):
        v = rng.standard_normal(x.shape)
        eps = 1e-4
        yp, _, _ = oracle.step_n(cfg, x + eps * v, 1, tn, dt)
        ym, _, _ = oracle.step_n(cfg, x - eps * v, 1, tn, dt)
        fd = np.sum(mu * (yp - ym)) / (2 * eps)
        ad = np.sum(xbar * v)
        assert abs(fd - ad) <= 1e-6 * max(abs(fd), np.sum(np.abs(mu * (yp - ym))) / (2 * eps)), (fd, ad)
    # parameter directions
    for k in range(oracle.n_params(cfg)):
        h = 1e-6
        cp, dp = _perturb(cfg, k, h)
        cm, dm = _perturb(cfg, k, -h)
        yp, _, _ = oracle.step_n(cp, x, 1, tn, dt)
        ym, _, _ = oracle.step_n(cm, x, 1, tn, dt)
        fd = np.sum(mu * (yp - ym)) / (dp - dm)
        scale = np.sum(np.abs(mu * (yp - ym))) / abs(dp - dm) + 1e-300
        assert abs(fd - gbar[k]) <= 1e-5 * scale + 1e-12 * abs(fd), (_params(cfg)[k], fd, gbar[k])


def _loss(cfg, T0, n, t0, target):
    _, tr, _ = oracle.step_n(cfg, T0, n, t0, cfg["dt"], want_energy=False)
    return float(np.sum(cfg["dt"] * (tr[:, 1] - target) ** 2))


def test_adjoint_gradient_matches_central_differences():
    cfg = _case(nr=16, nz=12)
    n = 160
    t0 = 1.0e-3 - 80 * cfg["dt"]
    T0 = inputs.initial_field(cfg, "smooth", seed=2)
    target = inputs.target_waveform(cfg, t0 + cfg["dt"] * np.arange(1, n + 1))
    loss, grad, dT0 = oracle.adjoint(cfg, T0, n, t0, cfg["dt"], target, ckpt=37)
    assert abs(loss - _loss(cfg, T0, n, t0, target)) <= 1e-12 * loss
    for k in range(oracle.n_params(cfg)):
        h = 1e-6
        cp, dp = _perturb(cfg, k, h)
        cm, dm = _perturb(cfg, k, -h)
        fd = (_loss(cp, T0, n, t0, target) - _loss(cm, T0, n, t0, target)) / (dp - dm)
        assert abs(fd - grad[k]) <= 1e-5 * abs(fd) + 1e-9 * loss, (_params(cfg)[k], fd, grad[k])
    # dJ/dT0: random directions over the whole field, and the largest components
    # (eps = 1e-3 K: smaller steps are limited by the rounding of the loss)
    rng = np.random.default_rng(3)
    for _ in range(3):
        v = rng.standard_normal(T0.shape)
        eps = 1e-3
        fd = (_loss(cfg, T0 + eps * v, n, t0, target) - _loss(cfg, T0 - eps * v, n, t0, target)) / (2 * eps)
        ad = float(np.sum(dT0 * v))
        assert abs(fd - ad) <= 1e-5 * np.sum(np.abs(dT0 * v)), (fd, ad)
    for flat in np.argsort(-np.abs(dT0).ravel())[:4]:
        j, i = np.unravel_index(flat, T0.shape)
        eps = 1e-3
        Tp, Tm = T0.copy(), T0.copy()
        Tp[j, i] += eps
        Tm[j, i] -= eps
        fd = (_loss(cfg, Tp, n, t0, target) - _loss(cfg, Tm, n, t0, target)) / (2 * eps)
        assert abs(fd - dT0[j, i]) <= 1e-5 * abs(fd), (j, i, fd, dT0[j, i])


def test_adjoint_checkpoint_interval_invariance():
    cfg = _case(nr=14, nz=9)
    n = 50
    T0 = inputs.initial_field(cfg, "smooth", seed=5)
    target = np.full(n, 30.0)
    ref = oracle.adjoint(cfg, T0, n, 0.0, cfg["dt"], target, ckpt=1)
    for ck in (7, 50, 1000):
        got = oracle.adjoint(cfg, T0, n, 0.0, cfg["dt"], target, ckpt=ck)
        assert got[0] == ref[0]
        assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])
