"""Seeded synthetic workloads for the explicit-implicit heat-conduction step.

This module only *describes* problems (plain dicts) and draws seeded initial
fields; it contains none of the scheme's arithmetic, so both the CUDA path and
the CPU oracle can take their inputs from it.

A problem dict holds:
  layers         list of per-layer dicts, innermost (r = 0) first:
                 thickness [m], rho [kg/m^3], lam_model (0 const, 1 power
                 law lam0 (T/t_ref)^lam_b), lam0 [W/m/K], lam_b, cap_model
                 (0 const, 1 c0 (T/t_ref)^3 / (1 + (T/theta)^3)), c0 [J/kg/K],
                 theta [K], t_ref [K], lam_scale, cap_scale
  nr, nz         radial / axial node counts (boundary nodes included)
  length         axial extent [m]
  bc_rmax, bc_z0, bc_zmax   0 Neumann, 1 Dirichlet at t_dirichlet [K]
  placement      0 vertex nodes (paper), 1 half-cell ghost nodes
  face_rule      0 lambda(mean T), 1 mean of nodal lambda
  interface_rule 0 paper's first-order interface rows, 1 conservative
  source         {layer, q0 [W/m^3], t_period, t_on, t_start [s],
                  waveform (0 rectangle, 1 tanh edges), edge_w [s], g_model, g_ref}
  dt             time step [s]

The workloads follow the synthetic configurations the solver is measured on:
a 4-layer 64x128 cylinder, the 5-layer 512x4096 production case with +/-10 %
jittered properties (seed 0), a batched design sweep of 256 ragged instances
(seed 1) and the 5-layer 256x1024 case with smoothed pulse edges used for
gradients.  Time steps are the largest "round" values under the axial
stability bound of the explicit z-direction (Eq. (stability_condition)),
because the scheme is explicit in z.
"""
from __future__ import annotations

import copy
import json
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_CALIB = os.path.join(_HERE, "calibration.json")

T_INIT = 20.0  # K, initial and Dirichlet temperature of the workloads

# 4-layer cylinder: core, insulator, heater, jacket (radial thickness in m)
_BASE_LAYERS = [
    dict(thickness=0.10e-3, rho=7900.0, lam0=15.0, lam_b=1.0, c0=5.0, theta=60.0),
    dict(thickness=0.02e-3, rho=1400.0, lam0=0.5, lam_b=0.5, c0=20.0, theta=40.0),
    dict(thickness=0.05e-3, rho=8900.0, lam0=100.0, lam_b=1.2, c0=2.0, theta=80.0),
    dict(thickness=0.10e-3, rho=7900.0, lam0=15.0, lam_b=1.0, c0=5.0, theta=60.0),
]
_OUTER_LAYER = dict(thickness=0.05e-3, rho=2700.0, lam0=2.0, lam_b=0.8, c0=10.0, theta=50.0)
HEATER = 2  # 0-based index of the heater layer


def heater_q0() -> float:
    """Heater amplitude [W/m^3] calibrated on the 64x128 case (surface peak 45 K).

    Written by ``oracle/calibrate_q0.py``; the value is an input of every
    workload, not a result of the solver under test.
    """
    with open(_CALIB) as f:
        return float(json.load(f)["q0_W_m3"])


def _layer(d: dict) -> dict:
    out = dict(lam_model=1, cap_model=1, t_ref=20.0, lam_scale=1.0, cap_scale=1.0)
    out.update(d)
    return out


def _base(nr, nz, layers, dt, q0, t_on=1e-3, t_period=10e-3) -> dict:
    return dict(
        layers=[_layer(l) for l in layers], nr=nr, nz=nz, length=10e-3,
        bc_rmax=0, bc_z0=0, bc_zmax=1, t_dirichlet=T_INIT,
        placement=0, face_rule=0, interface_rule=0,
        source=dict(layer=HEATER, q0=q0, t_period=t_period, t_on=t_on, t_start=0.0,
                    waveform=0, edge_w=0.0, g_model=0, g_ref=0.0),
        dt=dt,
    )


def small_case(q0: float | None = None) -> dict:
    """4 layers (0.10/0.02/0.05/0.10 mm), 64x128, 1 ms pulse every 10 ms, dt 0.5 us."""
    if q0 is None:
        q0 = heater_q0()
    cfg = _base(64, 128, _BASE_LAYERS, 5.0e-7, q0)
    cfg["name"] = "4-layer r-z cylinder 64x128 (fp64)"
    cfg["n_steps_full"] = 40000  # 20 ms = 2 pulses
    return cfg


def production_case(seed: int = 0, nr: int = 512, nz: int = 4096) -> dict:
    """5 layers, 512x4096, properties jittered +/-10 % (lam0, b, c0, theta per
    layer, layer-major, uniform, numpy default_rng(seed)), dt 0.4 ns."""
    rng = np.random.default_rng(seed)
    layers = copy.deepcopy(_BASE_LAYERS) + [dict(_OUTER_LAYER)]
    for ly in layers:
        for key in ("lam0", "lam_b", "c0", "theta"):
            ly[key] = ly[key] * float(rng.uniform(0.9, 1.1))
    cfg = _base(nr, nz, layers, 4.0e-10, heater_q0())
    cfg["name"] = f"5-layer r-z cylinder {nr}x{nz}, jittered seed {seed}"
    return cfg


def batched_cases(seed: int = 1, n: int = 256) -> list[dict]:
    """Design sweep: n instances, Nr log-uniform in [64,512], Nz log-uniform in
    [256,2048], thickness +/-30 %, lam0/c0 +/-10 %, heater amplitude +/-40 %,
    pulse duration uniform in [0.5, 2] ms.  Draw order per instance: nr, nz,
    5 thickness factors, 5 lam0 factors, 5 c0 factors, amplitude, duration.
    dt is left to the caller (per-instance stability bound)."""
    rng = np.random.default_rng(seed)
    q0 = heater_q0()
    out = []
    for k in range(n):
        nr = int(round(math.exp(rng.uniform(math.log(64), math.log(512)))))
        nz = int(round(math.exp(rng.uniform(math.log(256), math.log(2048)))))
        layers = copy.deepcopy(_BASE_LAYERS) + [dict(_OUTER_LAYER)]
        for ly in layers:
            ly["thickness"] *= float(rng.uniform(0.7, 1.3))
        for ly in layers:
            ly["lam0"] *= float(rng.uniform(0.9, 1.1))
        for ly in layers:
            ly["c0"] *= float(rng.uniform(0.9, 1.1))
        amp = float(rng.uniform(0.6, 1.4))
        dur = float(rng.uniform(0.5e-3, 2.0e-3))
        cfg = _base(nr, nz, layers, 0.0, q0 * amp, t_on=dur)
        cfg["name"] = f"sweep instance {k} ({nr}x{nz})"
        out.append(cfg)
    return out


def adjoint_case(nr: int = 256, nz: int = 1024, dt: float = 6.25e-9) -> dict:
    """5 layers (nominal properties), tanh pulse edges of 20 us, 2 pulses / 20 ms."""
    layers = copy.deepcopy(_BASE_LAYERS) + [dict(_OUTER_LAYER)]
    cfg = _base(nr, nz, layers, dt, heater_q0())
    cfg["source"].update(waveform=1, edge_w=20e-6)
    cfg["name"] = f"5-layer r-z cylinder {nr}x{nz}, smoothed pulses"
    return cfg


_GOLDEN = os.path.join(os.path.dirname(_HERE), "tests", "golden", "paper_material_fits.json")


def paper_case(nr: int = 256, nz: int = 201, stepped: bool = False) -> dict:
    """The paper's cryogenic cell (Section 5): copper core 1.2 mm, insulator
    0.05 mm, graphite heater 0.05 mm, outer insulator 1 um; length 5 cm;
    polynomial fits of c_V and lambda (Tables a_coefs, b_coefs), converted
    from cgs to SI; Joule source chi(T) I(t)^2 / S_2^2 with chi = 1.8 / sqrt(T)
    Ohm cm, I0 = 363 mA and the transient turn-on (waveform 2); 1 ms pulse
    every 25 ms; T0 = 4.2 K.  Rectangular r-z domain, or with `stepped` the
    outer layers on z <= z_0 = 4 cm only and the copper core alone up to the
    helium end (the working surface r = r_max spans z in [0, z_0])."""
    with open(_GOLDEN) as f:
        fit = json.load(f)
    r_cm = fit["radii_cm"]
    thick_cm = [r_cm["r0"], r_cm["r1"] - r_cm["r0"], r_cm["r2"] - r_cm["r1"],
                r_cm["rmax"] - r_cm["r2"]]
    layers = []
    for m in range(4):
        layers.append(dict(thickness=thick_cm[m] * 1e-2, rho=fit["rho_g_cm3"][m] * 1e3,
                           lam_model=2, lam_poly=[100.0 * b for b in fit["lam_b0_b1_b2_b3_b4"][m]],
                           cap_model=2, cap_poly=[1e3 * a for a in fit["cap_a0_a1_a2_a3"][m]],
                           t_ref=1.0, theta=1.0, lam_scale=1.0, cap_scale=1.0))
    run = fit["run"]
    s2 = math.pi * ((r_cm["r2"] * 1e-2) ** 2 - (r_cm["r1"] * 1e-2) ** 2)  # heater cross-section, m^2
    chi0 = fit["chi_ohm_cm_sqrtK"] * 1e-2                                     # Ohm m sqrt(K)
    q0 = chi0 * run["I0_A"] ** 2 / s2 ** 2          # X = q0 s(t) / sqrt(T), W/m^3
    cfg = dict(layers=layers, nr=nr, nz=nz, length=fit["z_cm"]["zmax"] * 1e-2,
               bc_rmax=0, bc_z0=0, bc_zmax=1, t_dirichlet=run["T0_K"], placement=0,
               face_rule=0, interface_rule=0,
               source=dict(layer=2, q0=q0, t_period=run["t_prd_s"], t_on=run["t_src_s"],
                           t_start=0.0, waveform=2, edge_w=run["tau_s"], g_model=1, g_ref=1.0),
               dt=run["tau_s"], t_guard=(run["T0_K"], 60.0))
    if stepped:
        cfg["step"] = dict(layers=1, z=fit["z_cm"]["z0"] * 1e-2)
    cfg["name"] = f"paper cryogenic cell {nr}x{nz} (polynomial materials, transient source)"
    return cfg


def target_waveform(cfg: dict, t: np.ndarray) -> np.ndarray:
    """Surface-temperature target: 42 K while the nominal pulse window is open,
    28 K while it is closed."""
    src = cfg["source"]
    u = np.asarray(t) - src["t_start"]
    phase = np.mod(u, src["t_period"])
    return np.where((u >= 0) & (phase < src["t_on"]), 42.0, 28.0)


def initial_field(cfg: dict, kind: str = "uniform", seed: int = 0,
                  amplitude: float = 5.0) -> np.ndarray:
    """(nz, nr) FP64 field: uniform T_INIT, or T_INIT + amplitude * u with u a
    smooth seeded field in [0, 1] (a few low cosine modes in r and z)."""
    nz, nr = cfg["nz"], cfg["nr"]
    if kind == "uniform":
        return np.full((nz, nr), T_INIT)
    rng = np.random.default_rng(seed)
    x = np.linspace(0.0, 1.0, nr)[None, :]
    y = np.linspace(0.0, 1.0, nz)[:, None]
    u = np.zeros((nz, nr))
    for a in range(4):
        for b in range(4):
            u += rng.normal() / (1 + a + b) * np.cos(math.pi * a * x) * np.cos(math.pi * b * y)
    u = (u - u.min()) / max(u.max() - u.min(), 1e-300)
    return T_INIT + amplitude * u
