"""Python access to the FP64 CPU oracle in ``oracle/ccell_oracle.c``.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this module.  The CUDA product path
(``paper_1408_5853_gb300``) never imports it and shares no code with it.

The oracle computes the explicit-implicit time step of Section 3 of the paper
(Eqs. (scheme_eq)-(cc_first_3)) with plain FP64 loops; see the header of
``ccell_oracle.c`` for the equations and the readings it takes.

A problem is described by a plain dict (see ``paper_1408_5853_gb300.inputs``);
this module marshals it into the oracle's own C struct.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ccell_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libccell_oracle.so")
MAX_LAYERS = 8

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, OpenMP if present)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found to build the oracle")
    base = [cc, "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
            _SRC, "-o", _SO + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


class Problem(ctypes.Structure):
    L = MAX_LAYERS
    _fields_ = [
        ("n_layers", ctypes.c_int),
        ("thickness", ctypes.c_double * L),
        ("nr", ctypes.c_int), ("nz", ctypes.c_int),
        ("length", ctypes.c_double),
        ("bc_rmax", ctypes.c_int), ("bc_z0", ctypes.c_int), ("bc_zmax", ctypes.c_int),
        ("t_dirichlet", ctypes.c_double),
        ("placement", ctypes.c_int),
        ("face_rule", ctypes.c_int), ("interface_rule", ctypes.c_int),
        ("rho", ctypes.c_double * L),
        ("lam_model", ctypes.c_int * L),
        ("lam0", ctypes.c_double * L), ("lam_b", ctypes.c_double * L),
        ("cap_model", ctypes.c_int * L),
        ("c0", ctypes.c_double * L), ("theta", ctypes.c_double * L),
        ("t_ref", ctypes.c_double * L),
        ("lam_scale", ctypes.c_double * L), ("cap_scale", ctypes.c_double * L),
        ("lam_poly", (ctypes.c_double * 5) * L),
        ("cap_poly", (ctypes.c_double * 4) * L),
        ("src_layer", ctypes.c_int),
        ("q0", ctypes.c_double),
        ("t_period", ctypes.c_double), ("t_on", ctypes.c_double), ("t_start", ctypes.c_double),
        ("waveform", ctypes.c_int),
        ("edge_w", ctypes.c_double),
        ("g_model", ctypes.c_int),
        ("g_ref", ctypes.c_double),
        ("step_layers", ctypes.c_int),
        ("z_step", ctypes.c_double),
    ]


def _load():
    global _lib
    if _lib is None:
        # CCELL_ORACLE_SO lets the mutation tests load a deliberately broken build
        lib = ctypes.CDLL(os.environ.get("CCELL_ORACLE_SO") or build())
        P = ctypes.POINTER(Problem)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.or_grid.argtypes = [P, dp, dp, ip, ip]
        lib.or_grid.restype = ctypes.c_int
        lib.or_outline.argtypes = [P, dp, ip, ip, ip]
        lib.or_outline.restype = ctypes.c_int
        lib.or_line_rows.argtypes = [P, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp,
                                     dp, dp, dp, ip]
        lib.or_line_rows.restype = ctypes.c_int
        lib.or_step_n.argtypes = [P, dp, ctypes.c_long, ctypes.c_double, ctypes.c_double, dp, dp]
        lib.or_step_n.restype = ctypes.c_int
        lib.or_step_adi_n.argtypes = [P, dp, ctypes.c_long, ctypes.c_double, ctypes.c_double, dp]
        lib.or_step_adi_n.restype = ctypes.c_int
        lib.or_tau_stab.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_int]
        lib.or_tau_stab.restype = ctypes.c_double
        lib.or_waveform.argtypes = [P, ctypes.c_double]
        lib.or_waveform.restype = ctypes.c_double
        lib.or_step_vjp.argtypes = [P, dp, dp, dp, ctypes.c_double, ctypes.c_double, dp, dp]
        lib.or_step_vjp.restype = ctypes.c_int
        lib.or_adjoint.argtypes = [P, dp, ctypes.c_long, ctypes.c_double, ctypes.c_double, dp,
                                   ctypes.c_int, dp, dp, dp]
        lib.or_adjoint.restype = ctypes.c_int
        lib.or_num_threads.restype = ctypes.c_int
        lib.or_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def problem(cfg: dict) -> Problem:
    """Marshal a problem dict into the oracle's C struct."""
    p = Problem()
    layers = cfg["layers"]
    if not 1 <= len(layers) <= MAX_LAYERS:
        raise ValueError("1..8 layers")
    p.n_layers = len(layers)
    for m, ly in enumerate(layers):
        p.thickness[m] = ly["thickness"]
        p.rho[m] = ly["rho"]
        p.lam_model[m] = ly.get("lam_model", 1)
        p.lam0[m] = ly.get("lam0", 0.0)
        p.lam_b[m] = ly.get("lam_b", 0.0)
        p.cap_model[m] = ly.get("cap_model", 1)
        p.c0[m] = ly.get("c0", 0.0)
        p.theta[m] = ly.get("theta", 1.0)
        p.t_ref[m] = ly.get("t_ref", 20.0)
        p.lam_scale[m] = ly.get("lam_scale", 1.0)
        p.cap_scale[m] = ly.get("cap_scale", 1.0)
        for k, v in enumerate(ly.get("lam_poly", [0.0] * 5)):
            p.lam_poly[m][k] = v
        for k, v in enumerate(ly.get("cap_poly", [0.0] * 4)):
            p.cap_poly[m][k] = v
    p.nr, p.nz = cfg["nr"], cfg["nz"]
    p.length = cfg["length"]
    p.bc_rmax = cfg.get("bc_rmax", 0)
    p.bc_z0 = cfg.get("bc_z0", 0)
    p.bc_zmax = cfg.get("bc_zmax", 1)
    p.t_dirichlet = cfg.get("t_dirichlet", 20.0)
    p.placement = cfg.get("placement", 0)
    p.face_rule = cfg.get("face_rule", 0)
    p.interface_rule = cfg.get("interface_rule", 0)
    src = cfg.get("source")
    if src is None:
        p.src_layer = -1
    else:
        p.src_layer = src["layer"]
        p.q0 = src["q0"]
        p.t_period = src["t_period"]
        p.t_on = src["t_on"]
        p.t_start = src.get("t_start", 0.0)
        p.waveform = src.get("waveform", 0)
        p.edge_w = src.get("edge_w", 0.0)
        p.g_model = src.get("g_model", 0)
        p.g_ref = src.get("g_ref", 0.0)
    step = cfg.get("step")
    if step is not None:
        p.step_layers = step["layers"]
        p.z_step = step["z"]
    return p


def grid(cfg: dict) -> dict:
    """Node positions r[nr], z[nz], radial node classes and segment layers."""
    lib = _load()
    p = problem(cfg)
    r = np.zeros(cfg["nr"])
    z = np.zeros(cfg["nz"])
    cls = np.zeros(cfg["nr"], dtype=np.int32)
    seg = np.zeros(cfg["nr"], dtype=np.int32)
    rc = lib.or_grid(ctypes.byref(p), _dp(r), _dp(z), _ip(cls), _ip(seg))
    if rc != 0:
        raise ValueError("oracle rejected the grid description")
    return {"r": r, "z": z, "rclass": cls, "seg": seg}


def outline(cfg: dict) -> tuple:
    """(i_step, j_narrow) of the stepped outline: the lines j >= j_narrow end at
    the radial node i_step; a rectangle gives (nr - 1, nz)."""
    lib = _load()
    p = problem(cfg)
    g = grid(cfg)
    i_step = np.zeros(1, dtype=np.int32)
    j_narrow = np.zeros(1, dtype=np.int32)
    if lib.or_outline(ctypes.byref(p), _dp(g["z"]), _ip(g["rclass"]), _ip(i_step),
                      _ip(j_narrow)) != 0:
        raise ValueError("oracle rejected the outline")
    return int(i_step[0]), int(j_narrow[0])


def line_rows(cfg: dict, T: np.ndarray, j: int, t: float, dt: float) -> tuple:
    """Rows (a, b, c, f) of the tridiagonal system of line j that one step from
    T at time t solves (row i: a_i x_{i-1} + b_i x_i + c_i x_{i+1} = f_i)."""
    lib = _load()
    p = problem(cfg)
    T = np.ascontiguousarray(T, dtype=np.float64)
    a, b, c, f = (np.zeros(cfg["nr"]) for _ in range(4))
    n = np.zeros(1, dtype=np.int32)
    if lib.or_line_rows(ctypes.byref(p), _dp(T), int(j), float(t), float(dt), _dp(a), _dp(b),
                        _dp(c), _dp(f), _ip(n)) != 0:
        raise ValueError("oracle rejected the line")
    k = int(n[0])
    return a[:k], b[:k], c[:k], f[:k]


def step_n(cfg: dict, T: np.ndarray, n_steps: int, t0: float, dt: float,
           want_trace: bool = True, want_energy: bool = True):
    """Run n_steps of the scheme.  Returns (T_new, trace[n,2] or None, energy[5] or None).

    energy = (stored heat dE, source Q, Dirichlet-edge flux, interface-edge
    flux, Neumann-edge flux), each summed over the steps.
    """
    lib = _load()
    p = problem(cfg)
    T = np.ascontiguousarray(T, dtype=np.float64).copy()
    if T.shape != (cfg["nz"], cfg["nr"]):
        raise ValueError(f"T must have shape (nz, nr) = {(cfg['nz'], cfg['nr'])}")
    trace = np.zeros((n_steps, 2)) if want_trace else None
    energy = np.zeros(5) if want_energy else None
    rc = lib.or_step_n(ctypes.byref(p), _dp(T), int(n_steps), float(t0), float(dt),
                       _dp(trace) if trace is not None else None,
                       _dp(energy) if energy is not None else None)
    if rc != 0:
        raise ValueError("oracle rejected the problem")
    return T, trace, energy


def step_adi_n(cfg: dict, T: np.ndarray, n_steps: int, t0: float, dt: float,
               want_trace: bool = True):
    """Run n_steps of the Peaceman-Rachford ADI variant (two half steps of
    dt/2: implicit in r, then implicit in z).  Returns (T_new, trace[n,2] or None)."""
    lib = _load()
    p = problem(cfg)
    T = np.ascontiguousarray(T, dtype=np.float64).copy()
    if T.shape != (cfg["nz"], cfg["nr"]):
        raise ValueError(f"T must have shape (nz, nr) = {(cfg['nz'], cfg['nr'])}")
    trace = np.zeros((n_steps, 2)) if want_trace else None
    rc = lib.or_step_adi_n(ctypes.byref(p), _dp(T), int(n_steps), float(t0), float(dt),
                           _dp(trace) if trace is not None else None)
    if rc != 0:
        raise ValueError("oracle rejected the problem")
    return T, trace


def n_params(cfg: dict) -> int:
    """Parameters of the adjoint: q0, t_on, lam_scale[L], cap_scale[L]."""
    return 2 + 2 * len(cfg["layers"])


def step_vjp(cfg: dict, x: np.ndarray, y: np.ndarray, mu: np.ndarray, tn: float, dt: float):
    """Adjoint of one step from x (T^n) to y (T^{n+1}) for mu = dJ/dT^{n+1}.
    Returns (dJ/dT^n, dJ/dtheta)."""
    lib = _load()
    p = problem(cfg)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    mu = np.ascontiguousarray(mu, dtype=np.float64).copy()
    xbar = np.zeros_like(x)
    gbar = np.zeros(n_params(cfg))
    if lib.or_step_vjp(ctypes.byref(p), _dp(x), _dp(y), _dp(mu), float(tn), float(dt),
                       _dp(xbar), _dp(gbar)) != 0:
        raise ValueError("oracle rejected the problem")
    return xbar, gbar


def adjoint(cfg: dict, T0: np.ndarray, n_steps: int, t0: float, dt: float, target: np.ndarray,
            ckpt: int = 256):
    """Loss J = sum_n dt (Sbar_n - target_n)^2 and its gradient with respect to
    theta = (q0, t_on, lam_scale[], cap_scale[]) and to T0."""
    lib = _load()
    p = problem(cfg)
    T0 = np.ascontiguousarray(T0, dtype=np.float64)
    target = np.ascontiguousarray(target, dtype=np.float64)
    if target.shape != (n_steps,):
        raise ValueError("target must have n_steps entries")
    loss = np.zeros(1)
    grad = np.zeros(n_params(cfg))
    dT0 = np.zeros_like(T0)
    if lib.or_adjoint(ctypes.byref(p), _dp(T0), int(n_steps), float(t0), float(dt), _dp(target),
                      int(ckpt), _dp(loss), _dp(grad), _dp(dT0)) != 0:
        raise ValueError("oracle rejected the problem")
    return float(loss[0]), grad, dT0


def tau_stab(cfg: dict, t_lo: float, t_hi: float, n_samples: int = 257) -> float:
    """Eq. (stability_condition): (min eta^2 / 2) * min over layers and T of rho c / lambda."""
    return _load().or_tau_stab(ctypes.byref(problem(cfg)), t_lo, t_hi, n_samples)


def waveform(cfg: dict, t: float) -> float:
    return _load().or_waveform(ctypes.byref(problem(cfg)), float(t))


def num_threads() -> int:
    return _load().or_num_threads()


def set_threads(n: int) -> None:
    _load().or_set_threads(int(n))


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
