"""Thin Python binding of the C ABI in ``include/ccell.h`` (libccell.so).

Argument marshalling only: every step of the time step runs in the CUDA
kernels of ``csrc/``.  PyTorch provides device memory and streams.  Importing
this module loads the CUDA library and fails loudly if it is missing; there is
no CPU fallback.

Low-level functions carry the C names (``cc_create_geometry``,
``cc_set_materials``, ``cc_set_source``, ``cc_set_dt``, ``cc_step_n``, ``cc_step_adi_n``,
``cc_sync``, ``cc_adjoint``, ``cc_adjoint_vjp``, ``cc_set_launch``, ``cc_get_launch``,
``cc_autotune``, ``cc_destroy``, ``cc_step_n_noalloc``, ``cc_query_grid``, ``cc_query_outline``,
``cc_query_tiles``, ``cc_tau_stab``, ``cc_status_string``, ``cc_kernel_launches``,
``cc_measure_fp64_rate``).  ``Solver``
builds a context from the problem dicts of ``inputs``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MAX_LAYERS = 8
FP64, MIXED = 0, 1

CC_OK, CC_EINVAL, CC_ENOMEM, CC_ECUDA, CC_EUNSTABLE = 0, -1, -2, -3, -4
CC_ETIMEOUT, CC_ENONFINITE, CC_ESTATE, CC_EUNSUPPORTED = -5, -6, -7, -8

_d = ctypes.c_double
_i = ctypes.c_int32


class GeometryDesc(ctypes.Structure):
    _fields_ = [
        ("n_layers", _i), ("thickness_m", _d * MAX_LAYERS), ("nr", _i), ("nz", _i),
        ("length_m", _d), ("bc_rmax", _i), ("bc_z0", _i), ("bc_zmax", _i),
        ("t_dirichlet_K", _d), ("placement", _i), ("precision", _i), ("face_rule", _i),
        ("interface_rule", _i), ("t_guard_lo_K", _d), ("t_guard_hi_K", _d),
        ("step_layers", _i), ("z_step_m", _d),
    ]


class Material(ctypes.Structure):
    _fields_ = [
        ("rho", _d), ("lam_model", _i), ("lam0", _d), ("lam_b", _d), ("cap_model", _i),
        ("c0", _d), ("theta", _d), ("t_ref", _d), ("lam_scale", _d), ("cap_scale", _d),
        ("lam_poly", _d * 5), ("cap_poly", _d * 4),
    ]


class Source(ctypes.Structure):
    _fields_ = [
        ("layer", _i), ("q0", _d), ("t_period", _d), ("t_on", _d), ("t_start", _d),
        ("waveform", _i), ("edge_w", _d), ("g_model", _i), ("g_ref", _d),
    ]


class CCError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {cc_status_string(status)} ({status})")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        path = _build.build()
    lib = ctypes.CDLL(path)
    vp, dp = ctypes.c_void_p, ctypes.POINTER(_d)
    lib.cc_create_geometry.argtypes = [ctypes.POINTER(GeometryDesc), _i, ctypes.POINTER(vp)]
    lib.cc_set_materials.argtypes = [vp, _i, ctypes.POINTER(Material)]
    lib.cc_set_source.argtypes = [vp, _i, ctypes.POINTER(Source)]
    lib.cc_set_dt.argtypes = [vp, _i, _d]
    lib.cc_step_n.argtypes = [vp, vp, ctypes.c_int64, _d, _d, vp, vp, vp]
    lib.cc_step_adi_n.argtypes = [vp, vp, ctypes.c_int64, _d, _d, vp, vp]
    lib.cc_sync.argtypes = [vp, vp]
    lib.cc_adjoint.argtypes = [vp, vp, ctypes.c_int64, _d, _d, vp, _i, vp, vp, vp, vp]
    lib.cc_destroy.argtypes = [vp]
    lib.cc_query_grid.argtypes = [ctypes.POINTER(GeometryDesc), dp, dp, ctypes.POINTER(_i)]
    lib.cc_query_outline.argtypes = [ctypes.POINTER(GeometryDesc), ctypes.POINTER(_i),
                                     ctypes.POINTER(_i)]
    ip = ctypes.POINTER(_i)
    lib.cc_query_tiles.argtypes = [ctypes.POINTER(GeometryDesc), _i, _i, _i, _i, ip, _i, ip, ip,
                                   ip, ip]
    lib.cc_query_tiles.restype = ctypes.c_int
    lib.cc_tau_stab.argtypes = [vp, _i, dp]
    lib.cc_status_string.argtypes = [ctypes.c_int]
    lib.cc_status_string.restype = ctypes.c_char_p
    lib.cc_kernel_launches.restype = ctypes.c_int64
    lib.cc_step_n_noalloc.argtypes = [ctypes.POINTER(GeometryDesc), ctypes.POINTER(Material),
                                      ctypes.POINTER(Source), vp, ctypes.c_int64, _d, _d, vp,
                                      vp, vp]
    lib.cc_step_n_noalloc.restype = ctypes.c_int
    lib.cc_set_launch.argtypes = [vp, _i, _i, _i]
    lib.cc_set_launch.restype = ctypes.c_int
    lib.cc_get_launch.argtypes = [vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)]
    lib.cc_get_launch.restype = ctypes.c_int
    lib.cc_autotune.argtypes = [vp, vp, _i, ctypes.POINTER(ctypes.c_float), vp]
    lib.cc_autotune.restype = ctypes.c_int
    lib.cc_adjoint_vjp.argtypes = [vp, vp, ctypes.c_int64, _d, _d, vp, _i, vp, vp, vp]
    lib.cc_adjoint_vjp.restype = ctypes.c_int
    lib.cc_measure_fp64_rate.argtypes = [vp, ctypes.c_int64, _i, dp, dp, vp]
    lib.cc_measure_fp64_rate.restype = ctypes.c_int
    for name in ("cc_create_geometry", "cc_set_materials", "cc_set_source", "cc_set_dt",
                 "cc_step_n", "cc_step_adi_n", "cc_sync", "cc_adjoint", "cc_destroy",
                 "cc_query_grid", "cc_query_outline", "cc_tau_stab"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int, what: str) -> None:
    if status != CC_OK:
        raise CCError(status, what)


# ---------------------------------------------------------------------------
# C names
# ---------------------------------------------------------------------------
def cc_status_string(status: int) -> str:
    return _load().cc_status_string(int(status)).decode()


def cc_kernel_launches() -> int:
    return int(_load().cc_kernel_launches())


def cc_measure_fp64_rate(scratch_ptr: int, scratch_len: int, iters: int, stream_ptr) -> tuple:
    """(FP64 FMAs per second, seconds of the timed launch) of the current GPU."""
    rate, sec = _d(0.0), _d(0.0)
    _check(_load().cc_measure_fp64_rate(ctypes.c_void_p(scratch_ptr), scratch_len, iters,
                                        ctypes.byref(rate), ctypes.byref(sec),
                                        ctypes.c_void_p(stream_ptr)), "cc_measure_fp64_rate")
    return rate.value, sec.value


def cc_create_geometry(descs) -> ctypes.c_void_p:
    arr = (GeometryDesc * len(descs))(*descs)
    ctx = ctypes.c_void_p()
    _check(_load().cc_create_geometry(arr, len(descs), ctypes.byref(ctx)), "cc_create_geometry")
    return ctx


def cc_set_materials(ctx, instance: int, materials) -> None:
    arr = (Material * len(materials))(*materials)
    _check(_load().cc_set_materials(ctx, instance, arr), "cc_set_materials")


def cc_set_source(ctx, instance: int, source: Source) -> None:
    _check(_load().cc_set_source(ctx, instance, ctypes.byref(source)), "cc_set_source")


def cc_set_dt(ctx, instance: int, dt: float) -> None:
    _check(_load().cc_set_dt(ctx, instance, float(dt)), "cc_set_dt")


def cc_step_adi_n(ctx, T_ptr: int, n_steps: int, t0: float, dt: float, trace_ptr,
                  stream_ptr) -> None:
    _check(_load().cc_step_adi_n(ctx, T_ptr, int(n_steps), float(t0), float(dt), trace_ptr,
                                 stream_ptr), "cc_step_adi_n")


def cc_step_n(ctx, T_ptr: int, n_steps: int, t0: float, dt: float, trace_ptr, energy_ptr,
              stream_ptr) -> None:
    _check(_load().cc_step_n(ctx, T_ptr, int(n_steps), float(t0), float(dt), trace_ptr,
                             energy_ptr, stream_ptr), "cc_step_n")


def cc_sync(ctx, stream_ptr) -> None:
    _check(_load().cc_sync(ctx, stream_ptr), "cc_sync")


def cc_adjoint(ctx, T0_ptr, n_steps, t0, dt, target_ptr, ckpt_every, loss_ptr, grad_ptr,
               dT0_ptr, stream_ptr) -> None:
    _check(_load().cc_adjoint(ctx, T0_ptr, int(n_steps), float(t0), float(dt), target_ptr,
                              int(ckpt_every), loss_ptr, grad_ptr, dT0_ptr, stream_ptr),
           "cc_adjoint")


def cc_set_launch(ctx, mode: int, threads: int, rows_per_lane: int) -> None:
    _check(_load().cc_set_launch(ctx, int(mode), int(threads), int(rows_per_lane)),
           "cc_set_launch")


def cc_get_launch(ctx) -> tuple:
    m, t, r = _i(), _i(), _i()
    _check(_load().cc_get_launch(ctx, ctypes.byref(m), ctypes.byref(t), ctypes.byref(r)),
           "cc_get_launch")
    return m.value, t.value, r.value


def cc_autotune(ctx, T_ptr: int, n_trial: int, stream_ptr) -> float:
    best = ctypes.c_float()
    _check(_load().cc_autotune(ctx, T_ptr, int(n_trial), ctypes.byref(best), stream_ptr),
           "cc_autotune")
    return best.value


def cc_adjoint_vjp(ctx, T0_ptr, n_steps, t0, dt, seed_ptr, ckpt_every, grad_ptr, dT0_ptr,
                   stream_ptr) -> None:
    _check(_load().cc_adjoint_vjp(ctx, T0_ptr, int(n_steps), float(t0), float(dt), seed_ptr,
                                  int(ckpt_every), grad_ptr, dT0_ptr, stream_ptr),
           "cc_adjoint_vjp")


def cc_step_n_noalloc(desc: GeometryDesc, materials_list, source_struct: Source, T_ptr: int,
                      n_steps: int, t0: float, dt: float, trace_ptr, energy_ptr,
                      stream_ptr) -> None:
    """One FP64 instance, no device allocation (scratch in a static device array)."""
    arr = (Material * len(materials_list))(*materials_list)
    _check(_load().cc_step_n_noalloc(ctypes.byref(desc), arr, ctypes.byref(source_struct), T_ptr,
                                     int(n_steps), float(t0), float(dt), trace_ptr, energy_ptr,
                                     stream_ptr), "cc_step_n_noalloc")


def cc_destroy(ctx) -> None:
    _check(_load().cc_destroy(ctx), "cc_destroy")


def cc_query_grid(desc: GeometryDesc):
    r = np.zeros(desc.nr)
    z = np.zeros(desc.nz)
    cls = np.zeros(desc.nr, dtype=np.int32)
    _check(_load().cc_query_grid(ctypes.byref(desc), r.ctypes.data_as(ctypes.POINTER(_d)),
                                 z.ctypes.data_as(ctypes.POINTER(_d)),
                                 cls.ctypes.data_as(ctypes.POINTER(_i))), "cc_query_grid")
    return r, z, cls


def cc_query_tiles(descs, threads: int, rows_per_lane: int, n_blocks: int):
    """CTA tiles of the step kernels for these descriptors: (tiles[n, 3] =
    (instance, j0, nl), cta[n_blocks + 1] or None, lanes per instance,
    shared-memory bytes of the largest tile)."""
    arr = (GeometryDesc * len(descs))(*descs)
    n = _i(0)
    _check(_load().cc_query_tiles(arr, len(descs), threads, rows_per_lane, n_blocks, None, 0,
                                  ctypes.byref(n), None, None, None), "cc_query_tiles")
    tiles = np.zeros((max(n.value, 1), 3), dtype=np.int32)
    cta = np.zeros(n_blocks + 1, dtype=np.int32)
    lanes = np.zeros(len(descs), dtype=np.int32)
    smem = _i(0)
    ip = ctypes.POINTER(_i)
    _check(_load().cc_query_tiles(arr, len(descs), threads, rows_per_lane, n_blocks,
                                  tiles.ctypes.data_as(ip), n.value, ctypes.byref(n),
                                  cta.ctypes.data_as(ip) if n_blocks > 0 else None,
                                  lanes.ctypes.data_as(ip), ctypes.byref(smem)),
           "cc_query_tiles")
    return tiles[:n.value], (cta if n_blocks > 0 else None), lanes, smem.value


def cc_query_outline(desc: GeometryDesc) -> tuple:
    """(i_step, j_narrow) of a stepped outline: the lines j >= j_narrow end at
    the radial node i_step; a rectangle gives (nr - 1, nz)."""
    i_step, j_narrow = _i(0), _i(0)
    _check(_load().cc_query_outline(ctypes.byref(desc), ctypes.byref(i_step),
                                    ctypes.byref(j_narrow)), "cc_query_outline")
    return i_step.value, j_narrow.value


def cc_tau_stab(ctx, instance: int) -> float:
    out = _d()
    _check(_load().cc_tau_stab(ctx, instance, ctypes.byref(out)), "cc_tau_stab")
    return out.value


# ---------------------------------------------------------------------------
# problem dicts -> C structs
# ---------------------------------------------------------------------------
def geometry_desc(cfg: dict, precision: int = FP64) -> GeometryDesc:
    d = GeometryDesc()
    d.n_layers = len(cfg["layers"])
    for m, ly in enumerate(cfg["layers"]):
        d.thickness_m[m] = ly["thickness"]
    d.nr, d.nz = cfg["nr"], cfg["nz"]
    d.length_m = cfg["length"]
    d.bc_rmax, d.bc_z0, d.bc_zmax = cfg.get("bc_rmax", 0), cfg.get("bc_z0", 0), cfg.get("bc_zmax", 1)
    d.t_dirichlet_K = cfg.get("t_dirichlet", 20.0)
    d.placement = cfg.get("placement", 0)
    d.precision = precision
    d.face_rule = cfg.get("face_rule", 0)
    d.interface_rule = cfg.get("interface_rule", 0)
    lo, hi = cfg.get("t_guard", (0.0, 0.0))
    d.t_guard_lo_K, d.t_guard_hi_K = lo, hi
    step = cfg.get("step")
    if step is not None:
        d.step_layers, d.z_step_m = step["layers"], step["z"]
    return d


def materials(cfg: dict) -> list:
    out = []
    for ly in cfg["layers"]:
        m = Material()
        m.rho = ly["rho"]
        m.lam_model = ly.get("lam_model", 1)
        m.lam0 = ly.get("lam0", 0.0)
        m.lam_b = ly.get("lam_b", 0.0)
        m.cap_model = ly.get("cap_model", 1)
        m.c0 = ly.get("c0", 0.0)
        m.theta = ly.get("theta", 1.0)
        m.t_ref = ly.get("t_ref", 20.0)
        m.lam_scale = ly.get("lam_scale", 1.0)
        m.cap_scale = ly.get("cap_scale", 1.0)
        for k, v in enumerate(ly.get("lam_poly", [0.0] * 5)):
            m.lam_poly[k] = v
        for k, v in enumerate(ly.get("cap_poly", [0.0] * 4)):
            m.cap_poly[k] = v
        out.append(m)
    return out


def source(cfg: dict) -> Source:
    s = Source()
    src = cfg.get("source")
    if src is None:
        s.layer = -1
        return s
    s.layer = src["layer"]
    s.q0 = src["q0"]
    s.t_period, s.t_on, s.t_start = src["t_period"], src["t_on"], src.get("t_start", 0.0)
    s.waveform = src.get("waveform", 0)
    s.edge_w = src.get("edge_w", 0.0)
    s.g_model = src.get("g_model", 0)
    s.g_ref = src.get("g_ref", 0.0)
    return s


class Solver:
    """A context over one or more problem dicts (instances)."""

    def __init__(self, cfgs, precision: int = FP64):
        if isinstance(cfgs, dict):
            cfgs = [cfgs]
        self.cfgs = list(cfgs)
        self.precision = precision
        self.ctx = cc_create_geometry([geometry_desc(c, precision) for c in self.cfgs])
        for k, c in enumerate(self.cfgs):
            cc_set_materials(self.ctx, k, materials(c))
            cc_set_source(self.ctx, k, source(c))
            if c.get("dt", 0.0) > 0.0:
                cc_set_dt(self.ctx, k, c["dt"])
        self.sizes = [c["nr"] * c["nz"] for c in self.cfgs]
        self.total = int(sum(self.sizes))

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == FP64 else torch.float32

    def step(self, T, n_steps: int, t0: float = 0.0, dt: float = 0.0, trace=None, energy=None,
             stream=None) -> None:
        """Advance the flat field ``T`` (all instances concatenated) in place."""
        import torch
        if not (T.is_cuda and T.is_contiguous() and T.dtype == self.dtype and T.numel() == self.total):
            raise ValueError("T must be a contiguous CUDA tensor of the context's dtype and size")
        for buf, n in ((trace, 2 * n_steps * len(self.cfgs)), (energy, 5 * len(self.cfgs))):
            if buf is not None and not (buf.is_cuda and buf.is_contiguous()
                                        and buf.dtype == torch.float64 and buf.numel() == n):
                raise ValueError("trace/energy must be contiguous CUDA float64 of the right size")
        st = stream if stream is not None else torch.cuda.current_stream()
        cc_step_n(self.ctx, T.data_ptr(), n_steps, t0, dt,
                  trace.data_ptr() if trace is not None else None,
                  energy.data_ptr() if energy is not None else None, st.cuda_stream)

    def step_adi(self, T, n_steps: int, t0: float = 0.0, dt: float = 0.0, trace=None,
                 stream=None) -> None:
        """Advance the FP64 field ``T`` in place by n_steps steps of the ADI
        variant (no stability bound on dt)."""
        import torch
        if not (T.is_cuda and T.is_contiguous() and T.dtype == torch.float64
                and T.numel() == self.total):
            raise ValueError("T must be a contiguous CUDA float64 tensor of the context's size")
        if trace is not None and not (trace.is_cuda and trace.is_contiguous()
                                      and trace.dtype == torch.float64
                                      and trace.numel() == 2 * n_steps * len(self.cfgs)):
            raise ValueError("trace must be contiguous CUDA float64 of the right size")
        st = stream if stream is not None else torch.cuda.current_stream()
        cc_step_adi_n(self.ctx, T.data_ptr(), n_steps, t0, dt,
                      trace.data_ptr() if trace is not None else None, st.cuda_stream)

    def set_launch(self, mode: int, threads: int = 128, rows_per_lane: int = 16) -> None:
        cc_set_launch(self.ctx, mode, threads, rows_per_lane)

    def get_launch(self) -> tuple:
        return cc_get_launch(self.ctx)

    def _check_field(self, T, dtype=None) -> None:
        """T must be this context's contiguous CUDA field (no CPU fallback)."""
        if not (T.is_cuda and T.is_contiguous() and T.dtype == (dtype or self.dtype)
                and T.numel() == self.total):
            raise ValueError("T must be a contiguous CUDA tensor of the context's dtype and size")

    def autotune(self, T, n_trial: int = 3, stream=None) -> float:
        """Pick the fastest launch shape on field T (restored); returns ms per step."""
        import torch
        self._check_field(T)
        st = stream if stream is not None else torch.cuda.current_stream()
        return cc_autotune(self.ctx, T.data_ptr(), n_trial, st.cuda_stream)

    # ---- parameters of the adjoint: (q0, t_on, lam_scale[L], cap_scale[L]) per instance
    def n_params(self, instance: int = 0) -> int:
        return 2 + 2 * len(self.cfgs[instance]["layers"])

    def get_params(self, instance: int = 0) -> list:
        c = self.cfgs[instance]
        src = c.get("source") or {"q0": 0.0, "t_on": 0.0}
        return ([src["q0"], src["t_on"]] + [ly.get("lam_scale", 1.0) for ly in c["layers"]]
                + [ly.get("cap_scale", 1.0) for ly in c["layers"]])

    def set_params(self, instance: int, theta) -> None:
        """Apply theta = (q0, t_on, lam_scale[], cap_scale[]) to one instance."""
        c = self.cfgs[instance]
        L = len(c["layers"])
        theta = [float(v) for v in theta]
        if c.get("source") is not None:
            c["source"] = dict(c["source"], q0=theta[0], t_on=theta[1])
            cc_set_source(self.ctx, instance, source(c))
        for m in range(L):
            c["layers"][m] = dict(c["layers"][m], lam_scale=theta[2 + m], cap_scale=theta[2 + L + m])
        cc_set_materials(self.ctx, instance, materials(c))

    def adjoint(self, T0, n_steps: int, t0: float, dt: float, target, ckpt_every: int = 256,
                want_dT0: bool = False, stream=None):
        """Loss sum_n dt (Sbar_n - target_n)^2 per instance, its gradient
        (per instance: q0, t_on, lam_scale[], cap_scale[]) and optionally dJ/dT0."""
        import torch
        self._check_field(T0, torch.float64)
        if target.numel() != n_steps * len(self.cfgs):
            raise ValueError("target must hold n_steps values per instance")
        dev = T0.device
        st = stream if stream is not None else torch.cuda.current_stream()
        loss = torch.zeros(len(self.cfgs), dtype=torch.float64, device=dev)
        grad = torch.zeros(sum(self.n_params(k) for k in range(len(self.cfgs))),
                           dtype=torch.float64, device=dev)
        dT0 = torch.zeros_like(T0) if want_dT0 else None
        target = target.contiguous().to(device=dev, dtype=torch.float64)
        cc_adjoint(self.ctx, T0.data_ptr(), n_steps, t0, dt, target.data_ptr(), ckpt_every,
                   loss.data_ptr(), grad.data_ptr(), dT0.data_ptr() if want_dT0 else None,
                   st.cuda_stream)
        return loss, grad, dT0

    def sync(self, stream=None) -> None:
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        cc_sync(self.ctx, st.cuda_stream)

    def tau_stab(self, instance: int = 0) -> float:
        return cc_tau_stab(self.ctx, instance)

    def close(self) -> None:
        if self.ctx is not None:
            cc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_fn():
    import torch

    class SurfaceTrace(torch.autograd.Function):
        """theta [n_inst, 2 + 2L] and T0 -> z-mean surface temperature after each
        step, [n_inst, n_steps].  Backward runs the reverse-time adjoint sweep on
        the GPU (checkpoint every ``ckpt`` steps, recompute in between)."""

        @staticmethod
        def forward(ctx, theta, T0, solver, n_steps, t0, dt, ckpt):
            for k in range(len(solver.cfgs)):
                solver.set_params(k, theta[k].tolist())
            T = T0.detach().clone()
            trace = torch.zeros(len(solver.cfgs) * n_steps * 2, dtype=torch.float64,
                                device=T0.device)
            solver.step(T, n_steps, t0, dt, trace, None)
            ctx.solver, ctx.n, ctx.t0, ctx.dt, ctx.ckpt = solver, n_steps, t0, dt, ckpt
            ctx.save_for_backward(theta, T0)
            return trace.view(len(solver.cfgs), n_steps, 2)[:, :, 1].clone()

        @staticmethod
        def backward(ctx, g):
            theta, T0 = ctx.saved_tensors
            sol = ctx.solver
            for k in range(len(sol.cfgs)):
                sol.set_params(k, theta[k].tolist())
            seed = g.detach().to(dtype=torch.float64).contiguous()
            grad = torch.zeros(theta.numel(), dtype=torch.float64, device=T0.device)
            dT0 = torch.zeros_like(T0)
            cc_adjoint_vjp(sol.ctx, T0.data_ptr(), ctx.n, ctx.t0, ctx.dt, seed.data_ptr(), ctx.ckpt,
                           grad.data_ptr(), dT0.data_ptr(), torch.cuda.current_stream().cuda_stream)
            sol.sync()
            return (grad.view(theta.shape).to(device=theta.device, dtype=theta.dtype), dT0,
                    None, None, None, None, None)

    return SurfaceTrace


def surface_trace(theta, T0, solver: "Solver", n_steps: int, t0: float = 0.0, dt: float = 0.0,
                  ckpt: int = 256):
    """Differentiable surface trace: see ``SurfaceTrace``.  theta has one row of
    (q0, t_on, lam_scale[], cap_scale[]) per instance (all instances must have
    the same number of layers); T0 is the flat FP64 field of all instances."""
    return _autograd_fn().apply(theta, T0, solver, n_steps, t0, dt, ckpt)
