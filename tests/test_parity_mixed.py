"""GPU parity of the mixed-precision path (FP32 state, properties and stencil;
FP64 elimination and energy sums) against the FP64 oracle.

Bar: max |dT| <= 1e-3 K over the field and the surface trace, on the same
seeded inputs (the oracle starts from the FP32-rounded initial field), plus
the energy identity of the scheme on the GPU's own energy terms.
"""
import numpy as np
import pytest

from gpu_helpers import oracle_cone, run_gpu
from oracle import oracle
from paper_1408_5853_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_K = 1e-3
MIXED = 1


def _f32(T):
    return np.asarray(T, dtype=np.float32).astype(np.float64)


def _cmp(cfg, T0, n, t0=0.0):
    T0 = _f32(T0)
    (Tg,), trg, eg = run_gpu(cfg, T0, n, t0=t0, precision=MIXED)
    To, tro, eo = oracle.step_n(cfg, T0, n, t0, cfg["dt"])
    err = np.max(np.abs(Tg - To))
    terr = np.max(np.abs(trg[0] - tro))
    assert err <= TOL_K, f"field max|dT| = {err:.3e} K"
    assert terr <= TOL_K, f"trace max|dT| = {terr:.3e} K"
    e = eg[0]
    assert abs(e[1] - eo[1]) <= 1e-5 * abs(eo[1]) + 1e-300
    assert abs(e[0] - e[1:].sum()) <= 1e-4 * max(abs(e[0]), abs(e[1]))
    return err, terr


def test_mixed_small_case_across_pulse_edge():
    cfg = inputs.small_case()
    T0 = inputs.initial_field(cfg, "smooth", seed=0)
    err, _ = _cmp(cfg, T0, 1001, t0=1e-3 - 500 * cfg["dt"])
    assert err < 1e-4   # far inside the bar on the 64 x 128 case


@pytest.mark.parametrize("nr,nz", [(3, 3), (9, 7), (37, 19), (100, 40), (300, 9), (512, 5)])
def test_mixed_ragged_sizes(nr, nz):
    cfg = inputs.small_case()
    if nr < 12:
        cfg["layers"] = cfg["layers"][:1] if nr < 5 else cfg["layers"][:2]
        cfg["source"]["layer"] = 0
    cfg.update(nr=nr, nz=nz)
    cfg["dt"] = min(5e-7, 0.5 * oracle.tau_stab(cfg, 20.0, 100.0))
    _cmp(cfg, inputs.initial_field(cfg, "smooth", seed=nr + nz), 9)


@pytest.mark.parametrize("variant", ["rmax_dirichlet", "z0_dirichlet", "face_rule_1",
                                     "interface_rule_1", "tanh_waveform"])
def test_mixed_flag_variants(variant):
    cfg = inputs.small_case()
    cfg.update(nr=45, nz=50)
    if variant == "rmax_dirichlet":
        cfg["bc_rmax"] = 1
    elif variant == "z0_dirichlet":
        cfg["bc_z0"] = 1
    elif variant == "face_rule_1":
        cfg["face_rule"] = 1
    elif variant == "interface_rule_1":
        cfg["interface_rule"] = 1
    elif variant == "tanh_waveform":
        cfg["source"].update(waveform=1, edge_w=2e-5)
    cfg["dt"] = min(5e-7, 0.5 * oracle.tau_stab(cfg, 20.0, 100.0))
    _cmp(cfg, inputs.initial_field(cfg, "smooth", seed=5), 40, t0=1e-3 - 20 * cfg["dt"])


@pytest.mark.parametrize("launch", [None, (1, 256, 16), (1, 64, 16)])
def test_mixed_production_size_sampled_lines(launch):
    """512 x 4096 in the default shape and in the persistent shapes the bench's
    autotuner picks for this workload."""
    cfg = inputs.production_case()
    T0 = _f32(inputs.initial_field(cfg, "smooth", seed=0))
    n, t0 = 24, 1e-3 - 12 * cfg["dt"]
    (Tg,), _, eg = run_gpu(cfg, T0, n, t0=t0, precision=MIXED, launch=launch)
    M = cfg["nz"] - 1
    for j in (0, 1, 2, 1000, 2047, M - 1, M):
        ref = oracle_cone(cfg, T0, j, n, t0, cfg["dt"])
        err = np.max(np.abs(Tg[j] - ref))
        assert err <= TOL_K, f"line {j}: max|dT| = {err:.3e} K"
