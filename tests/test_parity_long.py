"""GPU parity with the oracle at the workloads' own horizons, over the full field.

Short runs cannot show a fault that needs many steps to surface (a drift in
the FP64 sums of the trace and energy terms, a grid barrier of the persistent
launch that slips after thousands of steps, the FP32 state pair of the mixed
path).  These tests run the CUDA path for as long as the oracle allows on the
host and compare every node, every trace sample and the energy terms:

  * 4-layer 64 x 128 cylinder, the full 20 ms (40 000 steps of 0.5 us, two
    1 ms pulses): FP64 in every launch mode
    (<= 1e-9 K), the mixed path (<= 1e-3 K);
  * 5-layer 512 x 4096 production cylinder, 2 000 steps across the end of a
    pulse, all 4096 lines: FP64 in every launch mode (one launch per step with
    CTA tiles or warp-owned lines, persistent, persistent with the field
    resident in shared memory; <= 1e-9 K), the mixed path in the
    shape the autotuner picks (<= 1e-3 K), all against one oracle run from the
    FP32-rounded field;
  * the 256-instance design sweep (seed 1) in one context, mixed precision in
    the autotuned shape, 2 000 steps; 8 sampled instances against the oracle
    (<= 1e-3 K).

The step is Section 3 of the paper, Eqs. (scheme_eq)-(cc_first_3), with the
closures of Eqs. (first_oder_bc)-(T_ini_for_back_sweep).
"""
import numpy as np
import pytest

from gpu_helpers import run_gpu
from oracle import oracle
from paper_1408_5853_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_FP64_K = 1e-9
TOL_MIXED_K = 1e-3
FP64, MIXED = 0, 1


def _f32(T):
    return np.asarray(T, dtype=np.float32).astype(np.float64)


def _check(Tg, trg, eg, ref, tol, energy_rel):
    To, tro, eo = ref
    err = float(np.max(np.abs(Tg - To)))
    assert err <= tol, f"field max|dT| = {err:.3e} K"
    terr = float(np.max(np.abs(trg - tro)))
    assert terr <= tol, f"trace max|dT| = {terr:.3e} K"
    scale = max(abs(eo[0]), abs(eo[1]))
    eerr = float(np.max(np.abs(eg - eo))) / scale
    assert eerr <= energy_rel, f"energy rel err {eerr:.3e}"
    return err, terr


# ---------------------------------------------------------------- 64 x 128, 20 ms
@pytest.fixture(scope="module")
def small_20ms():
    cfg = inputs.small_case()
    n = int(round(20e-3 / cfg["dt"]))            # 40 000 steps
    T0 = inputs.initial_field(cfg, "uniform")     # 20 K, the configured start
    return cfg, T0, n, oracle.step_n(cfg, T0, n, 0.0, cfg["dt"])


@pytest.mark.parametrize("launch", [(0, 256, 16), (1, 256, 16), (2, 256, 16), (3, 256, 16),
                                    (4, 256, 16)])
def test_small_case_full_20ms_fp64(small_20ms, launch):
    cfg, T0, n, ref = small_20ms
    (Tg,), trg, eg = run_gpu(cfg, T0, n, launch=launch)
    _check(Tg, trg[0], eg[0], ref, TOL_FP64_K, 1e-9)
    assert ref[1][:, 0].max() > 44.0             # both pulses heat the surface near 45 K


def test_small_case_full_20ms_mixed(small_20ms):
    cfg, T0, n, ref = small_20ms                 # T0 = 20 K is exact in FP32
    (Tg,), trg, eg = run_gpu(cfg, T0, n, precision=MIXED)
    _check(Tg, trg[0], eg[0], ref, TOL_MIXED_K, 1e-4)


# ------------------------------------------------------------ 512 x 4096, 2000 steps
@pytest.fixture(scope="module")
def production_2000():
    cfg = inputs.production_case()
    n = 2000
    t0 = 1e-3 - 1000 * cfg["dt"]                 # the heater switches off mid-run
    T0 = _f32(inputs.initial_field(cfg, "smooth", seed=0))
    return cfg, T0, n, t0, oracle.step_n(cfg, T0, n, t0, cfg["dt"])


@pytest.mark.parametrize("launch", [(0, 256, 16), (1, 256, 16), (2, 256, 16), (3, 256, 16),
                                    (3, 128, 16), (4, 256, 16)])
def test_production_2000_steps_fp64_full_field(production_2000, launch):
    cfg, T0, n, t0, ref = production_2000
    (Tg,), trg, eg = run_gpu(cfg, T0, n, t0=t0, launch=launch)
    _check(Tg, trg[0], eg[0], ref, TOL_FP64_K, 1e-9)


@pytest.mark.parametrize("launch", ["autotune", (4, 384, 16), (4, 512, 16), (5, 512, 16)])
def test_production_2000_steps_mixed_full_field(production_2000, launch):
    cfg, T0, n, t0, ref = production_2000
    (Tg,), trg, eg = run_gpu(cfg, T0, n, t0=t0, precision=MIXED, launch=launch)
    err, _ = _check(Tg, trg[0], eg[0], ref, TOL_MIXED_K, 1e-4)
    assert err < 1e-5, err                       # far inside the bar at this horizon


# ------------------------------------------------- 256-instance sweep, 2000 steps
def test_batched_sweep_sampled_instances_2000_steps():
    cfgs = inputs.batched_cases(seed=1, n=256)
    for c in cfgs:                               # the bench's time steps
        c["dt"] = 0.9 * oracle.tau_stab(c, 20.0, 100.0)
    T0s = [inputs.initial_field(c, "uniform") for c in cfgs]
    n = 2000
    Tg, trg, eg = run_gpu(cfgs, T0s, n, precision=MIXED, launch="autotune")
    pick = np.random.default_rng(11).choice(len(cfgs), size=8, replace=False)
    for k in sorted(int(v) for v in pick):
        ref = oracle.step_n(cfgs[k], T0s[k], n, 0.0, cfgs[k]["dt"])
        _check(Tg[k], trg[k], eg[k], ref, TOL_MIXED_K, 1e-4)
