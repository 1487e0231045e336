"""Launch shapes of the time step on the GPU: one launch per step or all steps
in one cooperative launch with a bounded grid barrier, block sizes and lane
policies, the autotuner, the barrier timeout report, and CUDA-graph capture.
Results must not depend on the launch shape beyond rounding (FP64 bar:
1e-9 K against the oracle; mixed: 1e-3 K)."""
import os

import numpy as np
import pytest

from oracle import oracle
from paper_1408_5853_gb300 import inputs

pytestmark = pytest.mark.gpu


def _run(cfgs, T0s, n, precision, shape, t0=0.0):
    import torch
    from paper_1408_5853_gb300 import ccell
    sol = ccell.Solver(cfgs, precision=precision)
    if shape is not None:
        sol.set_launch(*shape)
    dt = torch.float64 if precision == 0 else torch.float32
    T = torch.tensor(np.concatenate([t.ravel() for t in T0s]), dtype=dt, device="cuda")
    tr = torch.zeros(len(cfgs) * n * 2, dtype=torch.float64, device="cuda")
    en = torch.zeros(len(cfgs) * 5, dtype=torch.float64, device="cuda")
    sol.step(T, n, t0, 0.0, tr, en)
    sol.sync()
    out = T.double().cpu().numpy()
    sol.close()
    return out, tr.view(len(cfgs), n, 2).cpu().numpy(), en.view(len(cfgs), 5).cpu().numpy()


SHAPES = [(1, 128, 16), (1, 256, 8), (1, 64, 4), (0, 64, 4), (0, 256, 8), (2, 256, 16),
          (2, 128, 8), (2, 64, 4), (4, 256, 16), (4, 128, 8), (4, 64, 4), (4, 384, 16),
          (4, 384, 4)]


# launch mode 5 (stores by the producers) is for mixed-precision contexts only
MIXED_ONLY = [(4, 512, 16), (4, 512, 4), (5, 512, 16), (5, 384, 16), (5, 256, 8), (5, 128, 16),
              (5, 64, 4)]


@pytest.mark.parametrize("shape,precision", [(s, p) for s in SHAPES for p in (0, 1)] +
                         [(s, 1) for s in MIXED_ONLY])
def test_launch_shapes_parity(shape, precision):
    cfgs = inputs.batched_cases(seed=1, n=5)
    T0s = []
    for k, c in enumerate(cfgs):
        c["dt"] = 0.9 * oracle.tau_stab(c, 20.0, 100.0)
        T0 = inputs.initial_field(c, "smooth", seed=k)
        if precision == 1:
            T0 = T0.astype(np.float32).astype(np.float64)
        T0s.append(T0)
    n = 13
    out, tr, en = _run(cfgs, T0s, n, precision, shape)
    tol = 1e-9 if precision == 0 else 1e-3
    ofs = 0
    for k, c in enumerate(cfgs):
        To, tro, eo = oracle.step_n(c, T0s[k], n, 0.0, c["dt"])
        nn = c["nr"] * c["nz"]
        assert np.max(np.abs(out[ofs:ofs + nn].reshape(To.shape) - To)) <= tol, k
        assert np.max(np.abs(tr[k] - tro)) <= tol, k
        ofs += nn


def test_persistent_small_case_matches_oracle():
    cfg = inputs.small_case()
    T0 = inputs.initial_field(cfg, "smooth", seed=3)
    n = 400
    t0 = 1e-3 - 200 * cfg["dt"]
    out, tr, en = _run([cfg], [T0], n, 0, (1, 128, 16), t0=t0)
    To, tro, eo = oracle.step_n(cfg, T0, n, t0, cfg["dt"])
    assert np.max(np.abs(out.reshape(To.shape) - To)) <= 1e-9
    assert np.max(np.abs(tr[0] - tro)) <= 1e-9
    assert np.max(np.abs(en[0] - eo)) <= 1e-9 * abs(eo[1])


@pytest.mark.parametrize("shape", [(3, 256, 16), (3, 128, 8), (3, 64, 4)])
def test_resident_mode_matches_oracle(shape):
    """Field resident in shared memory (one block per SM, boundary rows
    exchanged between steps): ragged sizes across the pulse end."""
    for nr, nz, seed in ((64, 128, 3), (100, 301, 4), (37, 700, 5)):
        cfg = inputs.small_case()
        cfg.update(nr=nr, nz=nz)
        cfg["dt"] = min(5e-7, 0.5 * oracle.tau_stab(cfg, 20.0, 100.0))
        T0 = inputs.initial_field(cfg, "smooth", seed=seed)
        n, t0 = 41, 1e-3 - 20 * cfg["dt"]
        out, tr, en = _run([cfg], [T0], n, 0, shape, t0=t0)
        To, tro, eo = oracle.step_n(cfg, T0, n, t0, cfg["dt"])
        assert np.max(np.abs(out.reshape(To.shape) - To)) <= 1e-9, (nr, nz)
        assert np.max(np.abs(tr[0] - tro)) <= 1e-9, (nr, nz)
        assert np.max(np.abs(en[0] - eo)) <= 1e-9 * abs(eo[1]), (nr, nz)


def test_barrier_timeout_is_reported():
    """A barrier that can never complete (test hook: one arrival too many
    expected, short wait) must end the kernel and surface as CC_ETIMEOUT."""
    from paper_1408_5853_gb300 import ccell
    cfg = inputs.small_case()
    T0 = inputs.initial_field(cfg)
    os.environ["CC_TEST_BARRIER_TIMEOUT"] = "1"
    try:
        for shape in ((1, 128, 16), (3, 128, 16)):   # grid barrier; neighbour step counters
            with pytest.raises(ccell.CCError) as e:
                _run([cfg], [T0], 5, 0, shape)
            assert e.value.status == ccell.CC_ETIMEOUT
    finally:
        del os.environ["CC_TEST_BARRIER_TIMEOUT"]
    # the GPU context stays usable afterwards
    out, _, _ = _run([cfg], [T0], 3, 0, (1, 128, 16))
    To, _, _ = oracle.step_n(cfg, T0, 3, 0.0, cfg["dt"])
    assert np.max(np.abs(out.reshape(To.shape) - To)) <= 1e-9


def test_autotune_keeps_field_and_picks_a_valid_shape():
    import torch
    from paper_1408_5853_gb300 import ccell
    cfgs = inputs.batched_cases(seed=1, n=8)
    for c in cfgs:
        c["dt"] = 0.9 * oracle.tau_stab(c, 20.0, 100.0)
    sol = ccell.Solver(cfgs, precision=ccell.MIXED)
    T0 = np.concatenate([inputs.initial_field(c, "smooth", seed=k).ravel()
                         for k, c in enumerate(cfgs)])
    T = torch.tensor(T0, dtype=torch.float32, device="cuda")
    keep = T.clone()
    ms = sol.autotune(T, n_trial=2)
    assert ms > 0.0
    mode, threads, rows = sol.get_launch()
    assert mode in (0, 1, 2, 4, 5) and threads in (64, 128, 256, 384, 512) and 2 <= rows <= 16
    assert torch.equal(T, keep)
    sol.close()


@pytest.mark.parametrize("mode,precision", [(0, 0), (1, 0), (2, 0), (3, 0), (4, 0), (4, 1), (5, 1)])
def test_cuda_graph_replay_equals_direct_call(mode, precision):
    import torch
    from paper_1408_5853_gb300 import ccell
    cfg = inputs.small_case()
    T0 = inputs.initial_field(cfg, "smooth", seed=8)
    n = 25
    sol = ccell.Solver(cfg, precision=precision)
    sol.set_launch(mode, 128, 16)
    Ta = torch.tensor(T0.ravel(), dtype=torch.float64 if precision == 0 else torch.float32,
                      device="cuda")
    tra = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    ena = torch.zeros(5, dtype=torch.float64, device="cuda")
    sol.step(Ta.clone(), n, 0.0, 0.0, tra, ena)   # warm-up: sizes the context's buffers
    torch.cuda.synchronize()
    Tb, trb, enb = Ta.clone(), torch.zeros_like(tra), torch.zeros_like(ena)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        sol.step(Tb, n, 0.0, 0.0, trb, enb)
    Tb.copy_(Ta)
    enb.zero_()
    g.replay()
    torch.cuda.synchronize()
    Tc, trc, enc = Ta.clone(), torch.zeros_like(tra), torch.zeros_like(ena)
    sol.step(Tc, n, 0.0, 0.0, trc, enc)
    sol.sync()
    assert torch.equal(Tb, Tc)
    # the z-mean of the trace is summed with FP64 atomics: equal up to summation order
    assert torch.allclose(trb, trc, rtol=1e-13, atol=0.0)
    assert torch.allclose(enb, enc, rtol=1e-12, atol=0.0)
    sol.close()


def test_measured_fp64_rate_is_plausible():
    """cc_measure_fp64_rate (the FP64-pipe roofline denominator): a positive,
    finite rate within the range of any FP64-capable GPU, repeatable within 20 %."""
    import torch
    from paper_1408_5853_gb300 import ccell
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    buf = torch.zeros(1024 * sms, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    r1, s1 = ccell.cc_measure_fp64_rate(buf.data_ptr(), buf.numel(), 2000, stream)
    r2, _ = ccell.cc_measure_fp64_rate(buf.data_ptr(), buf.numel(), 2000, stream)
    assert 1e10 < r1 < 1e14 and s1 > 0.0
    assert abs(r1 - r2) <= 0.2 * max(r1, r2)
    assert bool(torch.isfinite(buf).all())
    with pytest.raises(ccell.CCError):
        ccell.cc_measure_fp64_rate(buf.data_ptr(), 16, 10, stream)   # scratch too short
