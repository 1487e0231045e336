"""cc_step_n_noalloc against cc_step_n on the GPU.

cc_step_n_noalloc serves callers that cannot allocate device memory (an
embedding framework whose allocator owns the device, loops that forbid
allocation after start-up): it keeps its scratch in a static device array and
allocates nothing.  Its results must equal those of cc_step_n, within the FP64
parity tolerance of the other tests, on consecutive calls that reuse the
shared static array (an odd step count, an even one, then a different grid, so
stale contents of the previous call would show).

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TOL_K = 1e-9


def _run_pair(ccell, cfg, Ta, Tb, sol, n, t0, stream):
    import torch
    kw = dict(dtype=torch.float64, device="cuda")
    tra, ena = torch.zeros(2 * n, **kw), torch.zeros(5, **kw)
    trb, enb = torch.zeros(2 * n, **kw), torch.zeros(5, **kw)
    ccell.cc_step_n_noalloc(ccell.geometry_desc(cfg), ccell.materials(cfg), ccell.source(cfg),
                            Ta.data_ptr(), n, t0, cfg["dt"], tra.data_ptr(), ena.data_ptr(),
                            stream.cuda_stream)
    sol.step(Tb, n, t0, 0.0, trb, enb)
    sol.sync()
    torch.cuda.synchronize()
    assert torch.max(torch.abs(Ta - Tb)).item() <= TOL_K
    assert torch.max(torch.abs(tra - trb)).item() <= TOL_K
    e_a, e_b = ena.cpu().numpy(), enb.cpu().numpy()
    assert np.max(np.abs(e_a - e_b)) <= 1e-9 * max(abs(e_b[0]), abs(e_b[1]))


def test_noalloc_matches_step_n_on_consecutive_calls():
    import torch

    from paper_1408_5853_gb300 import ccell, inputs

    stream = torch.cuda.current_stream()
    cfg = inputs.small_case()
    T0 = inputs.initial_field(cfg, "smooth", seed=7)
    sol = ccell.Solver(cfg)
    Ta = torch.tensor(T0.ravel(), dtype=torch.float64, device="cuda")   # no-allocation path
    Tb = Ta.clone()                                                      # cc_step_n
    t0 = 1e-3 - 20 * cfg["dt"]   # the pulse switches off during the first call
    for n in (37, 64):
        _run_pair(ccell, cfg, Ta, Tb, sol, n, t0, stream)
        t0 += n * cfg["dt"]
    sol.close()

    # a different, ragged grid right after: the shared array must not leak state
    cfg2 = inputs.small_case()
    cfg2.update(nr=100, nz=41)
    T2 = inputs.initial_field(cfg2, "smooth", seed=8)
    sol2 = ccell.Solver(cfg2)
    Ta = torch.tensor(T2.ravel(), dtype=torch.float64, device="cuda")
    Tb = Ta.clone()
    _run_pair(ccell, cfg2, Ta, Tb, sol2, 25, 0.0, stream)
    sol2.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch

    from paper_1408_5853_gb300 import ccell, inputs

    cfg = inputs.production_case()          # 512 x 4096 = 2^21 nodes > 2^20
    T = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(ccell.CCError) as e:
        ccell.cc_step_n_noalloc(ccell.geometry_desc(cfg), ccell.materials(cfg),
                                ccell.source(cfg), T.data_ptr(), 1, 0.0, cfg["dt"], None, None,
                                torch.cuda.current_stream().cuda_stream)
    assert e.value.status == ccell.CC_EINVAL
