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


def _noalloc_vs_oracle(cfg, T0, n, t0):
    import torch

    from oracle import oracle
    from paper_1408_5853_gb300 import ccell

    kw = dict(dtype=torch.float64, device="cuda")
    T = torch.tensor(T0.ravel(), **kw)
    tr, en = torch.zeros(2 * n, **kw), torch.zeros(5, **kw)
    ccell.cc_step_n_noalloc(ccell.geometry_desc(cfg), ccell.materials(cfg), ccell.source(cfg),
                            T.data_ptr(), n, t0, cfg["dt"], tr.data_ptr(), en.data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    To, tro, eo = oracle.step_n(cfg, T0, n, t0, cfg["dt"])
    assert np.max(np.abs(T.cpu().numpy().reshape(To.shape) - To)) <= TOL_K
    assert np.max(np.abs(tr.view(n, 2).cpu().numpy() - tro)) <= TOL_K
    assert np.max(np.abs(en.cpu().numpy() - eo)) <= 1e-9 * max(abs(eo[0]), abs(eo[1]))


def test_noalloc_matches_oracle_half_cell_grid_dirichlet_face():
    """Half-cell placement (single layer) with a Dirichlet r_max, against the
    oracle: the grid, class and weight tables of this entry point come from
    the host code it shares with cc_step_n."""
    from oracle import oracle
    from paper_1408_5853_gb300 import inputs

    cfg = inputs.small_case()
    cfg["layers"] = cfg["layers"][2:3]
    cfg["layers"][0]["thickness"] = 0.3e-3
    cfg.update(nr=45, nz=50, placement=1, bc_rmax=1)
    cfg["source"]["layer"] = 0
    cfg["dt"] = min(5e-7, 0.5 * oracle.tau_stab(cfg, 20.0, 100.0))
    T0 = inputs.initial_field(cfg, "smooth", seed=5)
    _noalloc_vs_oracle(cfg, T0, 40, 1e-3 - 20 * cfg["dt"])


def test_noalloc_matches_oracle_transient_waveform():
    """The transient turn-on waveform (2), accepted as by cc_set_source, and a
    Dirichlet z = 0 face, against the oracle."""
    from paper_1408_5853_gb300 import inputs

    cfg = inputs.small_case()
    cfg.update(nr=70, nz=33, bc_z0=1)
    cfg["source"].update(waveform=2, edge_w=40 * cfg["dt"])
    T0 = inputs.initial_field(cfg, "smooth", seed=9)
    _noalloc_vs_oracle(cfg, T0, 60, 10e-3 - 10 * cfg["dt"])   # across a period start
