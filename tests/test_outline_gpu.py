"""GPU parity of the stepped outline r in [0, r_max(z)] (Section 2; the paper's
cell carries its outer layers on z in [0, z_0] only, Section 5) against the
oracle, through the C ABI.

FP64 bar: max |dT| <= 1e-9 K on every node and on the surface trace, energy
terms to 1e-9 relative; mixed bar: 1e-3 K.  Nodes outside the domain keep
their values bit for bit in both precisions.  The step sits mid-way, between
the last two lines, near the start, with every boundary and interface flag,
both launch modes, in ragged multi-instance contexts mixed with rectangles,
and on the paper's cell at the bench's size (512 x 1201, z_0 = 4 cm)."""
import numpy as np
import pytest

from gpu_helpers import run_gpu
from oracle import oracle
from paper_1408_5853_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_K = 1e-9


def stepped(layers=2, z_step=6e-3, nr=64, nz=128, **kw):
    cfg = inputs.small_case()
    cfg.update(nr=nr, nz=nz, **kw)
    cfg["step"] = dict(layers=layers, z=z_step)
    cfg["dt"] = min(5e-7, 0.5 * oracle.tau_stab(cfg, 20.0, 100.0))
    return cfg


def outside(cfg):
    i_s, j_n = oracle.outline(cfg)
    m = np.zeros((cfg["nz"], cfg["nr"]), dtype=bool)
    m[j_n:, i_s + 1:] = True
    return m


def _cmp64(cfg, T0, n, t0=0.0):
    (Tg,), trg, eg = run_gpu(cfg, T0, n, t0=t0)
    To, tro, eo = oracle.step_n(cfg, T0, n, t0, cfg["dt"])
    err = np.max(np.abs(Tg - To))
    assert err <= TOL_K, f"field max|dT| = {err:.3e} K"
    terr = np.max(np.abs(trg[0] - tro))
    assert terr <= TOL_K, f"trace max|dT| = {terr:.3e} K"
    scale = max(abs(eo[0]), abs(eo[1]), 1e-300)
    assert np.max(np.abs(eg[0] - eo)) / scale <= 1e-9, (eg[0], eo)
    out = outside(cfg)
    assert np.array_equal(Tg[out], T0[out])
    return Tg


@pytest.mark.parametrize("layers,z_step,flags", [
    (2, 6e-3, {}),
    (1, 9.95e-3, {}),                      # step between the last two lines
    (3, 0.2e-3, {}),                       # only lines 0..2 keep the full width
    (2, 6e-3, {"bc_rmax": 1}),
    (2, 6e-3, {"interface_rule": 1}),
    (2, 6e-3, {"face_rule": 1}),
    (1, 6e-3, {"bc_zmax": 0}),
    (2, 5e-3, {"nr": 300, "nz": 45}),      # several lane segments per line
])
def test_fp64_parity(layers, z_step, flags):
    cfg = stepped(layers, z_step, **flags)
    T0 = inputs.initial_field(cfg, "smooth", seed=layers)
    _cmp64(cfg, T0, 61, t0=1e-3 - 30 * cfg["dt"])


@pytest.mark.parametrize("layers,z_step,flags", [(2, 6e-3, {}), (1, 9.95e-3, {}),
                                                 (2, 6e-3, {"bc_rmax": 1}),
                                                 (3, 5e-3, {"nr": 300, "nz": 45})])
def test_mixed_parity(layers, z_step, flags):
    cfg = stepped(layers, z_step, **flags)
    T0 = inputs.initial_field(cfg, "smooth", seed=layers).astype(np.float32).astype(np.float64)
    (Tg,), trg, eg = run_gpu(cfg, T0, 200, t0=1e-3 - 100 * cfg["dt"], precision=1)
    To, tro, eo = oracle.step_n(cfg, T0, 200, 1e-3 - 100 * cfg["dt"], cfg["dt"])
    assert np.max(np.abs(Tg - To)) <= 1e-3
    assert np.max(np.abs(trg[0] - tro)) <= 1e-3
    e = eg[0]
    assert abs(e[1] - eo[1]) <= 1e-5 * abs(eo[1])
    assert abs(e[0] - e[1:].sum()) <= 1e-4 * max(abs(e[0]), abs(e[1]))
    out = outside(cfg)
    assert np.array_equal(Tg[out], T0[out])


@pytest.mark.parametrize("shape", [(1, 128, 16), (0, 64, 4), (1, 256, 8)])
@pytest.mark.parametrize("precision", [0, 1])
def test_launch_modes_with_rectangles_and_steps(shape, precision):
    import torch
    from paper_1408_5853_gb300 import ccell
    cfgs = inputs.batched_cases(seed=1, n=5)
    T0s = []
    for k, c in enumerate(cfgs):
        if k % 2 == 0:   # every other instance stepped, at a different height
            c["step"] = dict(layers=1 + k // 2, z=c["length"] * (0.3 + 0.2 * k / 4))
        c["dt"] = 0.9 * oracle.tau_stab(c, 20.0, 100.0)
        T0 = inputs.initial_field(c, "smooth", seed=k)
        if precision == 1:
            T0 = T0.astype(np.float32).astype(np.float64)
        T0s.append(T0)
    n = 13
    sol = ccell.Solver(cfgs, precision=precision)
    sol.set_launch(*shape)
    dt = torch.float64 if precision == 0 else torch.float32
    T = torch.tensor(np.concatenate([t.ravel() for t in T0s]), dtype=dt, device="cuda")
    tr = torch.zeros(len(cfgs) * n * 2, dtype=torch.float64, device="cuda")
    sol.step(T, n, 0.0, 0.0, tr, None)
    sol.sync()
    out = T.double().cpu().numpy()
    tr = tr.view(len(cfgs), n, 2).cpu().numpy()
    sol.close()
    tol = TOL_K if precision == 0 else 1e-3
    ofs = 0
    for k, c in enumerate(cfgs):
        To, tro, _ = oracle.step_n(c, T0s[k], n, 0.0, c["dt"], want_energy=False)
        nn = c["nr"] * c["nz"]
        Tg = out[ofs:ofs + nn].reshape(To.shape)
        assert np.max(np.abs(Tg - To)) <= tol, k
        assert np.max(np.abs(tr[k] - tro)) <= tol, k
        if "step" in c:
            m = outside(c)
            assert np.array_equal(Tg[m], T0s[k][m]), k
        ofs += nn


def test_paper_cell_with_its_outline():
    """The paper's cell at the bench's size and time step: 512 x 1201 over 5 cm,
    outer layers on z <= 4 cm only, the copper core alone to the helium end,
    from T = 4.2 K (Eq. (initcond)) through the first 0.05 ms of the pulse with
    the transient sub-steps tau* = tau/100, as a schedule of cc_step_n calls."""
    import torch
    from paper_1408_5853_gb300 import ccell, schedule
    cfg = inputs.paper_case(nr=512, nz=1201, stepped=True)
    cfg["t_guard"] = (4.2, 20.0)
    cfg["dt"] = 2.5e-7
    cfg["source"]["edge_w"] = cfg["dt"]
    chunks = schedule.transient_schedule(cfg["source"]["t_period"], cfg["dt"], 0.05e-3)
    sol = ccell.Solver(cfg)
    T = torch.full((cfg["nz"] * cfg["nr"],), 4.2, dtype=torch.float64, device="cuda")
    To = np.full((cfg["nz"], cfg["nr"]), 4.2)
    for t0, dt, n in chunks:
        tr = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
        sol.step(T, n, t0, dt, tr, None)
        To, tro, _ = oracle.step_n(cfg, To, n, t0, dt, want_energy=False)
        assert np.max(np.abs(tr.view(n, 2).cpu().numpy() - tro)) <= TOL_K
    sol.sync()
    Tg = T.cpu().numpy().reshape(To.shape)
    sol.close()
    assert np.max(np.abs(Tg - To)) <= TOL_K
    assert 6.0 < To.max() < 22.0
    assert np.all(Tg[outside(cfg)] == 4.2)


def test_rectangle_only_entry_points_refuse_steps():
    import torch
    from paper_1408_5853_gb300 import ccell
    cfg = stepped(2, 6e-3)
    sol = ccell.Solver(cfg)
    T = torch.tensor(inputs.initial_field(cfg).ravel(), device="cuda")
    with pytest.raises(ccell.CCError) as e:
        sol.step_adi(T, 2, 0.0, cfg["dt"])
    assert e.value.status == ccell.CC_EUNSUPPORTED
    with pytest.raises(ccell.CCError) as e:
        sol.adjoint(T, 4, 0.0, cfg["dt"], torch.zeros(4, dtype=torch.float64, device="cuda"))
    assert e.value.status == ccell.CC_EUNSUPPORTED
    sol.close()
