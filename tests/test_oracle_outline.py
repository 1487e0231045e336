"""Pins of the oracle's stepped outline, r in [0, r_max(z)] (Section 2): beyond
z_step only the innermost layers continue (the paper's cell carries its outer
layers on z in [0, z_0] only, Section 5).  No closed form exists for such a
domain, so it is pinned by facts that do not restate its code:

* a step beyond the end of the cylinder is the rectangle, bit for bit;
* nodes outside the domain keep their values and have no influence on the
  nodes inside (any values: the result inside is bit-identical);
* the discrete energy identity dE = Q + PhiD + PhiI + PhiN still closes to
  1e-12, with no interface defect for the conservative rule and no flux
  through Neumann closures; the step face takes no heat;
* with an outer layer of zero conductivity the core of the stepped cylinder
  evolves exactly as the core cylinder alone (a one-layer rectangle, pinned
  by the Bessel-Fourier and steady-state tests);
* a uniform field at the Dirichlet temperature is a fixed point (to the
  rounding of the line solves);
* the surface trace is the trapezoid mean over r = r_max of the full-width
  lines.
"""
import numpy as np
import pytest

from oracle import oracle
from paper_1408_5853_gb300 import inputs


def stepped(layers=2, z_step=6e-3, **kw):
    cfg = inputs.small_case()
    cfg.update(kw)
    cfg["step"] = dict(layers=layers, z=z_step)
    return cfg


def start_field(cfg, seed=3):
    T = inputs.initial_field(cfg, "smooth", seed=seed)
    T[0] = T[1]
    T[:, 0] = T[:, 1]
    T[-1] = cfg["t_dirichlet"]
    return T


def test_outline_hand_derived():
    # 63 cells over 0.10/0.02/0.05/0.10 mm: interfaces at nodes 23, 28, 40;
    # z_j = j * 10/127 mm: z_76 = 5.984 mm <= 6 mm < z_77 = 6.063 mm
    assert oracle.outline(stepped(2, 6e-3)) == (28, 77)
    assert oracle.outline(stepped(1, 6e-3)) == (23, 77)
    assert oracle.outline(stepped(3, 10e-3)) == (40, 128)
    # a line on the step face belongs to the full-width part
    cfg = inputs.paper_case(128, 301)   # z_j = j/6 mm over 5 cm
    cfg["step"] = dict(layers=1, z=0.04)
    assert oracle.outline(cfg)[1] == 241
    # refused: line 1 narrow, every layer kept, the half-cell placement
    for bad in (stepped(1, 0.05e-3), stepped(4, 5e-3), stepped(2, 5e-3, placement=1)):
        with pytest.raises(ValueError):
            oracle.outline(bad)


def test_step_beyond_the_end_is_the_rectangle():
    cfg = stepped(2, 0.5)
    rect = inputs.small_case()
    assert oracle.outline(cfg)[1] == 128      # no narrow line
    T = start_field(rect)
    a = oracle.step_n(cfg, T, 150, 0.0, cfg["dt"])
    b = oracle.step_n(rect, T, 150, 0.0, cfg["dt"])
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("layers,z_step", [(2, 6e-3), (1, 9.95e-3), (3, 2e-3)])
def test_outside_nodes_keep_values_and_do_not_act(layers, z_step):
    cfg = stepped(layers, z_step)
    i_s, j_n = oracle.outline(cfg)
    T = start_field(cfg)
    T1, tr1, e1 = oracle.step_n(cfg, T, 200, 0.0, cfg["dt"])
    out = np.zeros(T.shape, dtype=bool)
    out[j_n:, i_s + 1:] = True
    assert np.array_equal(T1[out], T[out])
    # other (finite) values outside change nothing inside
    T2 = T.copy()
    T2[out] = 20.0 + 50.0 * np.random.default_rng(7).random(out.sum())
    T3, tr3, e3 = oracle.step_n(cfg, T2, 200, 0.0, cfg["dt"])
    assert np.array_equal(T3[~out], T1[~out])
    assert np.array_equal(T3[out], T2[out])
    assert np.array_equal(tr3, tr1) and np.array_equal(e3, e1)


@pytest.mark.parametrize("interface_rule,bc_rmax,z_step",
                         [(0, 0, 6e-3), (1, 0, 6e-3), (1, 1, 6e-3), (1, 0, 9.95e-3),
                          (0, 1, 9.95e-3)])
def test_energy_identity_stepped(interface_rule, bc_rmax, z_step):
    cfg = stepped(3, z_step, interface_rule=interface_rule, bc_rmax=bc_rmax)
    i_s, j_n = oracle.outline(cfg)
    T = start_field(cfg)
    if bc_rmax == 0:
        T[:, -1] = T[:, -2]
        T[j_n:, i_s] = T[j_n:, i_s - 1]
    else:
        T[:, -1] = cfg["t_dirichlet"]
        T[j_n:, i_s] = cfg["t_dirichlet"]
    _, _, e = oracle.step_n(cfg, T, 600, 0.0, cfg["dt"])
    dE, Q, PD, PI, PN = e
    assert Q > 0
    assert abs(dE - Q - PD - PI - PN) <= 1e-12 * max(abs(Q), abs(dE))
    assert abs(PN) <= 1e-12 * abs(Q)          # Neumann closures carry no flux
    if interface_rule == 1:
        assert abs(PI) <= 1e-12 * abs(Q)      # conservative interface rows
    if bc_rmax == 1:
        assert abs(PD) > 1e-6 * abs(Q)


def _core_cases(nr=41, nz=48, z_step=4e-3):
    core = dict(thickness=0.30e-3, rho=7900.0, lam_model=1, lam0=15.0, lam_b=1.0,
                cap_model=1, c0=5.0, theta=60.0, t_ref=20.0)
    inert = dict(thickness=0.10e-3, rho=2700.0, lam_model=0, lam0=0.0, cap_model=0, c0=10.0)
    src = dict(layer=0, q0=2.0e9, t_period=1e-3, t_on=0.4e-3, t_start=0.0, waveform=0)
    base = dict(nz=nz, length=10e-3, bc_rmax=0, bc_z0=0, bc_zmax=1, t_dirichlet=20.0,
                placement=0, face_rule=0, interface_rule=0, source=src)
    two = dict(base, layers=[core, inert], nr=nr, step=dict(layers=1, z=z_step))
    one = dict(base, layers=[core], nr=31)
    return two, one


def test_inert_outer_layer_reduces_to_the_core_cylinder():
    two, one = _core_cases()
    g2, g1 = oracle.grid(two), oracle.grid(one)
    i_s, j_n = oracle.outline(two)
    assert i_s == 30 and 2 < j_n < 47
    np.testing.assert_allclose(g2["r"][:31], g1["r"], rtol=1e-15, atol=0.0)
    T = inputs.initial_field(two, "smooth", seed=5)
    T[0] = T[1]
    T[:, 0] = T[:, 1]
    T[-1] = 20.0
    T[:, i_s] = T[:, i_s - 1]
    tau = 0.5 * oracle.tau_stab(two, 20.0, 40.0)
    T2, _, _ = oracle.step_n(two, T, 300, 0.0, tau, want_trace=False, want_energy=False)
    T1, _, _ = oracle.step_n(one, T[:, :31].copy(), 300, 0.0, tau, want_trace=False,
                             want_energy=False)
    assert np.abs(T1 - 20.0).max() > 0.5          # the source heated the core
    assert np.abs(T2[:, :31] - T1).max() < 1e-11


def test_uniform_dirichlet_field_is_a_fixed_point():
    cfg = stepped(2, 6e-3)
    cfg["source"] = None
    T = np.full((cfg["nz"], cfg["nr"]), cfg["t_dirichlet"])
    T1, _, _ = oracle.step_n(cfg, T, 50, 0.0, cfg["dt"])
    assert np.abs(T1 - T).max() < 1e-11     # rounding of the line solves only


def test_trace_is_the_mean_over_the_full_width_surface():
    cfg = stepped(2, 6e-3)
    i_s, j_n = oracle.outline(cfg)
    z = oracle.grid(cfg)["z"]
    T1, tr, _ = oracle.step_n(cfg, start_field(cfg), 40, 0.0, cfg["dt"])
    zs, surf = z[:j_n], T1[:j_n, -1]
    mean = np.trapezoid(surf, zs) / (zs[-1] - zs[0])
    assert abs(tr[-1, 1] - mean) < 1e-12 * mean
    assert tr[-1, 0] == T1[0, -1]


def test_adi_and_adjoint_take_rectangles_only():
    cfg = stepped(2, 6e-3)
    T = start_field(cfg)
    with pytest.raises(ValueError):
        oracle.step_adi_n(cfg, T, 1, 0.0, cfg["dt"])
    with pytest.raises(ValueError):
        oracle.adjoint(cfg, T, 2, 0.0, cfg["dt"], np.zeros(2))
    # a step beyond the end is a rectangle
    oracle.step_adi_n(stepped(2, 0.5), T, 1, 0.0, cfg["dt"])
