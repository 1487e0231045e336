"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

No implementation of the paper exists to compare with, so the oracle is pinned
by closed forms, invariants, library routines and hand-derived values:

* grid partition (hand-derived largest-remainder counts);
* the rectangular waveform of Eq. (period) (half-open windows);
* uniform fixed point (no source, uniform T);
* exact discrete steady state of the axial operator, Eq. (Lambda_j), with
  constant lambda (quadratic profile is reproduced to rounding);
* Kirchhoff steady state with power-law lambda(T): second-order convergence;
* three-term Bessel-Fourier series J0 x cos (scipy.special): decay rates and
  second-order convergence of the full r-z step with cylindrical weights,
  Eq. (Lambda_i);
* the transient turn-on p^2(t) of Eq. (transient_function);
* two-layer radial steady state with a source and flux continuity at the
  layer border, Eqs. (sch), (cc_first_1)-(cc_first_3): first-order convergence
  to the analytic piecewise profile (swapping the two sides fails);
* uniform heating ODE rho c(T) dT/dt = X with the temperature-dependent heat
  capacity (scipy.integrate): first order in tau, Richardson limit;
* injected heat equals X * volume * time exactly (cylinder volume weights);
* the discrete energy identity dE = Q + PhiD + PhiI + PhiN to 1e-12;
* the stability bound Eq. (stability_condition): bounded below, grows above.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import oracle
from paper_1408_5853_gb300 import inputs


def single_layer(nr, nz, R=1.0, L=1.0, lam=1.0, rho=1.0, c=1.0, lam_model=0, lam_b=0.0,
                 cap_model=0, theta=1.0, t_ref=20.0, placement=1, bc=(0, 0, 0), t_d=20.0,
                 q0=None, t_on=None):
    cfg = dict(
        layers=[dict(thickness=R, rho=rho, lam_model=lam_model, lam0=lam, lam_b=lam_b,
                     cap_model=cap_model, c0=c, theta=theta, t_ref=t_ref)],
        nr=nr, nz=nz, length=L, bc_rmax=bc[0], bc_z0=bc[1], bc_zmax=bc[2], t_dirichlet=t_d,
        placement=placement, face_rule=0, interface_rule=0, source=None)
    if q0 is not None:
        cfg["source"] = dict(layer=0, q0=q0, t_period=1.0, t_on=1.0 if t_on is None else t_on,
                             t_start=0.0, waveform=0)
    return cfg


# ----------------------------------------------------------------------------
def test_grid_partition_hand_derived():
    # 64 nodes = 63 cells over 0.10/0.02/0.05/0.10 mm: ideal 23.33/4.67/11.67/23.33
    # -> floors 23/4/11/23 (61), two remainders .667 go to layers 1 and 2.
    g = oracle.grid(inputs.small_case(q0=1.0))
    assert list(np.nonzero(g["rclass"] == 2)[0]) == [23, 28, 40]
    assert g["rclass"][0] == 0 and g["rclass"][63] == 3
    assert g["r"][0] == 0.0 and abs(g["r"][63] - 0.27e-3) < 1e-18
    assert abs(g["r"][23] - 0.10e-3) < 1e-18 and abs(g["r"][40] - 0.17e-3) < 1e-18
    # 512 nodes over 0.10/0.02/0.05/0.10/0.05 mm: ideal 159.69/31.94/79.84/159.69/79.84
    # -> floors 159/31/79/159/79 (507); remainders order: 1, 2, 4 (tie -> lower), 0.
    cfg = inputs.production_case()
    for ly, t in zip(cfg["layers"], [0.10e-3, 0.02e-3, 0.05e-3, 0.10e-3, 0.05e-3]):
        ly["thickness"] = t
    g = oracle.grid(cfg)
    assert list(np.nonzero(g["rclass"] == 2)[0]) == [160, 192, 272, 431]
    z = g["z"]
    assert z[0] == 0.0 and abs(z[-1] - 10e-3) < 1e-18
    # the paper's cell, 64 nodes over 1.2/0.05/0.05/0.001 mm: ideal 58.11/2.42/2.42/0.05
    # -> floors 58/2/2/0, the 1 um insulator raised to the minimum of 2 cells (64),
    # the surplus cell taken from the largest layer: 57/2/2/2
    g = oracle.grid(inputs.paper_case(64, 41))
    assert list(np.nonzero(g["rclass"] == 2)[0]) == [57, 59, 61]


def test_rectangular_waveform_half_open():
    cfg = inputs.small_case(q0=1.0)   # 1 ms on, 10 ms period, Eq. (period)
    w = lambda t: oracle.waveform(cfg, t)
    assert w(0.0) == 1.0 and w(0.999e-3) == 1.0
    assert w(1.0e-3) == 0.0 and w(9.999e-3) == 0.0
    assert w(10.0e-3) == 1.0 and w(10.5e-3) == 1.0 and w(11.0e-3 + 1e-12) == 0.0
    assert w(-1e-9) == 0.0 and w(-9.5e-3) == 0.0      # no pulse before the first one
    cfg["source"]["t_start"] = 2e-3
    assert w(1.5e-3) == 0.0 and w(2e-3) == 1.0 and w(2.999e-3) == 1.0 and w(3e-3) == 0.0


def test_tanh_waveform_smooth_edges():
    cfg = inputs.adjoint_case(nr=8, nz=8)
    w = lambda t: oracle.waveform(cfg, t)
    assert abs(w(0.0) - 0.5) < 1e-12          # centre of the rising edge
    assert abs(w(0.5e-3) - 1.0) < 1e-12       # plateau
    assert abs(w(1.0e-3) - 0.5) < 1e-12       # centre of the falling edge
    assert abs(w(5e-3)) < 1e-12 and abs(w(10e-3) - 0.5) < 1e-12
    # continuous across the wrap point between pulses
    assert abs(w(5.5e-3 - 1e-12) - w(5.5e-3 + 1e-12)) < 1e-12
    # before the second pulse the rising edge of that pulse is the nearest one
    ew = cfg["source"]["edge_w"]
    assert abs(w(10e-3 - 2 * ew) - 0.5 * (1.0 + math.tanh(-2.0))) < 1e-12


def test_transient_turn_on_waveform():
    """Eq. (transient_function) with the exponent's sign read as negative:
    p^2 = 1 - exp(-(t - n t_prd)/(7 tau*)), tau* = tau/100, for the first tau
    of each period; then 1 while the pulse lasts (Eq. (period))."""
    cfg = inputs.small_case(q0=1.0)
    tau = 1e-5
    cfg["source"].update(waveform=2, edge_w=tau, t_period=25e-3, t_on=1e-3)
    w = lambda t: oracle.waveform(cfg, t)
    ts = tau / 100
    assert w(0.0) == 0.0                                       # switch-on
    assert abs(w(7 * ts) - (1 - math.exp(-1))) < 1e-15
    assert abs(w(0.5 * tau) - (1 - math.exp(-50 / 7))) < 1e-15
    assert w(tau) == 1.0 and w(0.5e-3) == 1.0                  # saturated
    assert w(1.0e-3) == 0.0 and w(24e-3) == 0.0                # pulse over
    assert w(25e-3 + 7 * ts) == pytest.approx(1 - math.exp(-1), abs=1e-9)  # next period


def test_uniform_fixed_point():
    cfg = inputs.small_case(q0=1.0)
    cfg["source"] = None
    T = np.full((cfg["nz"], cfg["nr"]), 20.0)
    T1, _, e = oracle.step_n(cfg, T, 50, 0.0, cfg["dt"])
    assert np.max(np.abs(T1 - T)) < 1e-12      # reproduced to rounding
    assert np.all(np.abs(e) < 1e-15)


# ----------------------------------------------------------------------------
def test_axial_steady_state_exact():
    """Constant lambda, uniform source, Neumann z=0 (half-cell ghost), Dirichlet z=L:
    T = T_D + X (L^2 - z^2) / (2 lambda) is reproduced by one step to rounding."""
    lam, X, L, TD = 3.0, 50.0, 1.0, 20.0
    cfg = single_layer(6, 17, L=L, lam=lam, placement=1, bc=(0, 0, 1), t_d=TD, q0=X)
    z = oracle.grid(cfg)["z"]
    Tz = TD + X * (L * L - z * z) / (2 * lam)
    T = np.repeat(Tz[:, None], cfg["nr"], axis=1)
    tau = 0.4 * oracle.tau_stab(cfg, 20.0, 40.0)
    T1, _, _ = oracle.step_n(cfg, T, 3, 0.0, tau)
    assert np.max(np.abs(T1 - T)) < 1e-12 * np.max(T)


def test_axial_steady_state_dirichlet_both_ends():
    """Constant lambda, uniform source, Dirichlet at z=0 and z=L (nodes on both
    faces): T = T_D + X z (L - z) / (2 lambda) is reproduced by one step to
    rounding."""
    lam, X, L, TD = 3.0, 50.0, 1.0, 20.0
    cfg = single_layer(6, 17, L=L, lam=lam, placement=1, bc=(0, 1, 1), t_d=TD, q0=X)
    z = oracle.grid(cfg)["z"]
    assert z[0] == 0.0 and abs(z[-1] - L) < 1e-15
    Tz = TD + X * z * (L - z) / (2 * lam)
    T = np.repeat(Tz[:, None], cfg["nr"], axis=1)
    tau = 0.4 * oracle.tau_stab(cfg, 20.0, 40.0)
    T1, _, _ = oracle.step_n(cfg, T, 3, 0.0, tau)
    assert np.max(np.abs(T1 - T)) < 1e-12 * np.max(T)


def test_radial_steady_state_dirichlet_rmax():
    """Constant lambda, uniform source, Dirichlet at r = R (a node on the
    boundary, half-cell ghost at the axis), insulated ends: the cylindrical
    3-point operator of Eq. (Lambda_i) is exact for T = T_D + X (R^2 - r^2) /
    (4 lambda), which one step reproduces to rounding."""
    lam, X, R, TD = 3.0, 50.0, 1.0, 20.0
    cfg = single_layer(9, 5, R=R, lam=lam, placement=1, bc=(1, 0, 0), t_d=TD, q0=X)
    r = oracle.grid(cfg)["r"]
    assert abs(r[-1] - R) < 1e-15 and abs(r[0] + r[1]) < 1e-15
    Tr = TD + X * (R * R - r * r) / (4 * lam)
    T = np.repeat(Tr[None, :], cfg["nz"], axis=0)
    tau = 0.4 * oracle.tau_stab(cfg, 20.0, 40.0)
    T1, _, _ = oracle.step_n(cfg, T, 3, 0.0, tau)
    assert np.max(np.abs(T1 - T)) < 1e-12 * np.max(T)


def _kirchhoff_error(M, b=1.2):
    lam0, Tr, X, L, TD = 2.0, 20.0, 400.0, 1.0, 20.0
    cfg = single_layer(3, M + 1, L=L, lam=lam0, lam_model=1, lam_b=b, t_ref=Tr,
                       placement=1, bc=(0, 0, 1), t_d=TD, q0=X)
    z = oracle.grid(cfg)["z"]
    exact = Tr * ((TD / Tr) ** (b + 1) + (b + 1) * X * (L * L - z * z) / (2 * lam0 * Tr)) ** (1 / (b + 1))
    T = np.repeat(exact[:, None], 3, axis=1)   # start near, converge to the discrete steady state
    tau = 0.45 * oracle.tau_stab(cfg, 20.0, 60.0)
    for _ in range(200):
        T1, _, _ = oracle.step_n(cfg, T, 400, 0.0, tau, want_trace=False, want_energy=False)
        done = np.max(np.abs(T1 - T)) < 1e-13
        T = T1
        if done:
            break
    return np.max(np.abs(T[1:, 1] - exact[1:]))


def test_kirchhoff_steady_state_second_order():
    e1, e2 = _kirchhoff_error(16), _kirchhoff_error(32)
    assert e2 < 5e-3
    assert 3.3 < e1 / e2 < 4.7, (e1, e2)


# ----------------------------------------------------------------------------
J11 = special.jn_zeros(1, 1)[0]   # first zero of J1: J0'(J11 r/R) = 0 at r = R


def _bessel_error(level):
    """Bessel-Fourier series T = T0 + sum_k a_k J0(j_{1,k} r/R) cos(m_k pi z/L)
    (three terms), Neumann on every face, constant kappa = lambda/(rho c) = 1:
    each term decays as exp(-(j_{1,k}^2/R^2 + m_k^2 pi^2/L^2) t)."""
    N = 8 * 2 ** level + 1
    cfg = single_layer(N + 1, N + 1, placement=1, bc=(0, 0, 0))
    g = oracle.grid(cfg)
    r, z = g["r"], g["z"]
    T0 = 20.0
    zeros = special.jn_zeros(1, 3)
    terms = [(1.0, zeros[0], 1), (0.3, zeros[1], 0), (-0.2, zeros[2], 2)]
    eta = z[2] - z[1]
    tau = 0.2 * eta * eta
    t_end = 0.02
    n = int(round(t_end / tau))
    tau = t_end / n
    u0 = sum(a * special.j0(k * r)[None, :] * np.cos(mz * math.pi * z)[:, None]
             for a, k, mz in terms)
    exact = T0 + sum(a * special.j0(k * r)[None, :] * np.cos(mz * math.pi * z)[:, None]
                     * math.exp(-(k ** 2 + (mz * math.pi) ** 2) * t_end) for a, k, mz in terms)
    T1, _, _ = oracle.step_n(cfg, T0 + u0, n, 0.0, tau, want_trace=False, want_energy=False)
    return np.max(np.abs(T1[1:-1, 1:-1] - exact[1:-1, 1:-1]))


def test_bessel_mode_second_order():
    e = [_bessel_error(k) for k in range(3)]
    assert e[2] < 5e-3, e
    assert 3.3 < e[1] / e[2] < 4.7, e


# ----------------------------------------------------------------------------
def _two_layer_radial(N, rule, swap=False):
    """Inner layer (radius a, lambda1, source X), outer (lambda2), Dirichlet T_D at R.
    Steady state: T = T_a + X (a^2 - r^2)/(4 lambda1) inside,
                  T = T_D + X a^2/(2 lambda2) ln(R/r) outside."""
    a, R, l1, l2, X, TD = 0.6, 1.0, 5.0, 0.5, 10.0, 20.0
    lay = lambda t, l: dict(thickness=t, rho=1.0, lam_model=0, lam0=l, cap_model=0, c0=1.0)
    cfg = dict(layers=[lay(a, l1), lay(R - a, l2)], nr=N + 1, nz=3, length=1.0,
               bc_rmax=1, bc_z0=0, bc_zmax=0, t_dirichlet=TD, placement=0,
               face_rule=0, interface_rule=rule,
               source=dict(layer=0, q0=X, t_period=1.0, t_on=1.0, t_start=0.0, waveform=0))
    if swap:  # deliberately wrong conductivities on the interface row sides
        cfg["layers"][0]["lam0"], cfg["layers"][1]["lam0"] = l2, l1
    r = oracle.grid(cfg)["r"]
    T, _, _ = oracle.step_n(cfg, np.full((3, N + 1), TD), 60, 0.0, 1e3, want_trace=False,
                            want_energy=False)
    Ta = TD + X * a * a / (2 * l2) * math.log(R / a)
    exact = np.where(r <= a, Ta + X * (a * a - r * r) / (4 * l1),
                     TD + X * a * a / (2 * l2) * np.log(R / np.maximum(r, 1e-300)))
    return np.max(np.abs(T[1] - exact)) / (Ta - TD)


@pytest.mark.parametrize("rule", [0, 1])
def test_two_layer_interface_first_order(rule):
    e = [_two_layer_radial(N, rule) for N in (40, 80, 160, 320)]
    # the paper states first order as a bound (Section 3); at least that is required
    assert e[-1] < 1e-2, e
    assert e[-2] / e[-1] > 1.8 and e[-3] / e[-2] > 1.8, e
    assert _two_layer_radial(160, rule, swap=True) > 0.5


# ----------------------------------------------------------------------------
def _uniform_heating(tau, cap_model=1):
    c0, theta, Tr, rho, X = 5.0, 60.0, 20.0, 7900.0, 4.0e7
    poly = [0.5, 0.1, 0.005, 1e-4]      # c = a0 + a1 T + a2 T^2 + a3 T^3 (Eq. (poly_cap))
    cfg = single_layer(5, 5, lam=10.0, rho=rho, c=c0, cap_model=cap_model, theta=theta,
                       t_ref=Tr, placement=0, bc=(0, 0, 0), q0=X)
    cfg["layers"][0]["cap_poly"] = poly
    t_end = 2e-3
    n = int(round(t_end / tau))
    T1, _, _ = oracle.step_n(cfg, np.full((5, 5), 20.0), n, 0.0, t_end / n,
                             want_trace=False, want_energy=False)
    if cap_model == 1:
        cap = lambda T: c0 * (T / Tr) ** 3 / (1 + (T / theta) ** 3)
    else:
        cap = lambda T: poly[0] + poly[1] * T + poly[2] * T ** 2 + poly[3] * T ** 3
    sol = integrate.solve_ivp(lambda t, y: [X / (rho * cap(y[0]))], (0, t_end), [20.0],
                              rtol=1e-12, atol=1e-12)
    return T1[2, 2], sol.y[0, -1]


@pytest.mark.parametrize("cap_model", [1, 2])
def test_uniform_heating_temperature_dependent_capacity(cap_model):
    a, exact = _uniform_heating(2e-6, cap_model)
    b, _ = _uniform_heating(1e-6, cap_model)
    assert abs(b - exact) < 0.6 * abs(a - exact)       # first order in tau
    rich = 2 * b - a                                    # Richardson limit
    assert abs(rich - exact) < 1e-4 * abs(exact - 20.0), (a, b, rich, exact)


def test_injected_heat_equals_cylinder_volume_times_X():
    R, L, X = 0.5, 2.0, 7.0
    cfg = single_layer(9, 9, R=R, L=L, placement=1, bc=(0, 0, 0), q0=X)
    tau = 1e-3
    cfg["source"].update(t_on=3 * tau - 1e-12, t_period=1.0)   # on for steps 0, 1, 2
    _, _, e = oracle.step_n(cfg, np.full((9, 9), 20.0), 10, 0.0, tau)
    assert abs(e[1] - 3 * tau * X * math.pi * R * R * L) < 1e-12 * e[1]


# ----------------------------------------------------------------------------
@pytest.mark.parametrize("interface_rule,face_rule", [(0, 0), (1, 0), (0, 1)])
def test_energy_identity_multilayer(interface_rule, face_rule):
    cfg = inputs.small_case()
    cfg.update(interface_rule=interface_rule, face_rule=face_rule)
    T = inputs.initial_field(cfg, "smooth", seed=3)
    T[0] = T[1]               # start from a field that satisfies the Neumann closures
    T[:, 0] = T[:, 1]
    T[:, -1] = T[:, -2]
    T[-1] = 20.0
    _, _, e = oracle.step_n(cfg, T, 600, 0.0, cfg["dt"])
    dE, Q, PD, PI, PN = e
    assert Q > 0 and dE > 0
    assert abs(dE - Q - PD - PI - PN) <= 1e-12 * max(abs(Q), abs(dE))
    assert abs(PN) <= 1e-12 * abs(Q)          # Neumann ghost edges carry no flux
    if interface_rule == 1:
        assert abs(PI) <= 1e-12 * abs(Q)      # conservative interface rows
    else:
        assert abs(PI) > 1e-9 * abs(Q)        # first-order interface defect


def test_energy_identity_dirichlet_both_ends():
    """Heat leaves through both Dirichlet faces z = 0 and z = z_max; the
    identity dE = Q + PhiD + PhiI + PhiN still closes to 1e-12."""
    cfg = inputs.small_case()
    cfg.update(bc_z0=1, interface_rule=1)
    T = inputs.initial_field(cfg, "smooth", seed=8)
    T[:, 0] = T[:, 1]
    T[:, -1] = T[:, -2]
    T[0] = 20.0
    T[-1] = 20.0
    _, _, e = oracle.step_n(cfg, T, 600, 0.0, cfg["dt"])
    dE, Q, PD, PI, PN = e
    assert abs(dE - Q - PD - PI - PN) <= 1e-12 * max(abs(Q), abs(dE))
    assert PD < -1e-3 * abs(Q)                # the warm field loses heat at both ends
    assert abs(PN) <= 1e-12 * abs(Q) and abs(PI) <= 1e-12 * abs(Q)


@pytest.mark.parametrize("variant", ["plain", "interface_rule_1", "rmax_dirichlet", "stepped"])
def test_line_sweep_equals_dense_solve(variant):
    """Brute force for the line solve: the sweep of Eqs. (front_sweep),
    (cc_first_3), (back_sweep) with its closures returns, on every line of a
    16-node cylinder with three interfaces, the dense solution (numpy, partial
    pivoting) of the rows it was given; the axis closure is exact."""
    cfg = inputs.small_case()
    cfg.update(nr=16, nz=10)
    if variant == "interface_rule_1":
        cfg["interface_rule"] = 1
    elif variant == "rmax_dirichlet":
        cfg["bc_rmax"] = 1
    elif variant == "stepped":
        cfg["step"] = dict(layers=2, z=5e-3)
    cfg["dt"] = 0.5 * oracle.tau_stab(cfg, 20.0, 100.0)
    assert list(np.nonzero(oracle.grid(cfg)["rclass"] == 2)[0]) == [5, 7, 10]
    T = inputs.initial_field(cfg, "smooth", seed=2)
    t = 1e-3 - 0.5 * cfg["dt"]                      # inside the pulse: the source is on
    T1, _, _ = oracle.step_n(cfg, T, 1, t, cfg["dt"], want_trace=False, want_energy=False)
    for j in range(1, cfg["nz"] - 1):
        a, b, c, f = oracle.line_rows(cfg, T, j, t, cfg["dt"])
        n = len(b)
        A = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
        assert a[0] == 0.0 and c[-1] == 0.0
        x = np.linalg.solve(A, f)
        assert np.max(np.abs(T1[j, :n] - x)) < 1e-11, (j, np.max(np.abs(T1[j, :n] - x)))
        assert T1[j, 0] == T1[j, 1]
        if variant != "rmax_dirichlet":
            assert abs(T1[j, n - 1] - T1[j, n - 2]) < 1e-11
    if variant == "stepped":
        assert len(oracle.line_rows(cfg, T, cfg["nz"] - 2, t, cfg["dt"])[1]) == 8


def test_no_dirichlet_face_no_dirichlet_flux():
    """With Neumann on every face (a start with T_0 != T_1 at z = 0), no heat
    is booked as Dirichlet flux and the identity still closes."""
    cfg = inputs.small_case()
    cfg.update(bc_zmax=0, interface_rule=1)
    T = inputs.initial_field(cfg, "smooth", seed=9)
    T[1] += 0.5                                # T_0 != T_1: heat through the ghost edge
    _, _, e = oracle.step_n(cfg, T, 1, 0.0, cfg["dt"])
    dE, Q, PD, PI, PN = e
    assert PD == 0.0
    assert abs(PN) > 1e-6 * abs(Q)
    assert abs(dE - Q - PD - PI - PN) <= 1e-12 * max(abs(Q), abs(dE))


def test_boundary_closures():
    cfg = inputs.small_case()
    T = inputs.initial_field(cfg, "smooth", seed=1)
    T1, tr, _ = oracle.step_n(cfg, T, 20, 0.0, cfg["dt"])
    assert np.array_equal(T1[:, 0], T1[:, 1])          # That_0 = That_1, Eq. (first_oder_bc)
    assert np.max(np.abs(T1[:, -1] - T1[:, -2])) < 1e-12 * 40
    assert np.array_equal(T1[0], T1[1])                # Neumann z = 0
    assert np.all(T1[-1] == 20.0)                      # Dirichlet z = z_max
    assert tr[-1, 0] == T1[0, -1]
    cfg["bc_z0"] = 1                                   # Dirichlet z = 0: the trace's
    T1, tr, _ = oracle.step_n(cfg, T, 3, 0.0, cfg["dt"])  # surface value is T_D
    assert np.all(T1[0] == 20.0) and np.all(tr[:, 0] == 20.0)


# ----------------------------------------------------------------------------
def _checkerboard_growth(frac):
    cfg = single_layer(4, 33, L=1.0, lam=1.0, placement=0, bc=(0, 0, 1), t_d=20.0)
    ts = oracle.tau_stab(cfg, 10.0, 30.0)
    j = np.arange(33)
    T = 20.0 + 1e-3 * ((-1.0) ** j)[:, None] * np.ones((1, 4))
    T[-1] = 20.0
    T1, _, _ = oracle.step_n(cfg, T, 400, 0.0, frac * ts, want_trace=False, want_energy=False)
    return np.max(np.abs(T1 - 20.0)) / 1e-3, ts


def test_stability_bound():
    g_lo, ts = _checkerboard_growth(0.95)
    g_hi, _ = _checkerboard_growth(1.05)
    # Eq. (stability_condition) with constant rho c / lambda = 1 and eta = 1/32
    assert abs(ts - 0.5 / 32 ** 2) < 1e-15
    assert g_lo <= 1.0
    assert g_hi > 10.0
