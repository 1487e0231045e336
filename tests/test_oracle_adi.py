"""Pins of the oracle's ADI variant (Peaceman-Rachford, two half steps of
tau/2: implicit in r, then implicit in z), the scheme the paper names as the
unconditionally stable alternative to its own (Section 3, after
Eq. (stability_condition)).  Pinned by facts that do not restate its formulas:

* second order in time (Richardson ratio 4 on a three-term Bessel-Fourier
  decay), converging to that exact series within the spatial error;
* stable and decaying at tau = 1000 x the explicit stability bound;
* its fixed point is the steady state of the paper's scheme (nonlinear
  materials, two layers with an interface, constant source): both schemes
  iterated to convergence agree;
* at small tau it approaches the paper's scheme (difference O(tau));
* a uniform field at the Dirichlet temperature without source is a fixed point.
"""
import math

import numpy as np
from scipy import special

from oracle import oracle
from test_oracle_pins import single_layer


def _bessel_case(N=33):
    cfg = single_layer(N + 1, N + 1, placement=1, bc=(0, 0, 0))
    g = oracle.grid(cfg)
    r, z = g["r"], g["z"]
    zeros = special.jn_zeros(1, 3)
    terms = [(1.0, zeros[0], 1), (0.3, zeros[1], 0), (-0.2, zeros[2], 2)]
    u = lambda t: sum(a * special.j0(k * r)[None, :] * np.cos(mz * math.pi * z)[:, None]
                      * math.exp(-(k ** 2 + (mz * math.pi) ** 2) * t) for a, k, mz in terms)
    return cfg, u, z[2] - z[1]


def test_adi_second_order_in_time_and_converges_to_series():
    cfg, u, eta = _bessel_case()
    t_end = 0.02
    res = {}
    for n in (10, 20, 40, 80):
        res[n], _ = oracle.step_adi_n(cfg, 20.0 + u(0.0), n, 0.0, t_end / n, want_trace=False)
    d = [np.abs(res[n] - res[2 * n]).max() for n in (10, 20, 40)]
    for k in range(2):
        assert 3.7 < d[k] / d[k + 1] < 4.3, d
    # the time steps are 4 and 0.5 x the explicit bound; the limit is the
    # exact series up to the spatial error of this grid (second order in h)
    err = np.abs(res[80] - (20.0 + u(t_end)))[1:-1, 1:-1].max()
    assert err < 1.5e-3, err
    assert t_end / 10 > 4.0 * 0.5 * eta * eta


def test_adi_stable_far_above_the_explicit_bound():
    cfg, u, eta = _bessel_case()
    tau = 1000.0 * 0.5 * eta * eta
    u0 = u(0.0)
    T, _ = oracle.step_adi_n(cfg, 20.0 + u0, 30, 0.0, tau, want_trace=False)
    assert np.all(np.isfinite(T))
    assert np.abs(T - 20.0).max() < 0.01 * np.abs(u0).max()


def _two_layer_case(nr=10, nz=12):
    lay = lambda t, l0, b, c0: dict(thickness=t, rho=2000.0, lam_model=1, lam0=l0, lam_b=b,
                                    cap_model=1, c0=c0, theta=50.0, t_ref=20.0)
    # unequal cell widths on the two sides of the interface (7 and 2 cells)
    return dict(layers=[lay(0.2e-3, 12.0, 1.0, 5.0), lay(0.05e-3, 2.0, 0.6, 9.0)],
                nr=nr, nz=nz, length=0.4e-3, bc_rmax=0, bc_z0=0, bc_zmax=1, t_dirichlet=20.0,
                placement=0, face_rule=0, interface_rule=0,
                source=dict(layer=0, q0=4e9, t_period=1.0, t_on=1.0, t_start=0.0, waveform=0))


def test_adi_fixed_point_is_the_steady_state_of_the_scheme():
    # both interface rules; Dirichlet on every face (heat leaves at r_max and z = 0 too)
    for rule, bcs in ((0, (0, 0, 1)), (1, (0, 0, 1)), (0, (1, 1, 1))):
        cfg = _two_layer_case()
        cfg["interface_rule"] = rule
        cfg["bc_rmax"], cfg["bc_z0"], cfg["bc_zmax"] = bcs
        ts = oracle.tau_stab(cfg, 20.0, 60.0)
        T = np.full((cfg["nz"], cfg["nr"]), 20.0)
        # the paper's scheme, small steps, to convergence
        Tm = T.copy()
        for _ in range(200):
            Tn, _, _ = oracle.step_n(cfg, Tm, 500, 0.0, 0.9 * ts, want_trace=False,
                                     want_energy=False)
            if np.abs(Tn - Tm).max() < 1e-12:
                Tm = Tn
                break
            Tm = Tn
        # ADI, steps of 200 x the bound
        Ta = T.copy()
        for _ in range(200):
            Tn, _ = oracle.step_adi_n(cfg, Ta, 50, 0.0, 200.0 * ts, want_trace=False)
            if np.abs(Tn - Ta).max() < 1e-12:
                Ta = Tn
                break
            Ta = Tn
        assert Tm.max() > 22.0  # the source heats well above the Dirichlet value
        assert np.abs(Ta - Tm).max() < 1e-9 * Tm.max(), (rule, np.abs(Ta - Tm).max())


def test_adi_approaches_the_scheme_at_small_tau():
    cfg = _two_layer_case()
    ts = oracle.tau_stab(cfg, 20.0, 60.0)
    T0 = np.full((cfg["nz"], cfg["nr"]), 20.0)
    t_end = 40 * ts
    diffs = []
    for n in (40, 80, 160):
        Ta, _ = oracle.step_adi_n(cfg, T0, n, 0.0, t_end / n, want_trace=False)
        Tm, _, _ = oracle.step_n(cfg, T0, n, 0.0, t_end / n, want_trace=False, want_energy=False)
        diffs.append(np.abs(Ta - Tm).max())
    assert diffs[0] > diffs[1] > diffs[2]
    assert diffs[1] / diffs[2] > 1.6, diffs   # at least first order in tau


def test_adi_uniform_dirichlet_field_is_a_fixed_point():
    cfg = _two_layer_case()
    cfg["source"] = None
    T0 = np.full((cfg["nz"], cfg["nr"]), 20.0)
    T, tr = oracle.step_adi_n(cfg, T0, 5, 0.0, 1e-3)
    assert np.abs(T - 20.0).max() < 1e-11   # rounding of the line solves only
    assert np.abs(tr - 20.0).max() < 1e-11
