"""The paper's own model data (Section 5) and the transient schedule (Section 3.1).

Checks of the reading of the printed tables, kept in tests/golden with their
citation: the conductivity table only makes sense with its columns read as
b4..b0 -- then the outer insulator's row is the constant
1e-3 W/(cm K) the text states and every fit is positive over 4.2-60 K.  The
heat-capacity table read as printed has the graphite fit turn negative near
22 K, inside the stated 4.2-60 K range; this is recorded, and runs of the paper
case stay below it.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1408_5853_gb300 import inputs, schedule

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_material_fits.json")


def _fit():
    with open(GOLDEN) as f:
        return json.load(f)


def test_conductivity_table_reading():
    fit = _fit()
    b = fit["lam_b0_b1_b2_b3_b4"]
    assert b[3] == [1.0e-3, 0.0, 0.0, 0.0, 0.0]        # lambda_3 = 1e-3 W/(cm K), stated in the text
    T = np.linspace(4.2, 60.0, 561)
    for m in range(4):
        lam = sum(b[m][k] * T ** k for k in range(5))
        assert np.all(lam > 0), m
    # copper at 20 K: the scale of a high-purity copper conductor (W/(cm K))
    assert 2.0 < sum(b[0][k] * 20.0 ** k for k in range(5)) < 3.0


def test_heat_capacity_table_as_printed():
    fit = _fit()
    a = fit["cap_a0_a1_a2_a3"]
    T = np.linspace(4.2, 60.0, 5601)
    for m in (0, 1, 3):
        assert np.all(sum(a[m][k] * T ** k for k in range(4)) > 0), m
    c2 = sum(a[2][k] * T ** k for k in range(4))
    first_negative = T[np.argmax(c2 <= 0)]
    assert 21.5 < first_negative < 22.5              # graphite fit negative above ~22 K


def test_paper_case_units_and_source():
    cfg = inputs.paper_case(nr=64, nz=41)
    fit = _fit()
    r = fit["radii_cm"]
    assert abs(sum(l["thickness"] for l in cfg["layers"]) - r["rmax"] * 1e-2) < 1e-15
    assert cfg["layers"][3]["lam_poly"][0] == pytest.approx(0.1)     # 1e-3 W/(cm K) in W/(m K)
    s2 = math.pi * ((r["r2"] * 1e-2) ** 2 - (r["r1"] * 1e-2) ** 2)
    # X = chi(T) I0^2 / S2^2 at 16 K: 1.8/4 Ohm cm = 4.5e-3 Ohm m
    X16 = cfg["source"]["q0"] * cfg["source"]["g_ref"] / math.sqrt(16.0)
    assert X16 == pytest.approx(4.5e-3 * 0.363 ** 2 / s2 ** 2, rel=1e-12)
    assert cfg["source"]["waveform"] == 2 and cfg["source"]["edge_w"] == 1e-5


def test_transient_schedule():
    ch = schedule.transient_schedule(t_period=25e-3, tau=1e-5, t_end=50e-3)
    assert ch[0][0] == 0.0 and ch[0][1] == pytest.approx(1e-7) and ch[0][2] == 100  # tau* = tau/100
    assert ch[1][0] == pytest.approx(1e-5) and ch[1][1] == 1e-5
    assert ch[2][0] == pytest.approx(25e-3) and ch[2][2] == 100
    total = sum(dt * n for _, dt, n in ch)
    assert total == pytest.approx(50e-3, rel=1e-9)
    for (t0, dt, n), (t1, _, _) in zip(ch, ch[1:]):
        assert t0 + dt * n == pytest.approx(t1, rel=1e-9, abs=1e-15)
