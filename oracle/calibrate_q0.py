"""Calibrate the heater amplitude q0 of the synthetic workloads.

TEST INFRASTRUCTURE (an input generator): it calls only the oracle.

The workloads ask for a heater amplitude "set so that the surface peaks near
45 K" without a number.  Reading taken: q0 is the value for which the maximum
over the 20 ms run (2 pulses of 1 ms every 10 ms) of the surface temperature
T(r_max, z=0) of the 4-layer 64x128 case equals 45.0 K (+/- 0.01 K), found by
regula falsi on the oracle.  The result is written to
``paper_1408_5853_gb300/calibration.json`` and read by the workload module.

Run:  python -m oracle.calibrate_q0
"""
from __future__ import annotations

import json
import os
import sys

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, _ROOT)

from oracle import oracle  # noqa: E402
from paper_1408_5853_gb300 import inputs  # noqa: E402

TARGET = 45.0


def surface_peak(q0: float) -> float:
    cfg = inputs.small_case(q0=q0)
    T = inputs.initial_field(cfg)
    _, trace, _ = oracle.step_n(cfg, T, cfg["n_steps_full"], 0.0, cfg["dt"], want_energy=False)
    return float(trace[:, 0].max())


def main() -> None:
    lo, hi = 5.0e9, 1.0e10
    flo, fhi = surface_peak(lo) - TARGET, surface_peak(hi) - TARGET
    assert flo < 0 < fhi, (flo, fhi)
    q = lo
    for _ in range(40):
        q = hi - fhi * (hi - lo) / (fhi - flo)
        f = surface_peak(q) - TARGET
        print(f"q0={q:.9e} peak-45={f:+.5f}")
        if abs(f) < 0.01:
            break
        if f < 0:
            lo, flo = q, f
        else:
            hi, fhi = q, f
    q = float(f"{q:.6e}")
    out = {
        "q0_W_m3": q,
        "surface_peak_K": surface_peak(q),
        "how": "oracle/calibrate_q0.py: regula falsi on the oracle so that the maximum "
               "surface temperature T(r_max, z=0) over 20 ms (2 pulses) of the 4-layer "
               "64x128 case is 45.0 K",
    }
    path = os.path.join(_ROOT, "paper_1408_5853_gb300", "calibration.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(out)


if __name__ == "__main__":
    main()
