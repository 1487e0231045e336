"""Time-step schedule of the transient turn-on model (Section 3.1).

At every switch-on t = t_start + n t_prd the paper advances the field with
the small step tau* = tau / 100 up to t_start + n t_prd + tau, then with tau up
to the next switch-on (the source waveform there is nu(t) p^2(t), waveform 2).
A schedule is a list of chunks (t0, dt, n_steps) to run in order, each one a
cc_step_n call.
"""
from __future__ import annotations


def transient_schedule(t_period: float, tau: float, t_end: float, t_start: float = 0.0,
                       sub: int = 100) -> list[tuple[float, float, int]]:
    """Chunks covering [t_start, t_end): `sub` steps of tau/sub after each
    switch-on, then steps of tau (the last chunk of a period is shortened to a
    whole number of steps that does not pass the next switch-on)."""
    if not (t_period > tau > 0.0) or sub < 1:
        raise ValueError("need t_period > tau > 0 and sub >= 1")
    out = []
    k = 0
    while True:
        on = t_start + k * t_period
        if on >= t_end:
            break
        out.append((on, tau / sub, sub))
        n_main = int((min(on + t_period, t_end) - (on + tau)) / tau + 1e-9)
        if n_main > 0:
            out.append((on + tau, tau, n_main))
        k += 1
    return out


def run_schedule(step, chunks) -> None:
    """Call step(t0, dt, n_steps) for every chunk, in order."""
    for t0, dt, n in chunks:
        step(t0, dt, n)
