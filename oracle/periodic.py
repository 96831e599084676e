"""Periodic-state criterion of the 0D waveforms, plain numpy (test infrastructure).

The paper runs its coupled simulations for several cardiac cycles and reads
the results once the waveforms repeat from beat to beat; it states no
numerical criterion.  The criterion used here (a fixed reading, the same on
both sides of every comparison) is the cycle-to-cycle change

    delta = max over the boundaries and over the waveforms W in
            {Q_u (boundary flow fed to the 0D model), mean gauge pressure}
            of  max_t |W(t) - W(t - T)| / max_t |W(t - T)|,

with t running over the last T steps of the record (the last beat) and
t - T over the beat before it; the state counts as periodic once
delta <= 0.01.  Fewer than 2 T recorded steps give delta = -1 (not enough
history); a waveform whose previous beat is identically zero is skipped.

Only ``tests/``, the smoke check and the benchmark's CPU-baseline leg may
use this module; it shares no code with the CUDA library.
"""
from __future__ import annotations

import numpy as np


def cycle_change(waves: np.ndarray, period: int) -> float:
    """Cycle-to-cycle change of one instance's waveform record.

    ``waves``: the oracle's record, one row per step,
    ``[t, (Q_u, P_mean - P_ref, chamber state, valve) per boundary]``.
    ``period``: beat length T in steps (>= 1).
    """
    w = np.asarray(waves, dtype=np.float64)
    T = int(period)
    if T < 1:
        raise ValueError("period must be >= 1")
    if w.ndim != 2 or (w.shape[1] - 1) % 4 != 0:
        raise ValueError("expected rows of 1 + 4 * n_boundaries values")
    if w.shape[0] < 2 * T:
        return -1.0
    nbc = (w.shape[1] - 1) // 4
    last = w[-T:]
    prev = w[-2 * T:-T]
    worst = 0.0
    for k in range(nbc):
        for col in (1 + 4 * k, 2 + 4 * k):          # Q_u and mean gauge pressure of boundary k
            num = 0.0
            den = 0.0
            for t in range(T):                       # plain loops: one beat against the one before
                num = max(num, abs(last[t, col] - prev[t, col]))
                den = max(den, abs(prev[t, col]))
            if den > 0.0:
                worst = max(worst, num / den)
    return worst
