"""Run a batch until every instance's 0D waveforms are periodic.

The criterion is the cycle-to-cycle change computed on the device by
``lbm_cycle_change``: for instance q with beat period T_q, at a step that
is a multiple of T_q, delta_q = max over its boundaries and over the
waveforms (boundary flow Q_u, mean gauge pressure) of
max_t |W(t) - W(t - T_q)| / max_t |W(t - T_q)| over the last beat.  The
instance counts as periodic at the first beat end with delta_q <= tol.
"""
from __future__ import annotations

import math
from functools import reduce

import numpy as np


def run_to_periodic(lat, periods, tol: float = 0.01, max_cycles: int = 20, chunk: int = 0,
                    on_chunk=None, history=None):
    """Advances ``lat`` (a :class:`Lattice`) until all instances are periodic
    or ``max_cycles`` beats of the longest period have run.

    Returns ``(cycles, steps)``: ``cycles[q]`` is the number of whole beats
    instance q had simulated when first found periodic (-1 if never), and
    ``steps`` the total steps taken.  ``chunk`` (default: gcd of the periods)
    is the stepping granularity; ``on_chunk(step)`` is called after each chunk.
    ``history`` (a dict, optional) receives for every instance the list of
    its cycle-to-cycle changes at each beat end until it is periodic.
    """
    periods = np.asarray(periods, dtype=np.int64)
    if chunk <= 0:
        chunk = int(reduce(math.gcd, [int(t) for t in periods]))
    n = periods.size
    cycles = np.full(n, -1, dtype=np.int64)
    start = lat.info().steps
    limit = start + int(max_cycles * periods.max())
    step = start
    while step < limit and (cycles < 0).any():
        lat.step(chunk)
        step += chunk
        if on_chunk is not None:
            on_chunk(step)
        at_end = ((step - start) % periods == 0) & (cycles < 0) & (step - start >= 2 * periods)
        if at_end.any():
            delta = lat.cycle_change(periods)
            ok = at_end & (delta >= 0) & (delta <= tol)
            cycles[ok] = (step - start) // periods[ok]
            if history is not None:
                for q in np.flatnonzero(at_end):
                    history.setdefault(int(q), []).append(float(delta[q]))
    return cycles, step - start
