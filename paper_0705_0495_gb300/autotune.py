"""Runtime autotuner of the cell-sort interval.

The sort runs on every particle-target step (every n1 steps) and, in
addition, every `sort_interval` steps: sorting more often keeps the particles
of a warp in fewer cells (cheaper charge deposition in the push) at the cost
of more sorts.  The tuner times a few RF-cycle fractions of the discharge for
each candidate interval (the divisors of n1, and 0 = only on particle-target
steps) on the GPU and returns the fastest.  The choice changes the slot order
and so the realisation of the random streams, not the method: the oracle
follows the same interval.
"""
import dataclasses

from . import o2pic


def candidates(n1):
    """Sort intervals worth timing for a particle-target interval n1."""
    if n1 <= 0:
        return [1, 2, 5, 10, 20]
    return sorted({k for k in range(1, n1 + 1) if n1 % k == 0} | {0})


def tune_sort_interval(discharge, tables, warm_steps=100, timed_steps=200, cands=None):
    """Time each candidate interval on `discharge` (a fresh simulation each,
    CUDA events on the library's stream); returns (best interval, {interval:
    ms per time step})."""
    import torch
    ms = {}
    for k in (cands if cands is not None else candidates(discharge.n1)):
        d = dataclasses.replace(discharge, sort_interval=k)
        sim = o2pic.Simulation([d], tables)
        try:
            sim.step(warm_steps)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(sim.stream)
            sim.step(timed_steps)
            e1.record(sim.stream)
            torch.cuda.synchronize()
            ms[k] = e0.elapsed_time(e1) / timed_steps
        finally:
            sim.close()
    best = min(ms, key=ms.get)
    return best, ms
