"""Runtime autotuners of the cell-sort interval and of the push's launch
shape (threads per block, slots per thread, blocks per SM).

The sort runs on every particle-target step (every n1 steps) and, in
addition, every `sort_interval` steps: sorting more often keeps the particles
of a warp in fewer cells (cheaper charge deposition in the push) at the cost
of more sorts.  The tuner times a few RF-cycle fractions of the discharge for
each candidate interval (the divisors of n1, and 0 = only on particle-target
steps) on the GPU and returns the fastest.  The choice changes the slot order
and so the realisation of the random streams, not the method: the oracle
follows the same interval.

The push is a persistent grid of blocks taking tickets of tiles; how many
blocks share an SM (1 up to what its registers and shared memory hold) trades
latency hiding against contention, and the shapes it is compiled for trade
threads per block (the per-block charge grid is shared by more or fewer
warps) against slots per thread (more independent work per thread, more
registers).  Its results depend on none of these, so the push tuner switches
them on one running simulation and times the candidates in interleaved
rounds (each round gives every candidate the next stretch of the discharge,
so a drift of the plasma favours none).  Both push tuners end on a whole RF
cycle, so that whole-cycle steps after them replay the captured cycle graph.
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
        sim = o2pic.Simulation([d], tables, numeric_budget=1.0 if d.gas_scheme else None)
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


def push_candidates(max_per_sm):
    """Blocks per SM worth timing for the push: every count that fits."""
    return list(range(1, max(1, int(max_per_sm)) + 1))


def tune_push_blocks(sim, steps=200, rounds=2, cands=None):
    """Time each blocks-per-SM count of the push on the running simulation
    `sim` (CUDA events on its stream, `steps` time steps per candidate and
    round after one untimed period for the new grid's graph); leaves the
    fastest set and returns (best, {count: ms per time step})."""
    import torch
    _, mx = sim.launch("push")
    cands = cands if cands is not None else push_candidates(mx)
    warm = max(2, min(steps, 64))
    tot = {k: 0.0 for k in cands}
    for _ in range(rounds):
        for k in cands:
            sim.set_launch(k)
            sim.step(warm)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(sim.stream)
            sim.step(steps)
            e1.record(sim.stream)
            torch.cuda.synchronize()
            tot[k] += e0.elapsed_time(e1)
    ms = {k: v / (rounds * steps) for k, v in tot.items()}
    best = min(ms, key=ms.get)
    sim.set_launch(best)
    sim.align_to_cycle()
    return best, ms


def shape_candidates(shapes):
    """(shape index, blocks per SM) pairs worth timing: every count that fits
    for every compiled shape; shapes as given by Simulation.launch_shapes()"""
    return [(k, b) for k, (_, _, mx) in enumerate(shapes) for b in push_candidates(mx)]


def tune_push_shape(sim, steps=200, rounds=2):
    """Time every (shape, blocks per SM) of the push on the running simulation
    `sim` as tune_push_blocks does; leaves the fastest set and returns
    ((threads, slots per thread, blocks per SM), {"threads x spt @ blocks":
    ms per time step})."""
    import torch
    shapes = sim.launch_shapes()
    cands = shape_candidates(shapes)
    warm = max(2, min(steps, 64))
    tot = {c: 0.0 for c in cands}
    for _ in range(rounds):
        for c in cands:
            sim.set_launch_shape(*c)
            sim.step(warm)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(sim.stream)
            sim.step(steps)
            e1.record(sim.stream)
            torch.cuda.synchronize()
            tot[c] += e0.elapsed_time(e1)
    ms = {c: v / (rounds * steps) for c, v in tot.items()}
    best = min(ms, key=ms.get)
    sim.set_launch_shape(*best)
    sim.align_to_cycle()
    nt, spt, _ = shapes[best[0]]
    return (nt, spt, best[1]), {f"{shapes[k][0]}x{shapes[k][1]}@{b}": v for (k, b), v in ms.items()}
