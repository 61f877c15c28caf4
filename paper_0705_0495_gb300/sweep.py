"""Batched run of the voltage sweep at 13.8 Pa (Sec. IV, Fig. Central) and of
the associative-detachment contrast at 150 V (Fig. Profiles).

All discharges of `inputs.sweep_13p8` advance together, one launch per kernel
for all of them.  After `cycles` RF cycles the densities are averaged over the
last `average_cycles` (the diagnostics sample every 10 steps) and reported at
x = L/2 (the bulk densities of Fig. Central) and as profiles (Fig. Profiles).

    python -m paper_0705_0495_gb300.sweep --cycles 1000 --average 50
"""
import argparse
import json
import time

import numpy as np

from . import inputs, o2pic


def run(cycles=1000, average_cycles=50, n_op=20000, seed=1, fp64=False):
    ds = inputs.sweep_13p8(n_op=n_op, seed=seed, fp64=fp64, rf_cycles=cycles)
    spc = ds[0].steps_per_cycle
    average_cycles = min(average_cycles, cycles)
    sim = o2pic.Simulation(ds, inputs.xs_tables())
    try:
        t0 = time.time()
        sim.step((cycles - average_cycles) * spc)
        for k in range(len(ds)):
            sim.diagnostics(k, reset=True)
        sim.step(average_cycles * spc)
        wall = time.time() - t0
        rows, profiles = [], []
        psteps = 0
        for k, d in enumerate(ds):
            g = sim.diagnostics(k)
            dens = g["dens_sum"] / max(g["n_samples"], 1)
            mid = d.n_cells // 2
            psteps += g["particle_steps"]
            rows.append({"U_rf": d.U_rf, "C": d.C_delta, "n_e": dens[0, mid], "n_O-": dens[1, mid],
                         "n_O2+": dens[2, mid], "superparticles": [sim.count(k, s) for s in range(3)],
                         "events": g["events"].tolist()})
            profiles.append(dens)
        return {"cycles": cycles, "average_cycles": average_cycles, "wall_s": wall,
                "particle_steps": psteps, "rows": rows}, profiles
    finally:
        sim.close()


def main():
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--cycles", type=int, default=1000)
    p.add_argument("--average", type=int, default=50)
    p.add_argument("--n-op", type=int, default=20000)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--profiles", default=None, help="write the averaged profiles to this .npz")
    a = p.parse_args()
    res, prof = run(a.cycles, a.average, a.n_op, a.seed)
    if a.profiles:
        np.savez(a.profiles, **{f"U{r['U_rf']:g}_C{r['C']:.3f}": pr for r, pr in zip(res["rows"], prof)})
    print(json.dumps(res))


if __name__ == "__main__":
    main()
