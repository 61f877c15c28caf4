#!/usr/bin/env python
"""Throughput of the PIC-MCC time step (push + deposit + MCC, with field
solve, births, sort and particle-target pass) on GB300, in particle-steps/s.

One bench step is one RF cycle of the workload (all time steps of the cycle).
Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead.
Multi-GPU (torchrun): every rank advances its own discharge (seed 1 + rank);
no data-path collective, weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_0705_0495_gb300 import inputs  # noqa: E402

METRIC = "particle-steps/s (push+deposit+MCC) and % HBM roofline, FP32/batched vs FP64"
UNIT = "particle-steps/s"
L2_BYTES = 129 * 1024 * 1024


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5, help="timed RF cycles")
    p.add_argument("--warmup", type=int, default=3, help="untimed RF cycles")
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="cfg4", choices=sorted(inputs.WORKLOADS))
    p.add_argument("--fp64", action="store_true", help="run the FP64 path on the workload")
    p.add_argument("--scale", type=float, default=1.0,
                   help="fraction of the workload's superparticles (same plasma density)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--n2", type=int, default=None,
                   help="intra-species Coulomb collisions every n2 steps on the workload (default: none)")
    p.add_argument("--gas-scheme", type=int, default=None, choices=[0, 1],
                   help="gas targets: 0 null-collision test (default), 1 the sequential scheme every n1 steps")
    p.add_argument("--no-autotune", action="store_true",
                   help="keep the workload's sort interval and the push grid's blocks per SM "
                        "instead of timing the candidates first")
    p.add_argument("--clocks-dir", default=None,
                   help="keep the raw nvidia-smi clock samples of the timed region in this directory")
    p.add_argument("--no-variants", action="store_true",
                   help="skip the FP64, batched-sweep, Coulomb and sequential-gas figures beside the main one")
    return p.parse_args()


def _workload(name, rank=0, fp64=False, scale=1.0):
    d = inputs.WORKLOADS[name](seed=1 + rank)
    if fp64:
        d.fp64 = True
    if scale != 1.0:
        # fewer superparticles of larger weight: the plasma density is unchanged
        d.n_op = max(2, int(d.n_op * scale) & ~1)
    return d


def _describe(d):
    return (f"{d.L * 100:g} cm gap, {d.n_cells} cells, O2 {d.p_Pa:g} Pa / {d.T_gas:g} K, "
            f"{d.U_rf:g} V at {d.f_rf / 1e6:g} MHz, dt = T_rf/{d.steps_per_cycle}, "
            f"{sum(d.n_init):.3g} superparticles (e {d.n_init[0]}, O- {d.n_init[1]}, "
            f"O2+ {d.n_init[2]}) at {d.n0_m3:g} m^-3, {'FP64' if d.fp64 else 'FP32 mixed'}")


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _traffic(push_slots_per_launch, shape):
    """DRAM bytes per push launch from a committed ncu capture, scaled by the
    slots a launch processes; null when the kernel source changed since the
    capture or the launch shape (threads, slots per thread, blocks per SM)
    differs from the captured one."""
    path = os.path.join(ROOT, "profiles", "k_push_traffic.json")
    src = os.path.join(ROOT, "paper_0705_0495_gb300", "csrc", "o2pic_push.cu")
    try:
        with open(path) as f:
            rec = json.load(f)
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if rec.get("source_sha256") != sha or list(rec.get("launch_shape", [])) != list(shape):
            return None
        return rec["dram_bytes_per_slot"] * push_slots_per_launch
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    out_dir = None  # where the raw samples go (default: the system's temporary directory)

    def __init__(self, index):
        import tempfile
        self.index = index
        self.proc = None
        self.out = os.path.join(Clocks.out_dir or tempfile.gettempdir(), f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.out), exist_ok=True)
            self.f = open(self.out, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.out):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            if self.index is not None and parts[0] != str(self.index):
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        items = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(items) and items[local_rank].isdigit():
            return int(items[local_rank])
        return None
    return local_rank


class OracleSample:
    """The FP64 oracle on a bounded sample of the workload: the same gap,
    grid, drive, gas and tables with the superparticles scaled down to about
    `target` (same plasma density), loaded once; each call advances `steps`
    time steps and returns (particle-steps, seconds)."""

    def __init__(self, name, target=5_000_000, steps=10, seed_offset=0):
        import oracle
        oracle.build()
        d = _workload(name, rank=seed_offset)
        total = sum(d.n_init)
        if total > target:
            d = _workload(name, scale=target / total)
        self.d = d
        self.steps = steps
        self.o = oracle.Oracle(d, inputs.xs_tables())
        self.text = (f"{name} discharge with {sum(d.n_init):.3g} superparticles (same plasma "
                     f"density), {steps} time steps per sample, 1 thread")

    def run(self):
        p0 = self.o.particle_steps
        t0 = time.perf_counter()
        self.o.step(self.steps)
        dt = time.perf_counter() - t0
        return self.o.particle_steps - p0, dt


def _oracle_worker(args):
    """one host core's share of the parallel CPU baseline: its own sample of
    the workload (another seed), `steps` time steps; (particle-steps, s)"""
    name, target, steps, k = args
    sys.path.insert(0, ROOT)
    smp = OracleSample(name, target=target, steps=steps, seed_offset=k)
    return smp.run()


def cpu_baseline_all_cores(name, target, steps):
    """The oracle on every host core at once: one independent sample per core
    (a spawned pool), the throughput summed over the cores and divided by
    the slowest core's time.  Returns (value, cores, text)."""
    import multiprocessing
    cores = os.cpu_count() or 1
    with multiprocessing.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(name, target, steps, k) for k in range(cores)])
    ps = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    return ps / dt, cores, (f"{cores} independent samples in parallel, one per host core, each a "
                            f"{name} discharge with about {target:.3g} superparticles (same plasma "
                            f"density, its own seed), {steps} time steps")


_REF = None


def _ref_init(name, target, steps, counter):
    """a reference-arm worker: its own sample of the workload (its own seed)"""
    global _REF
    sys.path.insert(0, ROOT)
    with counter.get_lock():
        k = counter.value
        counter.value += 1
    _REF = OracleSample(name, target=target, steps=steps, seed_offset=k)


def _ref_step(_):
    return _REF.run()


def run_reference(a, rank, world):
    """The reference arm: the FP64 oracle (the paper publishes no code) on the
    host cores, one independent bounded sample of the workload per core; a
    step advances every core's sample by 10 time steps, and the value is the
    particle-steps of all cores over the wall time."""
    if rank != 0:
        return
    import multiprocessing
    d = _workload(a.workload, scale=a.scale)
    cores = os.cpu_count() or 1
    target = min(2_000_000, sum(d.n_init))
    ctx = multiprocessing.get_context("spawn")
    counter = ctx.Value("i", 0)
    total_ps, total_t = 0, 0.0
    with ctx.Pool(cores, initializer=_ref_init, initargs=(a.workload, target, 10, counter)) as pool:
        for k in range(a.warmup + a.steps):
            t0 = time.perf_counter()
            res = pool.map(_ref_step, range(cores), chunksize=1)
            dt = time.perf_counter() - t0
            if k >= a.warmup:
                total_ps += sum(r[0] for r in res)
                total_t += dt
    value = total_ps / total_t
    text = (f"{cores} independent samples in parallel, one per host core, each a {a.workload} discharge "
            f"with about {target:.3g} superparticles (same plasma density, its own seed), 10 time "
            f"steps per bench step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * total_t / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{a.workload}: {_describe(d)}", "step": "bounded sample: " + text},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": text},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def reduce_over_ranks(values, ops, device):
    """Combine per-rank numbers: 'max' (the job's time is its slowest rank's)
    or 'sum' (work adds up over ranks).  Without a process group it is the
    identity."""
    import torch
    import torch.distributed as tdist
    out = []
    for v, op in zip(values, ops):
        t = torch.tensor([float(v)], dtype=torch.float64, device=device)
        if tdist.is_available() and tdist.is_initialized():
            tdist.all_reduce(t, op=tdist.ReduceOp.MAX if op == "max" else tdist.ReduceOp.SUM)
        out.append(float(t.item()))
    return out


def measure_variant(name, discharges, warm_steps, timed_steps, numeric_budget=None):
    """Particle-steps/s and the push's HBM fraction of another configuration
    (the FP64 path, the batched sweep), timed with CUDA events like the main
    figure; the state of each is far larger than L2."""
    import torch

    from paper_0705_0495_gb300 import o2pic
    sim = o2pic.Simulation(discharges, inputs.xs_tables(), numeric_budget=numeric_budget)
    try:
        sim.step(warm_steps)
        g0 = [sim.diagnostics(k) for k in range(len(discharges))]
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        sim.step(timed_steps)
        e1.record(sim.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ps = sum(sim.diagnostics(k)["particle_steps"] - g0[k]["particle_steps"] for k in range(len(discharges)))
        # the push's duration per launch, in the library's timing mode
        sim.set_timing(True)
        sim.timing(reset=True)
        sim.kernel_timing("coulomb", reset=True)
        sim.kernel_timing("sequential_gas", reset=True)
        r0 = [sim.diagnostics(k) for k in range(len(discharges))]
        sim.step(min(timed_steps, 200))
        kp = sim.kernel_timing("push")
        tm = sim.timing()
        r1 = [sim.diagnostics(k) for k in range(len(discharges))]
        peak, _ = _peaks()
        launches = max(1, tm["push_launches"])
        # the push of steps without diagnostics, against the method's bytes
        # (24 or 40 B per particle-step, 16 or 32 B per candidate)
        R = 8.0 if discharges[0].fp64 else 4.0
        live = sum(r1[k]["particle_steps"] - r0[k]["particle_steps"] for k in range(len(discharges))) / launches
        cands = sum(r1[k]["candidates"] - r0[k]["candidates"] for k in range(len(discharges))) / launches
        dur = kp["ms"] / 1e3 / max(1, kp["launches"])
        achieved = (live * (8.0 + 4.0 * R) + cands * 4.0 * R) / dur / 1e9 if dur > 0 else 0.0
        out = {"workload": name, "value": ps / (ms / 1e3), "unit": UNIT, "time_steps": timed_steps,
               "warmup_time_steps": warm_steps, "ms_per_time_step": ms / timed_steps,
               "push_hbm_frac": achieved / peak}
        g1 = sim.diagnostics(0)
        if g1["eq1_evaluations"] > 0:
            # Eq. 1 probabilities above 1 (clamped), per evaluation
            out["eq1_clamp_fraction"] = float(g1["violations"][1]) / g1["eq1_evaluations"]
        for kind in ("coulomb", "sequential_gas"):
            kc = sim.kernel_timing(kind)
            if kc["launches"] > 0 and kc["ms"] > 0:
                # the Coulomb pass or the sequential gas scheme: device time per
                # launch and the HBM fraction of its algorithmic bytes
                out[f"{kind}_ms_per_launch"] = kc["ms"] / kc["launches"]
                out[f"{kind}_hbm_frac"] = kc["bytes"] / (kc["ms"] / 1e3) / 1e9 / peak
        return out
    finally:
        sim.close()


def run_ours(a, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_0705_0495_gb300 import build as pbuild
    from paper_0705_0495_gb300 import o2pic

    dist = world > 1
    if dist:
        import torch.distributed as tdist
    torch.cuda.set_device(local_rank)
    if rank == 0:
        pbuild.build()
    if dist:
        tdist.barrier()
    d = _workload(a.workload, rank, a.fp64, a.scale)
    if a.n2 is not None:
        d.n2 = a.n2
    if a.gas_scheme is not None:
        d.gas_scheme = a.gas_scheme
    tabs = inputs.xs_tables()
    tune = None
    if not a.no_autotune:
        # the cell-sort interval: each candidate timed on this discharge
        from paper_0705_0495_gb300 import autotune
        best, ms = autotune.tune_sort_interval(d, tabs)
        d.sort_interval = best
        tune = {"chosen": best, "ms_per_time_step": {str(k): v for k, v in ms.items()}}
    sim = o2pic.Simulation([d], tabs, numeric_budget=1.0 if d.gas_scheme else None)
    push_tune = None
    if not a.no_autotune:
        # the push's launch shape: every (threads per block, slots per thread,
        # blocks per SM) timed on this simulation (results do not depend on it)
        best, pms = autotune.tune_push_shape(sim)
        push_tune = {"threads_per_block": best[0], "slots_per_thread": best[1], "blocks_per_sm": best[2],
                     "ms_per_time_step": pms}
    k_shape, b_shape = sim.launch_shape()
    shape_now = list(sim.launch_shapes()[k_shape][:2]) + [b_shape]
    spc = d.steps_per_cycle
    state_bytes = sum(d.n_init) * (12 + (16 if not d.fp64 else 32))
    flush = state_bytes < 4 * L2_BYTES
    scratch = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda") if flush else None

    def barrier():
        if dist:
            tdist.barrier()
        torch.cuda.synchronize()

    # whole RF cycles from a cycle boundary: each timed step is one replay of
    # the captured cycle graph
    sim.align_to_cycle()
    sim.step(a.warmup * spc)
    # the timed cycles run as the library runs them (one CUDA graph per
    # period of the step schedule); the push's own duration for the roofline
    # is taken afterwards, in the library's per-launch timing mode
    sim.set_timing(False)
    sim.timing(reset=True)
    g0 = sim.diagnostics(0)
    clocks = Clocks(_gpu_index(local_rank))
    clocks.start()
    stream = sim.stream
    total_ms = 0.0
    for k in range(a.steps):
        if flush:
            scratch.fill_(float(k))
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(spc)
        e1.record(stream)
        barrier()
        total_ms += e0.elapsed_time(e1)
    clk = clocks.stop()
    g1 = sim.diagnostics(0)
    launches_timed = sim.timing()["launches"]
    psteps = g1["particle_steps"] - g0["particle_steps"]
    total_ms_max, psteps_all = reduce_over_ranks([total_ms, psteps], ["max", "sum"], "cuda")
    value = psteps_all / (total_ms_max / 1e3)

    # roofline of the dominant kernel (the push): CUDA events around every
    # push launch on the library's stream, over one RF cycle (inputs larger
    # than L2, as above)
    peak, peak_kind = _peaks()
    sim.set_timing(True)
    sim.timing(reset=True)
    r0 = sim.diagnostics(0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(spc)
    e1.record(stream)
    torch.cuda.synchronize()
    cycle_ms_timed = e0.elapsed_time(e1)
    kp = sim.kernel_timing("push")        # the push of steps without diagnostics
    kd = sim.kernel_timing("push_diag")   # the push that also samples them
    tm = sim.timing()
    r1 = sim.diagnostics(0)
    sim.set_timing(False)
    launches = max(1, tm["push_launches"])
    live_per_launch = (r1["particle_steps"] - r0["particle_steps"]) / launches
    cands_per_launch = (r1["candidates"] - r0["candidates"]) / launches
    # algorithmic bytes of a push launch as the method needs them: cell,
    # offset and vx read and written per live particle (24 B in FP32, 40 B in
    # FP64), vy and vz read and written per null-collision candidate (16 or
    # 32 B); and the design's own count (every slot, the electrons' vy and vz
    # read for the energy-binned bound, the candidate list)
    R = 8.0 if d.fp64 else 4.0
    alg = live_per_launch * (8.0 + 4.0 * R) + cands_per_launch * 4.0 * R
    design = tm["push_bytes"] / launches
    dur_s = kp["ms"] / 1e3 / max(1, kp["launches"])
    achieved = alg / dur_s / 1e9 if dur_s > 0 else 0.0
    slots_per_launch = (r1["slots_visited"] - r0["slots_visited"]) / launches
    traffic = _traffic(slots_per_launch, shape_now)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_source": f"{peak_kind} HBM copy bandwidth",
            "kernel": "k_push (FP32, steps without diagnostics: 9 of 10 push launches)",
            "us_per_launch": dur_s * 1e6,
            "bytes_per_particle_step": alg / max(1.0, live_per_launch),
            "bytes_count": "24 B per particle-step (cell, offset, vx read and written) + 16 B per "
                           "null-collision candidate (vy, vz read and written)",
            "design_bytes_per_particle_step": design / max(1.0, live_per_launch),
            "design_frac": design / dur_s / 1e9 / peak if dur_s > 0 else 0.0,
            "diag_push_us_per_launch": 1e3 * kd["ms"] / max(1, kd["launches"]),
            "push_share_of_step_time": tm["push_ms"] / cycle_ms_timed if cycle_ms_timed > 0 else None,
            "launch_shape": {"threads_per_block": shape_now[0], "slots_per_thread": shape_now[1],
                             "blocks_per_sm": shape_now[2]}}

    e2e = None
    if not a.no_e2e:
        sim.set_timing(False)
        host = []
        h2d = 0
        for s in range(3):
            st = sim.get_state(0, s)
            pinned = {}
            for key in ("x", "vx", "vy", "vz"):
                t = torch.from_numpy(np.ascontiguousarray(st[key])).pin_memory()
                pinned[key] = t.numpy()
                h2d += t.numel() * 8
            al = torch.from_numpy(st["alive"].astype(np.int32)).pin_memory()
            pinned["alive"] = al.numpy()
            h2d += al.numel() * 4
            host.append(pinned)
        N = d.n_cells
        d2h = 8 * (3 * (N + 1) + (N + 1) + d.eedf_bins + 2 * d.iedf_bins
                   + d.fm_xbins * d.fm_bins + 40 + 1)
        ps_e2e = 0
        barrier()
        t0 = time.perf_counter()
        for k in range(a.steps):
            for s in range(3):
                h = host[s]
                sim.set_state(0, s, h["x"], h["vx"], h["vy"], h["vz"], h["alive"])
            gd0 = sim.diagnostics(0)
            sim.step(spc)
            gd1 = sim.diagnostics(0)
            ps_e2e += gd1["particle_steps"] - gd0["particle_steps"]
        barrier()
        te = time.perf_counter() - t0
        te_max, ps_e2e_all = reduce_over_ranks([te, ps_e2e], ["max", "sum"], "cuda")
        e2e = {"value": ps_e2e_all / te_max, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "path": "pic_set_state from pinned host arrays + pic_step(one RF cycle) + "
                       "pic_diagnostics read back, per step"}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        try:
            target = min(2_000_000, sum(d.n_init))
            val, cores, text = cpu_baseline_all_cores(a.workload, target, 30)
            cpu = {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": text,
                   "host_cores": os.cpu_count()}
        except Exception as ex:  # the baseline is reported, not required
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"failed: {ex}"}

    variants = None
    # the error against the FP64 oracle of each variant, with the tests that
    # establish it (FP32 replay: each step from the oracle's state within
    # 1e-5, at most 1e-4 of particle-steps with a flipped decision)
    REPLAY = "FP32 replay within 1e-5"
    accuracy = {
        "fp64": "step by step within 1e-9 of the gap and of the thermal speed, identical event counts "
                "(tests/test_gpu_parity.py); seed ensembles over 60 and over 1000 RF cycles within 3 standard "
                "errors (tests/test_gpu_long_horizon.py, tests/test_gpu_cfg5_long_horizon.py)",
        "batched": "each discharge of a batched handle equals its own oracle step by step within 1e-9 "
                   "(FP64, uneven discharges, tests/test_gpu_parity.py); the FP32 kernels are those of "
                   f"the single discharge ({REPLAY})",
        "coulomb": "FP64 step by step within 1e-9 (n2 = 1 and 3, ragged and oversized cells); "
                   f"{REPLAY}, one full-size step of this workload compared per cell; seed ensembles "
                   "within 3 standard errors (tests/test_gpu_parity.py, test_gpu_statistics.py)",
        "coulomb_inter": "FP64 step by step within 1e-9 (empty, single and oversized cells); "
                         f"{REPLAY}; seed ensembles within 3 standard errors "
                         "(tests/test_gpu_parity.py, test_gpu_statistics.py)",
        "sweep_13p8": "the seven discharges in one handle each equal their own oracle step by step "
                      "within 1e-9 (FP64, tests/test_gpu_parity.py)",
        "ion_subcycle": f"FP64 step by step within 1e-9 for k = 2 and 5; {REPLAY} (tests/test_gpu_parity.py)",
        "sequential_gas": "FP64 step by step within 1e-9 (chains (15) -> (16)/(17), frequent "
                          f"particle-target events); {REPLAY}, one full-size step of this workload "
                          "included; seed ensembles within 3 standard errors "
                          "(tests/test_gpu_parity.py, test_gpu_statistics.py)",
    }
    if rank == 0 and world == 1 and not a.no_variants:
        sim.close()
        sim = None
        variants = {}
        try:
            d64 = _workload(a.workload, fp64=True, scale=a.scale)
            variants["fp64"] = measure_variant(f"{a.workload} in FP64: {_describe(d64)}", [d64], 200, 400)
        except Exception as ex:
            variants["fp64"] = {"error": str(ex)}
        try:
            sweep = inputs.cfg3_sweep()
            variants["batched"] = measure_variant(
                "cfg3: 64 discharges (100-600 V x 5-50 Pa, 2.5-4 cm, 256/512 cells, 1e4-2e6 superparticles "
                f"each, {sum(sum(x.n_init) for x in sweep):.3g} total), FP32 mixed, one launch per kernel "
                "for all discharges", sweep, 200, sweep[0].steps_per_cycle)
        except Exception as ex:
            variants["batched"] = {"error": str(ex)}
        try:
            dc = _workload(a.workload, scale=a.scale)
            dc.n2 = dc.n1 if dc.n1 > 0 else 10
            variants["coulomb"] = measure_variant(
                f"{a.workload} with intra-species Coulomb collisions (1)-(3) every {dc.n2} steps "
                f"(ln Gamma {dc.coulomb_log:g}): {_describe(dc)}", [dc], 200, 400)
        except Exception as ex:
            variants["coulomb"] = {"error": str(ex)}
        try:
            dc = _workload(a.workload, scale=a.scale)
            dc.n2 = dc.n1 if dc.n1 > 0 else 10
            dc.coulomb_inter = True
            variants["coulomb_inter"] = measure_variant(
                f"{a.workload} with intra- and inter-species Coulomb collisions every {dc.n2} steps "
                f"(the Coulomb figures cover both passes): {_describe(dc)}", [dc], 200, 400)
        except Exception as ex:
            variants["coulomb_inter"] = {"error": str(ex)}
        try:
            sw = inputs.sweep_13p8()
            variants["sweep_13p8"] = measure_variant(
                "the 13.8 Pa sweep of Sec. IV: 7 discharges (2.5 cm, 128 cells, 75-300 V with C = 1/6, "
                "150 V with C = 0), 2e4 O2+ + 2e4 e/O- superparticles each at load, Coulomb every 10 "
                "steps, FP32 mixed, one launch per kernel for all", sw, 200, 2000)
        except Exception as ex:
            variants["sweep_13p8"] = {"error": str(ex)}
        try:
            dk = _workload(a.workload, scale=a.scale)
            dk.ion_subcycle = 5
            variants["ion_subcycle"] = measure_variant(
                f"{a.workload} with O- and O2+ pushed every {dk.ion_subcycle} steps over {dk.ion_subcycle} dt "
                f"(a throughput variant, not in the paper; value counts pushed particles, compare "
                f"ms_per_time_step): {_describe(dk)}", [dk], 200, 400)
        except Exception as ex:
            variants["ion_subcycle"] = {"error": str(ex)}
        try:
            dq = _workload(a.workload, scale=a.scale)
            dq.gas_scheme = 1
            variants["sequential_gas"] = measure_variant(
                f"{a.workload} with the sequential gas scheme (Table I in order every {dq.n1} steps, Eq. 1 "
                f"per channel) instead of the null-collision test: {_describe(dq)}", [dq], 200, 400,
                numeric_budget=1.0)
        except Exception as ex:
            variants["sequential_gas"] = {"error": str(ex)}
        for k, v in variants.items():
            if "error" not in v:
                v["accuracy"] = accuracy[k]

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms_max / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if d.fp64 else "f32",
            "data": "synthetic",
            "config": {
                "workload": f"{a.workload}: {_describe(d)}",
                "step": f"one RF cycle = {spc} time steps (sort and pair pass every "
                        f"{d.sort_interval or d.n1}/{d.n1} steps, diagnostics every {d.diag_every}"
                        + (f", Coulomb collisions every {d.n2}" if d.n2 > 0 else "")
                        + (", sequential gas scheme instead of the null-collision test" if d.gas_scheme else "")
                        + ")",
                "precision": ("FP64 throughout" if d.fp64 else
                              "FP32 particles, push and collisions; exact fixed-point charge "
                              "accumulation; FP64 Poisson, field and diagnostics"),
                # error against the FP64 oracle, as the parity tests establish it
                "accuracy": ("FP64 path: step by step within 1e-9 of the gap and of the thermal "
                             "speed with identical event counts; FP32 path: each step from the "
                             "oracle's state within 1e-5, at most 1e-4 of particle-steps with a "
                             "flipped decision (one full-size step of this workload included); "
                             "time-averaged densities, potential, EEDF and IEDF of FP32 and FP64 "
                             "seed ensembles within 3 standard errors of the oracle's "
                             "(tests/test_gpu_parity.py, test_gpu_statistics.py, "
                             "test_gpu_long_horizon.py, test_gpu_cfg5_long_horizon.py)"),
                "l2": ("inputs larger than L2: the particle state touched per time step "
                       f"({state_bytes / 1e6:.0f} MB) exceeds the 129 MB L2"
                       if not flush else "L2 flushed between timed iterations"),
                "parallelism": f"{world} GPU(s), one independent discharge per GPU",
                # the four tuned knobs: sort interval, threads per block, slots
                # per thread and blocks per SM of the push
                "autotune": {"sort_interval": d.sort_interval,
                             "push_threads_per_block": shape_now[0],
                             "push_slots_per_thread": shape_now[1],
                             "push_blocks_per_sm": shape_now[2],
                             "sort_interval_ms_per_time_step": (tune or {}).get("ms_per_time_step"),
                             "push_shape_ms_per_time_step": (push_tune or {}).get("ms_per_time_step")},
            },
            "roofline": roof,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clk,
            "gpu_launches": launches_timed,
            # one RF cycle is one CUDA graph: graph launches per bench step
            "cuda_graph": {"time_steps_per_graph": g1["graph_cycle_steps"],
                           "graph_launches_per_step": (g1["graph_launch_calls"] - g0["graph_launch_calls"]) / a.steps},
        }
        if variants:
            # the variants' workloads and accuracy first, their figures last
            # (FP64 and the batched sweep at the very end of the line)
            order = ["coulomb", "coulomb_inter", "sweep_13p8", "ion_subcycle", "sequential_gas", "batched", "fp64"]
            line["variant_workloads"] = {k: {"workload": v.get("workload"), "accuracy": v.get("accuracy")}
                                         for k, v in variants.items() if "error" not in v}
            keep = ("value", "ms_per_time_step", "push_hbm_frac", "coulomb_ms_per_launch", "coulomb_hbm_frac",
                    "sequential_gas_ms_per_launch", "sequential_gas_hbm_frac", "eq1_clamp_fraction", "error")
            line["variants"] = {k: {f: variants[k][f] for f in keep if f in variants[k]}
                                for k in order if k in variants}
        print(json.dumps(line), flush=True)
    if sim is not None:
        sim.close()


def main():
    a = _args()
    Clocks.out_dir = a.clocks_dir
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        if world > 1 and rank != 0:
            return
        run_reference(a, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
    try:
        run_ours(a, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as tdist
            tdist.destroy_process_group()


if __name__ == "__main__":
    main()
