"""Throughput of the PIC step (gather + push + MCC + deposit + field solve)
on the synthetic workload "mirror_128x512_1e7": 128 x 512 cells, 1e7
macro-electrons (FP32 particle path, FP64 field), mirror field B0 = 0.3 T,
-20 kV coaxial bias, 1e-5 mbar, cell sort every 20 steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload mirror_128x512_1e7 | scan_64x256_64sims]

``--workload scan_64x256_64sims`` times the parametric scan instead: 64
simulations of 64 x 256 cells (pressure x voltage x mirror field, 1e5 to 5e6
macro-electrons each, 8.15e7 in all) stepped as one batch.
``--workload unet_warmstart_128x512`` measures the learned field-solve warm
start: snapshots from 64 randomised simulations of the small workload's
physics on 128 x 512 cells, the U-Net's training throughput (TFLOP/s on the
BF16 tensor cores; K timed training steps after W warm-up steps), then the
trained net inside the loop against the previous-potential initial guess.
``--workload mirror_128x512_1e7_tables`` is the benchmark step with
tabulated cross sections (synthetic tables of 64 points: elastic,
ionisation and an energy-dependent anisotropy) instead of the analytic fits.
``--workload fluid_moments_128x512_1e7`` times the fluid-moment pass
(pic_moments_accumulate: twelve node moments of the 1e7 electrons after the
warm-up steps, accumulated on the GPU) in particles/s.
``--workload time_to_steady_64sims`` measures the wall time to steady state
of the 64-simulation scan at up-scaled pressure with a seed source, in the
batched FP32 form and in the plain FP64 form (one simulation after another,
cold-started solves); --steps is the step cap per simulation.

Prints one JSON line.  ``value`` is particle-steps/s with the particles
resident in HBM; ``e2e`` is the same metric through the C ABI from host
buffers (load from pinned host memory, K steps, diagnostics with the
density grid back to the host, all inside the timed region).  The
particle store (1e7 x 28 B read + 24 B written per step) exceeds the 129 MB
L2, so no flush is needed between steps.  ``--impl reference`` times the
CPU oracle on a bounded sample of the same workload.  Under torchrun each
rank runs an independent replica (weak scaling, no collective on the data
path); rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2206_14662_gb300.inputs import (cross_section_tables, scan_configs,  # noqa: E402
                                           seed_particles, workload)

WORKLOAD = "mirror_128x512_1e7"
LARGE = "mirror_256x1024_2e8"
SCAN = "scan_64x256_64sims"
UNET = "unet_warmstart_128x512"
STEADY = "time_to_steady_64sims"
TABLES = "mirror_128x512_1e7_tables"
SPLINE = "mirror_128x512_1e7_spline2"
TRAP = "trap_36x92_2e6"
ELLIPSE = (81e-3, 12e-3, 3e-3, 14e-3)


def trap_config(**kw):
    """The trap of Sec. II.B on a 36 x 92 grid: inner conductor 63.75 mm,
    outer cylinder 81 mm, z from -10 to 34 mm, the metal ellipse centred on
    the outer cylinder at z = 12 mm (semi-axes 3 mm in r, 14 mm in z),
    -30 kV bias, a uniform 0.28 T field (the paper's field map is not
    available), 0.1 mbar, degree-2 web splines."""
    base = dict(r_in=63.75e-3, r_out=81e-3, z_min=-10e-3, z_max=34e-3, nr=36, nz=92,
                v_inner=-30e3, v_outer=0.0, bfield_kind=0, b0=0.28, p_mbar=0.1,
                bspline_degree=2, ellipse=ELLIPSE, n_init=2_000_000, sort_every=20,
                source_rate=0.0)
    base.update(kw)
    return workload(WORKLOAD, **base)


def outside_ellipse(parts):
    r, z = parts[0], parts[1]
    keep = ((r - ELLIPSE[0]) / ELLIPSE[2]) ** 2 + ((z - ELLIPSE[1]) / ELLIPSE[3]) ** 2 > 1.0
    return [a[keep] for a in parts]
MOMENTS = "fluid_moments_128x512_1e7"
# algorithmic bytes per particle of the moment pass: cell 4 + offsets 8 +
# velocity 12 read (the node grids stay in L2)
BYTES_PER_PARTICLE_MOMENTS = 24
FALLBACK_BF16_TFLOPS = 1900.0
METRIC = "particle-steps/s (gather+push+MCC+deposit+field solve)"
# algorithmic bytes per particle-step of the fused particle kernel (FP32):
# read cell 4 + offsets 8 + velocity 12 + uid 4, write cell + offsets +
# velocity 24
BYTES_PER_PARTICLE_STEP = 52
FALLBACK_HBM_GBS = 6800.0


def graph_len(sort_every: int) -> int:
    """Steps per captured CUDA graph of pic_step for a sort period: lcm of
    the period and 2 (the two deposit buffers), doubled up to at least 8."""
    n = sort_every if sort_every % 2 == 0 else 2 * sort_every
    while n < 8:
        n *= 2
    return n


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def _peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for k in ("hbm_gbs", "hbm_GBps", "hbm"):
            if k in d:
                return float(d[k]), "measured"
    except Exception:
        pass
    return FALLBACK_HBM_GBS, "fallback"


def _peak_bf16():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for k in ("bf16_tflops", "bf16_TFLOPs", "bf16"):
            if k in d:
                return float(d[k]), "measured"
    except Exception:
        pass
    return FALLBACK_BF16_TFLOPS, "fallback"


def particle_kernel_sha() -> str:
    """SHA-256 over the sources the fused particle kernel is compiled from."""
    h = hashlib.sha256()
    for name in ("particle_step.cu", "pic_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2206_14662_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _traffic_record():
    """DRAM bytes per launch of the fused kernel from the committed ncu
    summary, valid only while the kernel source (particle_step.cu and the
    header it includes) is unchanged."""
    try:
        with open(os.path.join(ROOT, "profiles", "particle_step_traffic.json")) as f:
            rec = json.load(f)
        if rec.get("source_sha256") == particle_kernel_sha():
            return rec
    except Exception:
        pass
    return None


class Clocks:
    """nvidia-smi samples (every 100 ms) during the timed region; start()
    waits until the sampler has written its first line."""

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        dev = os.environ.get("LOCAL_RANK", "0")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", dev,
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 10 and os.path.getsize(self.path) == 0:
            time.sleep(0.05)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0])); mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def combine_ranks(sec, units, esec, e2e_units, device):
    """Whole-job figures of independent replicas: the slowest rank's times
    and the sum of the units every rank processed (collective on the
    default process group)."""
    import torch
    t = torch.tensor([sec, units, esec, e2e_units], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t[0:1], op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(t[2:3], op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(t[1:2])
    torch.distributed.all_reduce(t[3:4])
    return tuple(t.tolist())


def _inputs(args, rank):
    """(workload name, configurations, seeded particle arrays per
    simulation) of the run."""
    over = {} if args.warm_start is None else {"warm_start": args.warm_start}
    if args.workload == SCAN:
        cfgs = scan_configs(seed=1 + rank, **over)
        parts = [seed_particles(c, seed=1000 * (rank + 1) + k) for k, c in enumerate(cfgs)]
        return SCAN, cfgs, parts
    if args.workload == TRAP:
        cfg = trap_config(seed=1 + rank, **over)
        if args.particles:
            cfg["n_init"] = args.particles
        return TRAP, [cfg], [outside_ellipse(seed_particles(cfg))]
    name = LARGE if args.workload == LARGE else WORKLOAD
    cfg = workload(name, seed=1 + rank, **over)
    if args.particles:
        cfg["n_init"] = args.particles
    if args.workload == TABLES:
        E, sel, sio, xi = cross_section_tables(cfg["ion_E_th_eV"])
        cfg["xs"] = dict(E_eV=E, sigma_el=sel, sigma_io=sio, xi=xi)
        name = TABLES
    if args.workload == SPLINE:   # the weighted B-spline field of degree 2
        cfg["bspline_degree"] = 2
        name = SPLINE
    return name, [cfg], [seed_particles(cfg)]


def run_ours(args, ws, rank):
    import torch
    from paper_2206_14662_gb300._capi import Simulation

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    name, cfgs, parts = _inputs(args, rank)
    S = len(cfgs)
    n0 = sum(len(p[0]) for p in parts)
    pinned = []
    for p in parts:
        q = [torch.from_numpy(a).pin_memory() for a in p[:5]]
        q.append(torch.from_numpy(p[5].view(np.int64)).pin_memory())
        pinned.append(q)

    def pushed(sim):
        ds = [sim.diagnostics(sim=k) for k in range(S)]
        return sum(d["n_pushed"] for d in ds), ds[0]

    sim = Simulation(cfgs if S > 1 else cfgs[0])
    for k in range(S):
        sim.load_particles(*pinned[k], sim=k)
        xs = cfgs[k].get("xs")
        if xs is not None:   # tables stay with the simulation across loads
            sim.set_cross_sections(xs["E_eV"], xs["sigma_el"], xs["sigma_io"], xs["xi"], sim=k)
    sim.step(args.warmup)
    tune = None
    if args.autotune:
        # schedule, untimed: the sort periods that divide the timed step
        # count, so that the timed steps hold whole sort periods
        periods = [p for p in (5, 10, 20, 40, 80) if args.steps % graph_len(p) == 0]
        tune = sim.autotune(80, periods=periods or None)
    # start the timed region on a graph block (the steps are then replayed
    # graphs), after capturing the schedule's graphs untimed
    se = tune["sort_every"] if tune else cfgs[0]["sort_every"]
    gl = graph_len(se)
    at = sim.diagnostics()["step"]
    sim.step((gl - at % gl) % gl + 2 * gl)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()

    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks()
    u0, d0 = pushed(sim)
    clocks.start()
    torch.cuda.synchronize()
    ev0.record(stream)
    sim.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    u1, d1 = pushed(sim)
    ms = ev0.elapsed_time(ev1)
    units = u1 - u0
    launches = d1["kernels_launched"] - d0["kernels_launched"]

    # per-stage device time: the same workload continued with an event
    # between stages (kernels launched one by one while profiling)
    prof_steps = min(args.steps, 200)
    sim.profile_start()
    sim.step(prof_steps)
    prof = sim.profile_stop()
    u2, d2 = pushed(sim)
    prof_units = u2 - u1

    # end to end through the C ABI from host buffers
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_units = 0
    if args.e2e:
        for k in range(S):
            sim.load_particles(*pinned[k], sim=k)
        sim.step(args.steps)
        # the spline fields have no node deposit: their result is the
        # diagnostics record alone
        dens = name not in (SPLINE, TRAP)
        for k in range(S):   # a load resets the simulation's counters
            e2e_units += sim.diagnostics(density=dens, sim=k)["n_pushed"]
    t1 = time.perf_counter()
    sim.close()

    if ws > 1:
        sec, units, esec, e2e_units = combine_ranks(ms / 1e3, units, t1 - t0, e2e_units, "cuda")
    else:
        sec, esec = ms / 1e3, t1 - t0

    if rank != 0:
        return None
    value = units / sec
    peak, src = _peak_hbm()
    kern_ms = prof["particle_ms"] / max(1, prof["particle_launches"])
    per_launch_units = prof_units / max(1, prof["particle_launches"])
    achieved = BYTES_PER_PARTICLE_STEP * per_launch_units / (kern_ms * 1e-3) / 1e9
    traffic = _traffic_record() if S == 1 and name not in (TABLES, SPLINE, TRAP) else None
    cfg = cfgs[0]
    grid = f"{cfg['nr']}x{cfg['nz']}"
    nnodes = (cfg["nr"] + 1) * (cfg["nz"] + 1)
    live = int(round(units / args.steps))   # live particles per timed step
    if S == 1:
        config = {"workload": name if not args.particles else f"{name} (particles={n0})",
                  "particles": live, "particles_loaded": n0, "grid": grid,
                  "sort_every": tune["sort_every"] if tune else cfg["sort_every"],
                  "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                  "l2": f"inputs larger than L2 (particle store {live * 52 / 1e9:.2f} GB per step)"}
    else:
        config = {"workload": name, "simulations": S, "particles": live, "particles_loaded": n0,
                  "particles_min_max": [min(len(p[0]) for p in parts),
                                        max(len(p[0]) for p in parts)],
                  "grid": f"{S} x {grid}",
                  "sort_every": tune["sort_every"] if tune else cfg["sort_every"],
                  "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU, one batch",
                  "l2": f"inputs larger than L2 (particle store {n0 * 52 / 1e9:.1f} GB per step)"}
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "particle-steps/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": sec * 1e3 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 particles / f64 field",
        "data": "synthetic (seeded volume-uniform 1 eV Maxwellian load)" + (
            "; synthetic 64-point cross-section tables" if name == TABLES else ""),
        "config": config,
        "e2e": None if not args.e2e else {"value": e2e_units * ws / esec, "unit": "particle-steps/s",
                "h2d_bytes_per_step": int(n0 * 48 / args.steps),
                "d2h_bytes_per_step": int(S * (nnodes * 8 * (name not in (SPLINE, TRAP)) + 512)
                                          / args.steps)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm",
                     "kernel": ("k_particle_step_batch<float>" if S > 1 else
                                "k_particle_step<float, 1> (tables)" if name == TABLES else
                                "k_particle_step<float, 0, 2> (spline field)" if name == SPLINE else
                                "k_particle_step<float, 0, 2> (trap, web-spline field)" if name == TRAP else
                                "k_particle_step<float, 0>"),
                     "achieved": achieved,
                     "peak": peak, "peak_source": src, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": (traffic["dram_bytes_per_particle"] * per_launch_units) if traffic else None,
                     "traffic_source": (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of "
                                        f"{traffic['workload']}: {traffic['dram_bytes_per_particle']} "
                                        "B per particle-step, times this launch's particles")
                                       if traffic else None,
                     "kernel_ms_per_launch": kern_ms,
                     "bytes_per_particle_step": BYTES_PER_PARTICLE_STEP},
        "stage_ms_per_step": {"particle": prof["particle_ms"] / prof_steps,
                              "finalize": prof["finalize_ms"] / prof_steps,
                              "field": prof["field_ms"] / prof_steps,
                              "sort": prof["sort_ms"] / prof_steps,
                              "steps_profiled": prof_steps,
                              "note": "profiled pass after the timed region, kernels "
                                      "launched one by one"},
        "poisson": {"sweeps": d1["poisson_iters"], "relres": d1["poisson_relres"],
                    "relres_charge": d1["poisson_relres_charge"],
                    "warm_start": cfg.get("warm_start", 0)},
        "clocks": clk,
        "schedule": tune,
    }
    if args.cpu_baseline:
        if S == 1:
            # the oracle on at most 2e7 of the particles (a bounded sample)
            # (the spline oracle evaluates dense basis rows: a small sample)
            cap = 20_000 if name in (SPLINE, TRAP) else 20_000_000
            out["cpu_baseline"] = cpu_baseline(cfg, parts[0], name=name,
                                               n_sample=min(len(parts[0][0]), cap))
        else:
            # the oracle on the largest simulation of the scan, 4 steps
            k = int(np.argmax([len(p[0]) for p in parts]))
            out["cpu_baseline"] = cpu_baseline(cfgs[k], parts[k], steps=4, name=f"{name} (simulation {k})")
    return out


def run_moments(args, ws, rank):
    """The fluid-moment pass (Sec. IV.A): after the warm-up steps of the
    benchmark workload, K calls of pic_moments_accumulate over the resident
    particle store, each adding 1/K of the twelve node moments into one
    device array.  e2e: the exported state loaded from pinned host memory
    and K calls of pic_moments, each returning the grids to the host."""
    import torch
    from paper_2206_14662_gb300._capi import MOMENTS as NMOM
    from paper_2206_14662_gb300._capi import Simulation

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cfg = workload(WORKLOAD, seed=1 + rank)
    if args.particles:
        cfg["n_init"] = args.particles
    parts = seed_particles(cfg)
    shape = (NMOM, cfg["nr"] + 1, cfg["nz"] + 1)
    sim = Simulation(cfg)
    sim.load_particles(*parts)
    sim.step(args.warmup)
    # the walk's speed depends on how far the store has drifted from cell
    # order since the last sort (the store is cell-sorted every sort_every
    # steps; the seeded load itself is in random order)
    se = cfg["sort_every"]
    since_sort = args.warmup % se if args.warmup >= se else None
    n_live = int(sim.diagnostics()["n_particles"])
    acc = torch.zeros(shape, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        sim.moments_accumulate(acc, 1.0)
    acc.zero_()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks()
    clocks.start()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        sim.moments_accumulate(acc, 1.0 / args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    units = n_live * args.steps

    # end to end: the current state, in the simulation's cell order (export
    # returns uid order), from pinned host memory, then K calls returning
    # the moments to the host
    g = sim.export_particles()
    hr = (cfg["r_out"] - cfg["r_in"]) / cfg["nr"]
    hz = (cfg["z_max"] - cfg["z_min"]) / cfg["nz"]
    ir = np.clip(((g["r"] - cfg["r_in"]) / hr).astype(np.int64), 0, cfg["nr"] - 1)
    iz = np.clip(((g["z"] - cfg["z_min"]) / hz).astype(np.int64), 0, cfg["nz"] - 1)
    order = np.argsort(ir * (cfg["nz"] + 1) + iz, kind="stable")
    g = {k: v[order] for k, v in g.items()}
    host = [torch.from_numpy(np.ascontiguousarray(g[k])).pin_memory()
            for k in ("r", "z", "vr", "vt", "vz")]
    host.append(torch.from_numpy(np.ascontiguousarray(g["uid"]).view(np.int64)).pin_memory())
    n_e2e = len(g["uid"])
    e2e_units = 0
    esec = 0.0
    if args.e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.load_particles(*host)
        for _ in range(args.steps):
            sim.moments()
            e2e_units += n_e2e
        esec = time.perf_counter() - t0
    sim.close()

    if ws > 1:
        sec, units, esec, e2e_units = combine_ranks(ms / 1e3, units, esec, e2e_units, "cuda")
    else:
        sec = ms / 1e3
    if rank != 0:
        return None
    peak, src = _peak_hbm()
    kern_s = sec / args.steps
    achieved = BYTES_PER_PARTICLE_MOMENTS * n_live / kern_s / 1e9
    nnodes = shape[1] * shape[2]
    out = {
        "metric": "particles/s (fluid moments: n, n u, n <v v>, n <nu_d>, n <nu_io> on the nodes)",
        "value": units / sec, "unit": "particles/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sec * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 particles / f64 moments",
        "data": "synthetic (the benchmark workload after the warm-up steps)",
        "config": {"workload": MOMENTS if not args.particles else f"{MOMENTS} (particles={n_live})",
                   "particles": n_live, "grid": f"{cfg['nr']}x{cfg['nz']}",
                   "steps_since_sort": since_sort,
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": f"inputs larger than L2 (particle store read {n_live * 24 / 1e9:.2f} GB per pass)"},
        "e2e": None if not args.e2e else {
            "value": e2e_units / esec, "unit": "particles/s",
            "h2d_bytes_per_step": int(n_e2e * 48 / args.steps),
            "d2h_bytes_per_step": int(NMOM * nnodes * 8)},
        "gpu_launches": int(args.steps),
        "roofline": {"bound": "hbm", "kernel": "k_moments<float>", "achieved": achieved,
                     "peak": peak, "peak_source": src, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel_ms_per_launch": kern_s * 1e3,
                     "bytes_per_particle": BYTES_PER_PARTICLE_MOMENTS},
        "clocks": clk,
    }
    if args.cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_moments(cfg, g, n_sample=min(n_e2e, 1_000_000))
    return out


def cpu_baseline_moments(cfg, g, n_sample):
    """The oracle's moments (numpy, one thread) of the first n_sample
    particles of the state."""
    import oracle
    from oracle import fluid
    oracle.build()
    w = oracle.derived(cfg)["weight"]
    t0 = time.perf_counter()
    fluid.moments(cfg, *(g[k][:n_sample] for k in ("r", "z", "vr", "vt", "vz")), w)
    sec = time.perf_counter() - t0
    return {"value": n_sample / sec, "unit": "particles/s", "cores": 1, "kind": "oracle",
            "sample": f"moments of {n_sample} particles of {MOMENTS}", "seconds": sec}


def run_unet(args, ws, rank):
    """Training throughput of the warm-start U-Net and its effect in the
    loop (rank 0; other ranks exit)."""
    if rank != 0:
        return None
    import torch
    from paper_2206_14662_gb300 import warmstart
    from paper_2206_14662_gb300.inputs import unet_init_flat
    from paper_2206_14662_gb300.unet import UNet

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    c, H, W, B = 32, 128, 512, 16
    # 2e4 snapshots: 64 randomised simulations x 313 steps
    cfgs = warmstart.snapshot_configs(64, nr=H, nz=W, n_particles=10_000, seed=1)
    rho, phi, dphi = warmstart.collect(cfgs, steps=313, warmup=20)
    sc = warmstart.scales(rho, phi, dphi)
    net = UNet(c, H, W, B, precision=16)
    net.set_params(unet_init_flat(c, seed=3).astype(np.float32))
    # fixed mini-batches for the timed steps
    nb = 8
    xs = torch.empty((nb, B, H, W, 2), dtype=torch.float32, device="cuda")
    ts = torch.empty((nb, B, H, W), dtype=torch.float32, device="cuda")
    for i in range(nb):
        sl = slice(i * B, (i + 1) * B)
        xs[i, ..., 0] = rho[sl] / sc[0]
        xs[i, ..., 1] = phi[sl] / sc[1]
        ts[i] = dphi[sl] / sc[2]
    for i in range(args.warmup):
        net.train_step(xs[i % nb], ts[i % nb], lr=1e-3)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks()
    clocks.start()
    ev0.record()
    for i in range(args.steps):
        net.train_step(xs[i % nb], ts[i % nb], lr=1e-3)
    ev1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    tflops = warmstart.train_step_flops(c, H, W, B) / (ms * 1e-3) / 1e12
    # inference forward alone (batch 1, the in-loop size)
    inf = UNet(c, H, W, 1, precision=16)
    x1 = xs[0, :1].contiguous()
    for _ in range(5):
        inf.forward(x1)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(50):
        inf.forward(x1)
    ev1.record()
    torch.cuda.synchronize()
    fwd_ms = ev0.elapsed_time(ev1) / 50
    # train on all snapshots, then the A/B inside the loop
    net.set_params(unet_init_flat(c, seed=3).astype(np.float32))
    losses, base = warmstart.train(net, rho, phi, dphi, sc, epochs=2, lr=1e-3)
    losses, base = losses.cpu().numpy(), base.cpu().numpy()
    inf.set_params(net.get_params())
    ab = {}
    for n_part in (10_000, 1_000_000):
        cfg = warmstart.snapshot_configs(1, nr=H, nz=W, n_particles=n_part, seed=77)[0]
        t0 = time.perf_counter()
        prv = warmstart.evaluate(cfg, 50, warmup=20)
        t1 = time.perf_counter()
        lrn = warmstart.evaluate(cfg, 50, inf, sc, warmup=20)
        t2 = time.perf_counter()
        ab[f"particles_{n_part}"] = {
            "relres_init_median": {"previous": float(np.median(prv["relres_init"])),
                                   "learned": float(np.median(lrn["relres_init"]))},
            "sweeps_mean": {"previous": float(prv["sweeps"].mean()),
                            "learned": float(lrn["sweeps"].mean())},
            "relres_max": {"previous": float(prv["relres"].max()),
                           "learned": float(lrn["relres"].max())},
            "wall_s_70_steps": {"previous": t1 - t0, "learned": t2 - t1}}
    net.close()
    inf.close()
    peak, src = _peak_bf16()
    return {
        "metric": "U-Net training throughput (forward + data and weight gradients + Adam)",
        "value": tflops, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 (fp32 accumulation and master weights)",
        "data": "synthetic (snapshots of seeded simulations)",
        "config": {"workload": UNET, "base_channels": c, "grid": f"{H}x{W}", "batch": B,
                   "snapshots": int(rho.shape[0]),
                   "flop_per_step": warmstart.train_step_flops(c, H, W, B),
                   "l2": "activations and gradients of a batch exceed L2"},
        "e2e": None, "gpu_launches": None,
        "roofline": {"bound": "tensor",
                     "kernel": "k_conv3_tc (tcgen05) / k_gemm_fwd / k_gemm_wgrad (mma.sync) bf16",
                     "achieved": tflops, "peak": peak, "peak_source": src, "unit": "TFLOP/s",
                     "frac": tflops / peak, "traffic": None},
        "inference_forward_ms": fwd_ms,
        "inference_tflops": warmstart.forward_flops(c, H, W) / (fwd_ms * 1e-3) / 1e12,
        "training": {"epochs": 2, "loss_over_no_change_last64":
                     float(losses[-64:].mean() / base[-64:].mean())},
        "warm_start_ab": ab,
        "clocks": clk,
    }


def steady_configs():
    """The scan's 4 x 4 x 4 grid of voltage and field with the pressures
    scaled up to 1e-2 .. 1e-1 mbar (collision times of 30 to 700 steps),
    2e3 to 1e5 macro-electrons per simulation, room for 40 times the load,
    and a seed source of 1% of the initial load per collision time."""
    cfgs = scan_configs(n_sims=64, n_min=2_000, n_max=100_000)
    P = (1e-2, 2.15e-2, 4.64e-2, 1e-1)
    for k, c in enumerate(cfgs):
        c["p_mbar"] = P[(k // 16) % 4]
        c["capacity"] = 40 * c["n_init"] + 4096
    return cfgs


def run_steady(args, ws, rank):
    if rank != 0:
        return None
    import torch
    from paper_2206_14662_gb300 import steady
    from paper_2206_14662_gb300._capi import Simulation
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cfgs = steady_configs()
    with Simulation(cfgs) as sim:
        nus = [sim.diagnostics(sim=k)["nu_max"] for k in range(len(cfgs))]
    for c, nu in zip(cfgs, nus):
        c["source_rate"] = 0.01 * c["n_init"] * nu
    # the learned form's net: base width 8 (the scan's 64 x 256 grids), trained
    # on snapshots of the same 64 simulations (100 steps each after 20), not
    # counted in the time to steady
    from paper_2206_14662_gb300 import warmstart
    from paper_2206_14662_gb300.inputs import unet_init_flat
    from paper_2206_14662_gb300.unet import UNet
    t0 = time.perf_counter()
    nr, nz = cfgs[0]["nr"], cfgs[0]["nz"]
    rho, phi, dphi = warmstart.collect(cfgs, steps=100, warmup=20)
    sc = warmstart.scales(rho, phi, dphi)
    trainer = UNet(8, nr, nz, 16, precision=16)
    trainer.set_params(unet_init_flat(8, seed=5).astype(np.float32))
    losses, base = warmstart.train(trainer, rho, phi, dphi, sc, epochs=4, lr=1e-3)
    loss_ratio = float(losses[-64:].mean().item() / base[-64:].mean().item())
    net = UNet(8, nr, nz, len(cfgs), precision=16)
    net.set_params(trainer.get_params())
    trainer.close()
    del rho, phi, dphi
    train_s = time.perf_counter() - t0
    res = {}
    for form in ("batched", "learned", "plain"):
        stats = {}
        sec, st, pushed = steady.time_to_steady(cfgs, form, cap_steps=args.steps, net=net,
                                                scales=sc, stats=stats)
        done = [x for x in st if x is not None]
        res[form] = {"seconds": sec, "steady": len(done), "of": len(cfgs),
                     "median_steady_step": float(np.median(done)) if done else None,
                     "particle_steps": int(pushed),
                     "particle_steps_per_s": pushed / sec, "field_solve": stats}
    net.close()
    res["learned"]["net"] = {"base_channels": 8, "snapshots": 6400, "epochs": 4,
                             "train_seconds": train_s,
                             "loss_over_no_change_last64": loss_ratio}
    b, p = res["batched"], res["plain"]
    return {
        "metric": "time to steady state, 64-simulation scan (batched FP32 vs plain FP64)",
        "value": b["seconds"], "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": 0,
        "ms_per_step": None, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 particles / f64 field (batched); f64 (plain)",
        "data": "synthetic (seeded loads, seed source)",
        "config": {"workload": STEADY, "simulations": len(cfgs), "grid": "64 x 64x256",
                   "pressures_mbar": [1e-2, 2.15e-2, 4.64e-2, 1e-1],
                   "particles_min_max": [2000, 100000], "cap_steps": args.steps,
                   "detector": "window means of N, n_max, I_outer; two consecutive windows "
                               "within 2%; window max(2000 steps, 5/nu_max)"},
        "forms": res, "speedup": p["seconds"] / b["seconds"],
        "speedup_learned": p["seconds"] / res["learned"]["seconds"],
        "note": "simulations not steady by the cap count with the cap",
    }


def host_cores() -> int:
    """Cores this process may run on (nproc)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(cfg, parts, n_sample=None, steps=2, name=WORKLOAD):
    """The oracle as it stands on a bounded sample: the first n_sample
    particles of the load (all by default) with the full grid and field
    solve, ``steps`` steps, on all host cores (OpenMP over the particles'
    own steps; sums in particle order) and on one core.  The main figure is
    the all-core one; both give bitwise the same states."""
    import oracle
    oracle.build()
    sel = slice(None) if n_sample is None else slice(0, n_sample)
    res = {}
    for cores in (host_cores(), 1):
        oracle.set_threads(cores)
        o = oracle.OracleSim(cfg, *[a[sel] for a in parts])
        t0 = time.perf_counter()
        units = 0
        for _ in range(steps):
            units += o.n
            o.step()
        sec = time.perf_counter() - t0
        res[cores] = (units / sec, sec, oracle.threads())
    oracle.set_threads(host_cores())
    many, one = res[host_cores()], res[1]
    sample = (f"{steps} steps of {len(parts[0][sel])} particles of {name} "
              "(full grid, field solve included)")
    return {"value": many[0], "unit": "particle-steps/s", "cores": many[2], "kind": "oracle",
            "sample": sample, "seconds": many[1], "nproc": host_cores(),
            "single_core": {"value": one[0], "unit": "particle-steps/s", "cores": 1,
                            "seconds": one[1]}}


def run_reference(args, ws, rank):
    """The CPU oracle on a bounded sample of the workload: each step is one
    oracle step of 20 000 particles drawn from it, with the full grid and
    field solve."""
    if rank != 0:
        return None
    if args.workload == UNET:
        return run_reference_unet(args, ws)
    if args.workload == MOMENTS:
        return run_reference_moments(args, ws)
    import oracle
    oracle.build()
    name = args.workload
    # the scan: its largest simulation (the oracle runs one simulation)
    cfg = workload(name) if name in (WORKLOAD, LARGE) else (
        workload(WORKLOAD) if name in (TABLES, SPLINE) else scan_configs()[-1])
    if name == SPLINE:
        cfg["bspline_degree"] = 2
    if name == TRAP:
        cfg = trap_config()
    if name == TABLES:
        E, sel, sio, xi = cross_section_tables(cfg["ion_E_th_eV"])
        cfg["xs"] = dict(E_eV=E, sigma_el=sel, sigma_io=sio, xi=xi)
    # the spline and trap oracles evaluate dense basis rows per particle:
    # a small sample there
    # elsewhere at most 2e7 particle-steps over the whole run, at least
    # 20 000 particles per step
    n = 20_000 if name in (SPLINE, TRAP) else int(
        min(1_000_000, max(20_000, 2e7 // (args.steps + args.warmup))))
    oracle.set_threads(host_cores())
    cores = oracle.threads()
    parts = seed_particles(cfg, n=n)
    if name == TRAP:
        parts = outside_ellipse(parts)
        n = len(parts[0])
    o = oracle.OracleSim(cfg, *parts)
    for _ in range(args.warmup):
        o.step()
    t0 = time.perf_counter()
    units = 0
    for _ in range(args.steps):
        units += o.n
        o.step()
    sec = time.perf_counter() - t0
    v = units / sec
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "particle-steps/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "particles": n, "grid": f"{cfg['nr']}x{cfg['nz']}",
                       "parallelism": "cpu oracle, rank 0 only"},
            "cpu_baseline": {"value": v, "unit": "particle-steps/s", "cores": cores,
                             "kind": "oracle", "nproc": host_cores(),
                             "sample": f"{n} particles of {name} per step, full grid and field "
                                       "solve (OpenMP over the particles' own steps)"},
            "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def run_reference_moments(args, ws):
    """The oracle's moments (numpy) on a bounded sample: each step the
    moments of 200 000 seeded particles of the benchmark workload."""
    import oracle
    from oracle import fluid
    oracle.build()
    cfg = workload(WORKLOAD)
    n = 200_000
    r, z, vr, vt, vz, _ = seed_particles(cfg, n=n)
    w = oracle.derived(cfg)["weight"]
    steps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(steps):
        fluid.moments(cfg, r, z, vr, vt, vz, w)
    sec = time.perf_counter() - t0
    v = n * steps / sec
    return {"impl": "reference", "metric": "particles/s (fluid moments: n, n u, n <v v>, "
            "n <nu_d>, n <nu_io> on the nodes)", "value": v, "unit": "particles/s",
            "n_gpus": ws, "steps": steps, "warmup": 0, "ms_per_step": sec * 1e3 / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": MOMENTS, "particles": n,
                                            "grid": f"{cfg['nr']}x{cfg['nz']}",
                                            "parallelism": "cpu oracle, rank 0 only"},
            "cpu_baseline": {"value": v, "unit": "particles/s", "cores": 1, "kind": "oracle",
                             "sample": f"moments of {n} particles of {MOMENTS} per step"},
            "e2e": {"value": v, "unit": "particles/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def run_reference_unet(args, ws):
    """The FP64 U-Net oracle (numpy) on a bounded sample: forward and
    backward of one 128 x 512 image per step."""
    from oracle import unet as U
    from paper_2206_14662_gb300 import warmstart
    from paper_2206_14662_gb300.inputs import unet_init_flat
    c, H, W = 32, 128, 512
    p = U.unflatten(unet_init_flat(c, seed=3), c)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, H, W, 2))
    steps = max(1, min(args.steps, 2))
    t0 = time.perf_counter()
    for _ in range(steps):
        y, a = U.forward(p, x)
        U.backward(p, a, y / y.size)
    sec = (time.perf_counter() - t0) / steps
    v = warmstart.train_step_flops(c, H, W, 1) / sec / 1e12
    return {"impl": "reference", "metric": "U-Net training throughput (forward + data and "
            "weight gradients + Adam)", "value": v, "unit": "TFLOP/s", "n_gpus": ws,
            "steps": steps, "warmup": 0, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": UNET, "batch": 1, "grid": f"{H}x{W}"},
            "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": f"{steps} forward+backward of one image"},
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--workload", choices=[WORKLOAD, LARGE, SCAN, UNET, STEADY, TABLES, MOMENTS,
                                           SPLINE, TRAP],
                    default=WORKLOAD)
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the workload's sort period and the default kernel grid")
    ap.add_argument("--warm-start", type=int, choices=[0, 1], default=None,
                    help="override the field solve's initial guess (0 zero, 1 previous)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false",
                    help="skip the end-to-end pass (profiling captures)")
    ap.add_argument("--particles", type=int, default=0,
                    help="override the macro-electron count (profiling captures on a "
                         "smaller case; the reported workload is then not the benchmark's)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    ws, rank = _dist()
    if ws > 1 and args.impl == "ours":
        import torch
        torch.distributed.init_process_group("nccl")
        args.cpu_baseline = args.cpu_baseline and rank == 0 and False
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
    elif args.workload == UNET:
        out = run_unet(args, ws, rank)
    elif args.workload == STEADY:
        out = run_steady(args, ws, rank)
    elif args.workload == MOMENTS:
        out = run_moments(args, ws, rank)
    else:
        out = run_ours(args, ws, rank)
    if out is not None:
        print(json.dumps(out), flush=True)
    if ws > 1 and args.impl == "ours":
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
