"""Steady-state detection and the time-to-steady measurement.

Detector: the run is sampled every ``every`` steps (particle count N, peak
density n_max, current into the outer wall I_outer); sample means are taken
over consecutive windows of W steps; the run is steady when the means of two
consecutive complete windows agree within ``tol`` (relative) for every
quantity.  The paper's clouds breathe (Sec. III.A), so only time averages
can settle; W is chosen as max(2000 steps, 5 collision times).

time_to_steady() runs a set of simulations in one of two forms until each is
detected steady (or a step cap): "batched" (one handle stepping every
simulation together, FP32 particles, the field solve warm-started from the
previous potential, CUDA-graph blocks) or "plain" (one handle per
simulation, FP64 particles, cold-started solves, the simulations one after
another), and reports the wall time.
"""
from __future__ import annotations

import time

import numpy as np

from .inputs import seed_particles


class SteadyDetector:
    """Window means of a few quantities; steady when two consecutive
    complete windows agree within tol."""

    def __init__(self, window_steps: int, tol: float = 0.02, keys=("n", "n_max", "i_outer")):
        self.W = int(window_steps)
        self.tol = tol
        self.keys = keys
        self.sums = {}      # window index -> (count, sums)
        self.last = -1      # window of the last sample
        self.steady_step = None

    def add(self, step: int, **vals) -> bool:
        """Record the quantities at `step` (steps counted from the start,
        samples in increasing order); returns True once steady.  Windows
        before the one holding `step` are complete; the first time a sample
        falls in window w >= 2 the means of windows w - 2 and w - 1 are
        compared, and steady_step becomes the end of window w - 1."""
        if self.steady_step is not None:
            return True
        w = (step - 1) // self.W
        if w >= 2 and w != self.last and (w - 2) in self.sums and (w - 1) in self.sums:
            (c1, s1), (c2, s2) = self.sums[w - 2], self.sums[w - 1]
            m1, m2 = s1 / c1, s2 / c2
            scale = np.maximum(np.abs(m1), np.abs(m2))
            if np.all(np.abs(m2 - m1) <= self.tol * np.where(scale > 0, scale, 1.0)):
                self.steady_step = w * self.W
                return True
        c, s = self.sums.get(w, (0, np.zeros(len(self.keys))))
        self.sums[w] = (c + 1, s + np.array([float(vals[k]) for k in self.keys]))
        self.last = w
        return False


def window_steps(cfg: dict, nu_max: float, minimum: int = 2000) -> int:
    """max(minimum, 5 collision times 1 / nu_max), in steps."""
    tau = 1.0 / nu_max if nu_max > 0 else 0.0
    return int(max(minimum, np.ceil(5 * tau / cfg["dt"])))


def _sample(sim, k):
    d = sim.diagnostics(density=True, sim=k)
    return dict(n=d["n_particles"], n_max=d["n_peak"], i_outer=d["I_outer"]), d


def time_to_steady(cfgs: list[dict], form: str, cap_steps: int, samples_per_window: int = 10,
                   seed: int = 0, net=None, scales=None, stats: dict | None = None):
    """Run `cfgs` in the given form until every simulation is steady or has
    taken cap_steps; returns wall seconds, the per-simulation steady step
    (None if not reached) and the particle-steps advanced.  Form "learned"
    is "batched" with the net (batch = the simulations, H x W = nr x nz)
    supplying every solve's initial guess (warm_start = 2, `scales` the
    rho / phi / dphi scales of its training data).  `stats`, if given,
    receives the median initial relative residual and the mean sweeps of
    the field solves at the samples."""
    import torch
    from ._capi import Simulation
    S = len(cfgs)
    if form == "batched":
        cf = [dict(c, precision=32, warm_start=1) for c in cfgs]
    elif form == "learned":
        if net is None or scales is None:
            raise ValueError("the learned form needs a net and its scales")
        cf = [dict(c, precision=32, warm_start=2) for c in cfgs]
    elif form == "plain":
        cf = [dict(c, precision=64, warm_start=0) for c in cfgs]
    else:
        raise ValueError(form)
    parts = [seed_particles(c, seed=seed * 1000 + k) for k, c in enumerate(cf)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steady = [None] * S
    pushed = 0
    solve = {"relres_init": [], "sweeps": []}   # the field solves at the samples

    def note(d):
        solve["relres_init"].append(d["poisson_relres_init"])
        solve["sweeps"].append(d["poisson_iters"])
    if form in ("batched", "learned"):
        with Simulation(cf) as sim:
            for k, p in enumerate(parts):
                sim.load_particles(*p, sim=k)
            if form == "learned":
                sim.attach_unet(net, *scales)
            W = [window_steps(c, sim.diagnostics(sim=k)["nu_max"]) for k, c in enumerate(cf)]
            every = max(1, min(W) // samples_per_window)
            det = [SteadyDetector(w) for w in W]
            step = 0
            while step < cap_steps and any(s is None for s in steady):
                sim.step(every)
                step += every
                for k in range(S):
                    if steady[k] is None:
                        vals, d = _sample(sim, k)
                        note(d)
                        if det[k].add(step, **vals):
                            steady[k] = det[k].steady_step
            pushed = sum(sim.diagnostics(sim=k)["n_pushed"] for k in range(S))
            if form == "learned":
                sim.attach_unet(None, 1.0, 1.0, 1.0)
    else:
        for k in range(S):
            with Simulation(cf[k]) as sim:
                sim.load_particles(*parts[k])
                W = window_steps(cf[k], sim.diagnostics()["nu_max"])
                every = max(1, W // samples_per_window)
                det = SteadyDetector(W)
                step = 0
                while step < cap_steps:
                    sim.step(every)
                    step += every
                    vals, d = _sample(sim, 0)
                    note(d)
                    if det.add(step, **vals):
                        steady[k] = det.steady_step
                        break
                pushed += sim.diagnostics()["n_pushed"]
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    if stats is not None:
        stats["relres_init_median"] = float(np.median(solve["relres_init"])) if solve["sweeps"] else None
        stats["sweeps_mean"] = float(np.mean(solve["sweeps"])) if solve["sweeps"] else None
    return sec, steady, pushed
