"""The statistical steady-state case shared by the GPU test and its CPU
check (test code only; the oracle side runs in spawned worker processes).

Workload: the small coaxial gap (a = 1 mm, b = 10 mm, L = 40 mm, 32 x 64
cells, uniform B_z = 0.2 T, -10 kV) at the up-scaled pressure 0.3 mbar
(Sec. II.B: currents scale with the pressure, so a higher pressure reaches
the steady state in fewer steps), dt = 5 ps, 20 000 seeded electrons and a
volumetric seed source of 10 macro-electrons per step.  Elastic collisions
and ionisation balance the source against the wall losses within about
3000 steps; the statistics are time averages over the next 5000 steps,
sampled every 10 steps:
  n_max    the peak of the radial density profile: the charge of each
           radial node line over its volume (summed over z), averaged over
           the samples, then the largest over r;
  I_outer  electron current into the outer wall (A), from the absorbed
           weight over the window;
  N        mean number of macro-electrons.
"""
from __future__ import annotations

import numpy as np

EQUIL, WINDOW, EVERY = 3000, 5000, 10
SEEDS = (1, 2, 3, 4, 5)
QE = 1.602176634e-19


def config(seed: int, precision: int = 32) -> dict:
    from paper_2206_14662_gb300.inputs import workload
    dt = 5e-12
    return workload("coax_32x64_1e4", precision=precision, seed=seed, p_mbar=0.3, dt=dt,
                    n_init=20_000, source_rate=10.0 / dt, sort_every=20)


def radial_profile(cfg: dict, b_or_density, vol, is_density: bool) -> np.ndarray:
    """Charge per radial node line over its volume (electrons per m^3)."""
    nr, nz = cfg["nr"], cfg["nz"]
    v = vol.reshape(nr + 1, nz + 1)
    if is_density:
        q = (np.asarray(b_or_density).reshape(nr + 1, nz + 1) * v).sum(axis=1)
    else:
        q = (np.asarray(b_or_density).reshape(nr + 1, nz + 1) / -QE).sum(axis=1)
    return q / v.sum(axis=1)


def oracle_stats(seed: int, threads: int = 3) -> dict:
    """The oracle (FP64) on the case: time-averaged statistics."""
    import oracle
    from paper_2206_14662_gb300.inputs import seed_particles
    oracle.build()
    oracle.set_threads(threads)
    cfg = config(seed)
    cfg["nu_max"] = oracle.nu_max(cfg)   # derived once, not per seed-source call
    o = oracle.OracleSim(cfg, *seed_particles(cfg, seed=seed))
    vol = oracle.node_volumes(cfg)
    for _ in range(EQUIL):
        o.step()
    t0 = o.tally.copy()
    prof = np.zeros(cfg["nr"] + 1)
    N = 0.0
    for k in range(WINDOW):
        o.step()
        if (k + 1) % EVERY == 0:
            prof += radial_profile(cfg, o.b, vol, is_density=False)
            N += o.n
    ns = WINDOW // EVERY
    t1 = o.tally
    return {"n_max": float((prof / ns).max()), "N": N / ns,
            "I_outer": float((t1[oracle.T_ABS_OUTER] - t0[oracle.T_ABS_OUTER]) * QE /
                             (WINDOW * cfg["dt"])),
            "n_ionise": float(t1[oracle.T_N_IONISE] - t0[oracle.T_N_IONISE])}
