"""Helpers for the GPU-vs-oracle parity tests (test code only)."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2206_14662_gb300.inputs import seed_particles

# FP32 tolerance of the particle path: 1e-5 relative (positions in cells,
# velocities relative to the largest speed, deposits relative to the
# largest node charge); FP64: 1e-12.
TOL = {32: 1e-5, 64: 1e-12}
# a discrete decision (wall test, collision type) closer than this to its
# threshold may go either way in FP32 and is excluded from the comparison
AMBIGUOUS = {32: 1e-5, 64: 1e-13}


def make_gpu(cfg, parts, efield=None):
    from paper_2206_14662_gb300._capi import Simulation
    sim = Simulation(cfg)
    sim.load_particles(*parts)
    if efield is not None:
        sim.set_efield(*efield)
    return sim


def by_uid(d: dict) -> dict:
    order = np.argsort(d["uid"])
    return {k: v[order] for k, v in d.items()}


def compare_states(cfg, precision, g: dict, o: "oracle.OracleSim", margin=None,
                   uid_before=None, report=None, child_uid0=None, tol=None):
    """Compare GPU particles g (exported, sorted by uid) with the oracle's.
    Particles whose last decision was ambiguous (margin below the threshold)
    are excluded; if any was, children (uid >= child_uid0) are excluded too,
    since a flipped ionisation shifts the later children's uids.  Returns
    the number of ambiguous particles."""
    hr = (cfg["r_out"] - cfg["r_in"]) / cfg["nr"]
    hz = (cfg["z_max"] - cfg["z_min"]) / cfg["nz"]
    tol = TOL[precision] if tol is None else tol
    amb_uids = set()
    if margin is not None:
        amb = margin < AMBIGUOUS[precision]
        amb_uids = set(uid_before[amb].tolist())
    ou = o.uid
    gu = g["uid"]
    keep_o = np.array([u not in amb_uids for u in ou.tolist()], dtype=bool)
    keep_g = np.array([u not in amb_uids for u in gu.tolist()], dtype=bool)
    if amb_uids and child_uid0 is not None:
        keep_o &= ou < child_uid0
        keep_g &= gu < child_uid0
    assert np.array_equal(ou[keep_o], gu[keep_g]), "live particle sets differ"
    vmax = max(np.abs(o.vr).max(initial=0), np.abs(o.vt).max(initial=0), np.abs(o.vz).max(initial=0), 1.0)
    err = dict(
        r=np.abs(g["r"][keep_g] - o.r[keep_o]).max(initial=0) / hr,
        z=np.abs(g["z"][keep_g] - o.z[keep_o]).max(initial=0) / hz,
        vr=np.abs(g["vr"][keep_g] - o.vr[keep_o]).max(initial=0) / vmax,
        vt=np.abs(g["vt"][keep_g] - o.vt[keep_o]).max(initial=0) / vmax,
        vz=np.abs(g["vz"][keep_g] - o.vz[keep_o]).max(initial=0) / vmax,
    )
    if report is not None:
        report.update(err)
    for k, e in err.items():
        assert e <= tol, f"{k}: {e:.3e} > {tol:.1e}"
    return len(amb_uids)


def seeded(cfg, n, seed=3, margin_cells=0.0):
    return seed_particles(cfg, n=n, seed=seed, margin_cells=margin_cells)
