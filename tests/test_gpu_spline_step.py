"""Whole PIC steps on the weighted B-spline field (pic_config.bspline_degree:
Sec. II.A's weighted B-splines of arbitrary degree with particle shapes
from the same basis) against the oracle stepping the same particles in
its spline mode: FP64 steps with collisions and sorts, the potential at
the nodes, FP32 one step; graph replay agreeing with direct launches to
rounding (FP64)."""
import numpy as np
import pytest

import oracle
from paper_2206_14662_gb300.inputs import seed_particles, workload
from parity import by_uid, compare_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2206_14662_gb300 import build
    build.build()
    oracle.build()


def _cfg(precision, n, **kw):
    base = dict(precision=precision, bspline_degree=n, p_mbar=1.0, T0_eV=40.0, n_init=20_000,
                sort_every=3, source_rate=0.0, poisson_rtol=1e-12)
    base.update(kw)
    return workload("coax_32x64_1e4", **base)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_spline_steps_match_oracle(n):
    from paper_2206_14662_gb300._capi import PIC_GRID_PHI, Simulation
    cfg = _cfg(64, n)
    parts = seed_particles(cfg, n=8000, seed=20 + n)
    o = oracle.OracleSim(cfg, *parts)
    with Simulation(cfg) as sim:
        sim.load_particles(*parts)
        for _ in range(6):
            o.step()
        sim.step(6)
        g = by_uid(sim.export_particles())
        phi = sim.get_grid(PIC_GRID_PHI)
        d = sim.diagnostics()
    rep = {}
    compare_states(cfg, 64, g, o, report=rep, tol=1e-9)
    assert abs(d["n_elastic"] - o.tally[oracle.T_N_ELASTIC]) <= 1
    r, z = oracle.grid(cfg)
    R, Z = np.meshgrid(r, z, indexing="ij")
    want = o.spline.phi(o.coef, R.ravel(), Z.ravel())
    assert np.abs(phi - want).max() <= 1e-9 * np.abs(want).max()


def test_spline_step_fp32_one_step():
    cfg = _cfg(32, 2)
    parts = seed_particles(cfg, n=20_000 + 37, seed=5)
    from paper_2206_14662_gb300._capi import Simulation
    o = oracle.OracleSim(cfg, *parts)
    uid0, next0 = o.uid.copy(), o.uid_next
    res = o.step()
    with Simulation(cfg) as sim:
        sim.load_particles(*parts)
        sim.step(1)
        g = by_uid(sim.export_particles())
    amb = compare_states(cfg, 32, g, o, margin=res.margin, uid_before=uid0, child_uid0=next0)
    assert amb <= 5


@pytest.mark.parametrize("n", [1, 2, 3])
def test_spline_fp32_load_and_potential(n):
    """FP32 steps deposit through the block's fixed-point tile (integer warp
    sums and shared atomics, one FP64 atomic per coefficient and chunk):
    the potential at the nodes after the steps against the oracle's, to
    the FP32 positions' and the fixed-point unit's rounding.  The first
    load (at particle load) is the per-particle path, so the comparison
    after two steps covers the tile."""
    from paper_2206_14662_gb300._capi import PIC_GRID_PHI, Simulation
    cfg = _cfg(32, n, p_mbar=0.0)
    parts = seed_particles(cfg, n=20_000, seed=40 + n)
    o = oracle.OracleSim(cfg, *parts)
    with Simulation(cfg) as sim:
        sim.load_particles(*parts)
        for _ in range(2):
            o.step()
        sim.step(2)
        phi = sim.get_grid(PIC_GRID_PHI)
        d = sim.diagnostics()
    assert d["error"] == 0
    r, z = oracle.grid(cfg)
    R, Z = np.meshgrid(r, z, indexing="ij")
    want = o.spline.phi(o.coef, R.ravel(), Z.ravel())
    # the space-charge part of the potential: the difference to the
    # vacuum potential of the same walls
    vac = o.spline.phi(np.zeros_like(o.coef), R.ravel(), Z.ravel())
    err = np.abs(phi.ravel() - want).max()
    assert err <= 2e-5 * np.abs(want - vac).max(), err / np.abs(want - vac).max()


def test_spline_graph_replay_equals_direct():
    from paper_2206_14662_gb300._capi import Simulation
    cfg = _cfg(64, 2, n_init=30_000)
    parts = seed_particles(cfg, n=30_000, seed=8)
    out = []
    for k in (1, 24):   # one step at a time (direct) / blocks (graphs)
        with Simulation(cfg) as sim:
            sim.load_particles(*parts)
            for _ in range(24 // k):
                sim.step(k)
            out.append(by_uid(sim.export_particles()))
    a, b = out
    # FP64 atomics in the spline deposit make the sums order-dependent:
    # agreement to rounding, not bit for bit
    assert np.array_equal(a["uid"], b["uid"])
    for key in ("r", "z"):
        assert np.abs(a[key] - b[key]).max() <= 1e-9 * np.abs(a[key]).max()
