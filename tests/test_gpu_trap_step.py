"""Whole PIC steps in the paper's trap (Sec. II.B: the coaxial gap with a
filled metal ellipse on the outer cylinder; Sec. II.A: web-spline field):
pic_step with bspline_degree and the ellipse against the oracle stepping
the same particles on its web-spline field with absorption by the
ellipse: FP64 steps with collisions, the potential at the nodes, the
ellipse's absorbed weight."""
import numpy as np
import pytest

import oracle
from paper_2206_14662_gb300.inputs import seed_particles, workload
from parity import by_uid, compare_states

pytestmark = pytest.mark.gpu

ELL = (81e-3, 12e-3, 3e-3, 14e-3)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2206_14662_gb300 import build
    build.build()
    oracle.build()


def _trap(precision=64, **kw):
    base = dict(r_in=63.75e-3, r_out=81e-3, z_min=-10e-3, z_max=34e-3, nr=12, nz=30,
                v_inner=-20e3, v_outer=0.0, b0=0.2, bfield_kind=0, p_mbar=0.5, weight=2e4,
                T0_eV=50.0, dt=1e-11, source_rate=0.0, sort_every=3, bspline_degree=2,
                ellipse=ELL, precision=precision, n_init=6000)
    base.update(kw)
    return workload("coax_32x64_1e4", **base)


def _outside(parts):
    r, z = parts[0], parts[1]
    keep = ((r - ELL[0]) / ELL[2]) ** 2 + ((z - ELL[1]) / ELL[3]) ** 2 > 1.0
    return [a[keep] for a in parts]


def test_trap_steps_match_oracle():
    from paper_2206_14662_gb300._capi import PIC_GRID_PHI, Simulation
    cfg = _trap()
    parts = _outside(seed_particles(cfg, n=5000, seed=31))
    o = oracle.OracleSim(cfg, *parts)
    with Simulation(cfg) as sim:
        sim.load_particles(*parts)
        for _ in range(8):
            o.step()
        sim.step(8)
        g = by_uid(sim.export_particles())
        phi = sim.get_grid(PIC_GRID_PHI)
        d = sim.diagnostics()
    compare_states(cfg, 64, g, o, tol=1e-9)
    assert o.tally[oracle.T_ABS_ELLIPSE] > 0
    assert d["absorbed_ellipse"] == pytest.approx(o.tally[oracle.T_ABS_ELLIPSE], rel=1e-12)
    r, z = oracle.grid(cfg)
    R, Z = np.meshgrid(r, z, indexing="ij")
    ins = o.spline.geo.inside(R.ravel(), Z.ravel())
    want = o.spline.phi(o.coef, R.ravel(), Z.ravel())
    assert np.abs(phi[ins] - want[ins]).max() <= 1e-9 * np.abs(want[ins]).max()


def test_trap_fp32_load_and_potential():
    """FP32 steps in the trap deposit through the block's fixed-point tile:
    the potential inside the domain after two steps against the oracle's
    (no collisions, so both step the same particles)."""
    from paper_2206_14662_gb300._capi import PIC_GRID_PHI, Simulation
    cfg = _trap(32, p_mbar=0.0, n_init=20_000)
    parts = _outside(seed_particles(cfg, n=20_000, seed=33))
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
    ins = o.spline.geo.inside(R.ravel(), Z.ravel())
    want = o.spline.phi(o.coef, R.ravel(), Z.ravel())
    vac = o.spline.phi(np.zeros_like(o.coef), R.ravel(), Z.ravel())
    err = np.abs(phi.ravel()[ins] - want[ins]).max()
    assert err <= 2e-5 * np.abs(want[ins] - vac[ins]).max(), err
