"""Pins of the oracle's particle step in the paper's trap (Sec. II.B: the
coaxial gap with a filled metal ellipse on the outer cylinder, whose
current is reported separately): electrons whose straight (r, z) step
enters the ellipse are absorbed and tallied to it, a chord through its tip
counts, a near miss does not, the first crossing decides between the
ellipse and a wall, and the energy ledger of a collisional run in the
trap's web-spline field closes."""
import math

import numpy as np
import pytest

import oracle
from oracle import ME, QE
from paper_2206_14662_gb300.inputs import seed_particles, workload

ELL = (81e-3, 12e-3, 3e-3, 14e-3)


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _trap_cfg(**kw):
    base = dict(r_in=63.75e-3, r_out=81e-3, z_min=-10e-3, z_max=34e-3, nr=12, nz=30,
                v_inner=0.0, v_outer=0.0, b0=0.0, bfield_kind=0, p_mbar=1e-12,
                bspline_degree=2, ellipse=ELL, weight=1e-9, dt=1e-11, source_rate=0.0)
    base.update(kw)
    return workload("coax_32x64_1e4", **base)


def _one(cfg, r, z, vr, vz, vt=0.0):
    o = oracle.OracleSim(cfg, [r], [z], [vr], [vt], [vz], np.array([0], dtype=np.uint64))
    return o, o.step()


def test_head_on_entry_is_absorbed_by_the_ellipse():
    cfg = _trap_cfg()
    # 0.1 mm outside the ellipse's inner vertex (r = 78 mm, z = 12 mm),
    # moving outward 0.3 mm per step
    o, res = _one(cfg, 77.9e-3, 12e-3, 3e7, 0.0)
    assert res.event[0] == oracle.EV_WALL + 4
    assert o.n == 0
    assert res.tally[oracle.T_ABS_ELLIPSE] == pytest.approx(cfg["weight"])
    assert res.tally[oracle.T_ABS_OUTER] == 0.0
    assert res.tally[oracle.T_KE_ABSORBED] == pytest.approx(cfg["weight"] * 0.5 * ME * 9e14,
                                                             rel=1e-6)


def test_chord_and_near_miss():
    cfg = _trap_cfg(dt=1e-10)
    # along z at r = 78.01 mm, 0.01 mm inside the inner vertex (78 mm): the
    # ellipse spans |z - 12 mm| <= 1.14 mm there; a step from 10.5 to
    # 13.5 mm starts and ends outside and crosses it
    ends = [((78.01e-3 - ELL[0]) / ELL[2]) ** 2 + ((zz - ELL[1]) / ELL[3]) ** 2 - 1.0
            for zz in (10.5e-3, 13.5e-3)]
    assert min(ends) > 0
    o, res = _one(cfg, 78.01e-3, 10.5e-3, 0.0, 3e7)
    assert res.event[0] == oracle.EV_WALL + 4 and o.n == 0
    # the same step 0.01 mm outside the vertex misses it
    o, res = _one(cfg, 77.99e-3, 10.5e-3, 0.0, 3e7)
    assert res.event[0] < oracle.EV_WALL and o.n == 1
    assert res.tally[oracle.T_ABS_ELLIPSE] == 0.0


def test_first_crossing_between_wall_and_ellipse():
    cfg = _trap_cfg()
    # both steps end beyond the outer wall and inside the ellipse's
    # continuation; the first crossing along the segment decides
    # (0.6 mm out, 0.6 mm down from (80.6, 26.1) mm: ellipse at t ~ 0.25,
    # wall at t = 0.67)
    o, res = _one(cfg, 80.6e-3, 26.1e-3, 6e7, -6e7)
    assert res.event[0] == oracle.EV_WALL + 4
    assert res.tally[oracle.T_ABS_ELLIPSE] > 0 and res.tally[oracle.T_ABS_OUTER] == 0
    # (0.3 mm out, 1 mm down from (80.9, 26.5) mm: wall at t = 0.33, the
    # ellipse only after it)
    o, res = _one(cfg, 80.9e-3, 26.5e-3, 3e7, -1e8)
    assert res.event[0] == oracle.EV_WALL + 1
    assert res.tally[oracle.T_ABS_OUTER] > 0 and res.tally[oracle.T_ABS_ELLIPSE] == 0


def test_energy_ledger_in_the_trap():
    cfg = _trap_cfg(v_inner=-20e3, b0=0.2, p_mbar=0.5, weight=2e4, T0_eV=50.0)
    r, z, vr, vt, vz, uid = seed_particles(cfg, n=3000, seed=5)
    keep = ((r - ELL[0]) / ELL[2]) ** 2 + ((z - ELL[1]) / ELL[3]) ** 2 > 1.0
    o = oracle.OracleSim(cfg, r[keep], z[keep], vr[keep], vt[keep], vz[keep], uid[keep])
    ke0 = o.kinetic_energy()
    for _ in range(6):
        o.step()
    t = o.tally
    assert t[oracle.T_N_ELASTIC] > 0 and t[oracle.T_N_ABSORBED] > 0
    dke = o.kinetic_energy() - ke0
    budget = (t[oracle.T_WORK_E] - t[oracle.T_KE_ABSORBED] - t[oracle.T_ION_LOSS]
              - t[oracle.T_RECOIL_LOSS])
    assert dke == pytest.approx(budget, rel=1e-9, abs=1e-12 * abs(t[oracle.T_WORK_E]))
    # absorbed weight: walls and ellipse together equal the absorbed count
    absorbed = sum(t[k] for k in (oracle.T_ABS_INNER, oracle.T_ABS_OUTER, oracle.T_ABS_ZMIN,
                                  oracle.T_ABS_ZMAX, oracle.T_ABS_ELLIPSE))
    assert absorbed == pytest.approx(cfg["weight"] * t[oracle.T_N_ABSORBED])
