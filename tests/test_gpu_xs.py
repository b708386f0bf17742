"""Tabulated cross sections (Sec. II.A: elastic momentum-transfer and total
ionisation cross sections from tabulated data, the angle law's anisotropy
depending on the energy) through pic_set_cross_sections, against the CPU
oracle given the same tables: one collision-heavy step in a fixed field,
FP64 and FP32, uniform and mirror field; the majorant derived from the
tables; tables removed again restore the analytic run bit for bit; bad
tables are refused.  The tables are synthetic (inputs.cross_section_tables).
"""
import numpy as np
import pytest

import oracle
from paper_2206_14662_gb300.inputs import (cross_section_tables, random_field_node_arrays,
                                           seed_particles, workload)
from parity import TOL, by_uid, compare_states, make_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2206_14662_gb300 import build
    build.build()
    oracle.build()


def _cfg(precision, with_xi=True, **kw):
    base = dict(p_mbar=1.0, T0_eV=100.0, n_init=20_000, precision=precision, fixed_efield=1,
                sort_every=0)
    base.update(kw)
    cfg = workload("coax_32x64_1e4", **base)
    E, sel, sio, xi = cross_section_tables(cfg["ion_E_th_eV"], with_xi=with_xi)
    cfg["xs"] = dict(E_eV=E, sigma_el=sel, sigma_io=sio, xi=xi)
    return cfg


@pytest.mark.parametrize("precision,bkind,with_xi", [(64, 0, True), (64, 1, True), (32, 1, True),
                                                     (32, 0, False)])
def test_tabulated_step_matches_oracle(precision, bkind, with_xi):
    """One step from an identical state: particle states, children, event
    counts and the majorant agree with the oracle run on the same tables."""
    cfg = _cfg(precision, with_xi=with_xi, bfield_kind=bkind, p_mbar=3.0)
    n = 20_000 + 37
    parts = seed_particles(cfg, n=n, seed=3)
    er, ez = random_field_node_arrays(cfg, 3e5, seed=4)
    o = oracle.OracleSim(cfg, *parts, efield_nodes=(er, ez), solve_field=False)
    sim = make_gpu(cfg, parts, efield=(er, ez))
    xs = cfg["xs"]
    sim.set_cross_sections(xs["E_eV"], xs["sigma_el"], xs["sigma_io"], xs["xi"])
    uid0, next0 = o.uid.copy(), o.uid_next
    res = o.step()
    sim.step(1)
    d = sim.diagnostics()
    g = by_uid(sim.export_particles())
    sim.close()
    amb = compare_states(cfg, precision, g, o, margin=res.margin, uid_before=uid0,
                         child_uid0=next0)
    assert amb <= 3
    assert res.tally[oracle.T_N_ELASTIC] > 100 and res.tally[oracle.T_N_IONISE] > 5
    for key, slot in (("n_elastic", oracle.T_N_ELASTIC), ("n_ionise", oracle.T_N_IONISE),
                      ("n_absorbed", oracle.T_N_ABSORBED), ("n_candidates", oracle.T_N_CANDIDATE)):
        assert abs(d[key] - res.tally[slot]) <= amb, key
    assert d["nu_max"] == pytest.approx(o.P.nu_max, rel=1e-14)
    # the tables changed the collision rates: not the analytic majorant
    assert abs(d["nu_max"] / oracle.nu_max(dict(cfg, xs=None)) - 1.0) > 0.01


def test_removed_tables_restore_the_analytic_run():
    """Tables set and removed again before stepping: the FP32 run equals,
    bit for bit, the run that never had tables (graph-replayed steps)."""
    from paper_2206_14662_gb300._capi import PIC_GRID_PHI, Simulation
    cfg = _cfg(32, fixed_efield=0, n_init=30_000, sort_every=4)
    xs = cfg.pop("xs")
    out = []
    for with_tables in (False, True):
        with Simulation(cfg) as sim:
            sim.load_particles(*seed_particles(cfg))
            if with_tables:
                sim.set_cross_sections(xs["E_eV"], xs["sigma_el"], xs["sigma_io"], xs["xi"])
                assert sim.diagnostics()["nu_max"] != pytest.approx(oracle.nu_max(cfg), rel=1e-3)
                sim.set_cross_sections()
            sim.step(3)
            sim.step(21)
            out.append((by_uid(sim.export_particles()), sim.get_grid(PIC_GRID_PHI),
                        sim.diagnostics()))
    (ga, pa, da), (gb, pb, db) = out
    for k in ga:
        assert np.array_equal(ga[k], gb[k]), k
    assert np.array_equal(pa, pb)
    assert da["nu_max"] == db["nu_max"] and da["n_ionise"] == db["n_ionise"]


def test_tables_set_between_steps_take_effect():
    """Tables set after some steps change the collision rate from the next
    step on (the step graphs are rebuilt) and agree with the oracle from
    that state."""
    cfg = _cfg(64, n_init=8000)
    xs = cfg.pop("xs")
    parts = seed_particles(cfg, n=8000, seed=11)
    er, ez = random_field_node_arrays(cfg, 3e5, seed=12)
    sim = make_gpu(cfg, parts, efield=(er, ez))
    sim.step(8)
    g0 = by_uid(sim.export_particles())
    # children so far took the uids after the loaded ones
    uid_next8 = int(parts[5].max()) + 1 + int(sim.diagnostics()["n_ionise"])
    sim.set_cross_sections(xs["E_eV"], xs["sigma_el"], xs["sigma_io"], xs["xi"])
    sim.step(8)
    g = by_uid(sim.export_particles())
    d = sim.diagnostics()
    sim.close()
    # the oracle from the exported state of step 8 (uids as exported)
    o = oracle.OracleSim(dict(cfg, xs=xs), g0["r"], g0["z"], g0["vr"], g0["vt"], g0["vz"],
                         g0["uid"], efield_nodes=(er, ez), solve_field=False, step0=8,
                         uid_next=uid_next8)
    for _ in range(8):
        o.step()
    rep = {}
    compare_states(cfg, 64, g, o, report=rep)
    assert max(rep.values()) <= 1e-10


@pytest.mark.parametrize("bad", ["one_point", "not_increasing", "negative_sigma", "xi_one",
                                 "negative_energy"])
def test_bad_tables_are_refused(bad):
    from paper_2206_14662_gb300._capi import PicError, Simulation
    cfg = _cfg(32)
    xs = cfg.pop("xs")
    E, sel, sio, xi = (np.array(xs[k], dtype=float) for k in ("E_eV", "sigma_el", "sigma_io", "xi"))
    if bad == "one_point":
        E, sel, sio, xi = E[:1], sel[:1], sio[:1], xi[:1]
    elif bad == "not_increasing":
        E[5] = E[4]
    elif bad == "negative_sigma":
        sel[3] = -1e-21
    elif bad == "xi_one":
        xi[7] = 1.0
    else:
        E[0] = -1.0
    with Simulation(cfg) as sim:
        with pytest.raises(PicError):
            sim.set_cross_sections(E, sel, sio, xi)
        # the simulation still runs on its analytic cross sections
        assert sim.diagnostics()["nu_max"] == pytest.approx(oracle.nu_max(cfg), rel=1e-12)
