"""Batches of simulations (the paper's parametric scans over pressure,
voltage and magnetic field, Sec. III-IV) stepped together through the C ABI:
each simulation of a batch follows the CPU oracle run on its own, and
simulation 0 of a batch is bit-identical to the same simulation run alone.

The random streams of simulation k use Philox counter word 1 = k, the high
word of its particles' 64-bit identity; the oracle is given uids
(k << 32) | uid for that simulation.
"""
import numpy as np
import pytest

import oracle
from paper_2206_14662_gb300.inputs import (random_field_node_arrays, seed_particles,
                                           workload)
from parity import TOL, by_uid, compare_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2206_14662_gb300 import build
    build.build()
    oracle.build()


def _batch_cfgs(precision, ns=(900, 2500, 37, 4100), **kw):
    """Four simulations of the 32 x 64 coax that differ in pressure,
    voltage, field kind and strength and particle count (ragged counts, one
    far below a chunk)."""
    var = [dict(p_mbar=0.3, v_inner=-10e3, b0=0.2, bfield_kind=0),
           dict(p_mbar=1.0, v_inner=-5e3, b0=0.35, bfield_kind=1),
           dict(p_mbar=3.0, v_inner=-20e3, b0=0.1, bfield_kind=1),
           dict(p_mbar=0.1, v_inner=-15e3, b0=0.5, bfield_kind=0)]
    out = []
    for k, n in enumerate(ns):
        c = workload("coax_32x64_1e4", precision=precision, T0_eV=30.0, n_init=n, **var[k % 4])
        if n == 0:
            c["weight"] = 1.0e6   # an empty simulation needs an explicit weight
        c.update(kw)
        out.append(c)
    return out


def _parts(cfg, k):
    return seed_particles(cfg, n=cfg["n_init"], seed=100 + k)


def _oracle(cfg, k, parts, **kw):
    r, z, vr, vt, vz, uid = parts
    return oracle.OracleSim(cfg, r, z, vr, vt, vz, uid + (np.uint64(k) << np.uint64(32)), **kw)


def _export(sim, k):
    g = by_uid(sim.export_particles(sim=k))
    g["uid"] = g["uid"] + (np.uint64(k) << np.uint64(32))
    return g


def test_batch_self_consistent_fp64_matches_oracle():
    """Ten self-consistent steps (field solve on, counting sort every three
    steps) of a batch of four different simulations, FP64: each simulation's
    particles, potential and event counts follow its own oracle run."""
    from paper_2206_14662_gb300._capi import PIC_GRID_PHI, Simulation
    cfgs = _batch_cfgs(64, poisson_rtol=1e-12, poisson_maxit=8, sort_every=3)
    parts = [_parts(c, k) for k, c in enumerate(cfgs)]
    oracles = [_oracle(c, k, p) for k, (c, p) in enumerate(zip(cfgs, parts))]
    with Simulation(cfgs) as sim:
        for k, p in enumerate(parts):
            sim.load_particles(*p, sim=k)
        sim.step(10)
        got = [(_export(sim, k), sim.get_grid(PIC_GRID_PHI, sim=k), sim.diagnostics(sim=k))
               for k in range(len(cfgs))]
    for o in oracles:
        for _ in range(10):
            o.step()
    for k, (cfg, o, (g, phi, d)) in enumerate(zip(cfgs, oracles, got)):
        assert np.abs(phi - o.phi).max() <= 1e-10 * np.abs(o.phi).max(), k
        compare_states(cfg, 64, g, o, tol=1e-9)
        assert d["n_ionise"] == o.tally[oracle.T_N_IONISE], k
        assert d["n_elastic"] == o.tally[oracle.T_N_ELASTIC], k
        assert d["n_absorbed"] == o.tally[oracle.T_N_ABSORBED], k
        assert d["n_particles"] == len(o.uid), k
        assert d["poisson_relres"] <= cfgs[k]["poisson_rtol"]
    # the simulations did differ: collisions in the high-pressure ones
    assert sum(o.tally[oracle.T_N_IONISE] for o in oracles) > 0


def test_batch_one_step_fp32_fixed_field_matches_oracle():
    """One FP32 step in a fixed field per simulation (each its own field),
    with collisions and wall losses: particles, children and deposits of
    every simulation agree with the oracle within the FP32 tolerance."""
    from paper_2206_14662_gb300._capi import PIC_GRID_RHS, Simulation
    cfgs = _batch_cfgs(32, ns=(3000, 1024, 5000, 1), fixed_efield=1, sort_every=0,
                       T0_eV=100.0)
    for c in cfgs:
        c["p_mbar"] *= 3
    parts = [_parts(c, k) for k, c in enumerate(cfgs)]
    fields = [random_field_node_arrays(c, 3e5 * (k + 1), seed=20 + k) for k, c in enumerate(cfgs)]
    oracles, results, uid0, next0 = [], [], [], []
    for k, (c, p, f) in enumerate(zip(cfgs, parts, fields)):
        o = _oracle(c, k, p, efield_nodes=f, solve_field=False)
        uid0.append(o.uid.copy())
        next0.append(o.uid_next)
        results.append(o.step())
        oracles.append(o)
    with Simulation(cfgs) as sim:
        for k, (p, f) in enumerate(zip(parts, fields)):
            sim.load_particles(*p, sim=k)
            sim.set_efield(*f, sim=k)
        sim.step(1)
        got = [(_export(sim, k), sim.get_grid(PIC_GRID_RHS, sim=k), sim.diagnostics(sim=k))
               for k in range(len(cfgs))]
    n_ion = 0
    for k, (c, o, res, (g, b, d)) in enumerate(zip(cfgs, oracles, results, got)):
        amb = compare_states(c, 32, g, o, margin=res.margin, uid_before=uid0[k],
                             child_uid0=next0[k])
        assert amb <= 3, k
        for key, slot in (("n_elastic", oracle.T_N_ELASTIC), ("n_ionise", oracle.T_N_IONISE),
                          ("n_absorbed", oracle.T_N_ABSORBED)):
            assert abs(d[key] - res.tally[slot]) <= amb, (k, key)
        if amb == 0 and np.abs(res.b).max() > 0:
            assert np.abs(b - res.b).max() <= TOL[32] * np.abs(res.b).max(), k
        n_ion += res.tally[oracle.T_N_IONISE]
    assert n_ion > 0


def test_batch_simulation_zero_is_bitwise_a_single_run():
    """Simulation 0 of a batch draws the same random numbers and performs the
    same arithmetic as the simulation run alone: 40 FP32 steps (graph
    blocks, sorts) give bit-identical particles and potential."""
    from paper_2206_14662_gb300._capi import PIC_GRID_PHI, Simulation
    cfgs = _batch_cfgs(32, ns=(20_000, 7000, 50_000), sort_every=4, p_mbar=0.3, T0_eV=20.0)
    cfgs = [dict(c, nr=64, nz=256, bfield_kind=1) for c in cfgs]
    parts = [_parts(c, k) for k, c in enumerate(cfgs)]
    with Simulation(cfgs[0]) as one:
        one.load_particles(*parts[0])
        one.step(3)
        one.step(37)
        g1, phi1, d1 = by_uid(one.export_particles()), one.get_grid(PIC_GRID_PHI), one.diagnostics()
    with Simulation(cfgs) as sim:
        for k, p in enumerate(parts):
            sim.load_particles(*p, sim=k)
        sim.step(3)
        sim.step(37)
        gb, phib, db = (by_uid(sim.export_particles(sim=0)), sim.get_grid(PIC_GRID_PHI, sim=0),
                        sim.diagnostics(sim=0))
        d2 = sim.diagnostics(sim=2)
    for key in g1:
        assert np.array_equal(g1[key], gb[key]), key
    assert np.array_equal(phi1, phib)
    for key in ("n_particles", "n_elastic", "n_ionise", "n_absorbed", "n_pushed", "step"):
        assert d1[key] == db[key], key
    assert d2["n_pushed"] > 40 * 40_000 and d2["step"] == 40


def test_batch_edge_cases():
    """An empty simulation, one whose particles all leave in the first step
    and a capacity overflow in one simulation of a batch."""
    from paper_2206_14662_gb300._capi import PIC_ECAPACITY, PicError, Simulation
    cfgs = _batch_cfgs(32, ns=(0, 500, 3000), fixed_efield=1, sort_every=2)
    parts = [_parts(c, k) for k, c in enumerate(cfgs)]
    nn = (cfgs[0]["nr"] + 1) * (cfgs[0]["nz"] + 1)
    with Simulation(cfgs) as sim:
        for k, p in enumerate(parts):
            sim.load_particles(*p, sim=k)
        # simulation 1: a huge outward field empties it in one step
        sim.set_efield(np.full(nn, -1e12), np.zeros(nn), sim=1)
        sim.set_efield(np.zeros(nn), np.zeros(nn), sim=2)
        sim.step(4)
        d = [sim.diagnostics(sim=k) for k in range(3)]
    assert d[0]["n_particles"] == 0 and d[0]["n_pushed"] == 0
    assert d[1]["n_particles"] == 0 and d[1]["n_absorbed"] == 500
    assert d[2]["n_pushed"] >= 4 * 2900
    # a simulation with room for only a few children
    cfgs = _batch_cfgs(32, ns=(2000, 2000), fixed_efield=1, sort_every=0, p_mbar=30.0,
                       T0_eV=300.0)
    cfgs[1]["capacity"] = 2001
    parts = [_parts(c, k) for k, c in enumerate(cfgs)]
    with Simulation(cfgs) as sim:
        for k, p in enumerate(parts):
            sim.load_particles(*p, sim=k)
        sim.step(3)
        with pytest.raises(PicError) as ei:
            sim.diagnostics(sim=1)
        assert ei.value.code == PIC_ECAPACITY


def test_batch_with_seed_sources_matches_oracle():
    """Seed sources of different rates in the simulations of a batch (FP64,
    fixed per-simulation fields, collisions, a sort every two steps): the
    created particles of simulation k carry uids after its children and draw
    from its own streams (counter word 1 = k), as in the oracle."""
    from paper_2206_14662_gb300._capi import Simulation
    cfgs = _batch_cfgs(64, ns=(800, 1500, 300), fixed_efield=1, sort_every=2, T0_eV=20.0)
    rates = (11.4, 0.0, 3.7)
    for c, r in zip(cfgs, rates):
        c["source_rate"] = r / c["dt"]
    parts = [_parts(c, k) for k, c in enumerate(cfgs)]
    fields = [random_field_node_arrays(c, 2e5, seed=30 + k) for k, c in enumerate(cfgs)]
    oracles = [_oracle(c, k, p, efield_nodes=f, solve_field=False)
               for k, (c, p, f) in enumerate(zip(cfgs, parts, fields))]
    with Simulation(cfgs) as sim:
        for k, (p, f) in enumerate(zip(parts, fields)):
            sim.load_particles(*p, sim=k)
            sim.set_efield(*f, sim=k)
        sim.step(5)
        got = [(_export(sim, k), sim.diagnostics(sim=k)) for k in range(len(cfgs))]
    for o in oracles:
        for _ in range(5):
            o.step()
    for k, (cfg, o, (g, d)) in enumerate(zip(cfgs, oracles, got)):
        assert d["n_source"] == o.n_source, k
        compare_states(cfg, 64, g, o, tol=1e-10)
        assert d["ke_source_J"] == pytest.approx(o.ke_source, rel=1e-12, abs=1e-30), k
    assert oracles[0].n_source in (56, 57) and oracles[1].n_source == 0


def test_batch_self_consistent_fp32_follows_oracle():
    """Ten self-consistent FP32 steps of a batch (field solve on, sorts):
    each simulation's potential and particle positions follow its FP64
    oracle run within the FP32 tolerance."""
    from paper_2206_14662_gb300._capi import PIC_GRID_PHI, Simulation
    cfgs = _batch_cfgs(32, sort_every=3)
    parts = [_parts(c, k) for k, c in enumerate(cfgs)]
    oracles = [_oracle(c, k, p) for k, (c, p) in enumerate(zip(cfgs, parts))]
    with Simulation(cfgs) as sim:
        for k, p in enumerate(parts):
            sim.load_particles(*p, sim=k)
        sim.step(10)
        got = [(_export(sim, k), sim.get_grid(PIC_GRID_PHI, sim=k)) for k in range(len(cfgs))]
    for o in oracles:
        for _ in range(10):
            o.step()
    for k, (cfg, o, (g, phi)) in enumerate(zip(cfgs, oracles, got)):
        assert np.abs(phi - o.phi).max() <= 1e-5 * np.abs(o.phi).max(), k
        keep = np.isin(o.uid, g["uid"])
        assert keep.mean() > 0.995, k
        gi = np.searchsorted(g["uid"], o.uid[keep])
        hr = (cfg["r_out"] - cfg["r_in"]) / cfg["nr"]
        assert np.abs(g["r"][gi] - o.r[keep]).max() / hr <= 2e-5, k


def test_batch_autotuner_keeps_the_particles_bit_for_bit():
    """pic_autotune on a batch: the particles of every simulation equal
    those of the same number of steps with the default schedule."""
    from paper_2206_14662_gb300._capi import Simulation
    # the trials run thousands of steps: a low pressure and room to grow
    cfgs = _batch_cfgs(32, ns=(3000, 9000, 500), sort_every=20, p_mbar=0.01)
    for c in cfgs:
        c["capacity"] = 4 * c["n_init"] + 4096
    parts = [_parts(c, k) for k, c in enumerate(cfgs)]
    out = []
    for tune in (True, False):
        with Simulation(cfgs) as sim:
            for k, p in enumerate(parts):
                sim.load_particles(*p, sim=k)
            if tune:
                sim.step(3)
                sim.autotune(8)
                sim.step(5)
                steps = sim.diagnostics(sim=0)["step"]
            else:
                sim.step(steps)
            out.append([by_uid(sim.export_particles(sim=k)) for k in range(len(cfgs))])
    for a, b in zip(*out):
        for key in a:
            assert np.array_equal(a[key], b[key]), key
