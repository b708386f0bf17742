"""Fluid moments and force-balance terms (Sec. IV.A: the electron fluid's
forces from moments of the distribution function) through pic_moments and
pic_force_balance, against the oracle (oracle.fluid) on the same seeded
inputs: loaded states (scattered and clustered, so that both the per-lane
and the warp-summed accumulation run), a stepped state with absorbed
particles, tabulated cross sections, a batch member, FP64 and FP32; the
force terms and the fluid-model predictions (Sec. V) from the oracle's
moments; at the full mirror workload
(128 x 512 cells, 1e7 electrons) the partition-of-unity sums."""
import numpy as np
import pytest

import oracle
from oracle import fluid
from paper_2206_14662_gb300.inputs import (cross_section_tables, random_field_node_arrays,
                                           seed_particles, workload)
from parity import make_gpu

pytestmark = pytest.mark.gpu

# moments: per moment, relative to its largest node value.  FP64 differs
# from the oracle only in the order of the sums; FP32 stores offsets and
# velocities in FP32 and evaluates the collision rate in FP32.
MOM_TOL = {64: 1e-12, 32: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2206_14662_gb300 import build
    build.build()
    oracle.build()


def _cfg(precision, **kw):
    base = dict(precision=precision, fixed_efield=1, sort_every=0, T0_eV=20.0, n_init=40_000)
    base.update(kw)
    return workload("coax_32x64_1e4", **base)


def _compare_moments(got, want, tol):
    assert got.shape == want.shape
    for c in range(fluid.MOMENTS):
        scale = np.abs(want[c]).max()
        assert scale > 0, c
        err = np.abs(got[c] - want[c]).max() / scale
        assert err <= tol, (c, err)


def _clustered(cfg, n, seed):
    """n electrons in 6 cells, stored cell by cell."""
    rng = np.random.default_rng(seed)
    hr = (cfg["r_out"] - cfg["r_in"]) / cfg["nr"]
    hz = (cfg["z_max"] - cfg["z_min"]) / cfg["nz"]
    cells = np.array([(0, 0), (3, 7), (10, 30), (31, 63), (31, 0), (16, 40)])
    k = np.sort(rng.integers(0, len(cells), n))
    r = cfg["r_in"] + (cells[k, 0] + rng.uniform(0, 1, n)) * hr
    z = cfg["z_min"] + (cells[k, 1] + rng.uniform(0, 1, n)) * hz
    v = rng.normal(0, 3e6, (3, n))
    return r, z, v[0], v[1], v[2], np.arange(n, dtype=np.uint64)


def _drifted(cfg, n, seed):
    """n electrons as a cell-sorted store some steps after its sort: stored
    in the cell order of their positions, then each moved by up to two
    cells, so that 32-slot tiles hold a few cells each; a quarter of them
    in four crowded cells (tiles of one or two cells)."""
    rng = np.random.default_rng(seed)
    hr = (cfg["r_out"] - cfg["r_in"]) / cfg["nr"]
    hz = (cfg["z_max"] - cfg["z_min"]) / cfg["nz"]
    r = rng.uniform(cfg["r_in"], cfg["r_out"], n)
    z = rng.uniform(cfg["z_min"], cfg["z_max"], n)
    crowd = rng.random(n) < 0.25
    pick = rng.integers(0, 4, n)
    r[crowd] = cfg["r_in"] + (np.array([1, 2, cfg["nr"] // 2, cfg["nr"] - 1])[pick[crowd]]
                              + rng.uniform(0, 1, crowd.sum())) * hr
    z[crowd] = cfg["z_min"] + (np.array([0, 5, cfg["nz"] // 2, cfg["nz"] - 1])[pick[crowd]]
                               + rng.uniform(0, 1, crowd.sum())) * hz
    ir = np.minimum(((r - cfg["r_in"]) / hr).astype(np.int64), cfg["nr"] - 1)
    iz = np.minimum(((z - cfg["z_min"]) / hz).astype(np.int64), cfg["nz"] - 1)
    order = np.argsort(ir * (cfg["nz"] + 1) + iz, kind="stable")
    r, z = r[order], z[order]
    move = ~crowd[order]
    r[move] = np.clip(r[move] + rng.uniform(-2, 2, move.sum()) * hr, cfg["r_in"] + 1e-3 * hr,
                      cfg["r_out"] - 1e-3 * hr)
    z[move] = np.clip(z[move] + rng.uniform(-2, 2, move.sum()) * hz, cfg["z_min"] + 1e-3 * hz,
                      cfg["z_max"] - 1e-3 * hz)
    v = rng.normal(0, 3e6, (3, n))
    return r, z, v[0], v[1], v[2], np.arange(n, dtype=np.uint64)


def _layout(cfg, layout, n, seed):
    if layout == "scattered":
        return seed_particles(cfg, n=n, seed=seed)
    return (_clustered if layout == "clustered" else _drifted)(cfg, n, seed + 1)


@pytest.mark.parametrize("precision,layout,bkind", [(64, "scattered", 0), (64, "clustered", 1),
                                                    (32, "scattered", 1), (32, "clustered", 0),
                                                    (64, "drifted", 0), (32, "drifted", 1)])
def test_loaded_moments_match_oracle(precision, layout, bkind):
    cfg = _cfg(precision, bfield_kind=bkind)
    n = 20_000 + 37
    parts = _layout(cfg, layout, n, 21)
    sim = make_gpu(cfg, parts)
    got = sim.moments()
    w = sim.diagnostics()["weight"]
    sim.close()
    w_or = oracle.derived(cfg)["weight"]
    assert w == pytest.approx(w_or, rel=1e-14)
    want = fluid.moments(cfg, *parts[:5], w_or)
    _compare_moments(got, want, MOM_TOL[precision])


@pytest.mark.parametrize("precision", [64, 32])
def test_moments_on_the_widest_grid(precision):
    """nz = 4096 cells, the library's limit, and 300 radial cells: the walk
    packs the cell (ir, iz) in 32-bit sort keys."""
    cfg = _cfg(precision, nr=300, nz=4096)
    parts = _drifted(cfg, 30_000 + 11, 71)
    sim = make_gpu(cfg, parts)
    got = sim.moments()
    sim.close()
    want = fluid.moments(cfg, *parts[:5], oracle.derived(cfg)["weight"])
    _compare_moments(got, want, MOM_TOL[precision])


def test_empty_simulation_has_zero_moments():
    cfg = _cfg(64)
    parts = seed_particles(cfg, n=0, seed=1)
    sim = make_gpu(cfg, parts)
    M = sim.moments()
    sim.close()
    assert M.shape == (fluid.MOMENTS, cfg["nr"] + 1, cfg["nz"] + 1) and not M.any()


def test_stepped_moments_match_oracle():
    """After two steps in a fixed field (collisions, absorption at the
    walls, freed slots), FP64."""
    cfg = _cfg(64, p_mbar=3.0, T0_eV=60.0)
    n = 20_000
    parts = seed_particles(cfg, n=n, seed=31)
    er, ez = random_field_node_arrays(cfg, 3e5, seed=32)
    o = oracle.OracleSim(cfg, *parts, efield_nodes=(er, ez), solve_field=False)
    sim = make_gpu(cfg, parts, efield=(er, ez))
    amb = 0
    for _ in range(2):
        res = o.step()
        amb += int((res.margin < 1e-13).sum())
    sim.step(2)
    got = sim.moments()
    d = sim.diagnostics()
    sim.close()
    assert amb == 0
    assert d["n_absorbed"] > 0
    want = fluid.moments(cfg, o.r, o.z, o.vr, o.vt, o.vz, oracle.derived(cfg)["weight"])
    _compare_moments(got, want, 1e-11)


@pytest.mark.parametrize("precision", [64, 32])
def test_moments_with_tabulated_cross_sections(precision):
    cfg = _cfg(precision, T0_eV=80.0)
    E, sel, sio, xi = cross_section_tables(cfg["ion_E_th_eV"])
    parts = seed_particles(cfg, n=12_000, seed=41)
    sim = make_gpu(cfg, parts)
    sim.set_cross_sections(E, sel, sio, xi)
    got = sim.moments()
    sim.close()
    c_or = dict(cfg, xs=dict(E_eV=E, sigma_el=sel, sigma_io=sio, xi=xi))
    want = fluid.moments(c_or, *parts[:5], oracle.derived(cfg)["weight"])
    _compare_moments(got, want, MOM_TOL[precision])
    # the tables change the drag moment
    plain = fluid.moments(cfg, *parts[:5], oracle.derived(cfg)["weight"])
    assert np.abs(plain[10] - want[10]).max() > 1e-3 * np.abs(want[10]).max()


def test_batch_member_moments():
    from paper_2206_14662_gb300._capi import Simulation
    # batch members share geometry, step, solver settings and seed; the gas
    # pressure differs, and with it the drag moment
    cfgs = [_cfg(64, p_mbar=p) for p in (1.0, 4.0)]
    parts = [seed_particles(c, n=5000 + 700 * k, seed=50 + k) for k, c in enumerate(cfgs)]
    with Simulation(cfgs) as sim:
        for k in range(2):
            sim.load_particles(*parts[k], sim=k)
        got = [sim.moments(sim=k) for k in range(2)]
    for k in range(2):
        want = fluid.moments(cfgs[k], *parts[k][:5], oracle.derived(cfgs[k])["weight"])
        _compare_moments(got[k], want, MOM_TOL[64])


# force terms: relative to each term's largest magnitude.  Both sides work in
# FP64 from the same moments; the FP32 simulation holds E in FP32.
@pytest.mark.parametrize("precision,bkind", [(64, 0), (64, 1), (32, 1)])
def test_force_terms_match_oracle(precision, bkind):
    cfg = _cfg(precision, bfield_kind=bkind, b0=0.03)
    w = oracle.derived(cfg)["weight"]
    parts = seed_particles(cfg, n=30_000, seed=61)
    M = fluid.moments(cfg, *parts[:5], w)
    parts2 = seed_particles(cfg, n=30_000, seed=62)
    M_prev = fluid.moments(cfg, *parts2[:5], w)
    er, ez = random_field_node_arrays(cfg, 2e4, seed=63)
    sim = make_gpu(cfg, seed_particles(cfg, n=100, seed=64), efield=(er, ez))
    dt = 2e-12
    got = sim.force_balance(M, M_prev, dt)
    got0 = sim.force_balance(M)
    sim.close()
    want = fluid.force_terms(cfg, M, er, ez, M_prev=M_prev, dt_prev=dt)
    assert got.shape == want.shape == (7, 3, cfg["nr"] + 1, cfg["nz"] + 1)
    field_tol = 1e-10 if precision == 64 else 1e-6
    for t, name in enumerate(fluid.TERMS):
        for a in range(3):
            scale = np.abs(want[t, a]).max()
            if scale == 0:
                assert not got[t, a].any(), (name, a)
                continue
            tol = field_tol if name in ("F_E", "sum") else 1e-10
            err = np.abs(got[t, a] - want[t, a]).max() / scale
            assert err <= tol, (name, a, err)
    assert not got0[5].any()
    assert np.array_equal(got0[:5], got[:5])


def test_force_balance_argument_checks():
    from paper_2206_14662_gb300._capi import PicError
    cfg = _cfg(64)
    sim = make_gpu(cfg, seed_particles(cfg, n=100, seed=1))
    M = sim.moments()
    with pytest.raises(PicError):
        sim.force_balance(M, M, 0.0)
    with pytest.raises(PicError):
        sim.force_balance(M, M, -1.0)
    sim.close()


def test_full_size_partition_of_unity():
    """Mirror workload, 128 x 512 cells, 1e7 electrons, FP32, three solved
    steps: sum_i V_i M_c(i) = w sum_p g_c(v_p) over the live particles, to
    the FP32 arithmetic of the FP32 path."""
    cfg = workload("mirror_128x512_1e7")
    parts = seed_particles(cfg)
    sim = make_gpu(cfg, parts)
    sim.step(3)
    M = sim.moments()
    d = sim.diagnostics()
    g = sim.export_particles()
    sim.close()
    V = oracle.node_volumes(cfg).reshape(cfg["nr"] + 1, cfg["nz"] + 1)
    w = oracle.derived(cfg)["weight"]
    assert g["uid"].size > 0.5 * len(parts[0]) and d["error"] == 0
    vr, vt, vz = g["vr"], g["vt"], g["vz"]
    sums = [np.full(vr.size, 1.0), vr, vt, vz, vr * vr, vr * vt, vr * vz, vt * vt, vt * vz, vz * vz]
    for c, s in enumerate(sums):
        want = w * s.sum()
        got = (M[c] * V).sum()
        # FP32 simulation: products, short sums and w / V in FP32
        assert got == pytest.approx(want, rel=1e-6, abs=1e-6 * w * np.abs(s).sum()), c
    assert (M[10] >= 0).all() and M[10].sum() > 0
    assert (M[11] >= 0).all() and (M[11] <= M[10] * (1 + 1e-12)).all()


def test_force_balance_refuses_a_wrong_shape():
    cfg = _cfg(64)
    sim = make_gpu(cfg, seed_particles(cfg, n=10, seed=1))
    M = sim.moments()
    with pytest.raises(ValueError):
        sim.force_balance(M[:, :-1])
    with pytest.raises(ValueError):
        sim.force_balance(M, M[:10], 1e-12)
    sim.close()


@pytest.mark.parametrize("precision,bkind", [(64, 0), (64, 1), (32, 1)])
def test_fluid_model_matches_oracle(precision, bkind):
    """Fluid-Poisson model grids (pic_fluid_model) from the oracle's moments
    of a hot load (ionising speeds present) and a random node field."""
    cfg = _cfg(precision, bfield_kind=bkind, b0=0.05, T0_eV=120.0)
    w = oracle.derived(cfg)["weight"]
    parts = seed_particles(cfg, n=30_000, seed=71)
    M = fluid.moments(cfg, *parts[:5], w)
    assert M[11].sum() > 0
    er, ez = random_field_node_arrays(cfg, 3e5, seed=72)
    sim = make_gpu(cfg, seed_particles(cfg, n=100, seed=73), efield=(er, ez))
    got = sim.fluid_model(M)
    sim.close()
    want = fluid.fluid_model(cfg, M, er, ez)
    assert got.shape == want.shape == (9, cfg["nr"] + 1, cfg["nz"] + 1)
    tol = 1e-12 if precision == 64 else 1e-5
    for k, name in enumerate(fluid.FLUID_MODEL):
        scale = np.abs(want[k]).max()
        assert scale > 0, name
        err = np.abs(got[k] - want[k]).max() / scale
        assert err <= tol, (name, err)
    # the drift speeds reach the ionising range somewhere
    assert want[7].max() > 0


def test_accumulated_moments_average_snapshots():
    """pic_moments_accumulate adds scale x the moments into a device array:
    halves of a loaded state's moments sum to the oracle's; a time average
    of three snapshots equals the mean of three pic_moments calls."""
    import torch
    cfg = _cfg(64, fixed_efield=0, sort_every=2)
    parts = seed_particles(cfg, n=15_000, seed=81)
    sim = make_gpu(cfg, parts)
    shape = (fluid.MOMENTS, cfg["nr"] + 1, cfg["nz"] + 1)
    acc = torch.zeros(shape, dtype=torch.float64, device="cuda")
    sim.moments_accumulate(acc, 0.5)
    sim.moments_accumulate(acc, 0.5)
    got = acc.cpu().numpy()
    want = fluid.moments(cfg, *parts[:5], oracle.derived(cfg)["weight"])
    _compare_moments(got, want, MOM_TOL[64])
    acc.zero_()
    snaps = []
    for _ in range(3):
        sim.step(3)
        sim.moments_accumulate(acc, 1.0 / 3.0)
        snaps.append(sim.moments())
    avg = acc.cpu().numpy()
    _compare_moments(avg, sum(snaps) / 3.0, 1e-13)
    with pytest.raises(ValueError):
        sim.moments_accumulate(acc.float(), 1.0)
    with pytest.raises(ValueError):
        sim.moments_accumulate(acc.cpu(), 1.0)
    sim.close()
