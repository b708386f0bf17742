"""Pins of the CPU oracle against facts fixed by the paper's method and by
mathematics, independent of the oracle's own code (CPU only).

Each test names the passage it follows: the PIC cycle, Boris push, absorbing
walls and finite-element Poisson problem of Sec. II.A; the seed load of Sec.
II.A / III.A; the ExB drift u_theta = -E_r/B_z of Sec. IV.A; the collision
frequency n_n sigma v of Sec. IV.B; the Monte-Carlo collision module of
Sec. II.A.
"""
import os

import numpy as np
import pytest
from scipy import integrate, stats

from paper_2206_14662_gb300.inputs import seed_particles, workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def one_particle(oracle, cfg, r, z, vr, vt, vz, er=None, ez=None, uid=0):
    nn = (cfg["nr"] + 1) * (cfg["nz"] + 1)
    if er is None:
        er, ez = np.zeros(nn), np.zeros(nn)
    return oracle.OracleSim(cfg, [r], [z], [vr], [vt], [vz], [uid],
                            efield_nodes=(er, ez), solve_field=False)


# --------------------------------------------------------------- Philox

def test_philox_known_answers(oracle_mod):
    """Philox4x32-10 reproduces the published known-answer vectors."""
    n = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            out = oracle_mod.philox4x32_10(w[0:4], w[4:6])
            assert list(out) == w[6:10]
            n += 1
    assert n == 3


def test_philox_uniforms_chi2(oracle_mod):
    """Uniforms ((x >> 8) + 0.5) 2^-24 from consecutive counters pass a
    64-bin chi-square test and lie strictly inside (0, 1)."""
    u = []
    for c in range(4000):
        x = oracle_mod.philox4x32_10([c, 0, 17, 0], [1, 0])
        u.extend(((x >> 8).astype(np.float64) + 0.5) / 2 ** 24)
    u = np.array(u)
    assert u.min() > 0 and u.max() < 1
    counts, _ = np.histogram(u, bins=64, range=(0, 1))
    chi2 = ((counts - len(u) / 64) ** 2 / (len(u) / 64)).sum()
    assert stats.chi2.sf(chi2, 63) > 1e-4


# -------------------------------------------------------------- Poisson

def test_node_volumes_sum_to_gap_volume(oracle_mod):
    cfg = workload("coax_32x64_1e4")
    V = oracle_mod.node_volumes(cfg)
    a, b, L = cfg["r_in"], cfg["r_out"], cfg["z_max"] - cfg["z_min"]
    assert V.sum() == pytest.approx(np.pi * (b * b - a * a) * L, rel=1e-13)
    assert (V > 0).all()


def test_poisson_vacuum_exact_discrete(oracle_mod):
    """With no charge the discrete solution is z-independent and equals
    V_in + (V_out - V_in) S_i / S_nr, S_i = sum_{k<i} 1 / r_{k+1/2}: every
    bilinear element carries the same radial flux (r0 + r1)/(2h) dphi."""
    for name, nr, nz in (("coax_32x64_1e4", 32, 64), ("coax_32x64_1e4", 17, 9)):
        cfg = workload(name, nr=nr, nz=nz)
        phi = oracle_mod.poisson_solve(cfg, np.zeros((nr + 1) * (nz + 1))).reshape(nr + 1, nz + 1)
        r, _ = oracle_mod.grid(cfg)
        S = np.concatenate([[0.0], np.cumsum(2.0 / (r[1:] + r[:-1]))])
        exact = cfg["v_inner"] + (cfg["v_outer"] - cfg["v_inner"]) * S / S[-1]
        assert np.abs(phi - exact[:, None]).max() <= 1e-12 * abs(cfg["v_inner"])


def _order(errors):
    return np.log2(np.array(errors[:-1]) / np.array(errors[1:]))


def test_poisson_vacuum_continuum_second_order(oracle_mod):
    """phi(r) -> V_in + (V_out - V_in) ln(r/a)/ln(b/a) at second order."""
    errs = []
    for nr in (32, 64, 128):
        cfg = workload("coax_32x64_1e4", nr=nr, nz=8)
        phi = oracle_mod.poisson_solve(cfg, np.zeros((nr + 1) * 9)).reshape(nr + 1, 9)
        r, _ = oracle_mod.grid(cfg)
        a, b = cfg["r_in"], cfg["r_out"]
        cont = cfg["v_inner"] + (cfg["v_outer"] - cfg["v_inner"]) * np.log(r / a) / np.log(b / a)
        errs.append(np.abs(phi[:, 4] - cont).max())
    assert np.all(np.abs(_order(errs) - 2.0) < 0.1)


def test_poisson_uniform_charge_second_order(oracle_mod):
    """Uniform rho0 in the gap: b_i = rho0 V_i, and
    phi = -rho0 r^2 / (4 eps0) + C1 ln r + C2 with both Dirichlet values."""
    rho0 = -1.0e15 * oracle_mod.QE * 50
    errs = []
    for nr in (16, 32, 64, 128):
        cfg = workload("coax_32x64_1e4", nr=nr, nz=6)
        b = rho0 * oracle_mod.node_volumes(cfg)
        phi = oracle_mod.poisson_solve(cfg, b).reshape(nr + 1, 7)
        r, _ = oracle_mod.grid(cfg)
        a, bb = cfg["r_in"], cfg["r_out"]
        Va, Vb = cfg["v_inner"], cfg["v_outer"]
        p = lambda x: -rho0 * x * x / (4 * oracle_mod.EPS0)
        C1 = ((Vb - p(bb)) - (Va - p(a))) / np.log(bb / a)
        C2 = Va - p(a) - C1 * np.log(a)
        exact = p(r) + C1 * np.log(r) + C2
        assert np.ptp(phi, axis=1).max() < 1e-9 * np.abs(phi).max()   # z-independent
        errs.append(np.abs(phi[:, 3] - exact).max())
    assert np.all(np.abs(_order(errs) - 2.0) < 0.15)


def test_poisson_solution_satisfies_fem_system(oracle_mod):
    """A random right-hand side: phi meets the Dirichlet values and the
    interior rows of 2 pi eps0 (K_r (x) M_z + M_r (x) K_z) phi = b."""
    cfg = workload("coax_32x64_1e4", nr=12, nz=20)
    rng = np.random.default_rng(3)
    b = rng.standard_normal(13 * 21) * 1e-12
    phi = oracle_mod.poisson_solve(cfg, b)
    A = oracle_mod.fem_matrix(cfg).toarray()
    f = phi.reshape(13, 21)
    assert np.all(f[0] == cfg["v_inner"]) and np.all(f[-1] == cfg["v_outer"])
    res = (A @ phi - b).reshape(13, 21)[1:-1]
    assert np.abs(res).max() < 1e-10 * np.abs(b).max()
    assert oracle_mod.poisson_relres(cfg, b, phi) < 1e-13
    # the matrix is symmetric and its row sums vanish (constants are harmonic)
    assert np.abs(A - A.T).max() < 1e-25
    assert np.abs(A.sum(axis=1)).max() < 1e-22


def test_efield_vacuum_second_order(oracle_mod):
    """E_r -> (V_in - V_out) / (r ln(b/a)) at second order, E_z = 0.  The
    1/r field is steep at r = a = 1 mm, so the order is taken on fine grids
    (the one-sided wall difference is the largest error and is second order
    too; the order rises towards 2 as h shrinks)."""
    errs = []
    for nr in (128, 256, 512):
        cfg = workload("coax_32x64_1e4", nr=nr, nz=8)
        phi = oracle_mod.poisson_solve(cfg, np.zeros((nr + 1) * 9))
        er, ez = oracle_mod.efield(cfg, phi)
        r, _ = oracle_mod.grid(cfg)
        exact = (cfg["v_inner"] - cfg["v_outer"]) / (r * np.log(cfg["r_out"] / cfg["r_in"]))
        errs.append(np.abs(er.reshape(nr + 1, 9)[:, 4] - exact).max() / np.abs(exact).max())
        assert np.abs(ez).max() < 1e-6 * np.abs(er).max()
    orders = _order(errs)
    assert np.all(np.abs(orders - 2.0) < 0.15) and orders[1] > orders[0]


# -------------------------------------------------------------- deposit

def test_deposit_conserves_charge(oracle_mod):
    """sum_i b_i = q w N (partition of unity of the bilinear hats)."""
    cfg = workload("coax_32x64_1e4")
    r, z, *_ = seed_particles(cfg, n=20000)
    b = oracle_mod.deposit(cfg, r, z)
    w = oracle_mod.derived(cfg)["weight"]
    total = -oracle_mod.QE * w * len(r)
    assert abs(b.sum() - total) <= 1e-13 * abs(total)
    assert (b <= 0).all()


def test_deposit_on_a_node_goes_to_that_node(oracle_mod):
    cfg = workload("coax_32x64_1e4")
    rg, zg = oracle_mod.grid(cfg)
    b = oracle_mod.deposit(cfg, [rg[5]], [zg[9]])
    k = 5 * (cfg["nz"] + 1) + 9
    w = oracle_mod.derived(cfg)["weight"]
    assert b[k] == pytest.approx(-oracle_mod.QE * w, rel=1e-13)
    # a node coordinate may round to the far side of a cell edge: what lands
    # on the neighbours is rounding only
    assert np.abs(b).sum() - abs(b[k]) < 1e-13 * abs(b[k])


def test_deposit_density_of_uniform_load(oracle_mod):
    """A volume-uniform load of n0 deposits density ~ n0 on interior nodes."""
    cfg = workload("coax_32x64_1e4", nr=8, nz=8, n_init=400_000)
    r, z, *_ = seed_particles(cfg)
    n = oracle_mod.density(cfg, oracle_mod.deposit(cfg, r, z)).reshape(9, 9)
    inner = n[1:-1, 1:-1]
    assert abs(inner.mean() / cfg["n0"] - 1) < 0.01
    assert abs(n[0, 1:-1].mean() / cfg["n0"] - 1) < 0.05   # wall nodes too


# ------------------------------------------------------------------ push

def test_boris_gyration_closed_form(oracle_mod):
    """E = 0, uniform B: each step rotates the Cartesian velocity by
    2 atan(Omega dt / 2) and the positions close a polygon of radius
    (v_perp / Omega) sqrt(1 + (Omega dt / 2)^2).  The cylindrical push must
    reproduce that Cartesian orbit (|x_n|, and v in the local basis)."""
    cfg = workload("coax_32x64_1e4", p_mbar=0.0)
    QE, ME = oracle_mod.QE, oracle_mod.ME
    r0, v = 5e-3, 3e6
    s = one_particle(oracle_mod, cfg, r0, 0.0, 0.3 * v, 0.9 * v, 1e4)
    Om = QE * cfg["b0"] / ME
    dt = cfg["dt"]
    th = 2 * np.arctan(Om * dt / 2)
    v0 = complex(0.3 * v, 0.9 * v)
    R = abs(v0) / Om * np.sqrt(1 + (Om * dt / 2) ** 2)
    n = np.arange(1, 1001)
    # closed-form geometric sum of the rotated velocities
    vel = v0 * np.exp(1j * th * n)
    K = dt * v0 * np.exp(1j * th) / (np.exp(1j * th) - 1)
    x = r0 + K * (np.exp(1j * th * n) - 1)     # electron turns counter-clockwise
    centre = r0 - K
    rs, vrs, vts = [], [], []
    for _ in n:
        s.step()
        rs.append(s.r[0]); vrs.append(s.vr[0]); vts.append(s.vt[0])
    rs, vrs, vts = map(np.array, (rs, vrs, vts))
    assert np.abs(rs - np.abs(x)).max() < 1e-12 * r0
    loc = vel / (x / np.abs(x))
    assert np.abs(vrs - loc.real).max() < 1e-12 * v
    assert np.abs(vts - loc.imag).max() < 1e-12 * v
    assert np.abs(np.abs(x - centre) - R).max() < 1e-9 * R
    assert np.abs(np.hypot(vrs, vts) - abs(v0)).max() < 1e-12 * v


def test_exb_drift(oracle_mod):
    """Uniform E_r, uniform B_z on a thin annulus at r = 1 m: the drift is
    u_theta = -E_r / B_z (Sec. IV.A).  (a) v = E x B / B^2 is a fixed point
    of the Boris map; (b) from rest, the mean over whole Boris periods is the
    drift."""
    cfg = workload("coax_32x64_1e4", r_in=1.0, r_out=1.001, z_min=-0.01, z_max=0.01,
                   nr=4, nz=4, p_mbar=0.0, b0=0.1)
    Om = oracle_mod.QE * 0.1 / oracle_mod.ME
    P = 64
    cfg["dt"] = 2 * np.tan(np.pi / P) / Om          # exactly P steps per gyration
    Er = 1e3
    er, ez = np.full(25, Er), np.zeros(25)
    vd = -Er / cfg["b0"]
    s = one_particle(oracle_mod, cfg, 1.0005, 0.0, 0.0, vd, 0.0, er, ez)
    vt = []
    for _ in range(500):
        s.step(); vt.append(s.vt[0])
    assert np.abs(np.array(vt) / vd - 1).max() < 1e-5   # curvature, O(rho/r)
    s = one_particle(oracle_mod, cfg, 1.0005, 0.0, 0.0, 0.0, 0.0, er, ez)
    vt = []
    for _ in range(P * 50):
        s.step(); vt.append(s.vt[0])
    assert abs(np.mean(vt) / vd - 1) < 1e-5


def test_canonical_angular_momentum_mirror(oracle_mod):
    """Mirror field from A_theta = r B_z(z) / 2 and no E: the canonical
    momentum m r v_theta + q r A_theta oscillates boundedly with no drift."""
    cfg = workload("mirror_128x512_1e7", p_mbar=0.0)
    L = cfg["z_max"] - cfg["z_min"]
    QE, ME = oracle_mod.QE, oracle_mod.ME
    s = one_particle(oracle_mod, cfg, 5e-3, 0.0, 1e6, 2e6, 5e5)
    pt = []
    for _ in range(20000):
        s.step()
        Bz = cfg["b0"] * (1 + 0.5 * (2 * s.z[0] / L) ** 2)
        pt.append(ME * s.r[0] * s.vt[0] - QE * s.r[0] ** 2 * Bz / 2)
    pt = np.array(pt)
    scale = QE * 5e-3 ** 2 * cfg["b0"] / 2
    assert np.ptp(pt) / scale < 5e-3
    assert abs(pt[10000:].mean() - pt[:10000].mean()) / scale < 1e-5


def test_mirror_loss_cone(oracle_mod):
    """Mirror ratio 1.5: from the midplane, pitch angles below
    asin(sqrt(1/1.5)) = 54.7 deg escape through the ends, above are reflected."""
    cfg = workload("mirror_128x512_1e7", p_mbar=0.0)
    v = 5e6
    for deg, escapes in ((45, True), (52, True), (58, False), (70, False)):
        a = np.radians(deg)
        s = one_particle(oracle_mod, cfg, 5e-3, 0.0, v * np.sin(a), 0.0, v * np.cos(a))
        lost_at = None
        for k in range(16000):
            res = s.step()
            if s.n == 0:
                lost_at = res.event[0]
                break
        if escapes:
            assert lost_at in (oracle_mod.EV_WALL + 2, oracle_mod.EV_WALL + 3)
        else:
            assert lost_at is None


def test_absorption_first_crossing(oracle_mod):
    """A particle leaving through the corner is charged to the wall its
    straight (r, z) segment crosses first; the tally counts its weight."""
    cfg = workload("coax_32x64_1e4", p_mbar=0.0, b0=0.0)
    hz = (cfg["z_max"] - cfg["z_min"]) / cfg["nz"]
    b = cfg["r_out"]
    # crosses z_max first (t = 0.25) and r = b later (t = 0.5)
    s = one_particle(oracle_mod, cfg, b - 1e-6, cfg["z_max"] - 1e-6, 2e-6 / 1e-12, 0.0, 4e-6 / 1e-12)
    res = s.step()
    assert res.event[0] == oracle_mod.EV_WALL + 3
    assert res.tally[oracle_mod.T_ABS_ZMAX] == pytest.approx(oracle_mod.derived(cfg)["weight"])
    s = one_particle(oracle_mod, cfg, b - 1e-6, cfg["z_max"] - 4e-6, 4e-6 / 1e-12, 0.0, 2e-6 / 1e-12)
    assert s.step().event[0] == oracle_mod.EV_WALL + 1
    del hz


# ------------------------------------------------------------ collisions

def test_sigma_ion_fit(oracle_mod):
    cfg = workload("coax_32x64_1e4")
    E = np.linspace(0, 2000, 20001)
    s = np.array([oracle_mod.sigma_ion(cfg, e) for e in E])
    assert s[E <= 15.0].max() == 0.0
    assert E[np.argmax(s)] == pytest.approx(100.0, abs=0.1)
    assert s.max() == pytest.approx(1e-20, rel=1e-9)


def test_nu_max_is_a_majorant(oracle_mod):
    """n_n (sigma_el + sigma_io) v <= nu_max on [0, E_cap] (Sec. IV.B: the
    collision frequency n_n sigma v)."""
    cfg = workload("coax_32x64_1e4")
    P = oracle_mod.params(cfg)
    E_cap = 2 * abs(cfg["v_inner"])
    E = np.linspace(0, E_cap, 333_333)
    v = np.sqrt(2 * E * oracle_mod.QE / oracle_mod.ME)
    sig = np.array([oracle_mod.sigma_ion(cfg, e) for e in E[::37]])
    nu = P.n_gas * (cfg["sigma_el"] + sig) * v[::37]
    assert nu.max() <= P.nu_max
    assert nu.max() > P.nu_max / (1 + 2e-6) * (1 - 1e-4)


def _mono_energetic(oracle_mod, cfg, E_eV, N, seed):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((3, N))
    d /= np.linalg.norm(d, axis=0)
    sp = np.sqrt(2 * E_eV * oracle_mod.QE / oracle_mod.ME)
    nn = (cfg["nr"] + 1) * (cfg["nz"] + 1)
    uid = np.arange(N, dtype=np.uint64) + np.uint64(seed * N)
    s = oracle_mod.OracleSim(cfg, np.full(N, 5e-3), np.zeros(N), sp * d[0], sp * d[1], sp * d[2],
                             uid, efield_nodes=(np.zeros(nn), np.zeros(nn)), solve_field=False)
    return s, sp, d


def test_collision_counts_binomial(oracle_mod):
    """One step of N mono-energetic electrons: the elastic and ionisation
    counts are Binomial(N, P_null nu_k(E) / nu_max), nu_k = n_n sigma_k v."""
    cfg = workload("coax_32x64_1e4", p_mbar=10.0, elastic_recoil=0, dt=1e-13)
    N = 200_000
    for k, E_eV in enumerate((10.0, 50.0, 100.0, 300.0, 1000.0)):
        s, sp, _ = _mono_energetic(oracle_mod, cfg, E_eV, N, seed=k + 1)
        res = s.step()
        P = s.P
        p_null = 1 - np.exp(-P.nu_max * P.dt)
        for slot, nu in ((oracle_mod.T_N_ELASTIC, P.n_gas * cfg["sigma_el"] * sp),
                         (oracle_mod.T_N_IONISE, P.n_gas * oracle_mod.sigma_ion(cfg, E_eV) * sp)):
            p = p_null * nu / P.nu_max
            sd = np.sqrt(N * p * (1 - p))
            assert abs(res.tally[slot] - N * p) <= 4 * sd + 1e-9
        assert res.n_children == res.tally[oracle_mod.T_N_IONISE]


def _mu_cdf(xi):
    f = lambda m: (1 - xi * m) ** -2
    Z = integrate.quad(f, -1, 1)[0]
    return lambda x: np.array([integrate.quad(f, -1, t)[0] / Z for t in np.atleast_1d(x)])


@pytest.mark.parametrize("xi", [0.0, 0.5, 0.9])
def test_angle_law(oracle_mod, xi):
    """Scattering angle: cos chi has pdf ~ (1 - xi mu)^-2 (screened-Coulomb
    family of the cited analytic differential cross-section).  Mean against
    the closed form, full distribution against the numerically integrated
    CDF (KS), unit length, azimuth uniform."""
    rng = np.random.default_rng(11)
    vhat = np.array([0.3, -0.5, 0.81])
    vhat /= np.linalg.norm(vhat)
    n = 4000
    mus, phis = [], []
    e1 = np.cross(vhat, [0, 0, 1.0]); e1 /= np.linalg.norm(e1)
    e2 = np.cross(vhat, e1)
    for _ in range(n):
        d = oracle_mod.scatter_dir(vhat, rng.random(), rng.random(), xi)
        assert abs(np.linalg.norm(d) - 1) < 1e-12
        mus.append(d @ vhat)
        phis.append(np.arctan2(d @ e2, d @ e1))
    mus = np.array(mus)
    mean = 0.0 if xi == 0 else 1 / xi - (1 - xi ** 2) / (2 * xi ** 2) * np.log((1 + xi) / (1 - xi))
    sd = mus.std() / np.sqrt(n)
    assert abs(mus.mean() - mean) < 4 * sd
    assert stats.kstest(mus, _mu_cdf(xi)).pvalue > 1e-3
    assert stats.kstest((np.array(phis) + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-3


def test_opal_secondary_energy(oracle_mod):
    """Secondary energy: pdf ~ 1/(1 + (E2/B)^2) on [0, E_rem/2] (Opal-type
    energy sharing), checked against the numerically integrated CDF."""
    rng = np.random.default_rng(5)
    E_rem, B = 185.0, 10.0
    e2 = np.array([oracle_mod.opal_secondary(E_rem, B, u) for u in rng.random(4000)])
    assert e2.min() >= 0 and e2.max() <= E_rem / 2
    f = lambda e: 1 / (1 + (e / B) ** 2)
    Z = integrate.quad(f, 0, E_rem / 2)[0]
    cdf = lambda x: np.array([integrate.quad(f, 0, t)[0] / Z for t in np.atleast_1d(x)])
    assert stats.kstest(e2, cdf).pvalue > 1e-3


def test_ionisation_energy_bookkeeping(oracle_mod):
    """Per ionisation: E1 + E2 = E - E_ion, E2 <= (E - E_ion)/2, one child per
    event at the parent's position, child uids consecutive from uid_next in
    parent-uid order; the ion is not simulated (Sec. II.A)."""
    cfg = workload("coax_32x64_1e4", p_mbar=10.0, elastic_recoil=0, dt=1e-13,
                   sigma_el=1e-22)
    N = 50_000
    E_eV = 200.0
    s, sp, _ = _mono_energetic(oracle_mod, cfg, E_eV, N, seed=21)
    uid_before = s.uid.copy()
    next0 = s.uid_next
    res = s.step()
    ion = np.nonzero(res.event == oracle_mod.EV_IONISE)[0]
    assert len(ion) == res.n_children > 20
    parents_uid = uid_before[ion]
    assert np.all(np.diff(parents_uid.astype(np.int64)) > 0)
    children = np.arange(next0, next0 + len(ion), dtype=np.uint64)
    cidx = np.searchsorted(s.uid, children)
    pidx = np.searchsorted(s.uid, parents_uid)
    ME, QE = oracle_mod.ME, oracle_mod.QE
    KE = lambda i: 0.5 * ME * (s.vr[i] ** 2 + s.vt[i] ** 2 + s.vz[i] ** 2) / QE
    E1, E2 = KE(pidx), KE(cidx)
    E_rem = E_eV - cfg["ion_E_th_eV"]
    assert np.abs(E1 + E2 - E_rem).max() < 1e-12 * E_eV
    assert E2.max() <= E_rem / 2 * (1 + 1e-12)
    assert np.all(s.r[cidx] == s.r[pidx]) and np.all(s.z[cidx] == s.z[pidx])
    assert res.tally[oracle_mod.T_ION_LOSS] == pytest.approx(
        len(ion) * oracle_mod.derived(cfg)["weight"] * cfg["ion_E_th_eV"] * QE)


def test_energy_ledger(oracle_mod):
    """Over a self-consistent run with collisions and wall losses:
    KE_now - KE_0 = W_E - KE_absorbed - n_io E_ion - recoil loss, where W_E
    is the work of the two half kicks per step (the magnetic rotation and the
    frame rotation keep |v|)."""
    cfg = workload("coax_32x64_1e4", p_mbar=1.0, n_init=3000, T0_eV=50.0)
    parts = seed_particles(cfg)
    s = oracle_mod.OracleSim(cfg, *parts)
    for _ in range(60):
        s.step()
    t = s.tally
    assert t[oracle_mod.T_N_ABSORBED] > 0 and t[oracle_mod.T_N_ELASTIC] > 0
    scale = abs(t[oracle_mod.T_WORK_E]) + s.ke0 + t[oracle_mod.T_KE_ABSORBED]
    assert abs(s.ledger_residual()) < 1e-11 * scale


def test_seed_load_statistics():
    """The input recipe: volume-uniform r (r^2 uniform on [a^2, b^2]),
    uniform z, Maxwellian components of variance k T0 / m_e."""
    cfg = workload("coax_32x64_1e4")
    r, z, vr, vt, vz, uid = seed_particles(cfg, n=100_000)
    a, b = cfg["r_in"], cfg["r_out"]
    assert stats.kstest((r ** 2 - a * a) / (b * b - a * a), "uniform").pvalue > 1e-3
    assert stats.kstest((z - cfg["z_min"]) / (cfg["z_max"] - cfg["z_min"]), "uniform").pvalue > 1e-3
    sig = np.sqrt(cfg["T0_eV"] * 1.602176634e-19 / 9.1093837015e-31)
    for v in (vr, vt, vz):
        assert stats.kstest(v / sig, "norm").pvalue > 1e-3
    assert np.all(uid == np.arange(100_000))


# ------------------------------------------------------ seed source (II.A)

def test_seed_source_distribution(oracle_mod):
    """The volumetric seed source: r^2 uniform on [a^2, b^2] (uniform in
    volume), z uniform, each velocity component normal with variance
    e T0 / m_e, components uncorrelated."""
    oracle = oracle_mod
    import scipy.stats as ss
    cfg = workload("coax_32x64_1e4", T0_eV=4.0)
    k = 20000
    r, z, vr, vt, vz = oracle.source(cfg, k, uid0=123, step=7)
    a, b = cfg["r_in"], cfg["r_out"]
    assert (r > a).all() and (r < b).all()
    assert (z > cfg["z_min"]).all() and (z < cfg["z_max"]).all()
    assert ss.kstest((r * r - a * a) / (b * b - a * a), "uniform").pvalue > 1e-3
    assert ss.kstest((z - cfg["z_min"]) / (cfg["z_max"] - cfg["z_min"]), "uniform").pvalue > 1e-3
    vth = np.sqrt(oracle.QE * 4.0 / oracle.ME)
    for v in (vr, vt, vz):
        assert ss.kstest(v / vth, "norm").pvalue > 1e-3
    c = np.corrcoef(np.vstack([vr, vt, vz, r, z]))
    assert np.abs(c - np.eye(5)).max() < 4.0 / np.sqrt(k)


def test_seed_source_streams_and_counts(oracle_mod):
    """Source particles depend only on (seed, uid, step): the same call
    repeats, another step or uid differs; OracleSim injects
    floor(rate dt steps) particles (the fraction carried in FP64) with
    consecutive uids after the loaded ones, and the energy ledger accounts
    for the energy they bring."""
    oracle = oracle_mod
    cfg = workload("coax_32x64_1e4", fixed_efield=1, p_mbar=0.0)
    x1 = oracle.source(cfg, 5, 40, 3)
    assert all(np.array_equal(p, q) for p, q in zip(x1, oracle.source(cfg, 5, 40, 3)))
    assert not np.array_equal(x1[0], oracle.source(cfg, 5, 40, 4)[0])
    assert np.array_equal(x1[0][1:], oracle.source(cfg, 4, 41, 3)[0])
    cfg["source_rate"] = 0.37 / cfg["dt"]
    parts = seed_particles(cfg, n=50, margin_cells=4)
    nn = (cfg["nr"] + 1) * (cfg["nz"] + 1)
    o = oracle.OracleSim(cfg, *parts, efield_nodes=(np.zeros(nn), np.zeros(nn)), solve_field=False)
    for _ in range(100):
        o.step()
    assert abs(o.n_source - 37) <= 1
    assert np.array_equal(np.sort(o.uid)[-o.n_source:] if o.n_source else [],
                          np.arange(50, 50 + o.n_source, dtype=np.uint64))
    assert abs(o.ledger_residual()) <= 1e-12 * max(o.kinetic_energy(), 1e-30) + 1e-25


def test_cross_section_table_rule(oracle_mod):
    """Tabulated cross sections: the table's own values at its energies,
    the mean of two neighbours half-way between them, the end values held
    outside the table, and the constant xi when the table has none."""
    oracle = oracle_mod
    cfg = workload("coax_32x64_1e4")
    E = np.array([0.0, 10.0, 30.0, 100.0])
    sel = np.array([4e-20, 2e-20, 1e-20, 5e-21])
    sio = np.array([0.0, 0.0, 3e-21, 1e-21])
    xi = np.array([0.0, 0.2, 0.4, 0.5])
    cfg["xs"] = dict(E_eV=E, sigma_el=sel, sigma_io=sio, xi=xi)
    for k in range(4):
        assert oracle.xs_lookup(cfg, E[k]) == pytest.approx((sel[k], sio[k], xi[k]), rel=1e-15)
    for k in range(3):
        mid = 0.5 * (E[k] + E[k + 1])
        want = (0.5 * (sel[k] + sel[k + 1]), 0.5 * (sio[k] + sio[k + 1]), 0.5 * (xi[k] + xi[k + 1]))
        assert oracle.xs_lookup(cfg, mid) == pytest.approx(want, rel=1e-14)
    assert oracle.xs_lookup(cfg, -5.0) == pytest.approx((sel[0], sio[0], xi[0]))
    assert oracle.xs_lookup(cfg, 1e6) == pytest.approx((sel[-1], sio[-1], xi[-1]))
    cfg["xs"] = dict(E_eV=E, sigma_el=sel, sigma_io=sio, xi=None)
    assert oracle.xs_lookup(cfg, 20.0)[2] == cfg["xi_param"]


def test_dense_table_of_the_analytic_fit_gives_its_majorant(oracle_mod):
    """A table sampled finely from the config's analytic cross sections
    (constant elastic, the ionisation fit) interpolates them to within the
    linear-interpolation error h^2 max|f''| / 8 and gives the same
    collision majorant to 1e-5."""
    oracle = oracle_mod
    cfg = workload("coax_32x64_1e4", p_mbar=1.0)
    # up to the majorant's energy cap 2 |V_in - V_out|, beyond which the
    # table's last value would hold
    E_cap = 2.0 * abs(cfg["v_inner"] - cfg["v_outer"])
    E = np.unique(np.concatenate([np.linspace(0.0, E_cap, 40001), [cfg["ion_E_th_eV"]]]))
    sio = np.array([oracle.sigma_ion(cfg, e) for e in E])
    tab = dict(cfg, xs=dict(E_eV=E, sigma_el=np.full_like(E, cfg["sigma_el"]), sigma_io=sio))
    rng = np.random.default_rng(5)
    h = np.diff(E).max()
    for e in rng.uniform(0.0, E_cap, 200):
        se, si, _ = oracle.xs_lookup(tab, e)
        assert se == pytest.approx(cfg["sigma_el"], rel=1e-15)
        # second derivative of the fit is at most 2 sigma_pk / (E_pk - E_th)^2 in size
        bound = h * h / 8.0 * 2.0 * cfg["ion_sigma_pk"] / (cfg["ion_E_pk_eV"] - cfg["ion_E_th_eV"]) ** 2
        assert abs(si - oracle.sigma_ion(cfg, e)) <= bound + 1e-35
    assert oracle.nu_max(tab) == pytest.approx(oracle.nu_max(cfg), rel=1e-5)


def test_table_ionisation_needs_the_binding_energy(oracle_mod):
    """Ionisation counts only above the binding energy, whatever the table
    says: a table whose ionisation cross-section is large only below the
    threshold gives the elastic majorant."""
    oracle = oracle_mod
    cfg = workload("coax_32x64_1e4", p_mbar=1.0)
    Eth = cfg["ion_E_th_eV"]
    E = np.array([0.0, 0.5 * Eth, Eth, 2 * Eth, 1e5])
    sel = np.full(5, 1e-20)
    sio_low = np.array([1e-18, 1e-18, 0.0, 0.0, 0.0])
    a = oracle.nu_max(dict(cfg, xs=dict(E_eV=E, sigma_el=sel, sigma_io=sio_low)))
    b = oracle.nu_max(dict(cfg, xs=dict(E_eV=E, sigma_el=sel, sigma_io=np.zeros(5))))
    assert a == b
    # and above it the table counts
    c = oracle.nu_max(dict(cfg, xs=dict(E_eV=E, sigma_el=sel, sigma_io=sio_low[::-1])))
    assert c > 10 * a
