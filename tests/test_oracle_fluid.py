"""Pins of the oracle's fluid moments and force-balance terms (Sec. IV.A:
the forces on the electron fluid evaluated from moments of the
distribution function) against closed forms: a lone particle at a node or
inside a cell, the partition of unity, a counter-streaming pair's
pressure, rigid rotation, radial expansion, pressure fields whose
divergence is known, the Lorentz force against a plain cross product, the
drag of mono-energetic electrons, the inertia of two snapshots, the mirror
field's vanishing divergence and the isothermal Boltzmann equilibrium,
where the force balance sums to zero.  The fluid-Poisson model's
predictions (Sec. V) against the balance equations they solve."""
import numpy as np
import pytest

import oracle
from oracle import ME, QE, fluid
from paper_2206_14662_gb300.inputs import workload


@pytest.fixture(scope="module")
def cfg():
    oracle.build()
    return workload("coax_32x64_1e4", precision=64)


def _h(cfg):
    return ((cfg["r_out"] - cfg["r_in"]) / cfg["nr"], (cfg["z_max"] - cfg["z_min"]) / cfg["nz"])


def _shape(cfg):
    return cfg["nr"] + 1, cfg["nz"] + 1


def _vol(cfg):
    return oracle.node_volumes(cfg).reshape(_shape(cfg))


def test_lone_particle_on_a_node(cfg):
    """A particle on node (i, j): only that node sees it, with weight w / V_ij."""
    hr, hz = _h(cfg)
    i, j, w = 7, 11, 3.5e4
    r = cfg["r_in"] + i * hr
    z = cfg["z_min"] + j * hz
    v = (2e5, -3e5, 4e5)
    M = fluid.moments(cfg, [r], [z], [v[0]], [v[1]], [v[2]], w)
    V = _vol(cfg)[i, j]
    expect = [1, v[0], v[1], v[2], v[0] * v[0], v[0] * v[1], v[0] * v[2], v[1] * v[1],
              v[1] * v[2], v[2] * v[2]]
    for c, g in enumerate(expect):
        assert M[c, i, j] == pytest.approx(w * g / V, rel=1e-9)
        other = M[c].copy()
        other[i, j] = 0
        assert np.abs(other).max() <= 1e-9 * abs(M[c, i, j])


def test_particle_at_a_cell_centre_splits_evenly(cfg):
    hr, hz = _h(cfg)
    i, j, w = 4, 20, 1.0
    r = cfg["r_in"] + (i + 0.5) * hr
    z = cfg["z_min"] + (j + 0.5) * hz
    M = fluid.moments(cfg, [r], [z], [0.0], [0.0], [0.0], w)
    V = _vol(cfg)
    for di in (0, 1):
        for dj in (0, 1):
            assert M[0, i + di, j + dj] * V[i + di, j + dj] == pytest.approx(0.25, rel=1e-12)
    assert np.count_nonzero(M[0]) == 4


def test_partition_of_unity(cfg):
    """sum_i V_i M_c(i) = w sum_p g_c(v_p) for every moment."""
    rng = np.random.default_rng(5)
    n, w = 3000, 2.0e3
    r = rng.uniform(cfg["r_in"], cfg["r_out"], n)
    z = rng.uniform(cfg["z_min"], cfg["z_max"], n)
    vr, vt, vz = rng.normal(0, 1e6, (3, n))
    M = fluid.moments(cfg, r, z, vr, vt, vz, w)
    V = _vol(cfg)
    el, io = oracle.nu_parts(cfg, np.sqrt(vr ** 2 + vt ** 2 + vz ** 2))
    assert io.sum() > 0
    g = [np.ones(n), vr, vt, vz, vr * vr, vr * vt, vr * vz, vt * vt, vt * vz, vz * vz, el + io, io]
    for c in range(fluid.MOMENTS):
        assert (M[c] * V).sum() == pytest.approx(w * g[c].sum(), rel=1e-10, abs=1e-9 * w * np.abs(g[c]).sum())


def test_counter_streaming_pair_pressure(cfg):
    """Two particles on one node with v_r = +-v: no flow, P_rr = m n v^2."""
    hr, hz = _h(cfg)
    i, j, v = 5, 5, 7e5
    r = cfg["r_in"] + i * hr
    z = cfg["z_min"] + j * hz
    M = fluid.moments(cfg, [r, r], [z, z], [v, -v], [0, 0], [0, 0], 1.0)
    n, u, P = fluid._fluid(M)
    assert u[0, i, j] == 0.0
    assert P[0, i, j] == pytest.approx(ME * n[i, j] * v * v, rel=1e-12)
    assert P[3, i, j] == 0.0 and P[5, i, j] == 0.0


def test_nu_drag_is_the_elastic_rate_below_threshold(cfg):
    n_gas = oracle.derived(cfg)["n_gas"]
    E_eV = 0.5 * cfg["ion_E_th_eV"]
    v = np.sqrt(2 * E_eV * QE / ME)
    assert oracle.nu_drag(cfg, [v])[0] == pytest.approx(n_gas * cfg["sigma_el"] * v, rel=1e-13)
    # above threshold ionisation adds its own rate
    E2 = 3 * cfg["ion_E_th_eV"]
    v2 = np.sqrt(2 * E2 * QE / ME)
    extra = n_gas * oracle.sigma_ion(cfg, E2) * v2
    assert extra > 0
    assert oracle.nu_drag(cfg, [v2])[0] == pytest.approx(n_gas * cfg["sigma_el"] * v2 + extra,
                                                         rel=1e-13)


def _moments_of(cfg, n, u, vv=None):
    """Moments from prescribed fields n, u (3 arrays) and n <v v> (6; cold
    fluid n u u when None), nu_d = 0."""
    M = np.zeros((fluid.MOMENTS,) + _shape(cfg))
    M[0] = n
    M[1:4] = n * u
    pairs = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))
    for k, (a, b) in enumerate(pairs):
        M[4 + k] = n * u[a] * u[b] if vv is None else vv[k]
    return M


def _RZ(cfg):
    r, z = oracle.grid(cfg)
    return np.meshgrid(r, z, indexing="ij")


def _zero_e(cfg):
    return np.zeros(_shape(cfg)), np.zeros(_shape(cfg))


def test_rigid_rotation_inertia(cfg):
    """u_theta = Omega r, uniform n: F_i = (m n Omega^2 r, 0, 0) exactly (the
    centrifugal term), no pressure in a cold fluid."""
    R, Z = _RZ(cfg)
    n0, Om = 1e15, 3e7
    u = np.array([np.zeros_like(R), Om * R, np.zeros_like(R)])
    M = _moments_of(cfg, np.full_like(R, n0), u)
    T = fluid.force_terms(cfg, M, *_zero_e(cfg))
    scale = ME * n0 * Om ** 2 * R.max()
    assert np.abs(T[2, 0] - ME * n0 * Om ** 2 * R).max() <= 1e-10 * scale
    assert np.abs(T[2, 1]).max() <= 1e-10 * scale and np.abs(T[2, 2]).max() <= 1e-10 * scale
    assert np.abs(T[3]).max() <= 1e-6 * scale


def test_radial_expansion_inertia(cfg):
    """u_r = U r: F_i,r = -m n U^2 r; with u_theta = W as well, the
    Coriolis-like term gives F_i,theta = -m n (u_r W / r) = -m n U W."""
    R, _ = _RZ(cfg)
    n0, U, W = 2e15, 1e7, 4e4
    u = np.array([U * R, np.full_like(R, W), np.zeros_like(R)])
    T = fluid.force_terms(cfg, _moments_of(cfg, np.full_like(R, n0), u), *_zero_e(cfg))
    s = ME * n0 * U * U * R.max()
    assert np.abs(T[2, 0] - (-ME * n0 * U * U * R + ME * n0 * W * W / R)).max() <= 1e-9 * s
    assert np.abs(T[2, 1] + ME * n0 * U * W).max() <= 1e-9 * s


def test_isotropic_pressure_linear_in_r_and_z(cfg):
    """P = (a + b r + c z) I at rest: -div P = (-b, 0, -c) (the hoop term
    P_tt / r cancels (1/r) d(r P_rr)/dr's P / r)."""
    R, Z = _RZ(cfg)
    a, b, c = 1e3, 2e5, -3e4
    p = a + b * R + c * Z
    n = np.full_like(R, 1e15)
    zero = np.zeros_like(R)
    vv = np.array([p, zero, zero, p, zero, p]) / ME
    T = fluid.force_terms(cfg, _moments_of(cfg, n, [zero, zero, zero], vv), *_zero_e(cfg))
    s = abs(b) + abs(c)
    assert np.abs(T[3, 0] + b).max() <= 1e-7 * s
    assert np.abs(T[3, 1]).max() <= 1e-7 * s
    assert np.abs(T[3, 2] + c).max() <= 1e-7 * s


def test_off_diagonal_pressure_terms(cfg):
    """P_rt = k / r: (1/r^2) d(r^2 P_rt)/dr = k / r^2; P_rz = c z: the r
    component gains -c, the z component -c z / r."""
    R, Z = _RZ(cfg)
    k, c = 5.0, 7e4
    n = np.full_like(R, 1e15)
    zero = np.zeros_like(R)
    vv = np.array([zero, k / R, c * Z, zero, zero, zero]) / ME
    T = fluid.force_terms(cfg, _moments_of(cfg, n, [zero, zero, zero], vv), *_zero_e(cfg))
    s = np.abs(k / R ** 2).max() + c
    assert np.abs(T[3, 1] + k / R ** 2).max() <= 1e-7 * s
    assert np.abs(T[3, 0] + c).max() <= 1e-7 * s
    assert np.abs(T[3, 2] + c * Z / R).max() <= 1e-7 * s


@pytest.mark.parametrize("bkind", [0, 1])
def test_lorentz_force_is_the_cross_product(cfg, bkind):
    c = dict(cfg, bfield_kind=bkind, b0=0.05)
    rng = np.random.default_rng(9)
    shp = _shape(c)
    n = rng.uniform(1e14, 1e15, shp)
    u = rng.normal(0, 1e5, (3,) + shp)
    T = fluid.force_terms(c, _moments_of(c, n, u), *_zero_e(c))
    Br, Bz = fluid.magnetic_field(c)
    B = np.stack([Br, np.zeros_like(Br), Bz], axis=-1)
    F = -QE * n[..., None] * np.cross(np.moveaxis(u, 0, -1), B)
    assert np.allclose(np.moveaxis(T[1], 0, -1), F, rtol=1e-12, atol=1e-12 * np.abs(F).max())


def test_mirror_field_is_divergence_free(cfg):
    c = dict(cfg, bfield_kind=1, b0=0.1)
    Br, Bz = fluid.magnetic_field(c)
    hr, hz = _h(c)
    R, _ = _RZ(c)
    div = fluid._d(R * Br, hr, 0) / R + fluid._d(Bz, hz, 1)
    assert np.abs(div).max() <= 1e-9 * c["b0"] / hz
    assert Bz.min() == pytest.approx(c["b0"])


def test_drag_and_inertia_terms(cfg):
    """F_d = -m n <nu_d> u for a mono-energetic beam; F_a = m n du / dt."""
    R, _ = _RZ(cfg)
    n0, nu = 1e15, 2.5e8
    u = np.array([np.full_like(R, 1e5), np.full_like(R, -2e5), np.full_like(R, 3e5)])
    M = _moments_of(cfg, np.full_like(R, n0), u)
    M[10] = n0 * nu
    u2 = u * 1.5
    M2 = _moments_of(cfg, np.full_like(R, n0), u2)
    M2[10] = n0 * nu
    dt = 1e-11
    T = fluid.force_terms(cfg, M2, *_zero_e(cfg), M_prev=M, dt_prev=dt)
    for a in range(3):
        assert np.allclose(T[4, a], -ME * n0 * nu * u2[a], rtol=1e-12)
        assert np.allclose(T[5, a], ME * n0 * (u2[a] - u[a]) / dt, rtol=1e-9)
    # the sum carries F_a with the minus sign
    assert np.allclose(T[6], T[2] + T[0] + T[1] + T[3] + T[4] - T[5], rtol=1e-12, atol=0)
    # no previous state: F_a = 0
    assert not fluid.force_terms(cfg, M2, *_zero_e(cfg))[5].any()


def test_boltzmann_equilibrium_balances(cfg):
    """An isothermal electron gas at rest in a uniform axial field, n =
    n0 exp(q E_z z / kT) and P = n kT I, is in equilibrium: F_E + F_p = 0
    (up to the second-order differences)."""
    R, Z = _RZ(cfg)
    kT = 5.0 * QE
    Ez = 250.0   # n varies by e^(+-1) over the length
    n = 1e15 * np.exp(-QE * Ez * Z / kT)
    zero = np.zeros_like(R)
    p = n * kT
    vv = np.array([p, zero, zero, p, zero, p]) / ME
    T = fluid.force_terms(cfg, _moments_of(cfg, n, [zero, zero, zero], vv), zero, np.full_like(R, Ez))
    scale = np.abs(T[0, 2]).max()
    assert scale > 0
    assert np.abs(T[6]).max() <= 1e-3 * scale
    assert np.abs(T[0, 2] + T[3, 2]).max() <= 1e-3 * scale
    # a dropped factor in either term breaks the balance
    assert np.abs(T[0, 2] + 0.9 * T[3, 2]).max() > 0.05 * scale


def test_empty_nodes_have_no_flow(cfg):
    shp = _shape(cfg)
    M = np.zeros((fluid.MOMENTS,) + shp)
    T = fluid.force_terms(cfg, M, np.ones(shp), np.ones(shp))
    assert not T.any()


def _fm_moments(cfg, n, nu_d, nu_io):
    shp = _shape(cfg)
    M = np.zeros((fluid.MOMENTS,) + shp)
    M[0] = n
    M[10] = n * nu_d
    M[11] = n * nu_io
    return M


def test_fluid_model_solves_the_azimuthal_balance(cfg):
    """u_r of the model satisfies the azimuthal balance it came from,
    m u_r (1/r) d(r u_theta)/dr = -q u_r B_z - m nu_d u_theta, with the left
    side replaced through Gauss's law by -m u_r q n / (eps0 B_z) and
    u_theta = -E_r / B_z; below and above the Brillouin density."""
    c = dict(cfg, b0=0.2, bfield_kind=0)
    rng = np.random.default_rng(3)
    shp = _shape(c)
    q, m = -QE, ME
    n_brillouin = fluid.EPS0 * c["b0"] ** 2 / ME
    n = rng.uniform(0.05, 3.0, shp) * n_brillouin
    nu_d = rng.uniform(1e6, 1e8, shp)
    Er = rng.normal(0, 1e5, shp)
    out = fluid.fluid_model(c, _fm_moments(c, n, nu_d, 0.3 * nu_d), Er, np.zeros(shp))
    u_t, u_r = out[0], out[3]
    assert np.allclose(u_t, -Er / c["b0"], rtol=1e-14)
    lhs = -m * u_r * q * n / (fluid.EPS0 * c["b0"])
    rhs = -q * u_r * c["b0"] - m * nu_d * u_t
    assert np.abs(lhs - rhs).max() <= 1e-9 * np.abs(rhs).max()


def test_fluid_model_peak_density(cfg):
    """omega_p,max^2 = Omega_c^2 nu_io / (nu_io + nu_d): half Omega_c^2 when
    the two frequencies are equal, zero without ionisation; n_max gives
    back omega_p,max through omega_p^2 = e^2 n / (eps0 m)."""
    c = dict(cfg, b0=0.25, bfield_kind=0)
    shp = _shape(c)
    n = np.full(shp, 1e15)
    nu = np.full(shp, 3e7)
    Oc2 = (QE * c["b0"] / ME) ** 2
    out = fluid.fluid_model(c, _fm_moments(c, n, nu, nu), np.zeros(shp), np.zeros(shp))
    assert np.allclose(out[4], Oc2 / 2, rtol=1e-14)
    assert np.allclose(QE ** 2 * out[5] / (fluid.EPS0 * ME), out[4], rtol=1e-14)
    assert np.allclose(out[1], nu, rtol=1e-15) and np.allclose(out[2], nu, rtol=1e-15)
    out0 = fluid.fluid_model(c, _fm_moments(c, n, nu, 0 * nu), np.zeros(shp), np.zeros(shp))
    assert not out0[4].any() and not out0[5].any()
    # empty nodes: no ratios
    empty = fluid.fluid_model(c, _fm_moments(c, 0 * n, nu, nu), np.ones(shp), np.ones(shp))
    assert not empty[1:6].any() and not empty[8].any()


def test_fluid_model_drift_frequencies(cfg):
    """Collision frequencies at the E x B drift speed: with a uniform B_z
    and a radial field the drift is |E_r| / B_z; below the ionisation
    threshold nu_d = n_gas sigma_el v, above it the fit
    sigma_pk 2 s / (1 + s^2), s = (E - E_th) / (E_pk - E_th), adds."""
    c = dict(cfg, b0=0.1, bfield_kind=0)
    shp = _shape(c)
    n_gas = oracle.derived(c)["n_gas"]
    # a speed below and one above threshold
    E_lo, E_hi = 0.4 * c["ion_E_th_eV"], 4.0 * c["ion_E_th_eV"]
    v_lo, v_hi = np.sqrt(2 * E_lo * QE / ME), np.sqrt(2 * E_hi * QE / ME)
    Er = np.where(np.arange(shp[1])[None, :] % 2 == 0, v_lo, -v_hi) * c["b0"] * np.ones(shp)
    out = fluid.fluid_model(c, _fm_moments(c, np.ones(shp), np.ones(shp), np.ones(shp)), Er,
                            np.zeros(shp))
    lo, hi = out[:, :, 0], out[:, :, 1]
    assert np.allclose(lo[6], n_gas * c["sigma_el"] * v_lo, rtol=1e-12)
    assert not lo[7].any()
    s = (E_hi - c["ion_E_th_eV"]) / (c["ion_E_pk_eV"] - c["ion_E_th_eV"])
    sig_io = c["ion_sigma_pk"] * 2 * s / (1 + s * s)
    assert np.allclose(hi[7], n_gas * sig_io * v_hi, rtol=1e-12)
    assert np.allclose(hi[6], n_gas * (c["sigma_el"] + sig_io) * v_hi, rtol=1e-12)


def test_fluid_model_drift_speed_in_the_mirror(cfg):
    """|E x B| / |B|^2 with B_r != 0: against the component formula
    |E_z B_r - E_r B_z| / (B_r^2 + B_z^2), below threshold (pure elastic)."""
    c = dict(cfg, b0=0.5, bfield_kind=1, sigma_el=1e-20)
    shp = _shape(c)
    rng = np.random.default_rng(4)
    Er, Ez = rng.normal(0, 3e4, (2,) + shp)
    Br, Bz = fluid.magnetic_field(c)
    vd = np.abs(Ez * Br - Er * Bz) / (Br ** 2 + Bz ** 2)
    assert (0.5 * ME * vd ** 2 / QE < c["ion_E_th_eV"]).all()
    n_gas = oracle.derived(c)["n_gas"]
    out = fluid.fluid_model(c, _fm_moments(c, np.ones(shp), np.ones(shp), np.ones(shp)), Er, Ez)
    assert np.allclose(out[6], n_gas * 1e-20 * vd, rtol=1e-12)
    assert np.allclose(out[8], -fluid.EPS0 * Er * 1.0, rtol=1e-15)


def test_rigid_rotor_equilibrium_balances():
    """Electrons on the circular orbits of the coaxial vacuum field and a
    uniform B (each with the slow root of m v^2/r + q v B + q E_r = 0): the
    force terms evaluated from their moments sum to nearly zero (the
    verification of Sec. IV.A), while F_E and F_B are each far larger."""
    c = dict(workload("coax_32x64_1e4", precision=64), nr=24, nz=6, b0=0.3, bfield_kind=0,
             v_inner=-2e3, v_outer=0.0, p_mbar=1e-12)   # inside the Brillouin limit
    a, b = c["r_in"], c["r_out"]
    rng = np.random.default_rng(12)
    npart = 200_000
    r = np.sqrt(a * a + rng.uniform(0, 1, npart) * (b * b - a * a))
    z = rng.uniform(c["z_min"], c["z_max"], npart)
    Er_of = lambda rr: (c["v_inner"] - c["v_outer"]) / (rr * np.log(b / a))
    q, B = -QE, c["b0"]
    E = Er_of(r)
    v = (-q * B - np.sqrt((q * B) ** 2 - 4 * (ME / r) * q * E)) / (2 * ME / r)
    assert np.all(np.abs(ME * v * v / r + q * v * B + q * E) <= 1e-9 * np.abs(q * E))
    M = fluid.moments(c, r, z, np.zeros(npart), v, np.zeros(npart), 1e3)
    R, _ = _RZ(c)
    T = fluid.force_terms(c, M, Er_of(R), np.zeros_like(R))
    inner = (slice(2, -2), slice(1, -1))   # away from the walls and the z ends
    FE, FB, S = T[0, 0][inner], T[1, 0][inner], T[6, 0][inner]
    scale = np.abs(FE).max()
    assert np.abs(FB).max() > 0.9 * scale
    # the centrifugal term is ~2% of F_E here, the sum (discretisation and
    # sampling) ~0.3%: a dropped or mis-signed term cannot pass
    assert np.abs(T[2, 0][inner]).max() > 1e-2 * scale
    assert np.abs(S).max() <= 6e-3 * scale
    assert np.abs(T[6, 1][inner]).max() <= 1e-6 * scale   # no azimuthal force
    # the fluid-Poisson model's drift u_theta = -E_r / B_z (Sec. V.A) is the
    # electrons' mean azimuthal velocity up to the centrifugal correction
    # (m u^2 / r against q E_r: about 2 % here); with next to no gas the
    # predicted radial drift is negligible
    F = fluid.fluid_model(c, M, Er_of(R), np.zeros_like(R))
    u_t = M[2][inner] / M[0][inner]
    rel = np.abs(F[0][inner] - u_t) / np.abs(u_t)
    assert rel.max() <= 4e-2 and rel.max() >= 2e-3
    assert np.abs(F[3][inner]).max() <= 1e-9 * np.abs(u_t).max()
