"""Pins of the oracle's weighted B-spline field of degree n (Sec. II.A:
finite elements on weighted B-splines of arbitrary degree; particles deposit with
and feel the same basis): Cox-de Boor values against the closed forms of
low degrees, partition of unity and Marsden's identity, derivatives
against differences, the 1D mass and stiffness matrices against the
cardinal B-spline of degree 2n + 1 (truncated-power formula), the coaxial
vacuum potential V ln(b/r)/ln(b/a) at the optimal rate h^(n+1),
exact reproduction of a manufactured solution that lies in the space,
the field energy (eps0/2) int |grad phi|^2 dV against half the particles'
sum q phi(x_p), and an oracle step pushed by the spline field."""
import math

import numpy as np
import pytest

import oracle
from oracle import ME, QE
from oracle.bspline import EPS0, SplineField, bspline_basis, cell_quadrature, knots
from paper_2206_14662_gb300.inputs import seed_particles, workload


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _cfg(n, nr=16, nz=12, **kw):
    return workload("coax_32x64_1e4", nr=nr, nz=nz, bspline_degree=n, **kw)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_partition_of_unity_and_marsden(n):
    t = knots(n, 0.0, 1.0, 7)
    x = np.random.default_rng(n).uniform(0.0, 7.0, 300)
    B = bspline_basis(n, t, x)
    assert np.abs(B.sum(axis=1) - 1.0).max() <= 1e-14
    assert (B >= 0).all()
    # Marsden: (x - y)^n = sum_i prod_{k=1..n} (t_{i+k} - y) N_i(x)
    y = 0.37
    psi = np.array([np.prod(t[i + 1:i + n + 1] - y) for i in range(B.shape[1])])
    assert np.abs(B @ psi - (x - y) ** n).max() <= 1e-11 * 7.0 ** n


def test_low_degree_closed_forms():
    t1 = knots(1, 0.0, 1.0, 4)
    x = np.array([0.25, 1.0, 2.6])
    B1 = bspline_basis(1, t1, x)
    # knots t_k = k - n: degree-1 function i is the hat on grid point i
    assert B1[0, 0] == pytest.approx(0.75) and B1[0, 1] == pytest.approx(0.25)
    assert B1[1, 1] == pytest.approx(1.0) and B1[2, 2] == pytest.approx(0.4)
    t2 = knots(2, 0.0, 1.0, 4)
    assert np.allclose(bspline_basis(2, t2, [2.0])[0, 2:4], [0.5, 0.5])
    assert np.allclose(bspline_basis(2, t2, [2.5])[0, 2:5], [0.125, 0.75, 0.125])
    t3 = knots(3, 0.0, 1.0, 4)
    # cubic function i is centred on grid point i - 1
    assert np.allclose(bspline_basis(3, t3, [2.0])[0, 2:5], [1 / 6, 2 / 3, 1 / 6])


@pytest.mark.parametrize("n", [1, 2, 3])
def test_derivatives_match_differences(n):
    t = knots(n, 0.0, 0.5, 6)
    x = np.random.default_rng(7).uniform(0.01, 2.99, 50)
    x = x[np.abs(x / 0.5 - np.round(x / 0.5)) > 1e-3]   # away from knots (n = 1 kinks)
    d = 1e-6
    fd = (bspline_basis(n, t, x + d) - bspline_basis(n, t, x - d)) / (2 * d)
    assert np.abs(bspline_basis(n, t, x, deriv=True) - fd).max() <= 1e-6


def _cardinal(m, x, deriv=0):
    """Centred cardinal B-spline of order m (degree m - 1) or its
    derivative, by the truncated-power formula."""
    deg = m - 1 - deriv
    s = sum((-1) ** k * math.comb(m, k) * max(x + m / 2 - k, 0.0) ** deg for k in range(m + 1))
    return s / math.factorial(deg)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_z_matrices_are_cardinal_spline_values(n):
    """Away from the ends, int b_j b_{j+s} dz = h M_{2n+2}(s) and
    int b_j' b_{j+s}' dz = -M''_{2n+2}(s) / h."""
    F = SplineField(_cfg(n, nz=16))
    h = F.hz
    j = F.mz // 2
    for s in range(0, n + 1):
        assert F.M_z[j, j + s] == pytest.approx(h * _cardinal(2 * n + 2, s), rel=1e-12)
        assert F.K_z[j, j + s] == pytest.approx(-_cardinal(2 * n + 2, s, deriv=2) / h,
                                                rel=1e-10, abs=1e-12 / h)
    assert F.M_z[j, j + n + 1] == 0.0
    for M in (F.K_r, F.M_r, F.K_z, F.M_z):
        assert np.allclose(M, M.T, rtol=0, atol=1e-14 * np.abs(M).max())
    assert np.linalg.eigvalsh(F.M_r).min() > 0


@pytest.mark.parametrize("n", [1, 2, 3])
def test_vacuum_coax_converges_at_order_n_plus_1(n):
    errs = []
    for nr in (32, 64):
        cfg = _cfg(n, nr=nr, nz=4)
        F = SplineField(cfg)
        c = F.solve(np.zeros((F.mr, F.mz)))
        a, b = cfg["r_in"], cfg["r_out"]
        r = np.linspace(a, b, 2001)
        exact = cfg["v_outer"] + (cfg["v_inner"] - cfg["v_outer"]) * np.log(b / r) / np.log(b / a)
        errs.append(np.abs(F.phi(c, r, np.full_like(r, 0.004)) - exact).max())
    # the walls hold their potentials exactly
    assert F.phi(c, np.array([a, b]), np.zeros(2)) == pytest.approx([cfg["v_inner"], cfg["v_outer"]])
    rate = math.log2(errs[0] / errs[1])
    assert n + 0.8 <= rate <= n + 1.3, rate


@pytest.mark.parametrize("n", [1, 2, 3])
def test_manufactured_solution_in_the_space_is_exact(n):
    """phi* = phi_D(r) + w(r) p(r) q(z) with p, q polynomials of degree n
    lies in the discrete space; with rho = -eps0 lap phi* (cylindrical) and
    the flux eps0 d_n phi* through the z ends added to the load (the weak
    form's boundary term; the solver's ends are natural), the Galerkin
    solution is phi* itself, and E = -grad phi*."""
    import sympy as sy
    cfg = _cfg(n, nr=10, nz=8)
    F = SplineField(cfg)
    a, b = cfg["r_in"], cfg["r_out"]
    L = cfg["z_max"] - cfg["z_min"]
    r, z = sy.symbols("r z")
    s = (r - a) / (b - a)
    p = sum(sy.Rational(k + 2, k + 1) * (-s) ** k for k in range(n + 1))
    q = sum(sy.Rational(3, k + 2) * (z / L) ** k for k in range(n + 1))
    phi_D = cfg["v_inner"] + (cfg["v_outer"] - cfg["v_inner"]) * s
    w = (r - a) * (b - r) / (b - a)
    amp = 1e3 / ((b - a) / 4)
    phi = phi_D + amp * w * p * q
    lap = sy.diff(phi, r, 2) + sy.diff(phi, r) / r + sy.diff(phi, z, 2)
    rho = sy.lambdify((r, z), -EPS0 * lap, "numpy")
    f = F.rhs_density(lambda R, Z: rho(R, Z) + 0 * R)
    # + int eps0 (d phi*/dn) w b_i b_j 2 pi r dr over z = z_max (n = +z)
    # and z = z_min (n = -z)
    dphidz = sy.lambdify((r, z), sy.diff(phi, z), "numpy")
    rq, wr = cell_quadrature(a, F.hr, cfg["nr"], n + 4)
    Wb, _ = F.r_functions(rq)
    for zb, sign in ((cfg["z_max"], 1.0), (cfg["z_min"], -1.0)):
        flux = sign * EPS0 * dphidz(rq, np.full_like(rq, zb)) * 2 * np.pi * rq * wr
        bz = bspline_basis(n, F.tz, [zb])[0]   # (the knots extend past both ends)
        f += np.outer(Wb.T @ flux, bz)
    c = F.solve(f)
    rng = np.random.default_rng(3)
    rs = rng.uniform(a, b, 200)
    zs = rng.uniform(cfg["z_min"], cfg["z_max"], 200)
    want = sy.lambdify((r, z), phi, "numpy")(rs, zs)
    got = F.phi(c, rs, zs)
    assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max()
    er, ez = F.efield(c, rs, zs)
    er_want = sy.lambdify((r, z), -sy.diff(phi, r), "numpy")(rs, zs)
    ez_want = sy.lambdify((r, z), -sy.diff(phi, z), "numpy")(rs, zs)
    scale = np.abs(er_want).max()
    assert np.abs(er - er_want).max() <= 1e-8 * scale
    assert np.abs(ez - ez_want).max() <= 1e-8 * scale


@pytest.mark.parametrize("n", [1, 2, 3])
def test_field_energy_equals_particle_potential_sum(n):
    """With the walls grounded: (eps0/2) int |grad phi|^2 dV (quadrature of
    the field) = (1/2) sum_p q w phi(x_p) (the deposit and the gather are
    the same basis)."""
    cfg = _cfg(n, nr=12, nz=10)
    F = SplineField(cfg)
    r, z, *_ = seed_particles(cfg, n=400, seed=9)
    qw = -QE * 1e5
    c = F.solve(F.deposit(r, z, qw), dirichlet=False)
    W_particles = 0.5 * qw * F.phi(c, r, z, dirichlet=False).sum()
    rq, wr = cell_quadrature(cfg["r_in"], F.hr, cfg["nr"], n + 3)
    zq, wz = cell_quadrature(cfg["z_min"], F.hz, cfg["nz"], n + 3)
    R, Z = np.meshgrid(rq, zq, indexing="ij")
    er, ez = F.efield(c, R.ravel(), Z.ravel(), dirichlet=False)
    dV = (2 * np.pi * wr * rq)[:, None] * wz[None, :]
    W_field = 0.5 * EPS0 * ((er ** 2 + ez ** 2).reshape(R.shape) * dV).sum()
    assert W_field > 0
    assert W_field == pytest.approx(W_particles, rel=1e-10)


def test_gather_is_the_gradient_of_the_potential():
    cfg = _cfg(2, nr=12, nz=10)
    F = SplineField(cfg)
    r, z, *_ = seed_particles(cfg, n=300, seed=4)
    c = F.solve(F.deposit(r, z, -QE * 1e5))
    rs, zs = r[:50], z[:50]
    d = 1e-8
    er, ez = F.efield(c, rs, zs)
    fr = -(F.phi(c, rs + d, zs) - F.phi(c, rs - d, zs)) / (2 * d)
    fz = -(F.phi(c, rs, zs + d) - F.phi(c, rs, zs - d)) / (2 * d)
    scale = max(np.abs(er).max(), np.abs(ez).max())
    assert np.abs(er - fr).max() <= 1e-5 * scale
    assert np.abs(ez - fz).max() <= 1e-5 * scale


def test_oracle_step_is_pushed_by_the_spline_field():
    """No collisions, no magnetic field: one step changes each velocity
    by q E(x^n) dt / m with E the spline field's gradient at the particle."""
    cfg = _cfg(2, nr=12, nz=10, p_mbar=1e-12, b0=0.0, source_rate=0.0)
    parts = seed_particles(cfg, n=200, seed=6)
    o = oracle.OracleSim(cfg, *parts)
    er, ez = o.spline.efield(o.coef, o.r, o.z)
    vr0, vz0, uid0 = o.vr.copy(), o.vz.copy(), o.uid.copy()
    res = o.step()
    keep = res.event < oracle.EV_WALL
    assert keep.sum() > 150
    k = -QE * cfg["dt"] / ME
    # the radial component also turns with the particle's azimuthal motion;
    # the axial one is exactly v_z + q E_z dt / m
    assert np.array_equal(o.uid, uid0[keep])
    assert np.allclose(o.vz, vz0[keep] + k * ez[keep], rtol=1e-12, atol=1e-9)
    assert np.abs(o.vr - (vr0[keep] + k * er[keep])).max() <= 0.05 * np.abs(vr0).max()
    # the deposit after the step is the spline deposit of the survivors
    assert np.allclose(o.b, o.spline.deposit(o.r, o.z, o.qw), rtol=1e-13, atol=0)
