"""Pins of the oracle's web-spline field (Sec. II.A: weighted extended
B-splines carry curved Dirichlet electrodes on a rectangular grid; Sec.
II.B: the coaxial gap with a filled ellipse on the outer cylinder) and of
the potential-well depth along magnetic field lines: with the walls on
grid lines and no ellipse it is the weighted B-spline field itself; with
walls between grid lines the coaxial vacuum potential converges at the
optimal rate; the extended basis reproduces polynomials on the domain;
the trap's vacuum field holds its electrode potentials and the maximum
principle and converges under refinement; the deposit and the field are
consistent (field energy); the well depth of closed-form profiles."""
import math

import numpy as np
import pytest

from oracle.bspline import SplineField, bspline_basis
from oracle.webspline import (EPS0, QE, Geometry, WebSplineField, field_line_r, paper_trap,
                              well_depth_along, well_depth_map)
from paper_2206_14662_gb300.inputs import seed_particles, workload


def _trap_field(n, nr, nz, **kw):
    geo = paper_trap()
    return WebSplineField(geo, n, geo.a, geo.b, nr, nz, **kw)


def test_straight_walls_on_grid_lines_give_the_weighted_spline_field():
    cfg = workload("coax_32x64_1e4", nr=10, nz=8, bspline_degree=2)
    geo = Geometry(cfg["r_in"], cfg["r_out"], cfg["z_min"], cfg["z_max"], cfg["v_inner"],
                   cfg["v_outer"])
    W = WebSplineField(geo, 2, cfg["r_in"], cfg["r_out"], 10, 8)
    assert not W.outer.any()
    F = SplineField(cfg)
    r, z, *_ = seed_particles(cfg, n=500, seed=3)
    f = F.deposit(r, z, -QE * 1e5)
    c_f2, c_web = F.solve(f), W.solve(f.ravel())
    assert np.abs(c_f2 - c_web).max() <= 1e-11 * np.abs(c_f2).max()


@pytest.mark.parametrize("n", [1, 2, 3])
def test_off_grid_coax_converges(n):
    errs = []
    a, b = 1e-3, 10e-3
    for nr in (32, 64):
        h = (b - a) / nr
        r_lo = a - 0.37 * h
        geo = Geometry(a, b, -2e-3, 2e-3, -1000.0, 0.0)
        W = WebSplineField(geo, n, r_lo, r_lo + (nr + 1) * h, nr + 1, 2)
        assert W.outer.any()
        c = W.solve(np.zeros(W.mr * W.mz))
        rr = np.linspace(a, b, 1001)
        exact = -1000.0 * np.log(b / rr) / np.log(b / a)
        errs.append(np.abs(W.phi(c, rr, np.zeros_like(rr)) - exact).max())
    assert math.log2(errs[0] / errs[1]) >= n + 0.6


@pytest.mark.parametrize("n", [2, 3])
def test_extended_basis_reproduces_polynomials(n):
    """q(r, z) of degree <= n in each variable: its B-spline coefficients
    on the inner indices, pushed through the extension, give q again on the
    domain (the Lagrange extension is exact for polynomial coefficients)."""
    W = _trap_field(n, 14, 30)
    assert W.outer.sum() > 10
    rng = np.random.default_rng(n)
    A = rng.normal(size=(n + 1, n + 1))
    s = lambda r: (r - W.r_lo) / (W.r_hi - W.r_lo)
    t = lambda z: (z - W.z0) / (W.z1 - W.z0)
    q = lambda r, z: sum(A[i, j] * s(r) ** i * t(z) ** j for i in range(n + 1) for j in range(n + 1))
    # full coefficients by least squares on the box (exact: q is in the span)
    rb = np.random.default_rng(9).uniform(W.r_lo, W.r_hi, 6000)
    zb = np.random.default_rng(8).uniform(W.z0, W.z1, 6000)
    Br, Bz = bspline_basis(n, W.tr, rb), bspline_basis(n, W.tz, zb)
    Phi = (Br[:, :, None] * Bz[:, None, :]).reshape(len(rb), -1)
    c_full = np.linalg.lstsq(Phi, q(rb, zb), rcond=None)[0]
    u = c_full.reshape(W.mr, W.mz)[W.inner]   # inner coefficients, row-major like T
    c_ext = W.T @ u
    # points of the domain inside the supports of the outer B-splines, where
    # the extension decides the value
    pts = []
    g = np.linspace(0.0, 1.0, 23)[1:-1]
    for (jr, jz) in np.argwhere(W.outer):
        R = W.tr[jr] + g * (n + 1) * W.hr
        Z = W.tz[jz] + g * (n + 1) * W.hz
        RR, ZZ = np.meshgrid(R, Z, indexing="ij")
        ok = W.geo.inside(RR, ZZ) & (RR < W.r_hi) & (ZZ < W.z1)
        pts.append(np.stack([RR[ok], ZZ[ok]], axis=1))
    pts = np.concatenate(pts)
    assert len(pts) > 50
    Pr, Pz = bspline_basis(n, W.tr, pts[:, 0]), bspline_basis(n, W.tz, pts[:, 1])
    Pb = (Pr[:, :, None] * Pz[:, None, :]).reshape(len(pts), -1)
    scale = np.abs(q(rb, zb)).max()
    assert np.abs(Pb @ c_ext - q(pts[:, 0], pts[:, 1])).max() <= 1e-9 * scale
    # the outer functions matter there: dropping them changes the value
    drop = np.where(W.outer.ravel(), 0.0, c_full)
    assert np.abs(Pb @ drop - q(pts[:, 0], pts[:, 1])).max() > 1e-6 * scale
    # and everywhere in the domain the extended basis gives q
    ins = W.geo.inside(rb, zb)
    assert np.abs(Phi[ins] @ c_ext - q(rb[ins], zb[ins])).max() <= 1e-9 * scale


def test_trap_vacuum_field():
    W = _trap_field(2, 24, 60)
    geo = W.geo
    c = W.solve(np.zeros(W.mr * W.mz))
    # electrode potentials: walls and the ellipse surface
    th = np.linspace(0.5 * np.pi, 1.5 * np.pi, 50)   # the half of the ellipse inside r < b
    r0, z0, dr, dz = geo.ellipse
    re, ze = r0 + dr * np.cos(th), z0 + dz * np.sin(th)
    assert np.abs(W.phi(c, re, ze) - geo.v_out).max() <= 1e-9 * abs(geo.v_in)
    zs = np.linspace(geo.z_min, geo.z_max, 30)
    assert np.abs(W.phi(c, np.full(30, geo.a), zs) - geo.v_in).max() <= 1e-9 * abs(geo.v_in)
    # maximum principle inside
    rng = np.random.default_rng(2)
    rr, zz = rng.uniform(geo.a, geo.b, 4000), rng.uniform(geo.z_min, geo.z_max, 4000)
    ins = geo.inside(rr, zz)
    v = W.phi(c, rr[ins], zz[ins])
    lo, hi = min(geo.v_in, geo.v_out), max(geo.v_in, geo.v_out)
    span = hi - lo
    assert v.min() >= lo - 1e-3 * span and v.max() <= hi + 1e-3 * span
    # self-convergence: 12x30 and 24x60 against 48x120
    W4 = _trap_field(2, 48, 120)
    c4 = W4.solve(np.zeros(W4.mr * W4.mz))
    W1 = _trap_field(2, 12, 30)
    c1 = W1.solve(np.zeros(W1.mr * W1.mz))
    ref = W4.phi(c4, rr[ins], zz[ins])
    e1 = np.abs(W1.phi(c1, rr[ins], zz[ins]) - ref).max()
    e2 = np.abs(v - ref).max()
    assert e2 < e1 / 3 and e2 <= 2e-3 * span


def test_trap_field_energy_equals_particle_sum():
    W = _trap_field(2, 16, 40)
    geo = W.geo
    rng = np.random.default_rng(4)
    r, z = rng.uniform(geo.a, geo.b, 3000), rng.uniform(geo.z_min, geo.z_max, 3000)
    keep = geo.inside(r, z)
    r, z = r[keep], z[keep]
    qw = -QE * 1e6
    c = W.solve(W.deposit(r, z, qw), dirichlet=False)
    W_particles = 0.5 * qw * W.phi(c, r, z, dirichlet=False).sum()
    er, ez = W.efield(c, W.qr, W.qz, dirichlet=False)
    W_field = 0.5 * EPS0 * ((er ** 2 + ez ** 2) * W.qw).sum()
    assert W_field > 0
    assert W_field == pytest.approx(W_particles, rel=1e-9)


def test_well_depth_of_closed_form_profiles():
    z = np.linspace(-1.0, 1.0, 2001)
    A, s, zc = 5.0, 0.3, 0.2
    U = A * np.exp(-((z - zc) / s) ** 2)
    d, k = well_depth_along(U)
    want = A - A * max(math.exp(-((-1.0 - zc) / s) ** 2), math.exp(-((1.0 - zc) / s) ** 2))
    assert d == pytest.approx(want, rel=1e-9) and abs(z[k] - zc) < 1e-3
    # two humps: the deeper well is the higher hump, limited by the higher side
    U2 = 3.0 * np.exp(-((z + 0.5) / 0.1) ** 2) + 5.0 * np.exp(-((z - 0.4) / 0.1) ** 2) + 0.5 * z
    d2, k2 = well_depth_along(U2)
    kmax = int(np.argmax(U2))
    assert k2 == kmax
    assert d2 == pytest.approx(U2[kmax] - max(U2[:kmax].min(), U2[kmax + 1:].min()))
    assert well_depth_along(z)[0] == 0.0   # monotonic: no well


def test_field_lines_and_well_map():
    bz = lambda z: 0.3 * (1.0 + 2.0 * (np.asarray(z) / 0.02) ** 2)
    z = np.linspace(-0.01, 0.01, 11)
    r = field_line_r(0.07, 0.0, z, bz)
    assert np.allclose(r ** 2 * bz(z), 0.07 ** 2 * bz(0.0), rtol=1e-14)
    # uniform field and a potential bump in z: U_d on every line
    geo = Geometry(0.06, 0.08, -0.01, 0.03, 0.0, 0.0)
    phi = lambda r, z: 100.0 * np.exp(-((z - 0.012) / 0.004) ** 2) + 0 * r
    d = well_depth_map(phi, geo.inside, lambda zz: np.full_like(np.asarray(zz, float), 0.28),
                       np.array([0.065, 0.07, 0.075]), 0.012, geo.z_min, geo.z_max)
    want = 100.0 * (1.0 - math.exp(-((0.03 - 0.012) / 0.004) ** 2))
    assert np.allclose(d, want, rtol=1e-6)
