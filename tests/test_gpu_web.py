"""The web-spline field on the GPU (pic_web_*: Sec. II.A's weighted
extended B-splines for curved electrodes, Sec. II.B's trap) against
oracle.webspline on the same seeded inputs: the deposit in the full basis,
the preconditioned CG solve (residual of the oracle's system, field at the
particles, iterations) and phi / E at the particles, for the paper's trap
and for walls between grid lines."""
import numpy as np
import pytest

import oracle
from oracle import QE
from oracle.webspline import Geometry, WebSplineField, paper_trap
from paper_2206_14662_gb300.inputs import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2206_14662_gb300 import build
    build.build()
    oracle.build()


def _case(name):
    if name == "trap":
        geo = paper_trap()
        return geo, geo.a, geo.b, 36, 92
    geo = Geometry(1e-3, 10e-3, -2e-3, 2e-3, -1000.0, 0.0)
    h = 9e-3 / 32
    return geo, 1e-3 - 0.37 * h, 1e-3 - 0.37 * h + 33 * h, 33, 8


@pytest.mark.parametrize("name,n", [("trap", 2), ("trap", 3), ("offgrid", 2)])
def test_web_field_matches_oracle(name, n):
    import torch
    from paper_2206_14662_gb300._capi import WebSolver
    geo, r_lo, r_hi, nr, nz = _case(name)
    W = WebSplineField(geo, n, r_lo, r_hi, nr, nz)
    cfg = workload("coax_32x64_1e4", r_in=geo.a, r_out=geo.b, z_min=geo.z_min, z_max=geo.z_max,
                   nz=nz, v_inner=geo.v_in, v_outer=geo.v_out)
    rng = np.random.default_rng(n)
    r = rng.uniform(geo.a, geo.b, 20000)
    z = rng.uniform(geo.z_min, geo.z_max, 20000)
    keep = geo.inside(r, z)
    r, z = r[keep], z[keep]
    qw = -QE * 1e7
    f_or = W.deposit(r, z, qw)
    c_or = W.solve(f_or)
    dev = torch.device("cuda")
    rt, zt = torch.from_numpy(r).to(dev), torch.from_numpy(z).to(dev)
    with WebSolver(cfg, geo.ellipse, r_lo, r_hi, nr, n) as S:
        f = S.deposit(rt, zt, qw)
        c, it, rel = S.solve(torch.from_numpy(f_or.reshape(S.mr, S.mz)).to(dev), rtol=1e-12)
        phi, er, ez = S.eval(torch.from_numpy(c_or.reshape(S.mr, S.mz)).to(dev), rt, zt)
        torch.cuda.synchronize()
    assert np.abs(f.cpu().numpy().ravel() - f_or).max() <= 1e-12 * np.abs(f_or).max()
    assert rel <= 1e-12 and it <= 60
    cg = c.cpu().numpy()
    # the inner coefficients satisfy the oracle's system; the field agrees
    u = cg.ravel()[W.inner.ravel()]
    rhs = W.T.T @ f_or - W.g
    assert np.linalg.norm(W.A @ u - rhs) <= 1e-10 * np.linalg.norm(rhs)
    want = W.phi(c_or, r, z)
    assert np.abs(W.phi(cg, r, z) - want).max() <= 1e-10 * np.abs(want).max()
    assert np.abs(phi.cpu().numpy() - want).max() <= 1e-12 * np.abs(want).max()
    er_or, ez_or = W.efield(c_or, r, z)
    scale = max(np.abs(er_or).max(), np.abs(ez_or).max())
    assert np.abs(er.cpu().numpy() - er_or).max() <= 1e-11 * scale
    assert np.abs(ez.cpu().numpy() - ez_or).max() <= 1e-11 * scale


def test_well_depth_matches_oracle():
    import torch
    from oracle.webspline import well_depth_map
    from paper_2206_14662_gb300._capi import WebSolver
    geo = paper_trap(v_in=-30e3, v_out=0.0)
    W = WebSplineField(geo, 2, geo.a, geo.b, 36, 92)
    c_or = W.solve(np.zeros(W.mr * W.mz))
    cfg = workload("coax_32x64_1e4", r_in=geo.a, r_out=geo.b, z_min=geo.z_min, z_max=geo.z_max,
                   nz=92, v_inner=geo.v_in, v_outer=geo.v_out)
    b0, L = 0.28 / 3, geo.z_max - geo.z_min
    bz = lambda z: b0 * (1 + 2 * ((np.asarray(z) - geo.z_min) / L) ** 2)
    rs = np.linspace(geo.a + 0.5e-3, geo.b - 0.2e-3, 60)
    z1 = 12e-3 - 14.5e-3
    want = well_depth_map(lambda r, z: W.phi(c_or, r, z), geo.inside, bz, rs, z1, geo.z_min,
                          geo.z_max, samples=1501)
    with WebSolver(cfg, geo.ellipse, geo.a, geo.b, 36, 2) as S:
        c = torch.from_numpy(c_or.reshape(S.mr, S.mz)).to("cuda")
        got, z_at = S.well_depth(c, rs, z1, samples=1501, bfield_kind=1, b0=b0,
                                 z_mid=geo.z_min, L=L)
    assert want.max() > 50.0
    assert np.abs(got - want).max() <= 1e-9 * want.max()


@pytest.mark.parametrize("name,n", [("trap", 2), ("offgrid", 3)])
def test_web_direct_solve_matches_oracle(name, n):
    import torch
    from paper_2206_14662_gb300._capi import WebSolver
    geo, r_lo, r_hi, nr, nz = _case(name)
    W = WebSplineField(geo, n, r_lo, r_hi, nr, nz)
    cfg = workload("coax_32x64_1e4", r_in=geo.a, r_out=geo.b, z_min=geo.z_min, z_max=geo.z_max,
                   nz=nz, v_inner=geo.v_in, v_outer=geo.v_out)
    rng = np.random.default_rng(7)
    r = rng.uniform(geo.a, geo.b, 5000)
    z = rng.uniform(geo.z_min, geo.z_max, 5000)
    keep = geo.inside(r, z)
    f_or = W.deposit(r[keep], z[keep], -QE * 1e7)
    c_or = W.solve(f_or)
    with WebSolver(cfg, geo.ellipse, r_lo, r_hi, nr, n) as S:
        c = S.solve_direct(torch.from_numpy(f_or.reshape(S.mr, S.mz)).to("cuda"))
        torch.cuda.synchronize()
    cg = c.cpu().numpy()
    want = W.phi(c_or, r[keep], z[keep])
    assert np.abs(W.phi(cg, r[keep], z[keep]) - want).max() <= 1e-10 * np.abs(want).max()
