"""The C library's web-spline assembly (host code for curved electrodes,
Sec. II.A / II.B) against the oracle, on the CPU: the extension matrix,
the inner functions, the sparse Galerkin matrix and the lift load for the
paper's trap (ellipse on the outer cylinder) and for walls between grid
lines, degrees 1 to 3."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle.webspline import Geometry, WebSplineField, paper_trap
from paper_2206_14662_gb300.inputs import workload


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2206_14662_gb300 import build
    build.build()
    oracle.build()


def _cases():
    trap = paper_trap()
    yield "trap", trap, trap.a, trap.b, 14, 30
    geo = Geometry(1e-3, 10e-3, -2e-3, 2e-3, -1000.0, 0.0)
    h = 9e-3 / 16
    yield "offgrid", geo, 1e-3 - 0.37 * h, 1e-3 - 0.37 * h + 17 * h, 17, 4


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("case", ["trap", "offgrid"])
def test_web_system_matches_oracle(case, n):
    from paper_2206_14662_gb300._capi import web_system
    name, geo, r_lo, r_hi, nr, nz = next(c for c in _cases() if c[0] == case)
    W = WebSplineField(geo, n, r_lo, r_hi, nr, nz)
    cfg = workload("coax_32x64_1e4", r_in=geo.a, r_out=geo.b, z_min=geo.z_min,
                   z_max=geo.z_max, nz=nz, v_inner=geo.v_in, v_outer=geo.v_out)
    got = web_system(cfg, geo.ellipse, r_lo, r_hi, nr, n)
    assert np.array_equal(got["inner_full"], np.flatnonzero(W.inner.ravel()))
    T = sp.csr_matrix((got["t_val"], got["t_col"], got["t_ptr"]),
                      shape=(got["mr"] * got["mz"], len(got["g"])))
    assert abs(T - W.T).max() <= 1e-12 * abs(W.T).max()
    A = sp.csr_matrix((got["a_val"], got["a_col"], got["a_ptr"]), shape=W.A.shape)
    assert (np.diff(got["a_col"][got["a_ptr"][0]:got["a_ptr"][1]]) > 0).all()
    assert abs(A - W.A).max() <= 1e-11 * abs(W.A).max()
    assert np.abs(got["g"] - W.g).max() <= 1e-11 * np.abs(W.g).max()
    # the matrix is symmetric positive definite
    assert abs(A - A.T).max() <= 1e-12 * abs(A).max()


def test_bad_arguments_are_refused():
    from paper_2206_14662_gb300._capi import PicError, web_system
    geo = paper_trap()
    cfg = workload("coax_32x64_1e4", r_in=geo.a, r_out=geo.b, z_min=geo.z_min,
                   z_max=geo.z_max, nz=30)
    with pytest.raises(PicError):
        web_system(cfg, geo.ellipse, geo.a + 1e-3, geo.b, 14, 2)   # grid inside the walls
    with pytest.raises(PicError):
        web_system(cfg, (0.081, 0.012, 0.0, 0.014), geo.a, geo.b, 14, 2)
    with pytest.raises(PicError):
        web_system(cfg, geo.ellipse, geo.a, geo.b, 14, 0)


@pytest.mark.parametrize("n", [2, 3])
def test_web_inverse_matches_numpy(n):
    """The dense inverse the direct solve keeps on the device, against
    numpy's inverse of the oracle's matrix."""
    from paper_2206_14662_gb300._capi import web_inverse
    geo = paper_trap()
    nr, nz = 10, 24
    W = WebSplineField(geo, n, geo.a, geo.b, nr, nz)
    cfg = workload("coax_32x64_1e4", r_in=geo.a, r_out=geo.b, z_min=geo.z_min,
                   z_max=geo.z_max, nz=nz, v_inner=geo.v_in, v_outer=geo.v_out)
    got = web_inverse(cfg, geo.ellipse, geo.a, geo.b, nr, n)
    A = W.A.toarray()
    want = np.linalg.inv(A)
    assert np.abs(got - got.T).max() == 0.0
    assert np.abs(got - want).max() <= 1e-8 * np.abs(want).max()
    assert np.abs(got @ A - np.eye(len(A))).max() <= 1e-8
