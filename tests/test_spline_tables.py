"""The C library's weighted B-spline tables (host code of the spline field,
Sec. II.A) against the oracle, on the CPU: the 1D matrices and the lift
vector from its own Gauss rule and span recurrence against oracle.bspline
(Cox-de Boor, numpy Gauss-Legendre), and the generalised eigenpairs of
(K_r, M_r) against their defining identities and scipy's eigh."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle.bspline import SplineField
from paper_2206_14662_gb300.inputs import workload


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2206_14662_gb300 import build
    build.build()
    oracle.build()


def _cfg(n, nr, nz):
    return workload("coax_32x64_1e4", nr=nr, nz=nz, bspline_degree=n)


@pytest.mark.parametrize("n,nr,nz", [(1, 8, 6), (2, 16, 12), (3, 12, 20), (5, 9, 7)])
def test_matrices_match_oracle(n, nr, nz):
    from paper_2206_14662_gb300._capi import spline_matrices
    cfg = _cfg(n, nr, nz)
    got = spline_matrices(cfg, n)
    F = SplineField(cfg)
    for k in ("K_r", "M_r", "g_r", "K_z", "M_z", "m_z"):
        want = getattr(F, k)
        assert got[k].shape == want.shape, k
        assert np.abs(got[k] - want).max() <= 1e-12 * np.abs(want).max(), k


@pytest.mark.parametrize("n,nr", [(1, 8), (2, 40), (3, 130)])
def test_eigenpairs(n, nr):
    from paper_2206_14662_gb300._capi import spline_eigen, spline_matrices
    cfg = _cfg(n, nr, 6)
    V, lam = spline_eigen(cfg, n)
    M = spline_matrices(cfg, n)
    Kr, Mr = M["K_r"], M["M_r"]
    mr = nr + n
    assert np.abs(V.T @ Mr @ V - np.eye(mr)).max() <= 1e-9
    D = V.T @ Kr @ V
    scale = np.abs(lam).max()
    assert np.abs(D - np.diag(lam)).max() <= 1e-9 * scale
    assert (np.diff(lam) >= 0).all() and lam[0] > 0
    want = scipy.linalg.eigh(Kr, Mr, eigvals_only=True)
    assert np.abs(lam - want).max() <= 1e-9 * scale


def test_bad_arguments_are_refused():
    from paper_2206_14662_gb300._capi import PicError, spline_matrices
    cfg = _cfg(2, 8, 6)
    for deg in (0, 6):
        with pytest.raises(PicError):
            spline_matrices(cfg, deg)
    with pytest.raises(PicError):
        spline_matrices(dict(cfg, nr=1), 2)
