"""The preconditioner of the device web-spline solve, checked as an
algorithm on the oracle's matrices (CPU): conjugate gradients on the
paper's trap (Sec. II.B) preconditioned with the enclosing box's weighted
B-spline solve, rescaled by D = sqrt(diag(P^T S P) / diag A), converges in
a few dozen iterations, nearly independent of the grid, to the sparse-LU
solution; without the rescaling it needs several times as many."""
import numpy as np
import pytest

from oracle.bspline import SplineField
from oracle.webspline import WebSplineField, paper_trap
from paper_2206_14662_gb300.inputs import workload


def _pcg(A, b, M, rtol=1e-12, maxit=3000):
    x = np.zeros_like(b)
    r = b.copy()
    z = M(r)
    p = z.copy()
    rz = r @ z
    bn = np.linalg.norm(b)
    for it in range(1, maxit + 1):
        q = A @ p
        al = rz / (p @ q)
        x += al * p
        r -= al * q
        if np.linalg.norm(r) <= rtol * bn:
            return x, it
        z = M(r)
        rzn = r @ z
        p = z + (rzn / rz) * p
        rz = rzn
    return x, maxit


def _setup(n, nr, nz):
    geo = paper_trap()
    W = WebSplineField(geo, n, geo.a, geo.b, nr, nz)
    S = SplineField(workload("coax_32x64_1e4", r_in=geo.a, r_out=geo.b, z_min=geo.z_min,
                             z_max=geo.z_max, nr=nr, nz=nz, bspline_degree=n))
    idx = np.flatnonzero(W.inner.ravel())
    return W, S, idx


def _box_pre(W, S, idx, scaled):
    d = np.sqrt(S.A.diagonal()[idx] / W.A.diagonal()) if scaled else np.ones(len(idx))

    def M(r):
        full = np.zeros(W.mr * W.mz)
        full[idx] = d * r
        return d * S.solve(full, dirichlet=False).ravel()[idx]
    return M


@pytest.mark.parametrize("n,nr,nz,max_it", [(2, 36, 92, 40), (3, 36, 92, 50), (2, 72, 184, 50)])
def test_rescaled_box_preconditioner(n, nr, nz, max_it):
    W, S, idx = _setup(n, nr, nz)
    b = -W.g
    x, it = _pcg(W.A, b, _box_pre(W, S, idx, True))
    ref = W._lu.solve(b)
    assert it <= max_it
    assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()
    if nr == 36:
        _, it_plain = _pcg(W.A, b, _box_pre(W, S, idx, False))
        assert it_plain >= 5 * it
