"""Weighted B-spline finite elements of degree n for the r-z Poisson
problem, with particle shapes taken from the same basis (arXiv 2206.14662,
Sec. II.A: the field solve uses weighted extended B-splines of arbitrary degree,
which put Dirichlet electrodes on a rectangular grid) -- plain numpy and
scipy, FP64.

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's
CPU baseline use this package.

Basis.  Uniform knots t_k = t0 + (k - n) h extend n cells past each end of
[a, b] (r) and [z_min, z_max] (z); the degree-n B-splines b_i whose support
meets the interval (nr + n of them in r, nz + n in z) come from the
Cox-de Boor recursion.  The Dirichlet walls r = a and r = b carry the
weight w(r) = (r - a)(b - r) / (b - a), which vanishes on them:

    phi(r, z) = phi_D(r) + sum_ij c_ij w(r) b_i(r) b_j(z),
    phi_D(r) = V_in + (V_out - V_in) (r - a) / (b - a).

The walls lie on grid lines, so every B-spline meeting the gap covers a
whole cell of it and no extension of outer B-splines is needed (the curved
electrode would need it).  The z ends are natural (Neumann) boundaries.

Galerkin system (weak form of -div(eps0 grad phi) = rho, volume element
2 pi r dr dz, test functions w b_i b_j):

    2 pi eps0 (K_r (x) M_z + M_r (x) K_z) c = f - 2 pi eps0 (g_r (x) m_z)

with K_r = int (w b_i)'(w b_k)' r dr, M_r = int w^2 b_i b_k r dr,
g_r = int phi_D' (w b_i)' r dr, K_z = int b_j' b_l' dz, M_z = int b_j b_l dz,
m_z = int b_j dz, by Gauss-Legendre quadrature on every cell (exact for
these polynomial integrands).  Macro-particles deposit with the basis
itself, f_ij = sum_p q w_p w(r_p) b_i(r_p) b_j(z_p), and feel the exact
gradient E = -grad phi at their position (matching shape functions).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from numpy.polynomial.legendre import leggauss
from scipy.sparse.linalg import splu

EPS0 = 8.8541878128e-12
QE = 1.602176634e-19


def bspline_basis(n: int, knots, x, deriv: bool = False) -> np.ndarray:
    """(len(x), len(knots) - n - 1) values of the degree-n B-splines
    N_{i,n} on `knots` at x by the Cox-de Boor recursion (or their first
    derivatives).  Each x must lie in [knots[0], knots[-1])."""
    x = np.asarray(x, dtype=float).reshape(-1, 1)
    t = np.asarray(knots, dtype=float)
    N = ((t[:-1] <= x) & (x < t[1:])).astype(float)   # degree 0
    last = n if deriv else n + 1
    for p in range(1, last):
        left = (x - t[:-p - 1]) / (t[p:-1] - t[:-p - 1]) * N[:, :-1]
        right = (t[p + 1:] - x) / (t[p + 1:] - t[1:-p]) * N[:, 1:]
        N = left + right
    if not deriv:
        return N
    if n == 0:
        return np.zeros((x.shape[0], len(t) - 1))
    return (n / (t[n:-1] - t[:-n - 1]) * N[:, :-1]
            - n / (t[n + 1:] - t[1:-n]) * N[:, 1:])


def knots(n: int, lo: float, h: float, cells: int) -> np.ndarray:
    """Uniform knots lo + (k - n) h, k = 0..cells + 2n."""
    return lo + (np.arange(cells + 2 * n + 1) - n) * h


def cell_quadrature(lo: float, h: float, cells: int, q: int):
    """Gauss-Legendre points and weights, q per cell, over [lo, lo + cells h]."""
    xg, wg = leggauss(q)
    left = lo + h * np.arange(cells)[:, None]
    pts = (left + 0.5 * h * (xg[None, :] + 1.0)).ravel()
    wts = np.tile(0.5 * h * wg, cells)
    return pts, wts


class SplineField:
    """The degree-n weighted B-spline field of a workload (cfg needs
    "bspline_degree" = n >= 1 beside the geometry and the wall voltages)."""

    def __init__(self, cfg: dict):
        n = int(cfg["bspline_degree"])
        if n < 1:
            raise ValueError("bspline_degree must be >= 1")
        self.n = n
        self.a, self.b = cfg["r_in"], cfg["r_out"]
        self.z0, self.z1 = cfg["z_min"], cfg["z_max"]
        self.nr, self.nz = cfg["nr"], cfg["nz"]
        self.hr = (self.b - self.a) / self.nr
        self.hz = (self.z1 - self.z0) / self.nz
        self.v_in, self.v_out = cfg["v_inner"], cfg["v_outer"]
        self.tr = knots(n, self.a, self.hr, self.nr)
        self.tz = knots(n, self.z0, self.hz, self.nz)
        self.mr, self.mz = self.nr + n, self.nz + n
        self.dphi_D = (self.v_out - self.v_in) / (self.b - self.a)

        # 1D matrices by quadrature (degree of the integrands <= 2n + 3)
        rq, wrq = cell_quadrature(self.a, self.hr, self.nr, n + 3)
        Wb, dWb = self.r_functions(rq)
        self.K_r = (dWb * (wrq * rq)[:, None]).T @ dWb
        self.M_r = (Wb * (wrq * rq)[:, None]).T @ Wb
        self.g_r = (dWb * (wrq * rq * self.dphi_D)[:, None]).sum(axis=0)
        zq, wzq = cell_quadrature(self.z0, self.hz, self.nz, n + 2)
        Bz, dBz = self.z_functions(zq)
        self.K_z = (dBz * wzq[:, None]).T @ dBz
        self.M_z = (Bz * wzq[:, None]).T @ Bz
        self.m_z = (Bz * wzq[:, None]).sum(axis=0)

        c = 2.0 * np.pi * EPS0
        self.A = (c * (sp.kron(sp.csr_matrix(self.K_r), sp.csr_matrix(self.M_z))
                       + sp.kron(sp.csr_matrix(self.M_r), sp.csr_matrix(self.K_z)))).tocsc()
        self.f_D = c * np.kron(self.g_r, self.m_z)
        self._lu = splu(self.A)

    # ---------------------------------------------------------- functions
    def weight(self, r):
        r = np.asarray(r, dtype=float)
        return (r - self.a) * (self.b - r) / (self.b - self.a), (self.a + self.b - 2.0 * r) / (self.b - self.a)

    def r_functions(self, r):
        """(w b_i, (w b_i)') at the points r: (len(r), mr) each."""
        B = bspline_basis(self.n, self.tr, r)
        dB = bspline_basis(self.n, self.tr, r, deriv=True)
        w, dw = self.weight(r)
        return w[:, None] * B, dw[:, None] * B + w[:, None] * dB

    def z_functions(self, z):
        """(b_j, b_j') at the points z: (len(z), mz) each."""
        return bspline_basis(self.n, self.tz, z), bspline_basis(self.n, self.tz, z, deriv=True)

    # -------------------------------------------------------------- solve
    def solve(self, f: np.ndarray, dirichlet: bool = True) -> np.ndarray:
        """Coefficients c (mr x mz) for the load vector f (mr x mz or
        flat); dirichlet=False solves with zero wall potentials."""
        rhs = np.asarray(f, dtype=float).ravel() - (self.f_D if dirichlet else 0.0)
        return self._lu.solve(rhs).reshape(self.mr, self.mz)

    def deposit(self, r, z, qw: float) -> np.ndarray:
        """f_ij = sum_p qw w(r_p) b_i(r_p) b_j(z_p): (mr, mz)."""
        Wb, _ = self.r_functions(r)
        Bz, _ = self.z_functions(z)
        return qw * (Wb.T @ Bz)

    def rhs_density(self, rho, q: int | None = None) -> np.ndarray:
        """f_ij = int rho w b_i b_j 2 pi r dr dz for a density function
        rho(R, Z) (arrays), by tensor Gauss quadrature with q points per
        cell and direction."""
        q = self.n + 4 if q is None else q
        rq, wr = cell_quadrature(self.a, self.hr, self.nr, q)
        zq, wz = cell_quadrature(self.z0, self.hz, self.nz, q)
        Wb, _ = self.r_functions(rq)
        Bz, _ = self.z_functions(zq)
        R, Z = np.meshgrid(rq, zq, indexing="ij")
        G = (2.0 * np.pi * wr * rq)[:, None] * rho(R, Z) * wz[None, :]
        return Wb.T @ G @ Bz

    # ---------------------------------------------------------- evaluate
    def phi(self, c, r, z, dirichlet: bool = True):
        Wb, _ = self.r_functions(r)
        Bz, _ = self.z_functions(z)
        val = ((Wb @ np.asarray(c).reshape(self.mr, self.mz)) * Bz).sum(axis=1)
        if dirichlet:
            val = val + self.v_in + self.dphi_D * (np.asarray(r, dtype=float) - self.a)
        return val

    def efield(self, c, r, z, dirichlet: bool = True):
        """E = -grad phi at the points (r, z): (E_r, E_z)."""
        C = np.asarray(c).reshape(self.mr, self.mz)
        Wb, dWb = self.r_functions(r)
        Bz, dBz = self.z_functions(z)
        er = -((dWb @ C) * Bz).sum(axis=1)
        if dirichlet:
            er = er - self.dphi_D
        ez = -((Wb @ C) * dBz).sum(axis=1)
        return er, ez
