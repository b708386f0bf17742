"""Weighted extended B-splines (web-splines) of degree n for the r-z
Poisson problem on domains with curved Dirichlet electrodes on a
rectangular grid (arXiv 2206.14662, Sec. II.A: the field solve uses
weighted extended B-splines, which carry curved Dirichlet surfaces on a
rectangular grid; Sec. II.B: the coaxial gap with a filled ellipse on the
outer cylinder) -- plain numpy and scipy, FP64.

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's
CPU baseline use this package.

Domain.  D = {a < r < b, z_min < z < z_max} minus an optional filled
ellipse ((r - r0)/dr)^2 + ((z - z0)/dz)^2 <= 1 (centred on the outer wall
in the paper's trap).  Dirichlet: V_in on r = a, V_out on r = b and on the
ellipse; natural (Neumann) ends in z.  The grid may be wider than [a, b]
(walls between grid lines).

Weight.  w_c = (r - a)(b - r)/(b - a) for the walls; with the ellipse,
w_e = s ((r - r0)^2/dr^2 + (z - z0)^2/dz^2 - 1), s = min(dr, dz)/2, and
the R-function conjunction w = w_c + w_e - sqrt(w_c^2 + w_e^2) (positive
exactly where both are).  Lift: phi_D = V_in + (V_out - V_in) t with
t = (r - a)/(r - a + w_o), w_o the conjunction of (b - r) and w_e (zero on
the outer metal), t = (r - a)/(b - a) without the ellipse.

Basis.  Tensor B-splines b_k (uniform knots extending n cells past the
grid) whose support meets D.  Inner: some grid cell of the support lies in
D (exact test for the walls and the convex ellipse); outer: the rest.  Each outer b_j is tied to the (n+1) x
(n+1) array I(j) of inner indices nearest to j, and the extended inner
functions are B_i = b_i + sum_{j: i in I(j)} e_ij b_j with the Lagrange
coefficients e_ij = prod_nu prod_{mu != i_nu} (j_nu - mu)/(i_nu - mu) over
the array's index range, so polynomials of degree <= n keep their
B-spline representation.  Trial and test space: w B_i.

Quadrature.  Gauss points per cell; cells met by the ellipse are split
into strips in r, and at each r-point the z-intervals inside D are exact
(the ellipse is explicit in z), each with its own Gauss points.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from numpy.polynomial.legendre import leggauss
from scipy.sparse.linalg import splu

from .bspline import bspline_basis, knots

EPS0 = 8.8541878128e-12
QE = 1.602176634e-19


class Geometry:
    """Coaxial walls a < b, z range, optional ellipse (r0, z0, dr, dz)."""

    def __init__(self, a, b, z_min, z_max, v_in, v_out, ellipse=None):
        self.a, self.b, self.z_min, self.z_max = a, b, z_min, z_max
        self.v_in, self.v_out = v_in, v_out
        self.ellipse = ellipse

    # ------------------------------------------------------------ weights
    def _w_e(self, r, z):
        r0, z0, dr, dz = self.ellipse
        s = 0.5 * min(dr, dz)
        e = ((r - r0) / dr) ** 2 + ((z - z0) / dz) ** 2 - 1.0
        return s * e, s * 2.0 * (r - r0) / dr ** 2, s * 2.0 * (z - z0) / dz ** 2

    @staticmethod
    def _conj(x, gx, y, gy):
        """R-conjunction x + y - sqrt(x^2 + y^2) and its gradient."""
        q = np.sqrt(x * x + y * y)
        qs = np.where(q > 0, q, 1.0)
        v = x + y - q
        g = [gx[k] + gy[k] - (x * gx[k] + y * gy[k]) / qs for k in range(2)]
        return v, g

    def weight(self, r, z):
        """(w, dw/dr, dw/dz)."""
        r = np.asarray(r, float)
        z = np.asarray(z, float)
        ab = self.b - self.a
        wc = (r - self.a) * (self.b - r) / ab
        gc = [(self.a + self.b - 2.0 * r) / ab, np.zeros_like(r)]
        if self.ellipse is None:
            return wc, gc[0], gc[1]
        we, ger, gez = self._w_e(r, z)
        v, g = self._conj(wc, gc, we, [ger, gez])
        return v, g[0], g[1]

    def lift(self, r, z):
        """(phi_D, d/dr, d/dz)."""
        r = np.asarray(r, float)
        z = np.asarray(z, float)
        dv = self.v_out - self.v_in
        if self.ellipse is None:
            ab = self.b - self.a
            return self.v_in + dv * (r - self.a) / ab, np.full_like(r, dv / ab), np.zeros_like(r)
        we, ger, gez = self._w_e(r, z)
        wo, go = self._conj(self.b - r, [-np.ones_like(r), np.zeros_like(r)], we, [ger, gez])
        x = r - self.a
        den = x + wo
        t = x / den
        tr = ((1.0) * den - x * (1.0 + go[0])) / den ** 2
        tz = (-x * go[1]) / den ** 2
        return self.v_in + dv * t, dv * tr, dv * tz

    def inside(self, r, z):
        r = np.asarray(r, float)
        z = np.asarray(z, float)
        ok = (r > self.a) & (r < self.b) & (z > self.z_min) & (z < self.z_max)
        if self.ellipse is not None:
            r0, z0, dr, dz = self.ellipse
            ok &= ((r - r0) / dr) ** 2 + ((z - z0) / dz) ** 2 > 1.0
        return ok

    def cell_state(self, r0, r1, z0, z1):
        """2: the closed cell [r0, r1] x [z0, z1] lies in the closure of D
        with interior points of D; 1: it meets D only in part; 0: it misses
        D.  Exact: the ellipse is convex (a cell inside it has its four
        corners inside) and its defining quadratic is least over the cell at
        the centre clamped into the cell."""
        tol = 1e-12 * (self.b - self.a)   # grid lines computed on the walls
        if r1 <= self.a + tol or r0 >= self.b - tol:
            return 0
        in_walls = r0 >= self.a - tol and r1 <= self.b + tol
        if self.ellipse is None:
            return 2 if in_walls else 1
        er, ez, dr, dz = self.ellipse
        e = lambda r, z: ((r - er) / dr) ** 2 + ((z - ez) / dz) ** 2
        ra, rb = max(r0, self.a), min(r1, self.b)
        corners = [e(r, z) for r in (ra, rb) for z in (z0, z1)]
        if max(corners) <= 1.0:
            return 0
        e_min = e(min(max(er, r0), r1), min(max(ez, z0), z1))
        return 2 if (in_walls and e_min >= 1.0) else 1

    def z_intervals(self, r, lo, hi):
        """Sub-intervals of [lo, hi] inside D at radius r (a < r < b)."""
        if self.ellipse is None:
            return [(lo, hi)]
        r0, z0, dr, dz = self.ellipse
        x = (r - r0) / dr
        if abs(x) >= 1.0:
            return [(lo, hi)]
        h = dz * np.sqrt(1.0 - x * x)
        out = []
        if lo < z0 - h:
            out.append((lo, min(hi, z0 - h)))
        if hi > z0 + h:
            out.append((max(lo, z0 + h), hi))
        return out


def _gauss(q):
    x, w = leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w   # on [0, 1]


class WebSplineField:
    """Web-spline field of degree n on a grid (r_lo, r_hi, nr) x (z_min,
    z_max, nz) for a Geometry."""

    def __init__(self, geo: Geometry, n: int, r_lo: float, r_hi: float, nr: int, nz: int,
                 extend: bool = True, strips: int = 8):
        self.geo, self.n = geo, n
        self.r_lo, self.r_hi, self.nr = r_lo, r_hi, nr
        self.z0, self.z1, self.nz = geo.z_min, geo.z_max, nz
        self.hr = (r_hi - r_lo) / nr
        self.hz = (self.z1 - self.z0) / nz
        self.tr = knots(n, r_lo, self.hr, nr)
        self.tz = knots(n, self.z0, self.hz, nz)
        self.mr, self.mz = nr + n, nz + n
        self._classify()
        self.T = self._extension(extend)
        self._quadrature(strips)
        self._assemble()

    # ------------------------------------------------------ classification
    def _cell_state(self):
        """Per grid cell: 2 entirely in D, 1 partly, 0 outside."""
        st = np.zeros((self.nr, self.nz), dtype=int)
        for i in range(self.nr):
            r0, r1 = self.r_lo + i * self.hr, self.r_lo + (i + 1) * self.hr
            for j in range(self.nz):
                st[i, j] = self.geo.cell_state(r0, r1, self.z0 + j * self.hz,
                                               self.z0 + (j + 1) * self.hz)
        return st

    def _classify(self):
        st = self._cell_state()
        self.cell_state = st
        n = self.n
        inner = np.zeros((self.mr, self.mz), dtype=bool)
        relevant = np.zeros((self.mr, self.mz), dtype=bool)
        for i in range(self.mr):
            ci = slice(max(i - n, 0), min(i, self.nr - 1) + 1)
            for j in range(self.mz):
                cj = slice(max(j - n, 0), min(j, self.nz - 1) + 1)
                sub = st[ci, cj]
                inner[i, j] = (sub == 2).any()
                relevant[i, j] = (sub >= 1).any()
        self.inner, self.relevant = inner, relevant
        self.outer = relevant & ~inner

    def _extension(self, extend):
        """Sparse T (full index -> inner index): B_i = sum_k T[k, i] b_k."""
        n = self.n
        idx = -np.ones((self.mr, self.mz), dtype=int)
        ii = np.argwhere(self.inner)
        idx[self.inner] = np.arange(len(ii))
        self.inner_index = idx
        self.n_inner = len(ii)
        rows, cols, vals = [], [], []
        for (i, j) in ii:   # b_i itself
            rows.append(i * self.mz + j)
            cols.append(idx[i, j])
            vals.append(1.0)
        if extend:
            for (jr, jz) in np.argwhere(self.outer):
                lr, lz = self._nearest_array(jr, jz)
                for al in range(n + 1):
                    er = _lagrange(jr, lr, al, n)
                    for be in range(n + 1):
                        ez = _lagrange(jz, lz, be, n)
                        rows.append(jr * self.mz + jz)
                        cols.append(idx[lr + al, lz + be])
                        vals.append(er * ez)
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.mr * self.mz, self.n_inner))

    def _nearest_array(self, jr, jz):
        """Lower corner (lr, lz) of the (n+1)^2 array of inner indices whose
        centre is nearest to (jr, jz)."""
        n = self.n
        best, arg = None, None
        for lr in range(max(0, jr - 3 * n - 3), min(self.mr - n, jr + 3 * n + 4)):
            for lz in range(max(0, jz - 3 * n - 3), min(self.mz - n, jz + 3 * n + 4)):
                if not self.inner[lr:lr + n + 1, lz:lz + n + 1].all():
                    continue
                d = (lr + 0.5 * n - jr) ** 2 + (lz + 0.5 * n - jz) ** 2
                if best is None or d < best:
                    best, arg = d, (lr, lz)
        if arg is None:
            raise RuntimeError("no inner array near an outer B-spline; refine the grid")
        return arg

    # ---------------------------------------------------------- quadrature
    def _quadrature(self, strips):
        q = self.n + 3
        ug, wg = _gauss(q)
        R, Z, W = [], [], []
        for i in range(self.nr):
            for j in range(self.nz):
                s = self.cell_state[i, j]
                if s == 0:
                    continue
                zlo, zhi = self.z0 + j * self.hz, self.z0 + (j + 1) * self.hz
                rlo = max(self.r_lo + i * self.hr, self.geo.a)
                rhi = min(self.r_lo + (i + 1) * self.hr, self.geo.b)
                if rhi <= rlo:
                    continue
                ns = 1 if (s == 2 and rlo == self.r_lo + i * self.hr and
                           rhi == self.r_lo + (i + 1) * self.hr) else strips
                for k in range(ns):
                    a0 = rlo + (rhi - rlo) * k / ns
                    h0 = (rhi - rlo) / ns
                    for ur, wr in zip(ug, wg):
                        r = a0 + ur * h0
                        for (za, zb) in self.geo.z_intervals(r, zlo, zhi):
                            R.append(np.full(q, r))
                            Z.append(za + ug * (zb - za))
                            W.append(wr * h0 * wg * (zb - za))
        self.qr = np.concatenate(R)
        self.qz = np.concatenate(Z)
        self.qw = np.concatenate(W) * 2.0 * np.pi * self.qr   # volume weights

    # ------------------------------------------------------------ assembly
    def _full_functions(self, r, z):
        """Sparse (P x mr mz) matrices of w b_k, d/dr, d/dz at the points."""
        n = self.n
        r = np.asarray(r, float)
        z = np.asarray(z, float)
        P = len(r)
        cr = np.clip(np.floor((r - self.r_lo) / self.hr).astype(int), 0, self.nr - 1)
        cz = np.clip(np.floor((z - self.z0) / self.hz).astype(int), 0, self.nz - 1)
        Br = bspline_basis(n, self.tr, r)
        dBr = bspline_basis(n, self.tr, r, deriv=True)
        Bz = bspline_basis(n, self.tz, z)
        dBz = bspline_basis(n, self.tz, z, deriv=True)
        w, wr, wz = self.geo.weight(r, z)
        rows, cols, v0, vr, vz = [], [], [], [], []
        ar = np.arange(P)
        for k in range(n + 1):
            ir = cr + k
            br, dbr = Br[ar, ir], dBr[ar, ir]
            for l in range(n + 1):
                jz = cz + l
                bz, dbz = Bz[ar, jz], dBz[ar, jz]
                rows.append(ar)
                cols.append(ir * self.mz + jz)
                v0.append(w * br * bz)
                vr.append((wr * br + w * dbr) * bz)
                vz.append((wz * bz + w * dbz) * br)
        rows, cols = np.concatenate(rows), np.concatenate(cols)
        shape = (P, self.mr * self.mz)
        mk = lambda v: sp.csr_matrix((np.concatenate(v), (rows, cols)), shape=shape)
        return mk(v0), mk(vr), mk(vz)

    def _assemble(self):
        F0, Fr, Fz = self._full_functions(self.qr, self.qz)
        W = sp.diags(self.qw)
        A_full = EPS0 * (Fr.T @ W @ Fr + Fz.T @ W @ Fz)
        _, pr, pz = self.geo.lift(self.qr, self.qz)
        g_full = EPS0 * (Fr.T @ (self.qw * pr) + Fz.T @ (self.qw * pz))
        self.A = (self.T.T @ A_full @ self.T).tocsc()
        self.g = self.T.T @ g_full
        self._lu = splu(self.A)

    # ------------------------------------------------------- solve / eval
    def deposit(self, r, z, qw) -> np.ndarray:
        """Load of point charges on rings, in the full basis (mr mz)."""
        F0, _, _ = self._full_functions(r, z)
        return qw * np.asarray(F0.sum(axis=0)).ravel()

    def rhs_density(self, rho) -> np.ndarray:
        """Load of a charge density rho(r, z), full basis, by the domain
        quadrature."""
        F0, _, _ = self._full_functions(self.qr, self.qz)
        return F0.T @ (self.qw * rho(self.qr, self.qz))

    def solve(self, f_full, dirichlet: bool = True) -> np.ndarray:
        """Full-basis coefficients c (mr x mz) of phi - phi_D."""
        rhs = self.T.T @ np.asarray(f_full, float).ravel() - (self.g if dirichlet else 0.0)
        u = self._lu.solve(rhs)
        return (self.T @ u).reshape(self.mr, self.mz)

    def phi(self, c, r, z, dirichlet: bool = True):
        F0, _, _ = self._full_functions(r, z)
        v = F0 @ np.asarray(c).ravel()
        if dirichlet:
            v = v + self.geo.lift(r, z)[0]
        return v

    def efield(self, c, r, z, dirichlet: bool = True):
        _, Fr, Fz = self._full_functions(r, z)
        cc = np.asarray(c).ravel()
        er, ez = -(Fr @ cc), -(Fz @ cc)
        if dirichlet:
            _, pr, pz = self.geo.lift(r, z)
            er, ez = er - pr, ez - pz
        return er, ez


def _lagrange(j, lo, alpha, n):
    """Value at index j of the Lagrange polynomial of node lo + alpha on the
    nodes lo .. lo + n."""
    v = 1.0
    for mu in range(n + 1):
        if mu != alpha:
            v *= (j - (lo + mu)) / (alpha - mu)
    return v


def paper_trap(v_in=-30e3, v_out=0.0):
    """Sec. II.B's geometry: inner conductor r_a = 63.75 mm, outer cylinder
    r_b = 81 mm, z from -10 to 34 mm, a filled ellipse centred on the outer
    cylinder at z = 12 mm with axes 14 mm (z) and 3 mm (r); the axes are
    read as semi-axes."""
    return Geometry(63.75e-3, 81e-3, -10e-3, 34e-3, v_in, v_out,
                    ellipse=(81e-3, 12e-3, 3e-3, 14e-3))


# -------------------------------------------------------- potential wells

def field_line_r(r1, z1, z, bz):
    """Radius along the magnetic field line through (r1, z1) at the axial
    positions z, for B derived from A_theta = r B_z(z) / 2 (the field of
    the step): r^2 B_z(z) is constant along a line."""
    return r1 * np.sqrt(bz(z1) / bz(np.asarray(z, float)))


def well_depth_along(U):
    """Depth of the deepest well of a sampled profile U(s) along a field
    line (Sec. II.B: a well is a local maximum U_max of the potential
    energy along the line; its depth is U_max minus the higher of the
    lowest values on either side of it, U_min).  Returns (depth, index of
    U_max); (0, -1) without an interior local maximum."""
    U = np.asarray(U, float)
    best, arg = 0.0, -1
    for k in range(1, len(U) - 1):
        if U[k] >= U[k - 1] and U[k] > U[k + 1]:
            d = U[k] - max(U[:k].min(), U[k + 1:].min())
            if d > best:
                best, arg = d, k
    return best, arg


def well_depth_map(phi, inside, bz, r_starts, z1, z_min, z_max, samples=2001):
    """U_d (eV, U = e phi with phi in V) on the field lines through
    (r, z1) for r in r_starts: each line is sampled on [z_min, z_max] and
    cut to the stretch around z1 that stays inside the domain."""
    z = np.linspace(z_min, z_max, samples)
    k1 = int(np.argmin(np.abs(z - z1)))
    out = np.zeros(len(r_starts))
    for m, r1 in enumerate(r_starts):
        r = field_line_r(r1, z1, z, bz)
        ins = inside(r, z)
        if not ins[k1]:
            continue
        lo = k1
        while lo > 0 and ins[lo - 1]:
            lo -= 1
        hi = k1
        while hi < len(z) - 1 and ins[hi + 1]:
            hi += 1
        out[m] = well_depth_along(phi(r[lo:hi + 1], z[lo:hi + 1]))[0]
    return out
