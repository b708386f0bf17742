// webspline.cu -- the web-spline system for curved electrodes (arXiv
// 2206.14662, Sec. II.A: weighted extended B-splines carry curved
// Dirichlet surfaces on a rectangular grid; Sec. II.B: the coaxial gap
// with a filled ellipse on the outer cylinder).  Host assembly: the sparse
// Galerkin matrix of the extended weighted basis and its lift vector, for
// a device solver to consume.
//
// Domain: a < r < b, z_min < z < z_max, minus an optional filled ellipse
// ((r - r0)/dr)^2 + ((z - z0)/dz)^2 <= 1; V_in on r = a, V_out on r = b
// and on the ellipse; natural ends in z.  The B-spline grid spans
// [r_lo, r_hi] x [z_min, z_max] (the walls may lie between grid lines).
// Weight: w_c = (r - a)(b - r)/(b - a), with the ellipse the R-function
// conjunction x + y - sqrt(x^2 + y^2) of w_c and w_e = s (e - 1), e the
// ellipse's quadratic, s = min(dr, dz)/2.  Lift: V_in + dV t,
// t = (r - a)/(r - a + w_o), w_o the conjunction of (b - r) and w_e
// (t = (r - a)/(b - a) without the ellipse).
// Basis: tensor B-splines of degree n whose support meets the domain;
// inner when a whole grid cell of the support lies in it (exact test: the
// ellipse is convex), outer otherwise; each outer b_j is carried by the
// (n+1)^2 array of inner indices nearest to it with the Lagrange
// coefficients of its index, so B_i = b_i + sum_j e_ij b_j keeps
// polynomials of degree <= n.  Trial and test functions w B_i.
// Quadrature: Gauss points on whole cells; cut cells in r-strips with the
// exact inside z-intervals at each r-point.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "pic.h"
#include "pic_internal.cuh"

namespace pic {
namespace web {

constexpr int kMaxDeg = PIC_SPLINE_MAX_DEGREE;

// the p + 1 non-zero uniform B-splines of degree p on a knot span at local
// coordinate u (triangular Cox-de Boor scheme, distances in units of the
// spacing) and their derivatives for spacing h
void span_basis_d(int p, double u, double h, double* N, double* dN) {
  double M[kMaxDeg + 1];
  auto basis = [](int q, double x, double* B) {
    B[0] = 1.0;
    for (int j = 1; j <= q; ++j) {
      double saved = 0.0;
      for (int r = 0; r < j; ++r) {
        const double tmp = B[r] / j;
        B[r] = saved + (r + 1 - x) * tmp;
        saved = (x + j - r - 1) * tmp;
      }
      B[j] = saved;
    }
  };
  basis(p, u, N);
  if (p == 0) {
    dN[0] = 0.0;
    return;
  }
  basis(p - 1, u, M);
  for (int r = 0; r <= p; ++r) dN[r] = ((r >= 1 ? M[r - 1] : 0.0) - (r <= p - 1 ? M[r] : 0.0)) / h;
}

void gauss01(int q, double* x, double* w) {   // Gauss-Legendre on [0, 1]
  for (int i = 0; i < q; ++i) {
    double t = std::cos(kPi * (i + 0.75) / (q + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= q; ++k) {
        const double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = q * (t * p1 - p0) / (t * t - 1.0);
      const double d = p1 / dp;
      t -= d;
      if (std::fabs(d) < 1e-16) break;
    }
    x[i] = 0.5 * (t + 1.0);
    w[i] = 1.0 / ((1.0 - t * t) * dp * dp);
  }
}

struct Geo {
  double a, b, z0, z1, v_in, v_out;
  bool ell;
  double er, ez, edr, edz;

  void w_e(double r, double z, double& v, double& gr, double& gz) const {
    const double s = 0.5 * std::min(edr, edz);
    v = s * (((r - er) / edr) * ((r - er) / edr) + ((z - ez) / edz) * ((z - ez) / edz) - 1.0);
    gr = s * 2.0 * (r - er) / (edr * edr);
    gz = s * 2.0 * (z - ez) / (edz * edz);
  }
  static void conj(double x, double gx0, double gx1, double y, double gy0, double gy1, double& v,
                   double& g0, double& g1) {
    const double q = std::sqrt(x * x + y * y), qs = q > 0 ? q : 1.0;
    v = x + y - q;
    g0 = gx0 + gy0 - (x * gx0 + y * gy0) / qs;
    g1 = gx1 + gy1 - (x * gx1 + y * gy1) / qs;
  }
  void weight(double r, double z, double& w, double& wr, double& wz) const {
    const double ab = b - a;
    const double wc = (r - a) * (b - r) / ab, gc = (a + b - 2.0 * r) / ab;
    if (!ell) {
      w = wc;
      wr = gc;
      wz = 0.0;
      return;
    }
    double v, gr, gz;
    w_e(r, z, v, gr, gz);
    conj(wc, gc, 0.0, v, gr, gz, w, wr, wz);
  }
  void lift(double r, double z, double& p, double& pr, double& pz) const {
    const double dv = v_out - v_in;
    if (!ell) {
      p = v_in + dv * (r - a) / (b - a);
      pr = dv / (b - a);
      pz = 0.0;
      return;
    }
    double v, gr, gz, wo, g0, g1;
    w_e(r, z, v, gr, gz);
    conj(b - r, -1.0, 0.0, v, gr, gz, wo, g0, g1);
    const double x = r - a, den = x + wo;
    p = v_in + dv * x / den;
    pr = dv * (den - x * (1.0 + g0)) / (den * den);
    pz = dv * (-x * g1) / (den * den);
  }
  int cell_state(double r0, double r1, double za, double zb) const {
    const double tol = 1e-12 * (b - a);
    if (r1 <= a + tol || r0 >= b - tol) return 0;
    const bool in_walls = r0 >= a - tol && r1 <= b + tol;
    if (!ell) return in_walls ? 2 : 1;
    auto e = [&](double r, double z) {
      return ((r - er) / edr) * ((r - er) / edr) + ((z - ez) / edz) * ((z - ez) / edz);
    };
    const double ra = std::max(r0, a), rb = std::min(r1, b);
    double cmax = 0.0;
    for (double r : {ra, rb})
      for (double z : {za, zb}) cmax = std::max(cmax, e(r, z));
    if (cmax <= 1.0) return 0;
    const double emin = e(std::min(std::max(er, r0), r1), std::min(std::max(ez, za), zb));
    return (in_walls && emin >= 1.0) ? 2 : 1;
  }
  // inside z-intervals of [lo, hi] at radius r; returns their count (<= 2)
  int z_intervals(double r, double lo, double hi, double* zl, double* zh) const {
    if (!ell || std::fabs((r - er) / edr) >= 1.0) {
      zl[0] = lo;
      zh[0] = hi;
      return 1;
    }
    const double x = (r - er) / edr, hh = edz * std::sqrt(1.0 - x * x);
    int k = 0;
    if (lo < ez - hh) { zl[k] = lo; zh[k] = std::min(hi, ez - hh); ++k; }
    if (hi > ez + hh) { zl[k] = std::max(lo, ez + hh); zh[k] = hi; ++k; }
    return k;
  }
};

}  // namespace web
}  // namespace pic

using namespace pic;

struct pic_web {
  web::Geo G;
  int n, nr, nz, mr, mz;
  double r_lo, hr, hz;
  std::vector<int> inner_full;                 // full index of inner function i
  std::vector<int> t_ptr, t_col;               // extension T: full row -> inner columns
  std::vector<double> t_val;
  std::vector<int> a_ptr, a_col;               // A (inner x inner, CSR, sorted columns)
  std::vector<double> a_val, g;                // g: lift load (inner)
};

namespace {

int build(pic_web* W, const pic_config* c, const double* ellipse, double r_lo, double r_hi,
          int nr, int n) {
  using namespace pic::web;
  W->G = Geo{c->r_in, c->r_out, c->z_min, c->z_max, c->v_inner, c->v_outer, ellipse != nullptr,
             ellipse ? ellipse[0] : 0.0, ellipse ? ellipse[1] : 0.0, ellipse ? ellipse[2] : 1.0,
             ellipse ? ellipse[3] : 1.0};
  W->n = n;
  W->nr = nr;
  W->nz = c->nz;
  W->mr = nr + n;
  W->mz = c->nz + n;
  W->r_lo = r_lo;
  W->hr = (r_hi - r_lo) / nr;
  W->hz = (c->z_max - c->z_min) / c->nz;
  const int mr = W->mr, mz = W->mz, NZ = W->nz;
  const Geo& G = W->G;
  // cells
  std::vector<int> st((size_t)nr * NZ);
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < NZ; ++j)
      st[(size_t)i * NZ + j] = G.cell_state(r_lo + i * W->hr, r_lo + (i + 1) * W->hr,
                                            G.z0 + j * W->hz, G.z0 + (j + 1) * W->hz);
  // functions: inner / outer
  std::vector<char> inner((size_t)mr * mz, 0), outer((size_t)mr * mz, 0);
  for (int i = 0; i < mr; ++i)
    for (int j = 0; j < mz; ++j) {
      bool any2 = false, any1 = false;
      for (int ci = std::max(i - n, 0); ci <= std::min(i, nr - 1); ++ci)
        for (int cj = std::max(j - n, 0); cj <= std::min(j, NZ - 1); ++cj) {
          const int s = st[(size_t)ci * NZ + cj];
          any2 |= s == 2;
          any1 |= s >= 1;
        }
      inner[(size_t)i * mz + j] = any2;
      outer[(size_t)i * mz + j] = any1 && !any2;
    }
  std::vector<int> idx((size_t)mr * mz, -1);
  for (int k = 0; k < mr * mz; ++k)
    if (inner[k]) {
      idx[k] = (int)W->inner_full.size();
      W->inner_full.push_back(k);
    }
  const int ni = (int)W->inner_full.size();
  if (ni == 0) return PIC_EINVAL;
  // extension T (rows: full functions, CSR)
  std::vector<std::vector<std::pair<int, double>>> trow((size_t)mr * mz);
  for (int k = 0; k < mr * mz; ++k)
    if (inner[k]) trow[k].push_back({idx[k], 1.0});
  for (int jr = 0; jr < mr; ++jr)
    for (int jz = 0; jz < mz; ++jz) {
      if (!outer[(size_t)jr * mz + jz]) continue;
      double best = -1.0;
      int lr = -1, lz = -1;
      for (int r0 = std::max(0, jr - 3 * n - 3); r0 < std::min(mr - n, jr + 3 * n + 4); ++r0)
        for (int z0 = std::max(0, jz - 3 * n - 3); z0 < std::min(mz - n, jz + 3 * n + 4); ++z0) {
          bool all = true;
          for (int a = 0; a <= n && all; ++a)
            for (int bb = 0; bb <= n && all; ++bb) all = inner[(size_t)(r0 + a) * mz + z0 + bb];
          if (!all) continue;
          const double d = (r0 + 0.5 * n - jr) * (r0 + 0.5 * n - jr) +
                           (z0 + 0.5 * n - jz) * (z0 + 0.5 * n - jz);
          if (best < 0 || d < best) {
            best = d;
            lr = r0;
            lz = z0;
          }
        }
      if (lr < 0) return PIC_EINVAL;   // grid too coarse for the geometry
      auto lag = [&](int j, int lo, int al) {
        double v = 1.0;
        for (int mu = 0; mu <= n; ++mu)
          if (mu != al) v *= (double)(j - (lo + mu)) / (al - mu);
        return v;
      };
      for (int al = 0; al <= n; ++al)
        for (int be = 0; be <= n; ++be)
          trow[(size_t)jr * mz + jz].push_back(
              {idx[(size_t)(lr + al) * mz + lz + be], lag(jr, lr, al) * lag(jz, lz, be)});
    }
  W->t_ptr.assign(1, 0);
  for (auto& row : trow) {
    for (auto& e : row) {
      W->t_col.push_back(e.first);
      W->t_val.push_back(e.second);
    }
    W->t_ptr.push_back((int)W->t_col.size());
  }
  // quadrature and assembly of A = T^T A_full T, g = T^T g_full
  const int q = n + 3, strips = 8;
  double xg[kMaxDeg + 4], wg[kMaxDeg + 4];
  gauss01(q, xg, wg);
  std::vector<std::map<int, double>> A(ni);
  W->g.assign(ni, 0.0);
  const int L = (n + 1) * (n + 1);
  std::vector<int> fi(L);
  std::vector<double> v0(L), vr(L), vz(L);
  auto point = [&](double r, double z, double wq) {
    const int cr = std::min(std::max((int)std::floor((r - r_lo) / W->hr), 0), nr - 1);
    const int cz = std::min(std::max((int)std::floor((z - G.z0) / W->hz), 0), NZ - 1);
    double Nr[kMaxDeg + 1], dNr[kMaxDeg + 1], Nz[kMaxDeg + 1], dNz[kMaxDeg + 1];
    span_basis_d(n, (r - r_lo) / W->hr - cr, W->hr, Nr, dNr);
    span_basis_d(n, (z - G.z0) / W->hz - cz, W->hz, Nz, dNz);
    double w, wr, wz, p, pr, pz;
    G.weight(r, z, w, wr, wz);
    G.lift(r, z, p, pr, pz);
    for (int k = 0; k <= n; ++k)
      for (int l = 0; l <= n; ++l) {
        const int m = k * (n + 1) + l;
        fi[m] = (cr + k) * mz + cz + l;
        v0[m] = w * Nr[k] * Nz[l];
        vr[m] = (wr * Nr[k] + w * dNr[k]) * Nz[l];
        vz[m] = (wz * Nz[l] + w * dNz[l]) * Nr[k];
      }
    const double c = kEps0 * wq * 2.0 * kPi * r;
    for (int m = 0; m < L; ++m) {
      const int f = fi[m];
      for (int e = W->t_ptr[f]; e < W->t_ptr[f + 1]; ++e) {
        const int i = W->t_col[e];
        const double ti = W->t_val[e];
        W->g[i] += ti * c * (vr[m] * pr + vz[m] * pz);
        for (int m2 = 0; m2 < L; ++m2) {
          const double a = c * (vr[m] * vr[m2] + vz[m] * vz[m2]);
          if (a == 0.0) continue;
          const int f2 = fi[m2];
          for (int e2 = W->t_ptr[f2]; e2 < W->t_ptr[f2 + 1]; ++e2)
            A[i][W->t_col[e2]] += ti * W->t_val[e2] * a;
        }
      }
    }
  };
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < NZ; ++j) {
      const int s = st[(size_t)i * NZ + j];
      if (s == 0) continue;
      const double c0 = r_lo + i * W->hr, c1 = r_lo + (i + 1) * W->hr;
      const double rlo = std::max(c0, G.a), rhi = std::min(c1, G.b);
      if (rhi <= rlo) continue;
      const double zlo = G.z0 + j * W->hz, zhi = G.z0 + (j + 1) * W->hz;
      const int ns = (s == 2 && rlo == c0 && rhi == c1) ? 1 : strips;
      for (int k = 0; k < ns; ++k) {
        const double a0 = rlo + (rhi - rlo) * k / ns, h0 = (rhi - rlo) / ns;
        for (int qr = 0; qr < q; ++qr) {
          const double r = a0 + xg[qr] * h0;
          double zl[2], zh[2];
          const int nint = G.z_intervals(r, zlo, zhi, zl, zh);
          for (int t = 0; t < nint; ++t)
            for (int qz = 0; qz < q; ++qz)
              point(r, zl[t] + xg[qz] * (zh[t] - zl[t]), wg[qr] * h0 * wg[qz] * (zh[t] - zl[t]));
        }
      }
    }
  W->a_ptr.assign(1, 0);
  for (int i = 0; i < ni; ++i) {
    for (auto& e : A[i]) {
      W->a_col.push_back(e.first);
      W->a_val.push_back(e.second);
    }
    W->a_ptr.push_back((int)W->a_col.size());
  }
  return PIC_OK;
}

}  // namespace

extern "C" {

int pic_web_create(const pic_config* cfg, const double* ellipse, double r_lo, double r_hi,
                   int nr, int degree, pic_web** out) {
  if (!out) return PIC_EINVAL;
  *out = nullptr;
  if (!cfg || degree < 1 || degree > PIC_SPLINE_MAX_DEGREE || nr < 2 || cfg->nz < 2 ||
      !(cfg->r_in > 0 && cfg->r_out > cfg->r_in && cfg->z_max > cfg->z_min) ||
      !(r_lo <= cfg->r_in && r_hi >= cfg->r_out && r_hi > r_lo))
    return PIC_EINVAL;
  if (ellipse && !(ellipse[2] > 0 && ellipse[3] > 0)) return PIC_EINVAL;
  pic_web* W = new pic_web();
  const int rc = build(W, cfg, ellipse, r_lo, r_hi, nr, degree);
  if (rc) {
    delete W;
    return rc;
  }
  *out = W;
  return PIC_OK;
}

void pic_web_free(pic_web* w) { delete w; }

int pic_web_sizes(const pic_web* w, int* n_inner, int64_t* nnz, int64_t* t_nnz, int* mr, int* mz) {
  if (!w) return PIC_EINVAL;
  if (n_inner) *n_inner = (int)w->inner_full.size();
  if (nnz) *nnz = (int64_t)w->a_val.size();
  if (t_nnz) *t_nnz = (int64_t)w->t_val.size();
  if (mr) *mr = w->mr;
  if (mz) *mz = w->mz;
  return PIC_OK;
}

int pic_web_export(const pic_web* w, int* a_ptr, int* a_col, double* a_val, double* g,
                   int* inner_full, int* t_ptr, int* t_col, double* t_val) {
  if (!w) return PIC_EINVAL;
  auto put = [](auto* dst, const auto& v) {
    if (dst) std::memcpy(dst, v.data(), v.size() * sizeof(v[0]));
  };
  put(a_ptr, w->a_ptr);
  put(a_col, w->a_col);
  put(a_val, w->a_val);
  put(g, w->g);
  put(inner_full, w->inner_full);
  put(t_ptr, w->t_ptr);
  put(t_col, w->t_col);
  put(t_val, w->t_val);
  return PIC_OK;
}

}  // extern "C"
