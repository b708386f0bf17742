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
__host__ __device__ inline void span_basis_d(int p, double u, double h, double* N, double* dN) {
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

  __host__ __device__ void w_e(double r, double z, double& v, double& gr, double& gz) const {
    const double s = 0.5 * fmin(edr, edz);
    v = s * (((r - er) / edr) * ((r - er) / edr) + ((z - ez) / edz) * ((z - ez) / edz) - 1.0);
    gr = s * 2.0 * (r - er) / (edr * edr);
    gz = s * 2.0 * (z - ez) / (edz * edz);
  }
  __host__ __device__ static void conj(double x, double gx0, double gx1, double y, double gy0, double gy1, double& v,
                   double& g0, double& g1) {
    const double q = sqrt(x * x + y * y), qs = q > 0 ? q : 1.0;
    v = x + y - q;
    g0 = gx0 + gy0 - (x * gx0 + y * gy0) / qs;
    g1 = gx1 + gy1 - (x * gx1 + y * gy1) / qs;
  }
  __host__ __device__ void weight(double r, double z, double& w, double& wr, double& wz) const {
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
  __host__ __device__ void lift(double r, double z, double& p, double& pr, double& pz) const {
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

namespace pic {
namespace web {
// device copies and work vectors of a web-spline system (pic_web_device)
struct Dev {
  cudaStream_t stream = nullptr;
  int device = 0;              // the device the arrays live on
  int *a_ptr = nullptr, *a_col = nullptr, *inner_full = nullptr;
  int *t_ptr = nullptr, *t_col = nullptr, *tt_ptr = nullptr, *tt_col = nullptr;
  double *a_val = nullptr, *g = nullptr, *t_val = nullptr, *tt_val = nullptr;
  double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  double *full = nullptr, *full2 = nullptr, *dots = nullptr;
  double* scale = nullptr;     // sqrt(diag S / diag A) on the inner functions
  double* inv = nullptr;       // A^-1 (n_inner x n_inner), pic_web_direct
  pic_spline* pre = nullptr;   // the enclosing box's solver: the preconditioner
};
}  // namespace web
}  // namespace pic

struct pic_web {
  pic_config box;            // the grid box as a config (walls at the grid's ends)
  pic::web::Dev* dev = nullptr;
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

// A^-1 of the SPD system: Cholesky A = L L^T, L^-1 by forward substitution,
// A^-1 = L^-T L^-1 (dense, row-major; false if A is not positive definite)
bool dense_inverse(const pic_web* W, std::vector<double>& inv) {
  const int n = (int)W->inner_full.size();
  std::vector<double> L((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int e = W->a_ptr[i]; e < W->a_ptr[i + 1]; ++e)
      if (W->a_col[e] <= i) L[(size_t)i * n + W->a_col[e]] = W->a_val[e];
  for (int j = 0; j < n; ++j) {   // right-looking Cholesky, column j
    double* Lj = &L[(size_t)j * n];
    double d = Lj[j];
    for (int k = 0; k < j; ++k) d -= Lj[k] * Lj[k];
    if (!(d > 0)) return false;
    d = std::sqrt(d);
    Lj[j] = d;
    for (int i = j + 1; i < n; ++i) {
      double* Li = &L[(size_t)i * n];
      double s = Li[j];
      for (int k = 0; k < j; ++k) s -= Li[k] * Lj[k];
      Li[j] = s / d;
    }
  }
  // X = L^-1 (lower), row by row: X[i][j] = (delta_ij - sum_{j<=k<i} L[i][k] X[k][j]) / L[i][i]
  std::vector<double> X((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    const double* Li = &L[(size_t)i * n];
    double* Xi = &X[(size_t)i * n];
    for (int k = 0; k < i; ++k) {
      const double lik = Li[k];
      if (lik == 0.0) continue;
      const double* Xk = &X[(size_t)k * n];
      for (int j = 0; j <= k; ++j) Xi[j] -= lik * Xk[j];
    }
    Xi[i] += 1.0;
    for (int j = 0; j <= i; ++j) Xi[j] /= Li[i];
  }
  // A^-1 = X^T X: entry (a, b) = sum_{k >= max(a, b)} X[k][a] X[k][b]
  inv.assign((size_t)n * n, 0.0);
  for (int k = 0; k < n; ++k) {
    const double* Xk = &X[(size_t)k * n];
    for (int a = 0; a <= k; ++a) {
      const double xa = Xk[a];
      if (xa == 0.0) continue;
      double* row = &inv[(size_t)a * n];
      for (int b = 0; b <= a; ++b) row[b] += xa * Xk[b];
    }
  }
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < a; ++b) inv[(size_t)b * n + a] = inv[(size_t)a * n + b];
  return true;
}

}  // namespace

extern "C" {

int pic_web_inverse(const pic_web* w, double* out) {
  if (!w || !out) return PIC_EINVAL;
  std::vector<double> inv;
  if (!dense_inverse(w, inv)) return PIC_ENOCONV;
  std::memcpy(out, inv.data(), inv.size() * sizeof(double));
  return PIC_OK;
}

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
  W->box = *cfg;
  W->box.r_in = r_lo;
  W->box.r_out = r_hi;
  W->box.nr = nr;
  const int rc = build(W, cfg, ellipse, r_lo, r_hi, nr, degree);
  if (rc) {
    delete W;
    return rc;
  }
  *out = W;
  return PIC_OK;
}

void pic_web_free(pic_web* w) {
  if (!w) return;
  if (w->dev) {
    pic::web::Dev* d = w->dev;
    for (void* ptr : {(void*)d->a_ptr, (void*)d->a_col, (void*)d->inner_full, (void*)d->t_ptr,
                      (void*)d->t_col, (void*)d->tt_ptr, (void*)d->tt_col, (void*)d->a_val,
                      (void*)d->g, (void*)d->t_val, (void*)d->tt_val, (void*)d->x, (void*)d->r,
                      (void*)d->z, (void*)d->p, (void*)d->q, (void*)d->full, (void*)d->full2,
                      (void*)d->dots, (void*)d->scale, (void*)d->inv})
      if (ptr) cudaFree(ptr);
    pic_spline_free(d->pre);
    delete d;
  }
  delete w;
}

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

// ------------------------------------------------------------------ device

namespace pic {
namespace web {

// y = A x, one warp per row (rows hold a few dozen entries)
__global__ void k_spmv(int rows, const int* __restrict__ ptr, const int* __restrict__ col,
                       const double* __restrict__ val, const double* __restrict__ x,
                       double* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  for (long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; row < rows;
       row += ((long long)gridDim.x * blockDim.x) >> 5) {
    double s = 0.0;
    for (int e = ptr[row] + lane; e < ptr[row + 1]; e += 32) s = fma(val[e], x[col[e]], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s;
  }
}

// y = M x for a dense row-major n x n matrix, one warp per row
__global__ void k_gemv(int n, const double* __restrict__ M, const double* __restrict__ x,
                       double* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  for (long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; row < n;
       row += ((long long)gridDim.x * blockDim.x) >> 5) {
    const double* m = M + row * (long long)n;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s = fma(m[j], x[j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s;
  }
}

// out[0] += a . b, out[1] += b . b (block sums, one atomic each)
__global__ void k_dots(int n, const double* __restrict__ a, const double* __restrict__ b,
                       double* out) {
  __shared__ double sa[32], sb[32];
  double ab = 0.0, bb = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    ab = fma(a[i], b[i], ab);
    bb = fma(b[i], b[i], bb);
  }
  for (int o = 16; o > 0; o >>= 1) {
    ab += __shfl_xor_sync(0xffffffffu, ab, o);
    bb += __shfl_xor_sync(0xffffffffu, bb, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sa[w] = ab; sb[w] = bb; }
  __syncthreads();
  if (w == 0) {
    ab = lane < (int)(blockDim.x >> 5) ? sa[lane] : 0.0;
    bb = lane < (int)(blockDim.x >> 5) ? sb[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      ab += __shfl_xor_sync(0xffffffffu, ab, o);
      bb += __shfl_xor_sync(0xffffffffu, bb, o);
    }
    if (lane == 0) {
      atomicAdd(out, ab);
      atomicAdd(out + 1, bb);
    }
  }
}

// y = alpha x + beta y
__global__ void k_axpby(int n, double alpha, const double* __restrict__ x, double beta,
                        double* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    y[i] = alpha * x[i] + beta * y[i];
}

// dst[idx[i]] = s[i] src[i] and dst[i] = s[i] src[idx[i]]
__global__ void k_scatter(int n, const int* __restrict__ idx, const double* __restrict__ s,
                          const double* __restrict__ src, double* __restrict__ dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[idx[i]] = s[i] * src[i];
}

__global__ void k_gather(int n, const int* __restrict__ idx, const double* __restrict__ s,
                         const double* __restrict__ src, double* __restrict__ dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = s[i] * src[idx[i]];
}

struct Grid {
  int n, nr, nz, mz;
  double r_lo, z0, hr, hz;
};

__device__ __forceinline__ int span(double x, double lo, double h, int cells, double& u) {
  int c = (int)floor((x - lo) / h);
  c = min(max(c, 0), cells - 1);
  u = (x - lo) / h - c;
  return c;
}

__global__ void k_web_deposit(Geo G, Grid D, const double* __restrict__ r,
                              const double* __restrict__ z, long long np, double qw,
                              double* __restrict__ f) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    double ur, uz, Nr[kMaxDeg + 1], dNr[kMaxDeg + 1], Nz[kMaxDeg + 1], dNz[kMaxDeg + 1];
    const int cr = span(r[p], D.r_lo, D.hr, D.nr, ur), cz = span(z[p], D.z0, D.hz, D.nz, uz);
    span_basis_d(D.n, ur, D.hr, Nr, dNr);
    span_basis_d(D.n, uz, D.hz, Nz, dNz);
    double w, wr, wz;
    G.weight(r[p], z[p], w, wr, wz);
    for (int k = 0; k <= D.n; ++k)
      for (int l = 0; l <= D.n; ++l)
        atomicAdd(f + (size_t)(cr + k) * D.mz + cz + l, qw * w * Nr[k] * Nz[l]);
  }
}

__global__ void k_web_eval(Geo G, Grid D, const double* __restrict__ c,
                           const double* __restrict__ r, const double* __restrict__ z,
                           long long np, int dirichlet, double* __restrict__ phi,
                           double* __restrict__ er, double* __restrict__ ez) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    double ur, uz, Nr[kMaxDeg + 1], dNr[kMaxDeg + 1], Nz[kMaxDeg + 1], dNz[kMaxDeg + 1];
    const int cr = span(r[p], D.r_lo, D.hr, D.nr, ur), cz = span(z[p], D.z0, D.hz, D.nz, uz);
    span_basis_d(D.n, ur, D.hr, Nr, dNr);
    span_basis_d(D.n, uz, D.hz, Nz, dNz);
    double w, wr, wz;
    G.weight(r[p], z[p], w, wr, wz);
    double s = 0.0, sr = 0.0, sz = 0.0;   // sum c b, d/dr, d/dz (without the weight)
    for (int k = 0; k <= D.n; ++k) {
      const double* row = c + (size_t)(cr + k) * D.mz + cz;
      for (int l = 0; l <= D.n; ++l) {
        s = fma(row[l], Nr[k] * Nz[l], s);
        sr = fma(row[l], dNr[k] * Nz[l], sr);
        sz = fma(row[l], Nr[k] * dNz[l], sz);
      }
    }
    double v = w * s, gr = wr * s + w * sr, gz = wz * s + w * sz;
    if (dirichlet) {
      double pl, pr, pz;
      G.lift(r[p], z[p], pl, pr, pz);
      v += pl;
      gr += pr;
      gz += pz;
    }
    if (phi) phi[p] = v;
    if (er) er[p] = -gr;
    if (ez) ez[p] = -gz;
  }
}

// the magnetic field of the step on the axis-parallel coordinate: B_z(z)
// uniform b0, or the mirror b0 (1 + 2 (z - z_mid)^2 / L^2); field lines
// keep r^2 B_z(z)
struct BzModel {
  int kind;
  double b0, z_mid, L;
  __device__ double operator()(double z) const {
    if (kind != 1) return b0;
    const double s = (z - z_mid) / L;
    return b0 * (1.0 + 2.0 * s * s);
  }
};

__device__ __forceinline__ bool geo_inside(const Geo& G, double r, double z) {
  bool ok = r > G.a && r < G.b && z > G.z0 && z < G.z1;
  if (G.ell) {
    const double x = (r - G.er) / G.edr, y = (z - G.ez) / G.edz;
    ok = ok && x * x + y * y > 1.0;
  }
  return ok;
}

__device__ __forceinline__ double web_phi(const Geo& G, const Grid& D, const double* c, double r,
                                          double z) {
  double ur, uz, Nr[kMaxDeg + 1], dNr[kMaxDeg + 1], Nz[kMaxDeg + 1], dNz[kMaxDeg + 1];
  const int cr = span(r, D.r_lo, D.hr, D.nr, ur), cz = span(z, D.z0, D.hz, D.nz, uz);
  span_basis_d(D.n, ur, D.hr, Nr, dNr);
  span_basis_d(D.n, uz, D.hz, Nz, dNz);
  double w, wr, wz, pl, pr, pz;
  G.weight(r, z, w, wr, wz);
  G.lift(r, z, pl, pr, pz);
  double s = 0.0;
  for (int k = 0; k <= D.n; ++k) {
    const double* row = c + (size_t)(cr + k) * D.mz + cz;
    for (int l = 0; l <= D.n; ++l) s = fma(row[l], Nr[k] * Nz[l], s);
  }
  return pl + w * s;
}

// Potential-well depth along field lines (one thread per line): samples
// z_k = z_min + k (z_max - z_min)/(S - 1), r_k = r1 sqrt(B_z(z1)/B_z(z_k));
// U = e phi (eV) on the stretch around the sample nearest z1 that stays
// in the domain; the deepest interior local maximum, its depth measured to
// the higher of the lowest values on either side.  scratch holds S doubles
// per line (the suffix minima).
__global__ void k_well_depth(Geo G, Grid D, BzModel B, const double* __restrict__ c,
                             const double* __restrict__ r_start, int lines, double z1, int S,
                             double* __restrict__ U, double* __restrict__ smin,
                             double* __restrict__ depth, double* __restrict__ z_at) {
  const int line = blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= lines) return;
  double* u = U + (size_t)line * S;
  double* sm = smin + (size_t)line * S;
  const double dz = (G.z1 - G.z0) / (S - 1);
  const double r1 = r_start[line], b1 = B(z1);
  int k1 = (int)floor((z1 - G.z0) / dz + 0.5);
  k1 = min(max(k1, 0), S - 1);
  depth[line] = 0.0;
  z_at[line] = nan("");
  auto rz = [&](int k, double& r, double& z) {
    z = G.z0 + k * dz;
    r = r1 * sqrt(b1 / B(z));
  };
  double r, z;
  rz(k1, r, z);
  if (!geo_inside(G, r, z)) return;
  int lo = k1, hi = k1;
  while (lo > 0) {
    rz(lo - 1, r, z);
    if (!geo_inside(G, r, z)) break;
    --lo;
  }
  while (hi < S - 1) {
    rz(hi + 1, r, z);
    if (!geo_inside(G, r, z)) break;
    ++hi;
  }
  for (int k = lo; k <= hi; ++k) {
    rz(k, r, z);
    u[k] = web_phi(G, D, c, r, z);   // U in eV for phi in V
  }
  double m = INFINITY;   // suffix minima: sm[k] = min U[k + 1 .. hi]
  for (int k = hi; k >= lo; --k) {
    sm[k] = m;
    m = fmin(m, u[k]);
  }
  double left = u[lo], best = 0.0;
  int arg = -1;
  for (int k = lo + 1; k < hi; ++k) {
    if (u[k] >= u[k - 1] && u[k] > u[k + 1]) {
      const double d = u[k] - fmax(left, sm[k]);
      if (d > best) {
        best = d;
        arg = k;
      }
    }
    left = fmin(left, u[k]);
  }
  depth[line] = best;
  if (arg >= 0) z_at[line] = G.z0 + arg * dz;
}

inline int blocks_for(long long n, int threads) {
  return (int)std::max<long long>(1, std::min<long long>((n + threads - 1) / threads, 152 * 8));
}

}  // namespace web
}  // namespace pic

extern "C" {

int pic_web_device(pic_web* w, void* cuda_stream) {
  using namespace pic::web;
  if (!w) return PIC_EINVAL;
  if (w->dev) return PIC_OK;
  Dev* d = new Dev();
  d->stream = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&d->device) != cudaSuccess) {
    delete d;
    return PIC_ECUDA;
  }
  w->dev = d;
  const int ni = (int)w->inner_full.size(), nf = w->mr * w->mz;
  // T^T (inner rows) from T (full rows)
  std::vector<int> tt_ptr(ni + 1, 0), tt_col(w->t_col.size());
  std::vector<double> tt_val(w->t_val.size());
  for (int c : w->t_col) ++tt_ptr[c + 1];
  for (int i = 0; i < ni; ++i) tt_ptr[i + 1] += tt_ptr[i];
  std::vector<int> fill(tt_ptr.begin(), tt_ptr.end() - 1);
  for (int row = 0; row < nf; ++row)
    for (int e = w->t_ptr[row]; e < w->t_ptr[row + 1]; ++e) {
      const int k = fill[w->t_col[e]]++;
      tt_col[k] = row;
      tt_val[k] = w->t_val[e];
    }
  bool ok = true;
  auto up = [&](auto*& dst, const auto& v) {
    using T = std::remove_reference_t<decltype(v[0])>;
    if (!ok) return;
    ok = cudaMalloc((void**)&dst, std::max<size_t>(v.size(), 1) * sizeof(T)) == cudaSuccess &&
         (v.empty() || cudaMemcpy(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) ==
                           cudaSuccess);
  };
  auto zeros = [&](double*& dst, size_t n) {
    if (!ok) return;
    ok = cudaMalloc((void**)&dst, std::max<size_t>(n, 1) * sizeof(double)) == cudaSuccess;
  };
  up(d->a_ptr, w->a_ptr);
  up(d->a_col, w->a_col);
  up(d->a_val, w->a_val);
  up(d->g, w->g);
  up(d->inner_full, w->inner_full);
  up(d->t_ptr, w->t_ptr);
  up(d->t_col, w->t_col);
  up(d->t_val, w->t_val);
  up(d->tt_ptr, tt_ptr);
  up(d->tt_col, tt_col);
  up(d->tt_val, tt_val);
  // preconditioner scale: sqrt(diag S / diag A), S the box system
  // 2 pi eps0 (K_r (x) M_z + M_r (x) K_z) on the inner functions; the web
  // functions near the ellipse carry a small weight, so without it the
  // box operator is far from A there
  {
    const int mr = w->mr, mz = w->mz;
    std::vector<double> Kr((size_t)mr * mr), Mr((size_t)mr * mr), Kz((size_t)mz * mz),
        Mz((size_t)mz * mz);
    if (pic_spline_matrices(&w->box, w->n, Kr.data(), Mr.data(), nullptr, Kz.data(), Mz.data(),
                            nullptr) != PIC_OK)
      return PIC_EINVAL;
    std::vector<double> sc(ni);
    for (int i = 0; i < ni; ++i) {
      const int f = w->inner_full[i], ir = f / mz, jz = f % mz;
      const double dS = 2.0 * kPi * kEps0 *
                        (Kr[(size_t)ir * mr + ir] * Mz[(size_t)jz * mz + jz] +
                         Mr[(size_t)ir * mr + ir] * Kz[(size_t)jz * mz + jz]);
      double dA = 0.0;
      for (int e = w->a_ptr[i]; e < w->a_ptr[i + 1]; ++e)
        if (w->a_col[e] == i) dA = w->a_val[e];
      sc[i] = dA > 0 ? std::sqrt(dS / dA) : 1.0;
    }
    up(d->scale, sc);
  }
  for (double** v : {&d->x, &d->r, &d->z, &d->p, &d->q}) zeros(*v, ni);
  zeros(d->full, nf);
  zeros(d->full2, nf);
  zeros(d->dots, 2);
  if (!ok) {
    cudaGetLastError();
    return PIC_ENOMEM;
  }
  return pic_spline_create(&w->box, w->n, cuda_stream, &d->pre);
}

int pic_web_solve(pic_web* w, const double* f_full, double* c_full, int dirichlet, double rtol,
                  int maxit, int* iters, double* relres) {
  using namespace pic::web;
  if (!w || !w->dev || !f_full || !c_full || !(rtol > 0) || maxit < 1) return PIC_EINVAL;
  Dev* d = w->dev;
  cudaStream_t st = d->stream;
  const int ni = (int)w->inner_full.size(), nf = w->mr * w->mz;
  const int bi = blocks_for(ni, 256);
  const int bw = blocks_for((long long)ni * 32, 256), bwf = blocks_for((long long)nf * 32, 256);
  double h[2];
  auto dots = [&](const double* a, const double* b) -> bool {
    cudaMemsetAsync(d->dots, 0, 2 * sizeof(double), st);
    k_dots<<<bi, 256, 0, st>>>(ni, a, b, d->dots);
    return cudaMemcpyAsync(h, d->dots, 2 * sizeof(double), cudaMemcpyDeviceToHost, st) ==
               cudaSuccess &&
           cudaStreamSynchronize(st) == cudaSuccess;
  };
  // preconditioner z = D P^T S^-1 P D r (S: the box's weighted B-spline
  // system, D the diagonal rescaling)
  auto precond = [&](const double* r, double* z) -> int {
    cudaMemsetAsync(d->full, 0, (size_t)nf * sizeof(double), st);
    k_scatter<<<bi, 256, 0, st>>>(ni, d->inner_full, d->scale, r, d->full);
    const int rc = pic_spline_solve(d->pre, d->full, d->full2, 0);
    k_gather<<<bi, 256, 0, st>>>(ni, d->inner_full, d->scale, d->full2, z);
    return rc;
  };
  // right-hand side b = T^T f - [dirichlet] g, held in r; x = 0
  k_spmv<<<bw, 256, 0, st>>>(ni, d->tt_ptr, d->tt_col, d->tt_val, f_full, d->r);
  if (dirichlet) k_axpby<<<bi, 256, 0, st>>>(ni, -1.0, d->g, 1.0, d->r);
  cudaMemsetAsync(d->x, 0, (size_t)ni * sizeof(double), st);
  if (!dots(d->r, d->r)) return PIC_ECUDA;
  const double bnorm = std::sqrt(h[1]);
  int it = 0;
  double res = bnorm > 0 ? 1.0 : 0.0;
  if (bnorm > 0) {
    if (int rc = precond(d->r, d->z)) return rc;
    cudaMemcpyAsync(d->p, d->z, (size_t)ni * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (!dots(d->r, d->z)) return PIC_ECUDA;
    double rz = h[0];
    for (it = 1; it <= maxit; ++it) {
      k_spmv<<<bw, 256, 0, st>>>(ni, d->a_ptr, d->a_col, d->a_val, d->p, d->q);
      if (!dots(d->q, d->p)) return PIC_ECUDA;
      const double alpha = rz / h[0];
      k_axpby<<<bi, 256, 0, st>>>(ni, alpha, d->p, 1.0, d->x);
      k_axpby<<<bi, 256, 0, st>>>(ni, -alpha, d->q, 1.0, d->r);
      if (!dots(d->r, d->r)) return PIC_ECUDA;
      res = std::sqrt(h[1]) / bnorm;
      if (res <= rtol) break;
      if (int rc = precond(d->r, d->z)) return rc;
      if (!dots(d->z, d->r)) return PIC_ECUDA;
      const double beta = h[0] / rz;
      rz = h[0];
      k_axpby<<<bi, 256, 0, st>>>(ni, 1.0, d->z, beta, d->p);
    }
    it = std::min(it, maxit);
  }
  // c = T x
  k_spmv<<<bwf, 256, 0, st>>>(nf, d->t_ptr, d->t_col, d->t_val, d->x, c_full);
  if (iters) *iters = it;
  if (relres) *relres = res;
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return PIC_ECUDA;
  return res <= rtol ? PIC_OK : PIC_ENOCONV;
}

int pic_web_set_stream(pic_web* w, void* cuda_stream) {
  if (!w || !w->dev) return PIC_EINVAL;
  w->dev->stream = (cudaStream_t)cuda_stream;
  return w->dev->pre ? pic_spline_set_stream(w->dev->pre, cuda_stream) : PIC_OK;
}

int pic_web_direct(pic_web* w) {
  using namespace pic::web;
  if (!w || !w->dev) return PIC_EINVAL;
  Dev* d = w->dev;
  if (d->inv) return PIC_OK;
  std::vector<double> inv;
  if (!dense_inverse(w, inv)) return PIC_ENOCONV;
  // on the device the system was built on, queued on its stream; the
  // inverse is published only once its copy has completed
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(d->device) != cudaSuccess)
    return PIC_ECUDA;
  const size_t bytes = inv.size() * sizeof(double);
  double* p = nullptr;
  int rc = PIC_OK;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
    rc = PIC_ENOMEM;
  } else if (cudaMemcpyAsync(p, inv.data(), bytes, cudaMemcpyHostToDevice, d->stream) !=
                 cudaSuccess ||
             cudaStreamSynchronize(d->stream) != cudaSuccess) {
    rc = PIC_ECUDA;
  }
  if (rc) {
    if (p) cudaFree(p);
    cudaGetLastError();
  } else {
    d->inv = p;
  }
  cudaSetDevice(prev);
  return rc;
}

int pic_web_solve_direct(pic_web* w, const double* f, double* c, int dirichlet) {
  using namespace pic::web;
  if (!w || !w->dev || !w->dev->inv || !f || !c) return PIC_EINVAL;
  Dev* d = w->dev;
  cudaStream_t st = d->stream;
  const int ni = (int)w->inner_full.size(), nf = w->mr * w->mz;
  const int bi = blocks_for(ni, 256);
  // b = T^T f - [dirichlet] g;  u = A^-1 b (one warp per row of the dense
  // inverse, kept in L2 across steps);  c = T u
  k_spmv<<<blocks_for((long long)ni * 32, 256), 256, 0, st>>>(ni, d->tt_ptr, d->tt_col, d->tt_val,
                                                              f, d->r);
  if (dirichlet) k_axpby<<<bi, 256, 0, st>>>(ni, -1.0, d->g, 1.0, d->r);
  k_gemv<<<blocks_for((long long)ni * 32, 256), 256, 0, st>>>(ni, d->inv, d->r, d->x);
  k_spmv<<<blocks_for((long long)nf * 32, 256), 256, 0, st>>>(nf, d->t_ptr, d->t_col, d->t_val,
                                                              d->x, c);
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

int pic_web_well_depth(pic_web* w, const double* c, const double* r_start, int lines, double z1,
                       int samples, int bfield_kind, double b0, double z_mid, double L,
                       double* depth, double* z_at) {
  using namespace pic::web;
  if (!w || !w->dev || !c || !r_start || lines < 1 || samples < 3 || !depth || !z_at ||
      !(b0 > 0) || (bfield_kind == 1 && !(L > 0)))
    return PIC_EINVAL;
  cudaStream_t st = w->dev->stream;
  const size_t cells = (size_t)lines * samples;
  double *dr = nullptr, *dU = nullptr, *dS = nullptr, *dd = nullptr, *dza = nullptr;
  int rc = PIC_OK;
  if (cudaMalloc(&dr, lines * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dU, cells * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dS, cells * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dd, lines * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dza, lines * sizeof(double)) != cudaSuccess)
    rc = PIC_ENOMEM;
  if (!rc && cudaMemcpyAsync(dr, r_start, lines * sizeof(double), cudaMemcpyHostToDevice, st) !=
                 cudaSuccess)
    rc = PIC_ECUDA;
  if (!rc) {
    const Grid D{w->n, w->nr, w->nz, w->mz, w->r_lo, w->G.z0, w->hr, w->hz};
    const BzModel B{bfield_kind, b0, z_mid, L};
    k_well_depth<<<(lines + 127) / 128, 128, 0, st>>>(w->G, D, B, c, dr, lines, z1, samples, dU,
                                                      dS, dd, dza);
    if (cudaMemcpyAsync(depth, dd, lines * sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(z_at, dza, lines * sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
      rc = PIC_ECUDA;
  }
  for (double* p : {dr, dU, dS, dd, dza})
    if (p) cudaFree(p);
  cudaGetLastError();
  return rc;
}

int pic_web_deposit(pic_web* w, const double* r, const double* z, int64_t n, double qw,
                    double* f_full) {
  using namespace pic::web;
  if (!w || !w->dev || n < 0 || (n > 0 && (!r || !z || !f_full))) return PIC_EINVAL;
  if (n == 0) return PIC_OK;
  const Grid D{w->n, w->nr, w->nz, w->mz, w->r_lo, w->G.z0, w->hr, w->hz};
  k_web_deposit<<<blocks_for(n, 256), 256, 0, w->dev->stream>>>(w->G, D, r, z, n, qw, f_full);
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

int pic_web_eval(pic_web* w, const double* c_full, const double* r, const double* z, int64_t n,
                 int dirichlet, double* phi, double* er, double* ez) {
  using namespace pic::web;
  if (!w || !w->dev || n < 0 || (n > 0 && (!c_full || !r || !z))) return PIC_EINVAL;
  if (n == 0) return PIC_OK;
  const Grid D{w->n, w->nr, w->nz, w->mz, w->r_lo, w->G.z0, w->hr, w->hz};
  k_web_eval<<<blocks_for(n, 256), 256, 0, w->dev->stream>>>(w->G, D, c_full, r, z, n,
                                                             dirichlet, phi, er, ez);
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

}  // extern "C"
