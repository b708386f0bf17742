// spline.cu -- the weighted B-spline field of degree n (arXiv 2206.14662,
// Sec. II.A: finite elements on weighted B-splines of arbitrary degree, which put
// the Dirichlet electrodes on a rectangular grid) with particle shapes from
// the same basis.
//
// Basis: uniform B-splines b_i of degree n on knots extending n cells past
// each end (nr + n functions in r, nz + n in z), the coaxial walls carried
// by the weight w(r) = (r - a)(b - r) / (b - a) and the linear lift
// phi_D(r) = V_in + (V_out - V_in)(r - a)/(b - a):
//   phi = phi_D(r) + sum_ij c_ij w(r) b_i(r) b_j(z).
// Galerkin system (volume element 2 pi r dr dz):
//   (K_r (x) M_z + M_r (x) K_z) c = f / (2 pi eps0) - g_r (x) m_z,
// K_r = int (w b_i)'(w b_k)' r dr, M_r = int w^2 b_i b_k r dr,
// g_r = int phi_D' (w b_i)' r dr, K_z, M_z the z stiffness and mass, m_z =
// int b_j dz (Gauss-Legendre quadrature per cell, exact here).
//
// Solver: fast diagonalisation along r, the shorter direction.  With the
// generalised eigenpairs K_r V = M_r V diag(lambda), V^T M_r V = I (host,
// at creation: Cholesky of M_r, cyclic Jacobi on L^-1 K_r L^-T), the system
// splits into one banded SPD system (lambda_k M_z + K_z) d_k = (V^T f')_k
// per r-mode k, solved with band Cholesky factors made at creation; then
// c = V d.  A direct FP64 solve: no iteration, no residual contract.
//
// Particles deposit f_ij += q w w(r_p) b_i(r_p) b_j(z_p) and are evaluated
// with the exact gradient E = -grad phi at their position.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pic.h"
#include "pic_internal.cuh"
#include "dfloat.cuh"

namespace pic {
namespace spl {

constexpr int kMaxDeg = PIC_SPLINE_MAX_DEGREE;
constexpr int kMaxModes = 1024;   // r functions: the Jacobi eigen solver grows as m^3 (~1 min at 1024)

// Gauss-Legendre rule of q points on [-1, 1]: the roots of P_q by Newton's
// method from cos(pi (i + 3/4) / (q + 1/2)), weights 2 / ((1 - x^2) P_q'(x)^2)
void gauss_legendre(int q, double* x, double* w) {
  for (int i = 0; i < q; ++i) {
    double t = std::cos(kPi * (i + 0.75) / (q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;   // P_0, P_1; recurrence up to P_q
      for (int k = 2; k <= q; ++k) {
        const double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double pq = q == 0 ? 1.0 : p1, pqm1 = q == 1 ? 1.0 : p0;
      dp = q * (t * pq - pqm1) / (t * t - 1.0);
      const double dt = pq / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

// The p + 1 B-splines of degree p that are non-zero on a knot span of
// uniform knots, at local coordinate u in [0, 1) (the triangular
// Cox-de Boor scheme with left/right knot distances u + j - 1 and j - u in
// units of the spacing, denominators j): N[r] belongs to the r-th function
// of the span.
template <typename T>
__host__ __device__ __forceinline__ void span_basis(int p, T u, T* N) {
  N[0] = T(1);
  for (int j = 1; j <= p; ++j) {
    T saved = T(0);
    for (int r = 0; r < j; ++r) {
      const T right = T(r + 1) - u, left = u + T(j - r - 1);
      const T tmp = N[r] / T(j);
      N[r] = saved + right * tmp;
      saved = left * tmp;
    }
    N[j] = saved;
  }
}

// values and derivatives (spacing h) of the span's degree-p functions:
// N'_{i,p} = (N_{i,p-1} - N_{i+1,p-1}) / h
template <typename T>
__host__ __device__ __forceinline__ void span_basis_d(int p, T u, T h, T* N, T* dN) {
  T M[kMaxDeg + 1];
  span_basis<T>(p, u, N);
  if (p == 0) {
    dN[0] = T(0);
    return;
  }
  span_basis<T>(p - 1, u, M);
  for (int r = 0; r <= p; ++r) {
    const T lo = r >= 1 ? M[r - 1] : T(0), hi = r <= p - 1 ? M[r] : T(0);
    dN[r] = (lo - hi) / h;
  }
}

struct Tables {
  int n, nr, nz, mr, mz;
  double a, b, z0, hr, hz, v_in, v_out, dphiD;
  std::vector<double> K_r, M_r, g_r, K_z, M_z, m_z;   // dense, row-major
  std::vector<double> V, lam;                          // mr x mr, mr
  std::vector<double> band;                            // the sweeps' scaled tables
  std::vector<double> gt;                              // segment responses (band_factors)
};

// The z sweeps run in kSpikeSeg segments of rows per mode (k_band_spike),
// kSpikeModes modes a block.
constexpr int kSpikeSeg = 32;
constexpr int kSpikeModes = 4;

int check(const pic_config* c, int n) {
  if (!c || n < 1 || n > kMaxDeg) return PIC_EINVAL;
  if (!(c->r_in > 0 && c->r_out > c->r_in && c->z_max > c->z_min)) return PIC_EINVAL;
  if (c->nr < 2 || c->nz < 2 || c->nr + n > kMaxModes || c->nz > 65535) return PIC_EINVAL;
  return PIC_OK;
}

void matrices(const pic_config* c, int n, Tables& T) {
  T.n = n;
  T.nr = c->nr;
  T.nz = c->nz;
  T.mr = c->nr + n;
  T.mz = c->nz + n;
  T.a = c->r_in;
  T.b = c->r_out;
  T.z0 = c->z_min;
  T.hr = (c->r_out - c->r_in) / c->nr;
  T.hz = (c->z_max - c->z_min) / c->nz;
  T.v_in = c->v_inner;
  T.v_out = c->v_outer;
  T.dphiD = (c->v_outer - c->v_inner) / (c->r_out - c->r_in);
  const int mr = T.mr, mz = T.mz;
  T.K_r.assign((size_t)mr * mr, 0.0);
  T.M_r.assign((size_t)mr * mr, 0.0);
  T.g_r.assign(mr, 0.0);
  T.K_z.assign((size_t)mz * mz, 0.0);
  T.M_z.assign((size_t)mz * mz, 0.0);
  T.m_z.assign(mz, 0.0);
  double xg[kMaxDeg + 4], wg[kMaxDeg + 4];
  double N[kMaxDeg + 1], dN[kMaxDeg + 1];
  // r: integrands of degree <= 2n + 3
  const int qr = n + 3;
  gauss_legendre(qr, xg, wg);
  const double ab = T.b - T.a;
  for (int cell = 0; cell < T.nr; ++cell) {
    for (int q = 0; q < qr; ++q) {
      const double u = 0.5 * (xg[q] + 1.0);
      const double r = T.a + (cell + u) * T.hr;
      const double wq = 0.5 * T.hr * wg[q] * r;
      span_basis_d<double>(n, u, T.hr, N, dN);
      const double w = (r - T.a) * (T.b - r) / ab, dw = (T.a + T.b - 2.0 * r) / ab;
      double F[kMaxDeg + 1], dF[kMaxDeg + 1];
      for (int k = 0; k <= n; ++k) {
        F[k] = w * N[k];
        dF[k] = dw * N[k] + w * dN[k];
      }
      for (int k = 0; k <= n; ++k) {
        T.g_r[cell + k] += wq * T.dphiD * dF[k];
        for (int l = 0; l <= n; ++l) {
          T.K_r[(size_t)(cell + k) * mr + cell + l] += wq * dF[k] * dF[l];
          T.M_r[(size_t)(cell + k) * mr + cell + l] += wq * F[k] * F[l];
        }
      }
    }
  }
  // z: integrands of degree <= 2n
  const int qz = n + 2;
  gauss_legendre(qz, xg, wg);
  for (int cell = 0; cell < T.nz; ++cell) {
    for (int q = 0; q < qz; ++q) {
      const double u = 0.5 * (xg[q] + 1.0);
      const double wq = 0.5 * T.hz * wg[q];
      span_basis_d<double>(n, u, T.hz, N, dN);
      for (int k = 0; k <= n; ++k) {
        T.m_z[cell + k] += wq * N[k];
        for (int l = 0; l <= n; ++l) {
          T.K_z[(size_t)(cell + k) * mz + cell + l] += wq * dN[k] * dN[l];
          T.M_z[(size_t)(cell + k) * mz + cell + l] += wq * N[k] * N[l];
        }
      }
    }
  }
}

// symmetric eigen-decomposition A = Q diag(e) Q^T by cyclic Jacobi rotations
// (A is overwritten); returns false if it did not converge
bool jacobi_eigen(std::vector<double>& A, int m, std::vector<double>& Q, std::vector<double>& e) {
  Q.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
  auto at = [&](int i, int j) -> double& { return A[(size_t)i * m + j]; };
  double diag = 0.0;
  for (int i = 0; i < m; ++i) diag += at(i, i) * at(i, i);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = i + 1; j < m; ++j) off += at(i, j) * at(i, j);
    if (off <= 1e-30 * diag) {
      e.resize(m);
      for (int i = 0; i < m; ++i) e[i] = at(i, i);
      return true;
    }
    for (int p = 0; p < m; ++p) {
      for (int q = p + 1; q < m; ++q) {
        const double apq = at(p, q);
        if (apq == 0.0) continue;
        // rotation that zeroes A[p][q]: tan(theta) = t with
        // t^2 + 2 t cot(2 theta) - 1 = 0, the smaller root
        const double theta = (at(q, q) - at(p, p)) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < m; ++k) {   // columns p, q
          const double akp = at(k, p), akq = at(k, q);
          at(k, p) = cs * akp - sn * akq;
          at(k, q) = sn * akp + cs * akq;
        }
        for (int k = 0; k < m; ++k) {   // rows p, q
          const double apk = at(p, k), aqk = at(q, k);
          at(p, k) = cs * apk - sn * aqk;
          at(q, k) = sn * apk + cs * aqk;
        }
        for (int k = 0; k < m; ++k) {
          const double qkp = Q[(size_t)k * m + p], qkq = Q[(size_t)k * m + q];
          Q[(size_t)k * m + p] = cs * qkp - sn * qkq;
          Q[(size_t)k * m + q] = sn * qkp + cs * qkq;
        }
      }
    }
  }
  return false;
}

// generalised eigenpairs of (K_r, M_r): V^T M_r V = I, V^T K_r V = diag(lam),
// ascending
bool eigen(Tables& T) {
  const int m = T.mr;
  // Cholesky M_r = L L^T (lower, dense)
  std::vector<double> L((size_t)m * m, 0.0);
  for (int j = 0; j < m; ++j) {
    for (int i = j; i < m; ++i) {
      double s = T.M_r[(size_t)i * m + j];
      for (int k = 0; k < j; ++k) s -= L[(size_t)i * m + k] * L[(size_t)j * m + k];
      if (i == j) {
        if (!(s > 0)) return false;
        L[(size_t)j * m + j] = std::sqrt(s);
      } else {
        L[(size_t)i * m + j] = s / L[(size_t)j * m + j];
      }
    }
  }
  // C = L^-1 K_r L^-T: X = L^-1 K_r (forward substitution per column), then
  // C = L^-1 X^T (X^T = K_r L^-T since K_r is symmetric)
  auto lsolve = [&](std::vector<double>& B) {   // B := L^-1 B, column by column
    for (int col = 0; col < m; ++col)
      for (int i = 0; i < m; ++i) {
        double s = B[(size_t)i * m + col];
        for (int k = 0; k < i; ++k) s -= L[(size_t)i * m + k] * B[(size_t)k * m + col];
        B[(size_t)i * m + col] = s / L[(size_t)i * m + i];
      }
  };
  std::vector<double> X = T.K_r;
  lsolve(X);
  std::vector<double> C((size_t)m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) C[(size_t)i * m + j] = X[(size_t)j * m + i];
  lsolve(C);
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) {
      const double s = 0.5 * (C[(size_t)i * m + j] + C[(size_t)j * m + i]);
      C[(size_t)i * m + j] = C[(size_t)j * m + i] = s;
    }
  std::vector<double> Q, e;
  if (!jacobi_eigen(C, m, Q, e)) return false;
  // V = L^-T Q (back substitution per column), eigenpairs sorted ascending
  std::vector<int> order(m);
  for (int i = 0; i < m; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return e[x] < e[y]; });
  T.V.assign((size_t)m * m, 0.0);
  T.lam.resize(m);
  for (int kk = 0; kk < m; ++kk) {
    const int col = order[kk];
    T.lam[kk] = e[col];
    for (int i = m - 1; i >= 0; --i) {
      double s = Q[(size_t)i * m + col];
      for (int k = i + 1; k < m; ++k) s -= L[(size_t)k * m + i] * T.V[(size_t)k * m + kk];
      T.V[(size_t)i * m + kk] = s / L[(size_t)i * m + i];
    }
  }
  return true;
}

// band Cholesky factors L_k of lam_k M_z + K_z (bandwidth n), as the two
// tables of the device sweeps, each laid out [j][d][k] at (j (n + 1) + d)
// mr + k: d = 0 holds 1 / L_k[j][j]; d >= 1 holds, in the forward table,
// L_k[j][j - d] / L_k[j][j] and, in the backward table (after the forward
// one), L_k[j + d][j] / L_k[j][j] (0 beyond the ends)
bool band_factors(Tables& T) {
  const int n = T.n, mz = T.mz, mr = T.mr;
  const size_t half = (size_t)mz * (n + 1) * mr;
  T.band.assign(2 * half, 0.0);
  std::vector<double> L((size_t)mz * (n + 1));
  for (int k = 0; k < mr; ++k) {
    const double lam = T.lam[k];
    for (int j = 0; j < mz; ++j) {
      for (int i = std::max(0, j - n); i <= j; ++i) {
        double s = lam * T.M_z[(size_t)j * mz + i] + T.K_z[(size_t)j * mz + i];
        for (int q = std::max(0, j - n); q < i; ++q)
          s -= L[(size_t)j * (n + 1) + (j - q)] * L[(size_t)i * (n + 1) + (i - q)];
        if (i == j) {
          if (!(s > 0)) return false;
          L[(size_t)j * (n + 1)] = std::sqrt(s);
        } else {
          L[(size_t)j * (n + 1) + (j - i)] = s / L[(size_t)i * (n + 1)];
        }
      }
    }
    for (int j = 0; j < mz; ++j) {
      const double inv = 1.0 / L[(size_t)j * (n + 1)];
      for (int d = 0; d <= n; ++d) {
        const size_t at = ((size_t)j * (n + 1) + d) * mr + k;
        T.band[at] = d == 0 ? inv : (d <= j ? L[(size_t)j * (n + 1) + d] * inv : 0.0);
        T.band[half + at] =
            d == 0 ? inv : (j + d < mz ? L[(size_t)(j + d) * (n + 1) + d] * inv : 0.0);
      }
    }
  }
  // per sweep, mode and segment: the segment's exit window (its last n
  // values in the sweep's order) for each unit entry window, the same
  // recurrence as the device's without the right-hand side
  const int S = (mz + kSpikeSeg - 1) / kSpikeSeg;
  T.gt.assign((size_t)2 * mr * kSpikeSeg * n * n, 0.0);
  std::vector<double> gw((size_t)n * n);
  for (int sw = 0; sw < 2; ++sw) {
    const double* tab = T.band.data() + sw * half;
    for (int k = 0; k < mr; ++k)
      for (int p = 0; p < kSpikeSeg; ++p) {
        const int lo = std::min(p * S, mz), hi = std::min(lo + S, mz);
        for (int m = 0; m < n; ++m)
          for (int i = 0; i < n; ++i) gw[(size_t)m * n + i] = i == m ? 1.0 : 0.0;
        for (int q = 0; q < hi - lo; ++q) {
          const int j = sw == 0 ? lo + q : hi - 1 - q;
          for (int m = 0; m < n; ++m) {
            double* w = gw.data() + (size_t)m * n;
            double v = 0.0;
            for (int d = n; d >= 1; --d) v = std::fma(-tab[((size_t)j * (n + 1) + d) * mr + k], w[d - 1], v);
            for (int d = n - 1; d >= 1; --d) w[d] = w[d - 1];
            w[0] = v;
          }
        }
        double* out = T.gt.data() + (((size_t)sw * mr + k) * kSpikeSeg + p) * n * n;
        for (int i = 0; i < n; ++i)
          for (int m = 0; m < n; ++m) out[(size_t)i * n + m] = gw[(size_t)m * n + i];
      }
  }
  return true;
}

// ---------------------------------------------------------------- device

struct Geo {
  int n, nr, nz, mr, mz;
  double a, b, z0, hr, hz, v_in, dphiD;
};

// the span of x (cells along one axis), clamped to the grid, and the local
// coordinate in it
__device__ __forceinline__ int span_of(double x, double lo, double h, int cells, double& u) {
  const double s = (x - lo) / h;
  int c = (int)floor(s);
  c = min(max(c, 0), cells - 1);
  u = s - c;
  return c;
}

// F' = f / (2 pi eps0) - [dirichlet] g_r (x) m_z
__global__ void k_lift(const double* __restrict__ f, const double* __restrict__ g_r,
                       const double* __restrict__ m_z, double scale, int dirichlet, int mr, int mz,
                       double* __restrict__ out) {
  const long long total = (long long)mr * mz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / mz), j = (int)(t % mz);
    out[t] = f[t] * scale - (dirichlet ? g_r[i] * m_z[j] : 0.0);
  }
}

constexpr int kTile = 16;   // the transforms' square tiles

// The transforms in double-float (FP32 pairs, ~2^-48 relative): C(m, n) =
// sum_k A(m, k) B(k, n), FP64 in and out, with the constant operand (the
// eigenvector matrix, V_IS_A: A, else B) stored as float2 (hi, lo) and the
// other converted once per tile load (sdf_split, sdf_fma).  On this part
// FP64 instructions take ~16 SM cycles a warp, so the FP64 tile GEMM was
// bound by the FP64 pipe (23 us a transform at 128 x 512); the
// double-float form runs on the FP32 pipes.
template <bool V_IS_A>
__global__ void k_gemm_df(int M, int N, int K, const void* __restrict__ A, long long sam,
                          long long sak, const void* __restrict__ B, long long sbk, long long sbn,
                          double* __restrict__ C, long long scm, long long scn) {
  __shared__ float2 As[kTile][kTile + 1], Bs[kTile][kTile + 1];
  const int tm = threadIdx.y, tn = threadIdx.x;
  const int m = blockIdx.y * kTile + tm, n = blockIdx.x * kTile + tn;
  float2 acc = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < K; k0 += kTile) {
    const int ka = k0 + tn, kb = k0 + tm;
    const bool oka = m < M && ka < K, okb = kb < K && n < N;
    if (V_IS_A) {
      As[tm][tn] = oka ? ((const float2*)A)[m * sam + ka * sak] : make_float2(0.f, 0.f);
      Bs[tm][tn] = okb ? sdf_split(((const double*)B)[kb * sbk + n * sbn]) : make_float2(0.f, 0.f);
    } else {
      As[tm][tn] = oka ? sdf_split(((const double*)A)[m * sam + ka * sak]) : make_float2(0.f, 0.f);
      Bs[tm][tn] = okb ? ((const float2*)B)[kb * sbk + n * sbn] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kTile; ++k) acc = sdf_fma(acc, As[tm][k], Bs[k][tn]);
    __syncthreads();
  }
  if (m < M && n < N) C[m * scm + n * scn] = (double)acc.x + (double)acc.y;
}

// Per r-mode k, forward and back substitution with the band factor's two
// scaled tables (band_factors): y_j = x_j / L[j][j] - sum_d (L[j][j - d] /
// L[j][j]) y_{j - d}, then c_j = y_j / L[j][j] - sum_d (L[j + d][j] /
// L[j][j]) c_{j + d}; the forward sweep reads x (the modes) and writes y to
// `tmp`, the backward sweep reads y and writes the solution back to x.
// Each sweep is split into P segments of rows per mode (the "SPIKE"
// partition of a banded triangular solve); a block holds MG modes x P
// segments, thread t mode t % MG and segment t / MG.  Phase 1: each
// (segment, mode) runs its rows from a zero entry window, keeping its last
// N values.  Phase 2: one thread per mode chains the segments in the
// sweep's order: the entry window of the next segment is that exit window
// plus the segment's responses to unit entry windows (gt, precomputed on
// the host from the same tables) applied to its own entry window.  Phase
// 3: each segment reruns its rows from its true entry window and stores
// them.  The dependency chain is 2 S + P steps instead of mz (S = mz / P
// rows a segment), and the work spreads over mr / MG blocks: on this part
// FP64 instructions take ~16 SM cycles a warp, so the number of SMs doing
// FP64, not latency alone, sets the time.  Segments hold the same rows in
// both sweeps, so the backward sweep reads the rows its own thread stored.
template <int N, int B, class F>
__device__ __forceinline__ void band_rows(const double* __restrict__ src,
                                          const double* __restrict__ tab, bool nc, int j0,
                                          int count, int step, int k, int mr, bool valid, F&& f) {
  constexpr int w = N + 1;
  double xc[B], bc[B][w], xn[B], bn[B][w];
  auto load = [&](int i0, double* xs, double (*bs)[w]) {
#pragma unroll
    for (int t = 0; t < B; ++t) {
      const int i = i0 + t;
      const bool ok = valid && i < count;
      const int j = j0 + i * step;
      xs[t] = ok ? (nc ? __ldg(src + (size_t)j * mr + k) : src[(size_t)j * mr + k]) : 0.0;
#pragma unroll
      for (int d = 0; d <= N; ++d) bs[t][d] = ok ? __ldg(tab + ((size_t)j * w + d) * mr + k) : 0.0;
    }
  };
  load(0, xc, bc);
  for (int i0 = 0; i0 < count; i0 += B) {
    load(i0 + B, xn, bn);
#pragma unroll
    for (int t = 0; t < B; ++t)
      if (i0 + t < count) f(j0 + (i0 + t) * step, xc[t], bc[t]);
#pragma unroll
    for (int t = 0; t < B; ++t) {
      xc[t] = xn[t];
#pragma unroll
      for (int d = 0; d <= N; ++d) bc[t][d] = bn[t][d];
    }
  }
}

// one row of a sweep on window win (win[d - 1] the value d rows back in
// the sweep's order): x / L[j][j] - sum_d t_d win[d - 1], oldest term first
template <int N>
__device__ __forceinline__ double band_step(double xs, const double* t, double* win) {
  double v = xs * t[0];
#pragma unroll
  for (int d = N; d >= 1; --d) v = fma(-t[d], win[d - 1], v);
#pragma unroll
  for (int d = N - 1; d >= 1; --d) win[d] = win[d - 1];
  win[0] = v;
  return v;
}

template <int N, int MG, int P, int B>
__global__ void __launch_bounds__(MG * P) k_band_spike(const double* __restrict__ band,
                                                      const double* __restrict__ gt, int mz,
                                                      int mr, double* __restrict__ x,
                                                      double* __restrict__ tmp) {
  __shared__ double ztail[P][MG][N], tin[P][MG][N];
  const int mi = threadIdx.x % MG, p = threadIdx.x / MG;
  const int k = blockIdx.x * MG + mi;
  const bool valid = k < mr;
  const int S = (mz + P - 1) / P;
  const int lo = min(p * S, mz), hi = min(lo + S, mz), count = hi - lo;
#pragma unroll 1
  for (int sw = 0; sw < 2; ++sw) {
    const bool fwd = sw == 0;
    const double* src = fwd ? x : tmp;
    const double* tab = band + (size_t)sw * mz * (N + 1) * mr;
    double* dst = fwd ? tmp : x;
    const int j0 = fwd ? lo : hi - 1, step = fwd ? 1 : -1;
    // phase 1
    double zw[N];
#pragma unroll
    for (int i = 0; i < N; ++i) zw[i] = 0.0;
    band_rows<N, B>(src, tab, fwd, j0, count, step, k, mr, valid,
                    [&](int, double xs, const double* t) { band_step<N>(xs, t, zw); });
#pragma unroll
    for (int i = 0; i < N; ++i) ztail[p][mi][i] = zw[i];
    __syncthreads();
    // phase 2
    if (p == 0 && valid) {
      double T[N];
#pragma unroll
      for (int i = 0; i < N; ++i) T[i] = 0.0;
      const double* g = gt + ((size_t)sw * mr + k) * P * N * N;
      for (int q = 0; q < P; ++q) {
        const int seg = fwd ? q : P - 1 - q;
        const double* gs = g + (size_t)seg * N * N;
        double Tn[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
          tin[seg][mi][i] = T[i];
          double v = ztail[seg][mi][i];
#pragma unroll
          for (int m = 0; m < N; ++m) v = fma(__ldg(gs + i * N + m), T[m], v);
          Tn[i] = v;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) T[i] = Tn[i];
      }
    }
    __syncthreads();
    // phase 3
    double win[N];
#pragma unroll
    for (int i = 0; i < N; ++i) win[i] = tin[p][mi][i];
    band_rows<N, B>(src, tab, fwd, j0, count, step, k, mr, valid,
                    [&](int j, double xs, const double* t) {
                      const double v = band_step<N>(xs, t, win);
                      if (valid) dst[(size_t)j * mr + k] = v;
                    });
    __syncthreads();   // the shared windows are rewritten by the next sweep
  }
}

__global__ void k_deposit(Geo G, const double* __restrict__ r, const double* __restrict__ z,
                          long long np, double qw, double* __restrict__ f) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    double ur, uz, Nr[kMaxDeg + 1], Nz[kMaxDeg + 1];
    const int cr = span_of(r[p], G.a, G.hr, G.nr, ur);
    const int cz = span_of(z[p], G.z0, G.hz, G.nz, uz);
    span_basis<double>(G.n, ur, Nr);
    span_basis<double>(G.n, uz, Nz);
    const double rp = r[p];
    const double w = (rp - G.a) * (G.b - rp) / (G.b - G.a);
    for (int k = 0; k <= G.n; ++k) {
      const double fk = qw * w * Nr[k];
      for (int l = 0; l <= G.n; ++l) atomicAdd(f + (size_t)(cr + k) * G.mz + cz + l, fk * Nz[l]);
    }
  }
}

__global__ void k_eval(Geo G, const double* __restrict__ c, const double* __restrict__ r,
                       const double* __restrict__ z, long long np, int dirichlet,
                       double* __restrict__ phi, double* __restrict__ er, double* __restrict__ ez) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    double ur, uz, Nr[kMaxDeg + 1], dNr[kMaxDeg + 1], Nz[kMaxDeg + 1], dNz[kMaxDeg + 1];
    const int cr = span_of(r[p], G.a, G.hr, G.nr, ur);
    const int cz = span_of(z[p], G.z0, G.hz, G.nz, uz);
    span_basis_d<double>(G.n, ur, G.hr, Nr, dNr);
    span_basis_d<double>(G.n, uz, G.hz, Nz, dNz);
    const double rp = r[p];
    const double w = (rp - G.a) * (G.b - rp) / (G.b - G.a);
    const double dw = (G.a + G.b - 2.0 * rp) / (G.b - G.a);
    double v = 0.0, gr = 0.0, gz = 0.0;
    for (int k = 0; k <= G.n; ++k) {
      const double* row = c + (size_t)(cr + k) * G.mz + cz;
      double s = 0.0, sd = 0.0;
      for (int l = 0; l <= G.n; ++l) {
        s = fma(row[l], Nz[l], s);
        sd = fma(row[l], dNz[l], sd);
      }
      v = fma(w * Nr[k], s, v);
      gr = fma(dw * Nr[k] + w * dNr[k], s, gr);
      gz = fma(w * Nr[k], sd, gz);
    }
    if (dirichlet) {
      v += G.v_in + G.dphiD * (rp - G.a);
      gr += G.dphiD;
    }
    if (phi) phi[p] = v;
    if (er) er[p] = -gr;
    if (ez) ez[p] = -gz;
  }
}

}  // namespace spl
}  // namespace pic

using namespace pic;

// the band solve of the modes x (mr x mz, row j at j mr) in place, tmp
// its intermediate
static int band_solve(int n, const double* band, const double* gt, int mz, int mr, double* x,
                      double* tmp, cudaStream_t st) {
  using namespace pic::spl;
  const int blocks = (mr + kSpikeModes - 1) / kSpikeModes, threads = kSpikeModes * kSpikeSeg;
  switch (n) {
    case 1: k_band_spike<1, kSpikeModes, kSpikeSeg, 4><<<blocks, threads, 0, st>>>(band, gt, mz, mr, x, tmp); break;
    case 2: k_band_spike<2, kSpikeModes, kSpikeSeg, 4><<<blocks, threads, 0, st>>>(band, gt, mz, mr, x, tmp); break;
    case 3: k_band_spike<3, kSpikeModes, kSpikeSeg, 4><<<blocks, threads, 0, st>>>(band, gt, mz, mr, x, tmp); break;
    case 4: k_band_spike<4, kSpikeModes, kSpikeSeg, 4><<<blocks, threads, 0, st>>>(band, gt, mz, mr, x, tmp); break;
    default: k_band_spike<kMaxDeg, kSpikeModes, kSpikeSeg, 4><<<blocks, threads, 0, st>>>(band, gt, mz, mr, x, tmp); break;
  }
  return PIC_OK;
}

struct pic_spline {
  spl::Geo G;
  cudaStream_t stream;
  double *g_r, *m_z, *band, *gt, *work, *modes;
  float2* Vdf;   // the eigenvector matrix as double-float (hi, lo)
};

extern "C" {

int pic_spline_matrices(const pic_config* cfg, int degree, double* K_r, double* M_r, double* g_r,
                        double* K_z, double* M_z, double* m_z) {
  if (int rc = spl::check(cfg, degree)) return rc;
  spl::Tables T;
  spl::matrices(cfg, degree, T);
  auto put = [](double* dst, const std::vector<double>& v) {
    if (dst) std::memcpy(dst, v.data(), v.size() * sizeof(double));
  };
  put(K_r, T.K_r);
  put(M_r, T.M_r);
  put(g_r, T.g_r);
  put(K_z, T.K_z);
  put(M_z, T.M_z);
  put(m_z, T.m_z);
  return PIC_OK;
}

int pic_spline_eigen(const pic_config* cfg, int degree, double* V, double* lambda) {
  if (int rc = spl::check(cfg, degree)) return rc;
  spl::Tables T;
  spl::matrices(cfg, degree, T);
  if (!spl::eigen(T)) return PIC_ENOCONV;
  if (V) std::memcpy(V, T.V.data(), T.V.size() * sizeof(double));
  if (lambda) std::memcpy(lambda, T.lam.data(), T.lam.size() * sizeof(double));
  return PIC_OK;
}

void pic_spline_free(pic_spline* s) {
  if (!s) return;
  if (s->Vdf) cudaFree(s->Vdf);
  for (double* p : {s->g_r, s->m_z, s->band, s->gt, s->work, s->modes})
    if (p) cudaFree(p);
  delete s;
}

int pic_spline_create(const pic_config* cfg, int degree, void* cuda_stream, pic_spline** out) {
  if (!out) return PIC_EINVAL;
  *out = nullptr;
  if (int rc = spl::check(cfg, degree)) return rc;
  spl::Tables T;
  spl::matrices(cfg, degree, T);
  if (!spl::eigen(T) || !spl::band_factors(T)) return PIC_ENOCONV;
  pic_spline* s = new pic_spline();
  s->G = spl::Geo{T.n, T.nr, T.nz, T.mr, T.mz, T.a, T.b, T.z0, T.hr, T.hz, T.v_in, T.dphiD};
  s->stream = (cudaStream_t)cuda_stream;
  const size_t cells = (size_t)T.mr * T.mz;
  // V as double-float: hi = V rounded to FP32, lo = the remainder rounded
  std::vector<float2> vdf(T.V.size());
  for (size_t i = 0; i < T.V.size(); ++i) {
    const float hi = (float)T.V[i];
    vdf[i] = make_float2(hi, (float)(T.V[i] - (double)hi));
  }
  bool ok = cudaMalloc(&s->Vdf, T.V.size() * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&s->g_r, T.g_r.size() * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&s->m_z, T.m_z.size() * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&s->band, T.band.size() * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&s->gt, T.gt.size() * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&s->work, cells * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&s->modes, cells * sizeof(double)) == cudaSuccess;
  ok = ok &&
       cudaMemcpy(s->Vdf, vdf.data(), vdf.size() * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(s->g_r, T.g_r.data(), T.g_r.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(s->m_z, T.m_z.data(), T.m_z.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(s->band, T.band.data(), T.band.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(s->gt, T.gt.data(), T.gt.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    pic_spline_free(s);
    cudaGetLastError();
    return PIC_ENOMEM;
  }
  *out = s;
  return PIC_OK;
}

int pic_spline_solve(pic_spline* s, const double* f, double* c, int dirichlet) {
  if (!s || !f || !c || (const double*)c == f) return PIC_EINVAL;
  const spl::Geo& G = s->G;
  const int mr = G.mr, mz = G.mz;
  const long long cells = (long long)mr * mz;
  const int blocks = (int)std::min<long long>((cells + 255) / 256, 152 * 8);
  spl::k_lift<<<blocks, 256, 0, s->stream>>>(f, s->g_r, s->m_z, 1.0 / (2.0 * kPi * kEps0),
                                            dirichlet, mr, mz, s->work);
  const dim3 tb(spl::kTile, spl::kTile);
  // modes[j][k] = sum_i F'[i][j] V[i][k]   (M = mz rows j, N = mr columns k)
  spl::k_gemm_df<false><<<dim3((mr + spl::kTile - 1) / spl::kTile, (mz + spl::kTile - 1) / spl::kTile),
                          tb, 0, s->stream>>>(mz, mr, mr, s->work, 1, mz, s->Vdf, mr, 1, s->modes,
                                              mr, 1);
  // the band sweeps use the lifted right-hand side's buffer (consumed by
  // the transform above) for their intermediate
  if (int rc = band_solve(G.n, s->band, s->gt, mz, mr, s->modes, s->work, s->stream)) return rc;
  // c[i][j] = sum_k V[i][k] modes[j][k]   (M = mr rows i, N = mz columns j)
  spl::k_gemm_df<true><<<dim3((mz + spl::kTile - 1) / spl::kTile, (mr + spl::kTile - 1) / spl::kTile),
                         tb, 0, s->stream>>>(mr, mz, mr, s->Vdf, mr, 1, s->modes, 1, mr, c, mz,
                                             1);
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

int pic_spline_deposit(pic_spline* s, const double* r, const double* z, int64_t n, double qw,
                       double* f) {
  if (!s || n < 0 || (n > 0 && (!r || !z || !f))) return PIC_EINVAL;
  if (n == 0) return PIC_OK;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 8);
  spl::k_deposit<<<blocks, 256, 0, s->stream>>>(s->G, r, z, n, qw, f);
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

int pic_spline_eval(pic_spline* s, const double* c, const double* r, const double* z, int64_t n,
                    int dirichlet, double* phi, double* er, double* ez) {
  if (!s || n < 0 || (n > 0 && (!c || !r || !z))) return PIC_EINVAL;
  if (n == 0) return PIC_OK;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 8);
  spl::k_eval<<<blocks, 256, 0, s->stream>>>(s->G, c, r, z, n, dirichlet, phi, er, ez);
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

int pic_spline_set_stream(pic_spline* s, void* cuda_stream) {
  if (!s) return PIC_EINVAL;
  s->stream = (cudaStream_t)cuda_stream;
  return PIC_OK;
}

int pic_spline_sizes(const pic_spline* s, int* mr, int* mz) {
  if (!s) return PIC_EINVAL;
  if (mr) *mr = s->G.mr;
  if (mz) *mz = s->G.mz;
  return PIC_OK;
}

}  // extern "C"
