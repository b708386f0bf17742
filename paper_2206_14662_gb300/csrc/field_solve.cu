// field_solve.cu -- field solve of the PIC step (arXiv 2206.14662, Sec.
// II.A: finite elements, Dirichlet on the metal walls, Neumann on the open
// z ends).
//
// The finite-element matrix on bilinear elements of the (r,z) grid is
//   A = 2 pi eps0 (K_r (x) M_z + M_r (x) K_z)
// with r-weighted 1D matrices K_r, M_r (tridiagonal) and plain 1D matrices
// K_z, M_z of the uniform z grid with natural (Neumann) end rows.  The
// solver works on A' = A / (2 pi eps0) and b' = b / (2 pi eps0).
//
// Split.  phi = phi_vac + phi_rho: phi_vac carries the wall potentials and
// solves the charge-free problem exactly (it is z-independent: one radial
// tridiagonal solve in FP64 on the host, once); phi_rho solves
// A'_II phi_rho = b'_I with zero wall values.  phi_rho is orders of
// magnitude smaller than phi_vac, so its residual has no cancellation
// against the vacuum field.
//
// Separable preconditioner S (FP32).  With W = diag(1/2, 1, ..., 1, 1/2)
// and the mirrored neighbour-sum operator Y,
//   K_z = W (2 I - Y) / h_z,   M_z = W h_z (4 I + Y) / 6,
// and the cosines cos(pi k j / M), k = 0..M, diagonalise Y.  A DCT-I along
// z therefore splits the interior problem into M + 1 SPD tridiagonal
// systems along r, (g_k K_r + f_k M_r) phihat_k = bhat_k, solved by
// pre-factored Thomas sweeps, and the inverse DCT-I returns the potential.
// The DCT-I of length M + 1 is the DFT of the even extension of length 2M;
// two r-lines share one complex FFT (radix 2, shared memory) as real and
// imaginary parts.  M not a power of two uses a direct O(M^2) transform.
//
// Refinement.  phi_rho <- phi_rho + S(r), r = b' - A' phi_rho, with phi_rho,
// b' and the residual held in double-float (hi + lo, about 48 bits): on
// this part the FP64 pipe runs at a small fraction of the FP32 rate, so the
// FP64-accurate residual is formed from FP32 pairs instead.  Each sweep
// contracts the error by roughly the FP32 condition-number factor of S.
// Sweeps stop once ||r|| / ||b'_I - A'_ID phi_D|| (the residual relative to
// the right-hand side with all wall potentials moved into it) is <= rtol;
// if the last allowed sweep has not reached it, PIC_ENOCONV is latched.
// ||r|| / ||b'_I|| (relative to the charge alone) is reported as well.
//
// Initial guess.  Cold (warm_start 0): phi_rho = 0, so the first sweep
// sets phi_rho = S(b').  Warm (warm_start 1): the previous solve's phi_rho
// is kept; one residual pass before the first sweep measures it (and ends
// the solve at once if it already meets rtol), and every sweep adds.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "field_common.cuh"

namespace pic {

// ------------------------------------------------------- double-float

float2 df_from(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}

// ---------------------------------------------------------------- tables

// vacuum solution of the wall potentials of cfg (kd, ko: K_r) and its
// radial node field, into H.vac, H.evac64, H.evac32
static void vacuum_host(const pic_config& cfg, const HostTables& H, double hr) {
  const int nr = cfg.nr, NI = nr - 1;
  const double *kd = H.kd, *ko = H.ko;
  // K_r restricted to the interior lines with the wall potentials moved to
  // the right-hand side (M_r and K_z drop out for a z-independent field);
  // its radial node field by the same differences as the particle field
  // (central, one-sided second order on the walls)
  double* vac = H.vac;
  vac[0] = cfg.v_inner;
  vac[nr] = cfg.v_outer;
  for (int ii = 0; ii < NI; ++ii) {
    const int i = ii + 1;
    double rhs = 0.0;
    if (i == 1) rhs -= ko[0] * cfg.v_inner;
    if (i == nr - 1) rhs -= ko[nr - 1] * cfg.v_outer;
    const double sub = ii > 0 ? ko[i - 1] : 0.0;
    const double den = kd[i] - (ii > 0 ? sub * H.tmp_cp[ii - 1] : 0.0);
    H.tmp_cp[ii] = ko[i] / den;
    H.tmp_y[ii] = (rhs - (ii > 0 ? sub * H.tmp_y[ii - 1] : 0.0)) / den;
  }
  double xn = 0.0;
  for (int ii = NI - 1; ii >= 0; --ii) {
    xn = H.tmp_y[ii] - H.tmp_cp[ii] * xn;
    vac[ii + 1] = xn;
  }
  for (int i = 0; i <= nr; ++i) {
    double d;
    if (i == 0) d = (-3.0 * vac[0] + 4.0 * vac[1] - vac[2]) / (2.0 * hr);
    else if (i == nr) d = (3.0 * vac[nr] - 4.0 * vac[nr - 1] + vac[nr - 2]) / (2.0 * hr);
    else d = (vac[i + 1] - vac[i - 1]) / (2.0 * hr);
    H.evac64[i] = -d;
    H.evac32[i] = (float)(-d);
  }
}

void field_tables_host(const pic_config& cfg, FieldTables& T, const HostTables& H) {
  const int nr = cfg.nr, nz = cfg.nz, M = nz, NI = nr - 1, M1 = M + 1;
  T.nr = nr; T.nz = nz; T.M = M; T.NI = NI;
  T.hr = (cfg.r_out - cfg.r_in) / nr;
  T.hz = (cfg.z_max - cfg.z_min) / nz;
  T.rtol = cfg.poisson_rtol;
  T.maxit = cfg.poisson_maxit > 0 ? cfg.poisson_maxit : 4;
  T.inv2hr_d = 0.5 / T.hr;
  T.inv2hz_d = 0.5 / T.hz;
  T.inv2hr = (float)T.inv2hr_d;
  T.inv2hz = (float)T.inv2hz_d;
  T.hz32 = (float)T.hz;
  T.warm = cfg.warm_start >= 1 ? 1 : 0;
  int l2 = 0;
  while ((1 << l2) < 2 * M) ++l2;
  // FFT path for M a power of two whose 2M-point complex line and its M
  // twiddles fit the default 48 KB of dynamic shared memory; otherwise the
  // direct transform
  T.log2N = ((1 << l2) == 2 * M && 3 * M * (int)sizeof(float2) <= 48 * 1024) ? l2 : -1;
  const double hr = T.hr, hz = T.hz;

  double *kd = H.kd, *ko = H.ko, *md = H.md, *mo = H.mo;
  for (int i = 0; i <= nr; ++i) kd[i] = ko[i] = md[i] = mo[i] = 0.0;
  for (int e = 0; e < nr; ++e) {
    const double r0 = cfg.r_in + e * hr, r1 = cfg.r_in + (e + 1) * hr;
    const double k = (r0 + r1) / (2.0 * hr);
    kd[e] += k; kd[e + 1] += k; ko[e] = -k;
    md[e] += hr / 12.0 * (3.0 * r0 + r1);
    md[e + 1] += hr / 12.0 * (r0 + 3.0 * r1);
    mo[e] = hr / 12.0 * (r0 + r1);
  }

  vacuum_host(cfg, H, hr);

  // per-mode Thomas factors of g_k K_r + f_k M_r on the interior lines
  for (int k = 0; k <= M; ++k) {
    const double lam = 2.0 * std::cos(kPi * k / M);
    const double g = hz * (4.0 + lam) / 6.0, f = (2.0 - lam) / hz;
    const double eps_k = (k == 0 || k == M) ? 0.5 : 1.0;
    H.scale[k] = (float)(2.0 * eps_k / M);
    double cprev = 0.0;
    for (int ii = 0; ii < NI; ++ii) {
      const int i = ii + 1;
      const double diag = g * kd[i] + f * md[i];
      const double sub = ii > 0 ? g * ko[i - 1] + f * mo[i - 1] : 0.0;
      const double sup = g * ko[i] + f * mo[i];
      const double den = diag - sub * cprev;
      const size_t o = (size_t)ii * M1 + k;
      H.ta[o] = (float)sub;
      H.tinv[o] = (float)(1.0 / den);
      H.tcp[o] = (float)(sup / den);
      cprev = sup / den;
    }
  }
  if (T.log2N > 0) {
    const int N = 2 * M;
    for (int m = 0; m < N / 2; ++m) {
      H.tw[2 * m] = (float)std::cos(2.0 * kPi * m / N);
      H.tw[2 * m + 1] = (float)-std::sin(2.0 * kPi * m / N);
    }
  } else {
    for (int m = 0; m < 2 * M; ++m) H.cos[m] = (float)std::cos(kPi * m / M);
  }
  for (int i = 0; i <= nr; ++i) {
    H.kd2[i] = df_from(kd[i]); H.ko2[i] = df_from(ko[i]);
    H.md2[i] = df_from(md[i]); H.mo2[i] = df_from(mo[i]);
  }
  T.mzd_end = df_from(hz / 3.0);
  T.mzd_in = df_from(2.0 * hz / 3.0);
  T.mzo = df_from(hz / 6.0);
  T.kzd_end = df_from(1.0 / hz);
  T.kzd_in = df_from(2.0 / hz);
  T.kzo = df_from(-1.0 / hz);
  T.nsim = 1;
}

int field_tables_upload(FieldTables& T, const HostTables& H, cudaStream_t stream) {
  const int nr = T.nr, M1 = T.M + 1, NI = T.NI;
  const size_t nn = (size_t)(nr + 1) * M1, tri = (size_t)NI * M1 * sizeof(float);
  const size_t rad = (size_t)(nr + 1);
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream) == cudaSuccess;
  };
  bool ok = true;
  if (T.log2N > 0) ok = ok && cp(T.tw32, H.tw, (size_t)2 * T.M * sizeof(float));
  else ok = ok && cp(T.cos32, H.cos, (size_t)2 * T.M * sizeof(float));
  ok = ok && cp(T.scale32, H.scale, M1 * sizeof(float)) && cp(T.tri_a, H.ta, tri) &&
       cp(T.tri_inv, H.tinv, tri) && cp(T.tri_cp, H.tcp, tri) &&
       cp(T.phi_vac, H.vac, rad * sizeof(double)) && cp(T.evac64, H.evac64, rad * sizeof(double)) &&
       cp(T.evac32, H.evac32, rad * sizeof(float)) && cp(T.kr_d, H.kd2, rad * sizeof(float2)) &&
       cp(T.kr_o, H.ko2, rad * sizeof(float2)) && cp(T.mr_d, H.md2, rad * sizeof(float2)) &&
       cp(T.mr_o, H.mo2, rad * sizeof(float2));
  const size_t ns = (size_t)T.nsim;
  ok = ok && cudaMemsetAsync(T.phir, 0, ns * nn * sizeof(float2), stream) == cudaSuccess &&
       cudaMemsetAsync(T.b2, 0, ns * nn * sizeof(float2), stream) == cudaSuccess &&
       cudaMemsetAsync(T.res, 0, ns * nn * sizeof(float), stream) == cudaSuccess;
  return ok ? PIC_OK : PIC_ECUDA;
}

int field_tables_build(const pic_config* cfgs, int nsim, FieldTables& T,
                       void* (*dev_alloc)(size_t, void*), void* ctx,
                       cudaStream_t stream) {
  const pic_config& cfg = cfgs[0];
  const int nr = cfg.nr, M = cfg.nz, NI = nr - 1, M1 = M + 1;
  const size_t S = (size_t)nsim;
  const size_t nn = (size_t)(nr + 1) * M1, tri = (size_t)NI * M1;
  std::vector<double> dbl(9 * (size_t)(nr + 1));
  std::vector<float> flt(3 * tri + M1 + 4 * (size_t)M + (nr + 1));
  std::vector<float2> f2(4 * (size_t)(nr + 1));
  HostTables H;
  H.kd = dbl.data(); H.ko = H.kd + nr + 1; H.md = H.ko + nr + 1; H.mo = H.md + nr + 1;
  H.vac = H.mo + nr + 1; H.evac64 = H.vac + nr + 1; H.tmp_cp = H.evac64 + nr + 1;
  H.tmp_y = H.tmp_cp + nr + 1;
  H.ta = flt.data(); H.tinv = H.ta + tri; H.tcp = H.tinv + tri; H.scale = H.tcp + tri;
  H.tw = H.scale + M1; H.cos = H.tw + 2 * (size_t)M; H.evac32 = H.cos + 2 * (size_t)M;
  H.kd2 = f2.data(); H.ko2 = H.kd2 + nr + 1; H.md2 = H.ko2 + nr + 1; H.mo2 = H.md2 + nr + 1;
  field_tables_host(cfg, T, H);
  T.nsim = nsim;

  auto al = [&](size_t bytes, void** dst) -> bool {
    *dst = dev_alloc(std::max<size_t>(bytes, 16), ctx);
    return *dst != nullptr;
  };
  bool ok = true;
  T.tw32 = nullptr; T.cos32 = nullptr;
  if (T.log2N > 0) ok = al((size_t)2 * M * sizeof(float), (void**)&T.tw32);
  else ok = al((size_t)2 * M * sizeof(float), (void**)&T.cos32);
  ok = ok && al(M1 * sizeof(float), (void**)&T.scale32) &&
       al(tri * sizeof(float), (void**)&T.tri_a) && al(tri * sizeof(float), (void**)&T.tri_inv) &&
       al(tri * sizeof(float), (void**)&T.tri_cp) &&
       al(S * (nr + 1) * sizeof(double), (void**)&T.phi_vac) &&
       al(S * (nr + 1) * sizeof(double), (void**)&T.evac64) &&
       al(S * (nr + 1) * sizeof(float), (void**)&T.evac32) &&
       al((nr + 1) * sizeof(float2), (void**)&T.kr_d) &&
       al((nr + 1) * sizeof(float2), (void**)&T.kr_o) &&
       al((nr + 1) * sizeof(float2), (void**)&T.mr_d) &&
       al((nr + 1) * sizeof(float2), (void**)&T.mr_o) &&
       al(S * nn * sizeof(float2), (void**)&T.b2) && al(S * nn * sizeof(float2), (void**)&T.phir) &&
       al(S * nn * sizeof(float), (void**)&T.res) && al(S * tri * sizeof(float), (void**)&T.bhat) &&
       al(S * tri * sizeof(float), (void**)&T.phihat);
  if (!ok) return PIC_ENOMEM;
  int rc = field_tables_upload(T, H, stream);
  // the vacuum solution of every further simulation (its own wall
  // potentials; the geometry is shared)
  const size_t rad = (size_t)(nr + 1);
  for (int k = 1; k < nsim && rc == PIC_OK; ++k) {
    if (cudaStreamSynchronize(stream) != cudaSuccess) { rc = PIC_ECUDA; break; }
    vacuum_host(cfgs[k], H, T.hr);
    if (cudaMemcpyAsync(T.phi_vac + k * rad, H.vac, rad * sizeof(double), cudaMemcpyHostToDevice,
                        stream) != cudaSuccess ||
        cudaMemcpyAsync(T.evac64 + k * rad, H.evac64, rad * sizeof(double),
                        cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaMemcpyAsync(T.evac32 + k * rad, H.evac32, rad * sizeof(float), cudaMemcpyHostToDevice,
                        stream) != cudaSuccess)
      rc = PIC_ECUDA;
  }
  if (rc == PIC_OK && cudaStreamSynchronize(stream) != cudaSuccess) rc = PIC_ECUDA;
  return rc;
}

// ---------------------------------------------------------------- prep

// node-pass blocks: up to 32 x 16 threads (launch_field_solve picks the shape)
constexpr int kNodeThreads = 512;
constexpr int kNodeWarps = kNodeThreads / 32;

template <bool FIX>
__global__ void __launch_bounds__(kNodeThreads) k_prep(ChargeIn in, FieldTables T, DevState* st) {
  const int M1 = T.M + 1, nr = T.nr;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int sim = blockIdx.z;
  st += sim;
  float nb = 0.f, nl = 0.f;
  if (i <= nr && j < M1) {
    const size_t o = (size_t)sim * (nr + 1) * M1 + (size_t)i * M1 + j;
    const float2 b = prep_node<FIX>(in, T, sim, o, i, j, nb, nl);
    if (i > 0 && i < nr) T.res[o] = b.x;
  }
  __shared__ float red[2][kNodeWarps];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, lane = tid & 31, w = tid >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nb += __shfl_xor_sync(0xffffffffu, nb, o);
    nl += __shfl_xor_sync(0xffffffffu, nl, o);
  }
  if (lane == 0) { red[0][w] = nb; red[1][w] = nl; }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, c = 0.0;
    for (int k = 0; k < (int)(blockDim.x * blockDim.y) / 32; ++k) { a += red[0][k]; c += red[1][k]; }
    if (a != 0.0) atomicAdd(&st->b2sum, a);
    if (c != 0.0) atomicAdd(&st->bl2sum, c);
    if (blockIdx.x == 0 && blockIdx.y == 0) {
      st->solve_done = 0;
      st->poisson_iters = 0;
    }
  }
}

// ---------------------------------------------------------------- DCT-I

// y_k = sum_{j=0}^{M} x_j cos(pi k j / M) for two lines at once, FP32.
// FWD: lines are interior r-lines 1..nr-1 of T.res, output
//      bhat[line][k] = scale_k y_k.
// INV: lines are rows of phihat, output phi_rho[line + 1][k] (+)= y_k in
//      double-float (the first sweep sets, later sweeps add).
template <bool FWD>
__global__ void __launch_bounds__(512)
k_dct32(FieldTables T, const DevState* st, int sweep) {
  const int sim = blockIdx.y;
  if ((sweep > 0 || T.warm) && *(volatile const int*)&st[sim].solve_done) return;
  extern __shared__ float2 sh[];   // N line values, then N/2 twiddles
  const int M = T.M, N = 2 * M, M1 = M + 1, NI = T.NI, log2N = T.log2N;
  const size_t nn = (size_t)(T.nr + 1) * M1, tri = (size_t)NI * M1;
  T.res += sim * nn; T.phir += sim * nn; T.bhat += sim * tri; T.phihat += sim * tri;
  float2* tw = sh + N;
  const int line0 = blockIdx.x * 2;
  const bool two = line0 + 1 < NI;
  const float* x = FWD ? T.res + (size_t)(line0 + 1) * M1 : T.phihat + (size_t)line0 * M1;
  const float* y = x + M1;
  // bit-reversed input order, gathered from global memory so that the
  // shared-memory writes are consecutive (a bit-reversed scatter puts a
  // warp's writes N/2 apart, all in one bank)
  for (int p = threadIdx.x; p < N; p += blockDim.x) {
    const int n = __brev(p) >> (32 - log2N);
    const int m = n <= M ? n : N - n;
    sh[p] = make_float2(x[m], two ? y[m] : 0.f);
    if (p < N / 2) tw[p] = T.tw32[p];
  }
  __syncthreads();
  for (int s = 1; s <= log2N; ++s) {
    for (int t = threadIdx.x; t < N / 2; t += blockDim.x) fft_butterfly(sh, tw, N, s, t);
    __syncthreads();
  }
  const float x0 = x[0], xM = x[M];
  const float y0 = two ? y[0] : 0.f, yM = two ? y[M] : 0.f;
  for (int k = threadIdx.x; k <= M; k += blockDim.x) {
    const float2 v = dct_out(sh[k], k, x0, xM, y0, yM);
    const float vx = v.x, vy = v.y;
    if (FWD) {
      T.bhat[(size_t)line0 * M1 + k] = vx * T.scale32[k];
      if (two) T.bhat[(size_t)(line0 + 1) * M1 + k] = vy * T.scale32[k];
    } else {
      const bool set = sweep == 0 && !T.warm;
      float2* p = T.phir + (size_t)(line0 + 1) * M1 + k;
      *p = set ? make_float2(vx, 0.f) : df_add(*p, make_float2(vx, 0.f));
      if (two) {
        p += M1;
        *p = set ? make_float2(vy, 0.f) : df_add(*p, make_float2(vy, 0.f));
      }
    }
  }
}

// direct O(M^2) DCT-I for M that is not a power of two; one line per block
template <bool FWD>
__global__ void k_dct32_direct(FieldTables T, const DevState* st, int sweep) {
  const int sim = blockIdx.y;
  if ((sweep > 0 || T.warm) && *(volatile const int*)&st[sim].solve_done) return;
  extern __shared__ float xs[];
  const int M = T.M, M1 = M + 1, line = blockIdx.x;
  const size_t nn = (size_t)(T.nr + 1) * M1, tri = (size_t)T.NI * M1;
  T.res += sim * nn; T.phir += sim * nn; T.bhat += sim * tri; T.phihat += sim * tri;
  const float* x = FWD ? T.res + (size_t)(line + 1) * M1 : T.phihat + (size_t)line * M1;
  for (int j = threadIdx.x; j <= M; j += blockDim.x) xs[j] = x[j];
  __syncthreads();
  for (int k = threadIdx.x; k <= M; k += blockDim.x) {
    float acc = 0.f;
    int m = 0;   // (k j) mod 2M
    for (int j = 0; j <= M; ++j) {
      acc += xs[j] * T.cos32[m];
      m += k;
      if (m >= 2 * M) m -= 2 * M;
    }
    if (FWD) {
      T.bhat[(size_t)line * M1 + k] = acc * T.scale32[k];
    } else {
      float2* p = T.phir + (size_t)(line + 1) * M1 + k;
      *p = sweep == 0 && !T.warm ? make_float2(acc, 0.f) : df_add(*p, make_float2(acc, 0.f));
    }
  }
}

// ------------------------------------------------------------- tridiag

// One thread per z-mode: forward and back substitution of the pre-factored
// Thomas recurrence along the interior r-lines (FP32).  A block holds 16
// consecutive modes (33 blocks on the 512-cell grid); its 256 threads first
// copy the columns it needs into shared memory, 16 rows at a time with four
// rows' loads in flight per thread, so the recurrence, run by the first
// half-warp, then reads only shared memory, eight rows' operands at a time
// ahead of their dependent chain.  Right-hand side, sub-diagonal and pivot
// serve the forward pass; the super-diagonal serves the backward pass.
constexpr int kTriModes = 16;
constexpr int kTriThreads = 256;
constexpr int kTriRows = kTriThreads / kTriModes;   // rows staged per pass
constexpr int kTriBatch = 8;                        // rows per register batch of the recurrence
__global__ void __launch_bounds__(kTriThreads) k_tridiag32(FieldTables T, const DevState* st,
                                                           int sweep) {
  const int sim = blockIdx.y;
  if ((sweep > 0 || T.warm) && *(volatile const int*)&st[sim].solve_done) return;
  extern __shared__ float sm[];
  const int M1 = T.M + 1, NI = T.NI;
  const size_t tri = (size_t)NI * M1;
  T.bhat += sim * tri; T.phihat += sim * tri;
  const int col = threadIdx.x % kTriModes, row0 = threadIdx.x / kTriModes;
  const int k = blockIdx.x * kTriModes + col;
  const bool in = k < M1;
  float* sb = sm;                    // NI x 16: right-hand side, then solution
  float* sa = sm + NI * kTriModes;   // NI x 16: sub-diagonal
  float* sd = sa + NI * kTriModes;   // NI x 16: 1 / pivot
  float* sc = sd + NI * kTriModes;   // NI x 16: super-diagonal / pivot
#pragma unroll 4
  for (int i = row0; i < NI; i += kTriRows) {
    const size_t o = (size_t)i * M1 + k;
    const int q = i * kTriModes + col;
    sb[q] = in ? T.bhat[o] : 0.f;
    sa[q] = in ? T.tri_a[o] : 0.f;
    sd[q] = in ? T.tri_inv[o] : 0.f;
    sc[q] = in ? T.tri_cp[o] : 0.f;
  }
  __syncthreads();
  if (threadIdx.x < kTriModes) {
    // the recurrence in batches of kTriBatch rows: the batch's operands
    // are loaded into registers before its dependent chain starts
    float y = 0.f;
    for (int i0 = 0; i0 < NI; i0 += kTriBatch) {
      float b[kTriBatch], a[kTriBatch], d[kTriBatch];
#pragma unroll
      for (int k = 0; k < kTriBatch; ++k) {
        const int o = min(i0 + k, NI - 1) * kTriModes + col;
        b[k] = sb[o];
        a[k] = sa[o];
        d[k] = sd[o];
      }
#pragma unroll
      for (int k = 0; k < kTriBatch; ++k) {
        if (i0 + k < NI) {
          y = thomas_fwd(b[k], a[k], d[k], y);
          sb[(i0 + k) * kTriModes + col] = y;
        }
      }
    }
    float xn = 0.f;
    for (int i0 = NI - 1; i0 >= 0; i0 -= kTriBatch) {
      float b[kTriBatch], c[kTriBatch];
#pragma unroll
      for (int k = 0; k < kTriBatch; ++k) {
        const int o = max(i0 - k, 0) * kTriModes + col;
        b[k] = sb[o];
        c[k] = sc[o];
      }
#pragma unroll
      for (int k = 0; k < kTriBatch; ++k) {
        if (i0 - k >= 0) {
          xn = thomas_bwd(b[k], c[k], xn);
          sb[(i0 - k) * kTriModes + col] = xn;
        }
      }
    }
  }
  __syncthreads();
  if (in) {
#pragma unroll 4
    for (int i = row0; i < NI; i += kTriRows)
      T.phihat[(size_t)i * M1 + k] = sb[i * kTriModes + col];
  }
}

// shared memory of k_tridiag32 (four NI x 16 float arrays); above the
// default 48 KB the kernel is opted in once
static size_t tridiag_smem(const FieldTables& T) {
  return (size_t)4 * T.NI * kTriModes * sizeof(float);
}

// ------------------------------------ residual, convergence test, E field

// PREP (the warm start's first pass): b' is formed here as in k_prep before
// the residual of the previous solution, so one pass replaces two.
template <typename Real, int PREP>
__global__ void __launch_bounds__(kNodeThreads)
k_residual(FieldTables T, typename Vec2<Real>::type* E, DevState* st, int sweep, int last,
           ChargeIn in) {
  const int sim = blockIdx.z;
  st += sim;
  if (sweep >= 0 && (sweep > 0 || T.warm) && *(volatile const int*)&st->solve_done) return;
  const int nr = T.nr, M = T.M, M1 = M + 1;
  const size_t nn = (size_t)(nr + 1) * M1;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  float nb = 0.f, nl = 0.f;
  // the solve's first kernel resets the stopping state (before this
  // block's completion is counted, so before the last block's test)
  if (PREP && threadIdx.x == 0 && threadIdx.y == 0 && blockIdx.x == 0 && blockIdx.y == 0) {
    st->solve_done = 0;
    st->poisson_iters = 0;
  }
  if (PREP && i <= nr && j <= M)
    prep_node<PREP == 1>(in, T, sim, (size_t)sim * nn + (size_t)i * M1 + j, i, j, nb, nl);
  T.phir += sim * nn; T.res += sim * nn; T.b2 += sim * nn; E += sim * nn;
  T.evac32 += sim * (nr + 1); T.evac64 += sim * (nr + 1);
  float rn = 0.f;
  if (i <= nr && j <= M) {
    const size_t o = (size_t)i * M1 + j;
    const float2* ph = T.phir;
    E[o] = node_field<Real>(T, ph, T.evac32, T.evac64, o, i, j);

    if (i > 0 && i < nr) {
      // r = b' - A' phi_rho in double-float
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int di = -1; di <= 1; ++di) {
        float2 mz, kz;
        node_mzkz(T, ph, o + (ptrdiff_t)di * M1, j, mz, kz);
        acc = df_add(acc, row_term(T, i, di, mz, kz));
      }
      const float2 r = df_add(T.b2[o], df_neg(acc));
      T.res[o] = r.x;
      rn = r.x * r.x;
    }
  }
  // block reduction, then the last block evaluates the stopping test
  __shared__ float red[3][kNodeWarps];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, lane = tid & 31, w = tid >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rn += __shfl_xor_sync(0xffffffffu, rn, o);
    if (PREP) {
      nb += __shfl_xor_sync(0xffffffffu, nb, o);
      nl += __shfl_xor_sync(0xffffffffu, nl, o);
    }
  }
  if (lane == 0) { red[0][w] = rn; red[1][w] = nb; red[2][w] = nl; }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, bsum = 0.0, lsum = 0.0;
    for (int k = 0; k < (int)(blockDim.x * blockDim.y) / 32; ++k) {
      a += red[0][k];
      bsum += red[1][k];
      lsum += red[2][k];
    }
    if (a != 0.0) atomicAdd(&st->r2sum, a);
    if (PREP && bsum != 0.0) atomicAdd(&st->b2sum, bsum);
    if (PREP && lsum != 0.0) atomicAdd(&st->bl2sum, lsum);
    __threadfence();
    const unsigned nb = gridDim.x * gridDim.y;
    if (atomicAdd(&st->solve_blocks_done, 1u) == nb - 1) {
      __threadfence();
      const double r2 = *(volatile double*)&st->r2sum;
      const double b2 = *(volatile double*)&st->b2sum;
      const double bl2 = *(volatile double*)&st->bl2sum;
      double rel, strict;
      solve_norms(r2, b2, bl2, rel, strict);
      if (solve_record(st, T, rel, strict, sweep, last)) {
        st->b2sum = 0.0;
        st->bl2sum = 0.0;
      }
      st->r2sum = 0.0;
      st->solve_blocks_done = 0u;
    }
  }
}

// phi = phi_vac + phi_rho (FP64), on demand
__global__ void k_phi_out(FieldTables T, double* phi, int sim) {
  const int M1 = T.M + 1;
  const int n = (T.nr + 1) * M1;
  const float2* ph = T.phir + (size_t)sim * n;
  const double* vac = T.phi_vac + (size_t)sim * (T.nr + 1);
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n; o += gridDim.x * blockDim.x) {
    const float2 p = ph[o];
    phi[o] = vac[o / M1] + ((double)p.x + (double)p.y);
  }
}

void launch_phi_out(const FieldTables& T, double* phi, cudaStream_t stream, int sim) {
  const int n = (T.nr + 1) * (T.M + 1);
  k_phi_out<<<(n + 255) / 256, 256, 0, stream>>>(T, phi, sim);
}

int field_solve_kernels(const FieldTables& T) { return 1 + 4 * T.maxit; }

template <typename Real>
void launch_field_solve(const FieldTables& T, const double* rhs, const unsigned long long* cnt,
                        double cnt_unit, const float2* cnt_units, unsigned long long* cnt_clear,
                        void* efield, DevState* st, cudaStream_t stream) {
  const int M1 = T.M + 1, S = T.nsim;
  // node passes: 32 x 16 blocks for one simulation (half the blocks, so
  // half the same-address norm atomics of the 32 x 8 shape: 37 against 40
  // us per solve in the graph-replayed 128 x 512 step); 32 x 8 for a
  // batch, whose many blocks fill the GPU better in the smaller shape
  const int by = S == 1 ? 16 : 8;
  dim3 blk(32, by), grd((M1 + 31) / 32, (T.nr + 1 + by - 1) / by, S);
  const double s0 = 1.0 / (2.0 * kPi * kEps0);
  if (tridiag_smem(T) > 48 * 1024)
    cudaFuncSetAttribute(k_tridiag32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tridiag_smem(T));
  const ChargeIn in{rhs, cnt, cnt ? df_from(cnt_unit * s0) : make_float2(0.f, 0.f), cnt_units,
                    s0, cnt_clear};
  using V2 = typename Vec2<Real>::type;
  if (T.warm) {
    // b' and the residual of the previous solution (the refinement's start)
    // in one pass; the stopping state is reset by the solve's first kernel
    if (cnt) k_residual<Real, 1><<<grd, blk, 0, stream>>>(T, (V2*)efield, st, -1, T.maxit == 0, in);
    else k_residual<Real, 2><<<grd, blk, 0, stream>>>(T, (V2*)efield, st, -1, T.maxit == 0, in);
  } else {
    if (cnt) k_prep<true><<<grd, blk, 0, stream>>>(in, T, st);
    else k_prep<false><<<grd, blk, 0, stream>>>(in, T, st);
  }
  for (int s = 0; s < T.maxit; ++s) {
    if (T.log2N > 0) {
      const int N = 2 * T.M;
      const int threads = std::min(512, std::max(32, N / 2));
      const size_t smem = (size_t)(N + N / 2) * sizeof(float2);
      const dim3 blocks((T.NI + 1) / 2, S);
      k_dct32<true><<<blocks, threads, smem, stream>>>(T, st, s);
      k_tridiag32<<<dim3((M1 + kTriModes - 1) / kTriModes, S), kTriThreads, tridiag_smem(T),
                    stream>>>(T, st, s);
      k_dct32<false><<<blocks, threads, smem, stream>>>(T, st, s);
    } else {
      const size_t smem = (size_t)M1 * sizeof(float);
      k_dct32_direct<true><<<dim3(T.NI, S), 256, smem, stream>>>(T, st, s);
      k_tridiag32<<<dim3((M1 + kTriModes - 1) / kTriModes, S), kTriThreads, tridiag_smem(T),
                    stream>>>(T, st, s);
      k_dct32_direct<false><<<dim3(T.NI, S), 256, smem, stream>>>(T, st, s);
    }
    k_residual<Real, 0><<<grd, blk, 0, stream>>>(T, (V2*)efield, st, s, s == T.maxit - 1,
                                                ChargeIn{});
  }
}

template void launch_field_solve<float>(const FieldTables&, const double*,
                                        const unsigned long long*, double, const float2*,
                                        unsigned long long*, void*, DevState*, cudaStream_t);
template void launch_field_solve<double>(const FieldTables&, const double*,
                                         const unsigned long long*, double, const float2*,
                                         unsigned long long*, void*, DevState*, cudaStream_t);

}  // namespace pic
