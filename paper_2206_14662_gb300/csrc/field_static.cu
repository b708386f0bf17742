// field_static.cu -- pic_solve_field_static: the FP64 field solve of
// pic_solve_field for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not
// wanted -- a host framework that owns every byte of device memory through
// its own pool, a plug-in that may only touch the buffers it is handed, or
// a long-running service that must not grow its device footprint per call.
// Such a caller passes the right-hand side and the output potential in its
// own device buffers; everything else the solve needs (transformed
// right-hand side, per-mode Thomas factors, FFT twiddles, node field,
// residual accumulators) lives in one file-scope device array,
// g_field_scratch, of fixed size.  Every GPU that loads the library holds
// that array (about 5 MB) until the process exits.
//
// The array is shared by all calls: each call clears what must start at
// zero (the residual accumulators) and overwrites the rest; calls whose GPU
// work overlaps (different streams, or several host threads) race on it and
// must be serialised by the caller.  The host-side tables are built in
// static host arrays as well, so concurrent calls from several host threads
// are not allowed either.  The first call on each device looks up the
// array's device address (cudaGetSymbolAddress) with that device current;
// make that first call before any stream capture.
#include <cmath>
#include <cstring>

#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int kMaxNodes = PIC_STATIC_MAX_NODES;
constexpr int kMaxM = 4096;                 // nz limit of the library
constexpr int kMaxRadial = kMaxNodes / 3;   // nr + 1 when nz = 2

// scratch layout, in doubles
constexpr size_t kOffBhat = 0;
constexpr size_t kOffPhihat = kOffBhat + kMaxNodes;
constexpr size_t kOffTriA = kOffPhihat + kMaxNodes;
constexpr size_t kOffTriInv = kOffTriA + kMaxNodes;
constexpr size_t kOffTriCp = kOffTriInv + kMaxNodes;
constexpr size_t kOffE = kOffTriCp + kMaxNodes;             // double2 per node
constexpr size_t kOffTw = kOffE + 2 * (size_t)kMaxNodes;    // double2, < kMaxM
constexpr size_t kOffCos = kOffTw + 2 * (size_t)kMaxM;      // 2M entries
constexpr size_t kOffScale = kOffCos + 2 * (size_t)kMaxM;   // M + 1 entries
constexpr size_t kOffRad = kOffScale + kMaxM + 8;           // 5 radial vectors
constexpr size_t kOffState = kOffRad + 5 * (size_t)(kMaxRadial + 1);
constexpr size_t kStateDoubles = (sizeof(DevState) + 7) / 8 + 1;
constexpr size_t kScratchDoubles = ((kOffState + kStateDoubles + 31) / 32) * 32;

static __device__ __align__(256) double g_field_scratch[kScratchDoubles];

// device address of g_field_scratch per device, looked up on first use
constexpr int kMaxDevices = 64;
double* g_scratch_dev[kMaxDevices];

// host staging of the tables (static: this entry point allocates nothing)
double h_tri_a[kMaxNodes], h_tri_inv[kMaxNodes], h_tri_cp[kMaxNodes];
double h_tw[2 * kMaxM], h_cos[2 * kMaxM], h_scale[kMaxM + 1];
double h_rad[5][kMaxRadial + 1];   // phi_vac, K_r diag, K_r off, M_r diag, M_r off
double h_tmp_cp[kMaxRadial + 1], h_tmp_y[kMaxRadial + 1];
double h_walls[2 * (kMaxM + 1)];

__global__ void k_static_walls(double* phi, const double* walls, int nr, int nzp) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nzp; j += gridDim.x * blockDim.x) {
    phi[j] = walls[j];
    phi[(size_t)nr * nzp + j] = walls[nzp + j];
  }
}

}  // namespace
}  // namespace pic

using namespace pic;

extern "C" int pic_solve_field_static(const pic_config* cfg, const double* b, double* phi,
                                      double* relres, void* cuda_stream) {
  if (!cfg || !b || !phi) return PIC_EINVAL;
  const pic_config& c = *cfg;
  if (!(c.r_in > 0 && c.r_out > c.r_in && c.z_max > c.z_min)) return PIC_EINVAL;
  if (c.nr < 2 || c.nz < 2 || c.nz > kMaxM || !(c.poisson_rtol > 0)) return PIC_EINVAL;
  const long long nodes = (long long)(c.nr + 1) * (c.nz + 1);
  if (nodes > kMaxNodes) return PIC_EINVAL;   // beyond the static scratch
  cudaStream_t stream = (cudaStream_t)cuda_stream;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PIC_ECUDA;
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_field_scratch) != cudaSuccess || !p) return PIC_ECUDA;
    g_scratch_dev[dev] = (double*)p;
  }
  double* S = g_scratch_dev[dev];

  // tables of the separable solve (the same construction as the handle's)
  const int nr = c.nr, M = c.nz, NI = nr - 1, M1 = M + 1;
  FieldTables T;
  std::memset(&T, 0, sizeof(T));
  T.nr = nr; T.nz = M; T.M = M; T.NI = NI;
  T.hr = (c.r_out - c.r_in) / nr;
  T.hz = (c.z_max - c.z_min) / M;
  T.rtol = c.poisson_rtol;
  int l2 = 0;
  while ((1 << l2) < 2 * M) ++l2;
  T.log2N = ((1 << l2) == 2 * M && 2 * M * (int)sizeof(double2) <= 48 * 1024) ? l2 : -1;
  const double hr = T.hr, hz = T.hz;
  double* vac = h_rad[0];
  double* kd = h_rad[1];
  double* ko = h_rad[2];
  double* md = h_rad[3];
  double* mo = h_rad[4];
  for (int i = 0; i <= nr; ++i) kd[i] = ko[i] = md[i] = mo[i] = 0.0;
  for (int e = 0; e < nr; ++e) {
    const double r0 = c.r_in + e * hr, r1 = c.r_in + (e + 1) * hr;
    const double k = (r0 + r1) / (2.0 * hr);
    kd[e] += k; kd[e + 1] += k; ko[e] = -k;
    md[e] += hr / 12.0 * (3.0 * r0 + r1);
    md[e + 1] += hr / 12.0 * (r0 + 3.0 * r1);
    mo[e] = hr / 12.0 * (r0 + r1);
  }
  vac[0] = c.v_inner;
  vac[nr] = c.v_outer;
  for (int ii = 0; ii < NI; ++ii) {
    const int i = ii + 1;
    double rhs = 0.0;
    if (i == 1) rhs -= ko[0] * c.v_inner;
    if (i == nr - 1) rhs -= ko[nr - 1] * c.v_outer;
    const double sub = ii > 0 ? ko[i - 1] : 0.0;
    const double den = kd[i] - (ii > 0 ? sub * h_tmp_cp[ii - 1] : 0.0);
    h_tmp_cp[ii] = ko[i] / den;
    h_tmp_y[ii] = (rhs - (ii > 0 ? sub * h_tmp_y[ii - 1] : 0.0)) / den;
  }
  double xn = 0.0;
  for (int ii = NI - 1; ii >= 0; --ii) {
    xn = h_tmp_y[ii] - h_tmp_cp[ii] * xn;
    vac[ii + 1] = xn;
  }
  for (int k = 0; k <= M; ++k) {
    const double lam = 2.0 * std::cos(kPi * k / M);
    const double g = hz * (4.0 + lam) / 6.0, f = (2.0 - lam) / hz;
    const double eps_k = (k == 0 || k == M) ? 0.5 : 1.0;
    h_scale[k] = 2.0 * eps_k / (M * 2.0 * kPi * kEps0);
    double cprev = 0.0;
    for (int ii = 0; ii < NI; ++ii) {
      const int i = ii + 1;
      const double diag = g * kd[i] + f * md[i];
      const double sub = ii > 0 ? g * ko[i - 1] + f * mo[i - 1] : 0.0;
      const double sup = g * ko[i] + f * mo[i];
      const double den = diag - sub * cprev;
      const size_t o = (size_t)ii * M1 + k;
      h_tri_a[o] = sub;
      h_tri_inv[o] = 1.0 / den;
      h_tri_cp[o] = sup / den;
      cprev = h_tri_cp[o];
    }
  }
  if (T.log2N > 0) {
    const int N = 2 * M;
    for (int m = 0; m < N / 2; ++m) {
      h_tw[2 * m] = std::cos(2.0 * kPi * m / N);
      h_tw[2 * m + 1] = -std::sin(2.0 * kPi * m / N);
    }
  } else {
    for (int m = 0; m < 2 * M; ++m) h_cos[m] = std::cos(kPi * m / M);
  }
  const int nzp = M + 1;
  for (int j = 0; j < nzp; ++j) {
    h_walls[j] = c.v_inner;
    h_walls[nzp + j] = c.v_outer;
  }

  T.bhat = S + kOffBhat;
  T.phihat = S + kOffPhihat;
  T.tri_a = S + kOffTriA;
  T.tri_invd = S + kOffTriInv;
  T.tri_cp = S + kOffTriCp;
  T.twiddle = (double2*)(S + kOffTw);
  T.costab = S + kOffCos;
  T.fwd_scale = S + kOffScale;
  T.phi_vac = S + kOffRad;
  T.kr_d = S + kOffRad + (kMaxRadial + 1);
  T.kr_o = S + kOffRad + 2 * (kMaxRadial + 1);
  T.mr_d = S + kOffRad + 3 * (kMaxRadial + 1);
  T.mr_o = S + kOffRad + 4 * (kMaxRadial + 1);
  double* E = S + kOffE;
  DevState* st = (DevState*)(S + kOffState);
  // the wall values are staged in the transformed-solution area, which the
  // solve overwrites only after the walls are copied into phi
  double* walls = T.phihat;

  const size_t tri = (size_t)NI * M1 * sizeof(double);
  const size_t rad = (size_t)(nr + 1) * sizeof(double);
  bool ok = cudaMemcpyAsync(T.tri_a, h_tri_a, tri, cudaMemcpyHostToDevice, stream) == cudaSuccess &&
            cudaMemcpyAsync(T.tri_invd, h_tri_inv, tri, cudaMemcpyHostToDevice, stream) == cudaSuccess &&
            cudaMemcpyAsync(T.tri_cp, h_tri_cp, tri, cudaMemcpyHostToDevice, stream) == cudaSuccess &&
            cudaMemcpyAsync(T.fwd_scale, h_scale, (size_t)M1 * sizeof(double), cudaMemcpyHostToDevice,
                            stream) == cudaSuccess &&
            cudaMemcpyAsync(T.phi_vac, vac, rad, cudaMemcpyHostToDevice, stream) == cudaSuccess &&
            cudaMemcpyAsync(T.kr_d, kd, rad, cudaMemcpyHostToDevice, stream) == cudaSuccess &&
            cudaMemcpyAsync(T.kr_o, ko, rad, cudaMemcpyHostToDevice, stream) == cudaSuccess &&
            cudaMemcpyAsync(T.mr_d, md, rad, cudaMemcpyHostToDevice, stream) == cudaSuccess &&
            cudaMemcpyAsync(T.mr_o, mo, rad, cudaMemcpyHostToDevice, stream) == cudaSuccess &&
            cudaMemcpyAsync(walls, h_walls, 2 * (size_t)nzp * sizeof(double), cudaMemcpyHostToDevice,
                            stream) == cudaSuccess &&
            cudaMemsetAsync(st, 0, sizeof(DevState), stream) == cudaSuccess;
  if (ok && T.log2N > 0)
    ok = cudaMemcpyAsync(T.twiddle, h_tw, (size_t)2 * M * sizeof(double), cudaMemcpyHostToDevice,
                         stream) == cudaSuccess;
  if (ok && T.log2N <= 0)
    ok = cudaMemcpyAsync(T.costab, h_cos, (size_t)2 * M * sizeof(double), cudaMemcpyHostToDevice,
                         stream) == cudaSuccess;
  if (!ok) return PIC_ECUDA;
  k_static_walls<<<(nzp + 255) / 256, 256, 0, stream>>>(phi, walls, nr, nzp);
  launch_field_solve<double>(T, const_cast<double*>(b), phi, E, nullptr, st, false, stream);
  if (cudaGetLastError() != cudaSuccess) return PIC_ECUDA;
  if (!relres) return PIC_OK;
  DevState s;
  if (cudaMemcpyAsync(&s, st, sizeof(DevState), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return PIC_ECUDA;
  *relres = s.relres_last;
  return s.err ? s.err : PIC_OK;
}
