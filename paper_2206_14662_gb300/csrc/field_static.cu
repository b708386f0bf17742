// field_static.cu -- pic_solve_field_static: the FP64 field solve of
// pic_solve_field for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not
// wanted -- a host framework that owns every byte of device memory through
// its own pool, a plug-in that may only touch the buffers it is handed, or
// a long-running service that must not grow its device footprint per call.
// Such a caller passes the right-hand side and the output potential in its
// own device buffers; everything else the solve needs (transformed
// right-hand side, per-mode Thomas factors, FFT twiddles, space-charge
// potential, node field, residual accumulators) lives in one file-scope
// device array, g_field_scratch, of fixed size.  Every GPU that loads the
// library holds that array (about 4 MB) until the process exits.
//
// The array is shared by all calls: each call clears what must start at
// zero (the residual accumulators, the space-charge potential) and
// overwrites the rest; calls whose GPU
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
// radial node lines nr + 1: the Thomas sweep's shared-memory columns
// (four (nr - 1) x 32 floats, at most 200 KB, the check at entry) admit
// nr <= 401
constexpr int kMaxRadial = 402;
static_assert(4LL * (kMaxRadial - 2) * 32 * 4 <= 200 * 1024 &&
                  4LL * (kMaxRadial - 1) * 32 * 4 > 200 * 1024,
              "kMaxRadial is the largest nr + 1 the Thomas limit admits");

// scratch layout: byte offsets, each region 256-byte aligned
constexpr size_t al256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kTri = (size_t)kMaxNodes * sizeof(float);          // (nr-1)(nz+1) floats
constexpr size_t kOffTriA = 0;
constexpr size_t kOffTriInv = kOffTriA + al256(kTri);
constexpr size_t kOffTriCp = kOffTriInv + al256(kTri);
constexpr size_t kOffBhat = kOffTriCp + al256(kTri);
constexpr size_t kOffPhihat = kOffBhat + al256(kTri);
constexpr size_t kOffRes = kOffPhihat + al256(kTri);
constexpr size_t kOffB2 = kOffRes + al256(kTri);
constexpr size_t kOffPhir = kOffB2 + al256((size_t)kMaxNodes * sizeof(float2));
constexpr size_t kOffE = kOffPhir + al256((size_t)kMaxNodes * sizeof(float2));
constexpr size_t kOffTw = kOffE + al256((size_t)kMaxNodes * sizeof(double2));
constexpr size_t kOffCos = kOffTw + al256((size_t)2 * kMaxM * sizeof(float));
constexpr size_t kOffScale = kOffCos + al256((size_t)2 * kMaxM * sizeof(float));
constexpr size_t kOffVac = kOffScale + al256((size_t)(kMaxM + 1) * sizeof(float));
constexpr size_t kOffEvac64 = kOffVac + al256((size_t)(kMaxRadial + 1) * sizeof(double));
constexpr size_t kOffEvac32 = kOffEvac64 + al256((size_t)(kMaxRadial + 1) * sizeof(double));
constexpr size_t kOffKd = kOffEvac32 + al256((size_t)(kMaxRadial + 1) * sizeof(float));
constexpr size_t kOffKo = kOffKd + al256((size_t)(kMaxRadial + 1) * sizeof(float2));
constexpr size_t kOffMd = kOffKo + al256((size_t)(kMaxRadial + 1) * sizeof(float2));
constexpr size_t kOffMo = kOffMd + al256((size_t)(kMaxRadial + 1) * sizeof(float2));
constexpr size_t kOffState = kOffMo + al256((size_t)(kMaxRadial + 1) * sizeof(float2));
constexpr size_t kScratchBytes = kOffState + al256(sizeof(DevState));

static __device__ __align__(256) double g_field_scratch[kScratchBytes / sizeof(double)];

// device address of g_field_scratch per device, looked up on first use
constexpr int kMaxDevices = 64;
char* g_scratch_dev[kMaxDevices];

// host staging of the tables (static: this entry point allocates nothing)
double h_kd[kMaxRadial + 1], h_ko[kMaxRadial + 1], h_md[kMaxRadial + 1], h_mo[kMaxRadial + 1];
double h_vac[kMaxRadial + 1], h_evac64[kMaxRadial + 1];
double h_tmp_cp[kMaxRadial + 1], h_tmp_y[kMaxRadial + 1];
float h_ta[kMaxNodes], h_tinv[kMaxNodes], h_tcp[kMaxNodes];
float h_scale[kMaxM + 1], h_tw[2 * kMaxM], h_cos[2 * kMaxM], h_evac32[kMaxRadial + 1];
float2 h_kd2[kMaxRadial + 1], h_ko2[kMaxRadial + 1], h_md2[kMaxRadial + 1], h_mo2[kMaxRadial + 1];

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
  if ((long long)4 * (c.nr - 1) * 32 * 4 > 200 * 1024) return PIC_EINVAL;   // Thomas columns
  if (c.nr + 1 > kMaxRadial) return PIC_EINVAL;   // (implied by the line above)
  cudaStream_t stream = (cudaStream_t)cuda_stream;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PIC_ECUDA;
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_field_scratch) != cudaSuccess || !p) return PIC_ECUDA;
    g_scratch_dev[dev] = (char*)p;
  }
  char* S = g_scratch_dev[dev];

  FieldTables T;
  std::memset(&T, 0, sizeof(T));
  HostTables H;
  H.kd = h_kd; H.ko = h_ko; H.md = h_md; H.mo = h_mo; H.vac = h_vac; H.evac64 = h_evac64;
  H.tmp_cp = h_tmp_cp; H.tmp_y = h_tmp_y; H.ta = h_ta; H.tinv = h_tinv; H.tcp = h_tcp;
  H.scale = h_scale; H.tw = h_tw; H.cos = h_cos; H.evac32 = h_evac32;
  H.kd2 = h_kd2; H.ko2 = h_ko2; H.md2 = h_md2; H.mo2 = h_mo2;
  field_tables_host(c, T, H);
  T.tri_a = (float*)(S + kOffTriA);
  T.tri_inv = (float*)(S + kOffTriInv);
  T.tri_cp = (float*)(S + kOffTriCp);
  T.bhat = (float*)(S + kOffBhat);
  T.phihat = (float*)(S + kOffPhihat);
  T.res = (float*)(S + kOffRes);
  T.b2 = (float2*)(S + kOffB2);
  T.phir = (float2*)(S + kOffPhir);
  T.tw32 = (float2*)(S + kOffTw);
  T.cos32 = (float*)(S + kOffCos);
  T.scale32 = (float*)(S + kOffScale);
  T.phi_vac = (double*)(S + kOffVac);
  T.evac64 = (double*)(S + kOffEvac64);
  T.evac32 = (float*)(S + kOffEvac32);
  T.kr_d = (float2*)(S + kOffKd);
  T.kr_o = (float2*)(S + kOffKo);
  T.mr_d = (float2*)(S + kOffMd);
  T.mr_o = (float2*)(S + kOffMo);
  void* E = S + kOffE;
  DevState* st = (DevState*)(S + kOffState);

  // every call clears what must start at zero: the solver state (residual
  // sums, counters) and the space-charge potential (zero on the walls, so
  // phi = phi_vac there, the wall potentials)
  if (field_tables_upload(T, H, stream) != PIC_OK ||
      cudaMemsetAsync(st, 0, sizeof(DevState), stream) != cudaSuccess)
    return PIC_ECUDA;
  launch_field_solve<double>(T, b, nullptr, 0.0, nullptr, nullptr, E, st, stream);
  launch_phi_out(T, phi, stream);
  if (cudaGetLastError() != cudaSuccess) return PIC_ECUDA;
  if (!relres) return PIC_OK;
  DevState s;
  if (cudaMemcpyAsync(&s, st, sizeof(DevState), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return PIC_ECUDA;
  *relres = s.relres_last;
  return s.err ? s.err : PIC_OK;
}
