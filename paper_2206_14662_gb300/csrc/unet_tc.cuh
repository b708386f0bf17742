// unet_tc.cuh -- the 3 x 3 convolution GEMM of the U-Net on the 5th-
// generation tensor cores (tcgen05.mma, kind::f16, BF16 operands, FP32
// accumulators in tensor memory).  Internal to unet.cu.
//
//   out[p, n] = epi( sum_{t < 9} sum_{k < K} X[src(p, t), k] * Wk[n * ldw + t * K + k] )
//
// with src(p, t) the 3 x 3 neighbour (dy, dx) = (t / 3 - 1, t % 3 - 1) of p,
// zero outside the image (the forward convolution, and its data gradient with
// the tap-reversed transposed weights).  One CTA computes an 8 x 16 block of
// pixels x all N output channels (N = 32, 64, 128 or 256): the accumulator is
// a 128-lane x N-column FP32 tile in tensor memory.
//
// Operand reuse: per 32-channel chunk the CTA stages its block's halo (10 x
// 16 pixels) three times, shifted by dx = -1, 0, +1, in shared memory.  The
// operand of tap (dy, dx) is then copy dx + 1 from row 16 (dy + 1) on: a
// descriptor offset, since a row of the block is 16 staged rows, two whole
// core-matrix groups.  Each activation is read 3.75x per chunk instead of
// once per tap (9x).  The taps' weights stream through a second ring.
// Layout of every staged tile: the canonical K-major layout without swizzle,
// 8-row x 16-byte core matrices, the four 8-element K chunks of a row group
// 128 bytes apart (the descriptor's leading byte offset), row groups 512
// bytes apart (its stride byte offset).
//
// The CTA is warp-specialised: four producer warps fill both rings with
// cp.async and signal each stage's "full" mbarrier as their copies land
// (cp.async.mbarrier.arrive); one lane of a fifth warp waits for them, issues
// the tap's two K = 16 MMAs and commits them to the stage's "empty" mbarrier,
// which lets the producers refill it.  No block barrier sits in the loop.
// The producer warps then read the accumulator out of tensor memory for the
// epilogue.  Every wait is bounded (about one second of SM clock): a wait
// that runs out sets *err, and the CTA still frees its tensor memory and
// returns.
#pragma once

#include <cstdint>

#include "unet_kernels.cuh"

namespace pic {
namespace unet {

constexpr int kTcM = 128;        // pixels per CTA = tensor-memory lanes
constexpr int kTcK = 32;         // channels per K-step
constexpr int kTcProducerWarps = 4;                     // one pixel row per thread
constexpr int kTcThreads = 32 * (kTcProducerWarps + 1);  // + the MMA warp
constexpr long long kTcWaitCycles = 2000000000LL;

// A CTA computes an 8 x 16 block of output pixels (128 = the MMA's M, one
// tensor-memory lane each) for all N output channels.
constexpr int kTcTileH = 8, kTcTileW = 16;
constexpr int kTcHaloRows = (kTcTileH + 2) * kTcTileW;     // 160 staged pixel rows
constexpr int kTcHaloBytes = kTcHaloRows * kTcK * 2;       // one shifted copy, 10 KB
constexpr int kTcABytes = 3 * kTcHaloBytes;                 // the three copies, 30 KB

// SA halo stages: 2 when there are several 32-channel chunks to overlap, 1
// for a single chunk (K = 32), which leaves room for more CTAs per SM
template <int N, int SA>
struct TcShape {
  static_assert(N == 32 || N == 64 || N == 128 || N == 256, "tensor-memory columns");
  static constexpr int kBBytes = N * kTcK * 2;   // one tap's weights for one chunk
  static constexpr int kBStages = N <= 64 ? 8 : 4;
  // A ring, B ring, then the barriers (A full/empty, B full/empty, done)
  // and the tensor-memory address
  static constexpr int kBarOff = SA * kTcABytes + kBStages * kBBytes;
  static constexpr int kSmemBytes = kBarOff + 16 * (SA + kBStages) + 8 + 16;
  // instruction descriptor: FP32 accumulator (bits 4-5 = 1), BF16 A and B
  // (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 (bits
  // 17-22), M >> 4 (bits 24-28)
  static constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                                     ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
};

// byte offset of (row, 8-element chunk) in a staged K-major tile
__device__ __forceinline__ int tc_off(int row, int chunk) {
  return (row >> 3) * 512 + chunk * 128 + (row & 7) * 16;
}

// shared-memory matrix descriptor of a staged tile starting at saddr: start
// address >> 4 (bits 0-13), leading byte offset 128 >> 4 (bits 16-29),
// stride byte offset 512 >> 4 (bits 32-45), descriptor version 1 (bits
// 46-47), base offset 0, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(512 >> 4) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void tc_mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool tc_mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      "  .reg .pred p;\n"
      "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "  selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool tc_mbar_wait(uint32_t bar, uint32_t parity) {
  if (tc_mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!tc_mbar_try(bar, parity))
    if (clock64() - t0 > kTcWaitCycles) return false;
  return true;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A(desc) * B(desc)^T, M = 128, K = 16, N from the descriptor
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n"
      "  .reg .pred p;\n"
      "  setp.ne.b32 p, %4, 0;\n"
      "  tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

// 32 consecutive FP32 columns of this thread's lane
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

template <int N, int SA>
__global__ void __launch_bounds__(kTcThreads)
k_conv3_tc(const bf16* __restrict__ X, int ldx, int K, const bf16* __restrict__ Wk, int ldw,
           Grid3 g, const float* __restrict__ bias, bf16* __restrict__ Y, int ldy, int epi,
           const bf16* __restrict__ act, int lda, int mask_from, int* __restrict__ err) {
  using Sh = TcShape<N, SA>;
  constexpr int SB = Sh::kBStages;
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  const uint32_t s0 = smem_u32(tc_smem);
  const uint32_t sB0 = s0 + SA * kTcABytes;
  const uint32_t afull = s0 + Sh::kBarOff, aempty = afull + 8 * SA;
  const uint32_t bfull = aempty + 8 * SA, bempty = bfull + 8 * SB, done = bempty + 8 * SB;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tc_smem + Sh::kBarOff + 16 * (SA + SB) + 8);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // the block: image b, rows y0 .. y0 + 7, columns x0 .. x0 + 15
  const int tiles_x = g.W / kTcTileW, tiles_y = g.H / kTcTileH;
  const int b = blockIdx.x / (tiles_x * tiles_y);
  const int rem = blockIdx.x % (tiles_x * tiles_y);
  const int y0 = (rem / tiles_x) * kTcTileH, x0 = (rem % tiles_x) * kTcTileW;
  const int kc = K / kTcK;

  if (warp == kTcProducerWarps) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
        "tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::"r"(smem_u32(tmem_slot)),
        "r"((uint32_t)N)
        : "memory");
    if (lane == 0) {
      for (int s = 0; s < SA; ++s) {
        tc_mbar_init(afull + 8 * s, 32 * kTcProducerWarps);
        tc_mbar_init(aempty + 8 * s, 1);
      }
      for (int s = 0; s < SB; ++s) {
        tc_mbar_init(bfull + 8 * s, 32 * kTcProducerWarps);
        tc_mbar_init(bempty + 8 * s, 1);
      }
      tc_mbar_init(done, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp < kTcProducerWarps) {
    // producers.  Per 32-channel chunk c: the block's halo (image rows
    // y0 - 1 .. y0 + 8, columns x0 .. x0 + 15) three times, shifted by
    // dx = -1, 0, +1 (copy d holds pixel (y0 - 1 + i, x0 + j + d - 1) at
    // row 16 i + j, zero outside the image); then per tap its weights.
    for (int c = 0; c < kc && ok; ++c) {
      const int sa = c % SA, ua = c / SA;
      if (ua > 0 && !tc_mbar_wait(aempty + 8 * sa, (uint32_t)(ua - 1) & 1u)) {
        ok = false;
        break;
      }
      unsigned char* A = tc_smem + sa * kTcABytes;
      const int c0 = c * kTcK;
      for (int r = tid; r < 3 * kTcHaloRows; r += 32 * kTcProducerWarps) {
        const int d = r / kTcHaloRows, m = r % kTcHaloRows;
        const int yy = y0 - 1 + m / kTcTileW, xx = x0 + m % kTcTileW + d - 1;
        const bool in = yy >= 0 && yy < g.H && xx >= 0 && xx < g.W;
        const bf16* xs = X + (in ? (((long long)b * g.H + yy) * g.W + xx) * ldx + c0 : 0);
        unsigned char* dst = A + d * kTcHaloBytes;
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) cp_async16(dst + tc_off(m, ch), xs + ch * 8, in);
      }
      asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(afull + 8 * sa)
                   : "memory");
      for (int t = 0; t < 9; ++t) {
        const int s = c * 9 + t, sb = s % SB, ub = s / SB;
        if (ub > 0 && !tc_mbar_wait(bempty + 8 * sb, (uint32_t)(ub - 1) & 1u)) {
          ok = false;
          break;
        }
        unsigned char* B = tc_smem + SA * kTcABytes + sb * Sh::kBBytes;
#pragma unroll
        for (int r = tid; r < N; r += 32 * kTcProducerWarps) {
          const bf16* ws = Wk + (size_t)r * ldw + t * K + c0;
#pragma unroll
          for (int ch = 0; ch < 4; ++ch) cp_async16(B + tc_off(r, ch), ws + ch * 8, true);
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bfull + 8 * sb)
                     : "memory");
      }
    }
    cp_async_wait<0>();
  } else if (lane == 0) {
    // the MMA thread: tap (dy, dx) reads copy dx + 1 from row 16 (dy + 1),
    // i.e. (dy + 1) x two core-matrix groups further
    for (int c = 0; c < kc && ok; ++c) {
      const int sa = c % SA;
      if (!tc_mbar_wait(afull + 8 * sa, (uint32_t)(c / SA) & 1u)) {
        ok = false;
        break;
      }
      for (int t = 0; t < 9; ++t) {
        const int s = c * 9 + t, sb = s % SB;
        if (!tc_mbar_wait(bfull + 8 * sb, (uint32_t)(s / SB) & 1u)) {
          ok = false;
          break;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_after();
        const int dy = t / 3 - 1, dx = t % 3 - 1;
        const uint32_t a = s0 + sa * kTcABytes + (dx + 1) * kTcHaloBytes + (dy + 1) * 1024;
        const uint32_t bb = sB0 + sb * Sh::kBBytes;
#pragma unroll
        for (int j = 0; j < 2; ++j)
          tc_mma(tmem, tc_desc(a + 256 * j), tc_desc(bb + 256 * j), Sh::kIdesc,
                 (c > 0 || t > 0 || j > 0) ? 1u : 0u);
        tc_commit(bempty + 8 * sb);
      }
      if (ok) tc_commit(aempty + 8 * sa);
    }
    if (ok) tc_commit(done);
  }
  if (warp < kTcProducerWarps) {
    // epilogue: warp w owns tensor-memory lanes 32 w .. 32 w + 31, i.e.
    // rows 2 w, 2 w + 1 of the block
    if (ok) ok = tc_mbar_wait(done, 0u);
    if (__all_sync(0xffffffffu, ok)) {
      tc_fence_after();
      const int m = warp * 32 + lane;
      const long long q = ((long long)b * g.H + y0 + m / kTcTileW) * g.W + x0 + m % kTcTileW;
#pragma unroll 1
      for (int n0 = 0; n0 < N; n0 += 32) {
        float v[32];
        tc_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)n0, v);
        if (epi == kBiasRelu || epi == kBias) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            v[j] += bias[n0 + j];
            if (epi == kBiasRelu) v[j] = fmaxf(v[j], 0.f);
          }
        } else if (epi == kMask) {
          const bf16* a = act + q * lda + n0;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (n0 + j >= mask_from && !(__bfloat162float(a[j]) > 0.f)) v[j] = 0.f;
        }
        uint4* out = reinterpret_cast<uint4*>(Y + q * ldy + n0);
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          __nv_bfloat162 h[4];
#pragma unroll
          for (int j = 0; j < 4; ++j)
            h[j] = __floats2bfloat162_rn(v[8 * cc + 2 * j], v[8 * cc + 2 * j + 1]);
          out[cc] = *reinterpret_cast<const uint4*>(h);
        }
      }
    } else {
      ok = false;
    }
  }
  if (!ok) atomicCAS(err, 0, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == kTcProducerWarps) {
    __syncwarp();   // (the warp's MMA lane rejoins before the aligned dealloc)
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)N)
                 : "memory");
  }
}

}  // namespace unet
}  // namespace pic
