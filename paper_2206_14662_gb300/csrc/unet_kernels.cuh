// unet_kernels.cuh -- kernels of the learned field-solve warm start (a
// four-level U-Net): implicit-GEMM convolutions on the BF16 tensor cores
// (mma.sync m16n8k16, FP32 accumulation), their FP32 reference forms for
// the test mode, and the small elementwise kernels.  Internal to unet.cu.
//
// Activations are (batch, H, W, channels) with the channel count padded to a
// multiple of 32 (padded channels hold zeros and have zero weights, so they
// stay zero through training).  Every GEMM here is
//   out[p, n] = sum_{t < taps} sum_{k < K} in[src(p, t), k] * Wk[n * ldw + t * K + k]
// over the pixels p of an iteration grid (batch, h, w), with a pixel map:
//   kConv3  3 x 3 correlation, src = (y + t/3 - 1, x + t%3 - 1) on the same
//           grid (zero outside), out at p
//   kUpFwd  transposed 2 x 2 convolution, one sub-grid t = 2 dy + dx per
//           launch: src = p on the coarse grid, out at (2y + dy, 2x + dx) on
//           the fine grid
//   kUpBwd  its data gradient: src(p, t) = (2y + t/2, 2x + t%2) on the fine
//           grid, out at p on the coarse grid
// and the weight gradient
//   dW[n][t * K + k] += sum_p G[gsrc(p, t), n] * X[xsrc(p, t), k]
// (kConv3: gsrc = p, xsrc = src(p, t); transposed convolution: gsrc = the
// fine-grid pixel of sub-grid t, xsrc = p).  Weight layouts: a 3 x 3 layer
// [out][9 * in] (tap-major), a transposed 2 x 2 layer [out][4 * in].
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace pic {
namespace unet {

using bf16 = __nv_bfloat16;

enum PixMap { kConv3 = 0, kUpFwd = 1, kUpBwd = 2 };

// Epilogues of the forward-type GEMM
enum Epi {
  kBiasRelu = 0,   // out = relu(acc + bias)
  kBias = 1,       // out = acc + bias
  kMask = 2,       // out = acc * (n < mask_from || act[p, n] > 0)
  kPlain = 3       // out = acc
};

struct Grid3 {
  int B, H, W;     // iteration grid (the GEMM's pixel rows)
};

// source pixel of iteration pixel p for tap t, or -1 outside the grid;
// fine-grid pixels for the transposed convolution's data gradient
__device__ __forceinline__ long long src_pixel(int map, long long p, int t, Grid3 g) {
  const int x = (int)(p % g.W);
  const long long q = p / g.W;
  const int y = (int)(q % g.H);
  const int b = (int)(q / g.H);
  if (map == kConv3) {
    const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
    if (yy < 0 || yy >= g.H || xx < 0 || xx >= g.W) return -1;
    return ((long long)b * g.H + yy) * g.W + xx;
  }
  if (map == kUpBwd) {
    const int yy = 2 * y + (t >> 1), xx = 2 * x + (t & 1);
    return ((long long)b * (2 * g.H) + yy) * (2 * g.W) + xx;
  }
  return p;   // kUpFwd
}

// output pixel of iteration pixel p (sub-grid t of the transposed
// convolution)
__device__ __forceinline__ long long dst_pixel(int map, long long p, int t, Grid3 g) {
  if (map != kUpFwd) return p;
  const int x = (int)(p % g.W);
  const long long q = p / g.W;
  const int y = (int)(q % g.H);
  const int b = (int)(q / g.H);
  return ((long long)b * (2 * g.H) + 2 * y + (t >> 1)) * (2 * g.W) + 2 * x + (t & 1);
}

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
// 16-byte global -> shared copy, zero-filled when !valid
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}
__device__ __forceinline__ void ldsm_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3,
                                        const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3,
                                          const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_u32(p)));
}
// D = A (16x16, row) * B (16x8, col) + D, BF16 inputs, FP32 accumulators
__device__ __forceinline__ void mma_bf16(float* d, unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// ------------------------------------------------- forward-type GEMM (mma)

// Block: 128 threads, BM = 64 pixels x BN output channels, K in steps of 32
// channels of one tap, two-stage cp.async pipeline.  Warps tile the block
// as (4 / (BN / 32)) x (BN / 32), each warp 32 channels wide.  Shared rows
// are padded to 40 elements (80 bytes) so that ldmatrix rows fall in
// distinct banks.
constexpr int kBM = 64, kBK = 32, kLds = 40;

template <int BN>
__global__ void __launch_bounds__(128)
k_gemm_fwd(const bf16* __restrict__ X, int ldx, int K, const bf16* __restrict__ Wk, int ldw,
           int taps, int map, int tap0, Grid3 g, const float* __restrict__ bias,
           bf16* __restrict__ Y, int ldy, int epi, const bf16* __restrict__ act, int lda,
           int mask_from) {
  constexpr int WN = BN / 32, WM = 4 / WN, MT = (kBM / WM) / 16;
  __shared__ __align__(16) bf16 sA[2][kBM * kLds];
  __shared__ __align__(16) bf16 sB[2][BN * kLds];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp / WN, wn = warp % WN;
  const long long P = (long long)g.B * g.H * g.W;
  const long long p0 = (long long)blockIdx.x * kBM;
  const int n0 = blockIdx.y * BN;
  const int kc = K / kBK;               // channel chunks per tap
  const int steps = taps * kc;

  auto load = [&](int stage, int s) {
    const int t = s / kc, c0 = (s % kc) * kBK;
    const int tap = tap0 + t;
    // A: 64 pixel rows x 32 channels = 256 chunks of 16 bytes
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int ch = tid + i * 128;
      const int row = ch >> 2, part = ch & 3;
      const long long p = p0 + row;
      long long sp = -1;
      if (p < P) sp = src_pixel(map, p, map == kUpFwd ? 0 : tap, g);
      const bf16* src = X + (sp < 0 ? 0 : sp * ldx + c0 + part * 8);
      cp_async16(&sA[stage][row * kLds + part * 8], src, sp >= 0);
    }
    // B: BN channel rows x 32 k
#pragma unroll
    for (int i = 0; i < BN / 32; ++i) {
      const int ch = tid + i * 128;
      const int row = ch >> 2, part = ch & 3;
      const bf16* src = Wk + (size_t)(n0 + row) * ldw + t * K + c0 + part * 8;
      cp_async16(&sB[stage][row * kLds + part * 8], src, true);
    }
  };

  float acc[MT][4][4];
#pragma unroll
  for (int a = 0; a < MT; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

  load(0, 0);
  cp_async_commit();
  for (int s = 0; s < steps; ++s) {
    const int cur = s & 1;
    if (s + 1 < steps) load(cur ^ 1, s + 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 16) {
      unsigned af[MT][4], bfr[4][2];
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        const int row = wm * (kBM / WM) + mt * 16 + (lane & 15);
        ldsm_x4(af[mt][0], af[mt][1], af[mt][2], af[mt][3],
                &sA[cur][row * kLds + kk + (lane >> 4) * 8]);
      }
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        const int row = wn * 32 + np * 16 + (lane & 7) + ((lane >> 4) << 3);
        unsigned r0, r1, r2, r3;
        ldsm_x4(r0, r1, r2, r3, &sB[cur][row * kLds + kk + ((lane >> 3) & 1) * 8]);
        bfr[2 * np][0] = r0; bfr[2 * np][1] = r1;
        bfr[2 * np + 1][0] = r2; bfr[2 * np + 1][1] = r3;
      }
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
          mma_bf16(acc[mt][nt], af[mt][0], af[mt][1], af[mt][2], af[mt][3], bfr[nt][0], bfr[nt][1]);
    }
    __syncthreads();
  }
  cp_async_wait<0>();

  // epilogue: accumulator (row g or g + 8, columns 2 (lane & 3) + 0/1)
  const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int mt = 0; mt < MT; ++mt) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long p = p0 + wm * (kBM / WM) + mt * 16 + gq + 8 * h;
      if (p >= P) continue;
      const long long q = dst_pixel(map, p, tap0, g);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int n = n0 + wn * 32 + nt * 8 + 2 * tq;
        float v0 = acc[mt][nt][2 * h], v1 = acc[mt][nt][2 * h + 1];
        if (epi == kBiasRelu || epi == kBias) {
          v0 += bias[n];
          v1 += bias[n + 1];
          if (epi == kBiasRelu) {
            v0 = fmaxf(v0, 0.f);
            v1 = fmaxf(v1, 0.f);
          }
        } else if (epi == kMask) {
          const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(act + q * lda + n);
          if (n >= mask_from && !(__bfloat162float(a.x) > 0.f)) v0 = 0.f;
          if (n + 1 >= mask_from && !(__bfloat162float(a.y) > 0.f)) v1 = 0.f;
        }
        *reinterpret_cast<__nv_bfloat162*>(Y + q * ldy + n) = __floats2bfloat162_rn(v0, v1);
      }
    }
  }
}

// ------------------------------------------------ weight gradient (mma)

// dW[n][t * K + k] += sum over the block's pixel range of
// G[gsrc(p), n] * X[xsrc(p), k]: M = 64 output channels n, N = 64 input
// channels k, K = pixels in steps of 32.  Both operands are staged pixel-
// major ([pixel][channel], rows padded to 72 elements) and read with
// ldmatrix.trans.  Each block adds its partial sums with FP32 atomics.
constexpr int kWM = 64, kWN = 64, kWK = 32, kWLds = 72;

__global__ void __launch_bounds__(128)
k_gemm_wgrad(const bf16* __restrict__ G, int ldg, const bf16* __restrict__ X, int ldx, int K,
             int N, int map, Grid3 g, long long pix_per_block, float* __restrict__ dW, int taps) {
  __shared__ __align__(16) bf16 sG[2][kWK * kWLds];
  __shared__ __align__(16) bf16 sX[2][kWK * kWLds];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;       // 2 x 2 warps of 32 x 32
  const int t = blockIdx.z % taps;
  const long long P = (long long)g.B * g.H * g.W;
  const long long pa = (long long)(blockIdx.z / taps) * pix_per_block;
  const long long pb = pa + pix_per_block < P ? pa + pix_per_block : P;
  const int m0 = blockIdx.y * kWM;               // output channels n
  const int k0 = blockIdx.x * kWN;               // input channels k
  const int steps = (int)((pb - pa + kWK - 1) / kWK);
  if (steps <= 0) return;

  auto load = [&](int stage, int s) {
    // 32 pixel rows x 64 channels for each operand: 256 chunks each
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int ch = tid + i * 128;
      const int row = ch >> 3, part = ch & 7;
      const long long p = pa + (long long)s * kWK + row;
      long long gp = -1, xp = -1;
      if (p < pb) {
        if (map == kConv3) {
          gp = p;
          xp = src_pixel(kConv3, p, t, g);
        } else {          // transposed convolution: G on the fine grid
          gp = dst_pixel(kUpFwd, p, t, g);
          xp = p;
        }
      }
      const bool vg = gp >= 0 && m0 + part * 8 < N, vx = xp >= 0 && k0 + part * 8 < K;
      cp_async16(&sG[stage][row * kWLds + part * 8], G + (vg ? gp * ldg + m0 + part * 8 : 0), vg);
      cp_async16(&sX[stage][row * kWLds + part * 8], X + (vx ? xp * ldx + k0 + part * 8 : 0), vx);
    }
  };

  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

  load(0, 0);
  cp_async_commit();
  for (int s = 0; s < steps; ++s) {
    const int cur = s & 1;
    if (s + 1 < steps) load(cur ^ 1, s + 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kWK; kk += 16) {
      unsigned af[2][4], bfr[4][2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        // A = G^T: rows n, columns pixels; stored [pixel][n]
        const int kr = kk + (lane & 7) + ((lane >> 4) << 3);
        const int mc = wm * 32 + mt * 16 + ((lane >> 3) & 1) * 8;
        ldsm_x4_t(af[mt][0], af[mt][1], af[mt][2], af[mt][3], &sG[cur][kr * kWLds + mc]);
      }
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        // B = X: rows pixels, columns k; stored [pixel][k]
        const int kr = kk + (lane & 7) + (((lane >> 3) & 1) << 3);
        const int nc = wn * 32 + np * 16 + (lane >> 4) * 8;
        unsigned r0, r1, r2, r3;
        ldsm_x4_t(r0, r1, r2, r3, &sX[cur][kr * kWLds + nc]);
        bfr[2 * np][0] = r0; bfr[2 * np][1] = r1;
        bfr[2 * np + 1][0] = r2; bfr[2 * np + 1][1] = r3;
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
          mma_bf16(acc[mt][nt], af[mt][0], af[mt][1], af[mt][2], af[mt][3], bfr[nt][0], bfr[nt][1]);
    }
    __syncthreads();
  }
  cp_async_wait<0>();
  const int gq = lane >> 2, tq = lane & 3;
  const int ldw = taps * K;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int n = m0 + wm * 32 + mt * 16 + gq + 8 * h;
      if (n >= N) continue;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int k = k0 + wn * 32 + nt * 8 + 2 * tq;
        if (k < K) {
          atomicAdd(dW + (size_t)n * ldw + t * K + k, acc[mt][nt][2 * h]);
          atomicAdd(dW + (size_t)n * ldw + t * K + k + 1, acc[mt][nt][2 * h + 1]);
        }
      }
    }
}

// Weight gradient of a 32 x 32 tile (layers with 32 input or output
// channels, where a 64 x 64 tile would idle half or more of its MMAs):
// stages of 64 pixels, each warp takes one 16-pixel slice of every stage
// and accumulates the whole tile, and the four partial tiles are summed in
// shared memory before the FP32 atomics.
constexpr int kW2K = 64, kW2Lds = 40;

__global__ void __launch_bounds__(128)
k_gemm_wgrad32(const bf16* __restrict__ G, int ldg, const bf16* __restrict__ X, int ldx, int K,
               int N, int map, Grid3 g, long long pix_per_block, float* __restrict__ dW,
               int taps) {
  __shared__ __align__(16) bf16 sm[2 * 2 * kW2K * kW2Lds];   // sG[2], sX[2]; partials after
  bf16* sG = sm;
  bf16* sX = sm + 2 * kW2K * kW2Lds;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int t = blockIdx.z % taps;
  const long long P = (long long)g.B * g.H * g.W;
  const long long pa = (long long)(blockIdx.z / taps) * pix_per_block;
  const long long pb = pa + pix_per_block < P ? pa + pix_per_block : P;
  const int m0 = blockIdx.y * 32;                // output channels n
  const int k0 = blockIdx.x * 32;                // input channels k
  const int steps = (int)((pb - pa + kW2K - 1) / kW2K);
  if (steps <= 0) return;

  auto load = [&](int stage, int st) {
    // 64 pixel rows x 32 channels for each operand: 256 chunks each
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int ch = tid + i * 128;
      const int row = ch >> 2, part = ch & 3;
      const long long p = pa + (long long)st * kW2K + row;
      long long gp = -1, xp = -1;
      if (p < pb) {
        if (map == kConv3) {
          gp = p;
          xp = src_pixel(kConv3, p, t, g);
        } else {
          gp = dst_pixel(kUpFwd, p, t, g);
          xp = p;
        }
      }
      const bool vg = gp >= 0 && m0 + part * 8 < N, vx = xp >= 0 && k0 + part * 8 < K;
      cp_async16(&sG[(stage * kW2K + row) * kW2Lds + part * 8],
                 G + (vg ? gp * ldg + m0 + part * 8 : 0), vg);
      cp_async16(&sX[(stage * kW2K + row) * kW2Lds + part * 8],
                 X + (vx ? xp * ldx + k0 + part * 8 : 0), vx);
    }
  };

  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

  load(0, 0);
  cp_async_commit();
  for (int st = 0; st < steps; ++st) {
    const int cur = st & 1;
    if (st + 1 < steps) load(cur ^ 1, st + 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const bf16* gs = sG + cur * kW2K * kW2Lds;
    const bf16* xs = sX + cur * kW2K * kW2Lds;
    const int kk = warp * 16;                    // this warp's pixel slice
    unsigned af[2][4], bfr[4][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int kr = kk + (lane & 7) + ((lane >> 4) << 3);
      const int mc = mt * 16 + ((lane >> 3) & 1) * 8;
      ldsm_x4_t(af[mt][0], af[mt][1], af[mt][2], af[mt][3], gs + kr * kW2Lds + mc);
    }
#pragma unroll
    for (int np = 0; np < 2; ++np) {
      const int kr = kk + (lane & 7) + (((lane >> 3) & 1) << 3);
      const int nc = np * 16 + (lane >> 4) * 8;
      unsigned r0, r1, r2, r3;
      ldsm_x4_t(r0, r1, r2, r3, xs + kr * kW2Lds + nc);
      bfr[2 * np][0] = r0; bfr[2 * np][1] = r1;
      bfr[2 * np + 1][0] = r2; bfr[2 * np + 1][1] = r3;
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
        mma_bf16(acc[mt][nt], af[mt][0], af[mt][1], af[mt][2], af[mt][3], bfr[nt][0], bfr[nt][1]);
    __syncthreads();
  }
  cp_async_wait<0>();
  // sum the four warps' tiles in shared memory (the staging area is free)
  float* part = reinterpret_cast<float*>(sm);    // [4][32][33]
  const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int m = mt * 16 + gq + 8 * h, k = nt * 8 + 2 * tq;
        part[(warp * 32 + m) * 33 + k] = acc[mt][nt][2 * h];
        part[(warp * 32 + m) * 33 + k + 1] = acc[mt][nt][2 * h + 1];
      }
  __syncthreads();
  const int ldw = taps * K;
  for (int e = tid; e < 32 * 32; e += 128) {
    const int m = e >> 5, k = e & 31;
    const float v = part[m * 33 + k] + part[(32 + m) * 33 + k] + part[(64 + m) * 33 + k] +
                    part[(96 + m) * 33 + k];
    if (m0 + m < N && k0 + k < K) atomicAdd(dW + (size_t)(m0 + m) * ldw + t * K + k0 + k, v);
  }
}

}  // namespace unet
}  // namespace pic
