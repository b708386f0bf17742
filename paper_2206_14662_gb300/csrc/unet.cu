// unet.cu -- the learned initial guess of the field solve: a four-level
// convolutional U-Net (base width c: 3 x 3 convolutions with ReLU, two per
// level at widths c, 2c, 4c, 8c, 2 x 2 average pooling, 2 x 2 transposed
// convolutions, skip connections concatenated after the upsampled
// channels, a 1 x 1 head to one channel), trained on the GPU by this file's
// forward and backward kernels with Adam.  The paper has no counterpart: it
// only warm-starts the field solve, which still iterates to the same
// residual bound (the solver still decides convergence).
//
// Precision: precision 16 keeps activations and weight copies in BF16 and
// runs every convolution on the tensor cores with FP32 accumulation (FP32
// master weights, gradients and Adam moments); precision 32 is a test mode
// with FP32 activations and plain FP32 GEMM loops.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "pic_internal.cuh"
#include "unet_kernels.cuh"
#include "unet_tc.cuh"

namespace pic {
namespace unet {

// ------------------------------------------------------- element access

__device__ __forceinline__ float ld(const float* p) { return *p; }
__device__ __forceinline__ float ld(const bf16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void st(float* p, float v) { *p = v; }
__device__ __forceinline__ void st(bf16* p, float v) { *p = __float2bfloat16_rn(v); }

// ------------------------------------------------- FP32 reference GEMMs

// the GEMMs of unet_kernels.cuh, one output per thread, FP32 (test mode)
__global__ void k_gemm_fwd_ref(const float* __restrict__ X, int ldx, int K,
                               const float* __restrict__ Wk, int ldw, int taps, int map, int tap0,
                               Grid3 g, const float* __restrict__ bias, float* __restrict__ Y,
                               int ldy, int epi, const float* __restrict__ act, int lda,
                               int mask_from, int N) {
  const long long P = (long long)g.B * g.H * g.W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P * N;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / N;
    const int n = (int)(i % N);
    float acc = 0.f;
    for (int t = 0; t < taps; ++t) {
      const long long sp = src_pixel(map, p, map == kUpFwd ? 0 : tap0 + t, g);
      if (sp < 0) continue;
      const float* x = X + sp * ldx;
      const float* w = Wk + (size_t)n * ldw + t * K;
      for (int k = 0; k < K; ++k) acc = fmaf(x[k], w[k], acc);
    }
    const long long q = dst_pixel(map, p, tap0, g);
    if (epi == kBiasRelu) acc = fmaxf(acc + bias[n], 0.f);
    else if (epi == kBias) acc += bias[n];
    else if (epi == kMask && n >= mask_from && !(act[q * lda + n] > 0.f)) acc = 0.f;
    Y[q * ldy + n] = acc;
  }
}

__global__ void k_gemm_wgrad_ref(const float* __restrict__ G, int ldg, const float* __restrict__ X,
                                 int ldx, int K, int N, int map, Grid3 g, float* __restrict__ dW,
                                 int taps) {
  const long long P = (long long)g.B * g.H * g.W;
  const long long total = (long long)N * taps * K;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(i / ((long long)taps * K));
    const int t = (int)((i / K) % taps);
    const int k = (int)(i % K);
    float acc = 0.f;
    for (long long p = 0; p < P; ++p) {
      long long gp, xp;
      if (map == kConv3) { gp = p; xp = src_pixel(kConv3, p, t, g); }
      else { gp = dst_pixel(kUpFwd, p, t, g); xp = p; }
      if (xp < 0) continue;
      acc = fmaf(G[gp * ldg + n], X[xp * ldx + k], acc);
    }
    dW[i] += acc;
  }
}

// ---------------------------------------------------- elementwise kernels

// network input: (rho, phi_prev) FP32 (batch, H, W, 2) into channels 0, 1
// of a 32-channel activation
template <typename T>
__global__ void k_pack_input(const float* __restrict__ x, T* __restrict__ y, long long P) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P * 32;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i >> 5;
    const int c = (int)(i & 31);
    st(y + i, c < 2 ? x[2 * p + c] : 0.f);
  }
}

// 2 x 2 mean of x (fine grid H x W, channel stride ldx) into y (C channels)
template <typename T>
__global__ void k_pool(const T* __restrict__ x, int ldx, T* __restrict__ y, int C, int B, int H,
                       int W) {
  const int h = H / 2, w = W / 2;
  const long long total = (long long)B * h * w * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long q = i / C;
    const int xx = (int)(q % w), yy = (int)((q / w) % h), b = (int)(q / ((long long)w * h));
    const long long p00 = ((long long)b * H + 2 * yy) * W + 2 * xx;
    const float s = ld(x + p00 * ldx + c) + ld(x + (p00 + 1) * ldx + c) +
                    ld(x + (p00 + W) * ldx + c) + ld(x + (p00 + W + 1) * ldx + c);
    st(y + i, 0.25f * s);
  }
}

// gradient of a skip activation s (post-ReLU): the part arriving through
// the concatenation (gcat, stride ldg) plus the pooled path's gradient gp
// (coarse grid) spread over its 2 x 2 block, times relu'(s)
template <typename T>
__global__ void k_pool_bwd_mask(const T* __restrict__ gcat, int ldg, const T* __restrict__ gp,
                                const T* __restrict__ s, int lds, T* __restrict__ out, int C, int B,
                                int H, int W) {
  const long long total = (long long)B * H * W * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long p = i / C;
    const int x = (int)(p % W), y = (int)((p / W) % H), b = (int)(p / ((long long)W * H));
    const long long q = ((long long)b * (H / 2) + y / 2) * (W / 2) + x / 2;
    float v = ld(gcat + p * ldg + c) + 0.25f * ld(gp + q * C + c);
    if (!(ld(s + p * lds + c) > 0.f)) v = 0.f;
    st(out + i, v);
  }
}

// head: y = b + sum_c a[p, c] w[c]
template <typename T>
__global__ void k_head_fwd(const T* __restrict__ a, int C, const float* __restrict__ w,
                           const float* __restrict__ b, float* __restrict__ y, long long P) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
       p += (long long)gridDim.x * blockDim.x) {
    float acc = b[0];
    for (int c = 0; c < C; ++c) acc = fmaf(ld(a + p * C + c), w[c], acc);
    y[p] = acc;
  }
}

// loss sum (y - t)^2 / (2N) and its gradient (y - t) / N
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ t,
                       float* __restrict__ gy, float* __restrict__ loss, long long P) {
  float acc = 0.f;
  const float inv = 1.f / (float)P;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
       p += (long long)gridDim.x * blockDim.x) {
    const float d = y[p] - t[p];
    gy[p] = d * inv;
    acc += d * d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, 0.5f * acc * inv);
}

// head gradient: g[p, c] = gy[p] w[c] relu'(a[p, c]); gw[c] += sum_p gy a,
// gb += sum_p gy (threads own channels, pixels split over the grid)
template <typename T>
__global__ void k_head_bwd(const T* __restrict__ a, int C, const float* __restrict__ w,
                           const float* __restrict__ gy, T* __restrict__ g, float* __restrict__ gw,
                           float* __restrict__ gb, long long P) {
  const int c = threadIdx.x % C, lanes = blockDim.x / C, sub = threadIdx.x / C;
  if (sub >= lanes) return;
  float sw = 0.f, sb = 0.f;
  for (long long p = (long long)blockIdx.x * lanes + sub; p < P; p += (long long)gridDim.x * lanes) {
    const float av = ld(a + p * C + c), gv = gy[p];
    st(g + p * C + c, av > 0.f ? gv * w[c] : 0.f);
    sw = fmaf(gv, av, sw);
    if (c == 0) sb += gv;
  }
  atomicAdd(gw + c, sw);
  if (c == 0) atomicAdd(gb, sb);
}

// bias gradient: gb[n] += sum_p g[p, n] (channel stride ldg, N channels)
template <typename T>
__global__ void k_colsum(const T* __restrict__ g, int ldg, int N, float* __restrict__ gb,
                         long long P) {
  const int n = threadIdx.x % N, lanes = blockDim.x / N, sub = threadIdx.x / N;
  if (sub >= lanes) return;
  float s = 0.f;
  for (long long p = (long long)blockIdx.x * lanes + sub; p < P; p += (long long)gridDim.x * lanes)
    s += ld(g + p * ldg + n);
  atomicAdd(gb + n, s);
}

// compute copies of a layer's weights: wc = w (precision of the
// activations), wt = the data-gradient layout [in][taps * out] with the taps
// reversed for a 3 x 3 layer
template <typename T>
__global__ void k_derive(const float* __restrict__ w, int cout, int taps, int cin, int flip,
                         T* __restrict__ wc, T* __restrict__ wt) {
  const long long total = (long long)cout * taps * cin;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int co = (int)(i / ((long long)taps * cin));
    const int t = (int)((i / cin) % taps);
    const int ci = (int)(i % cin);
    const float v = w[i];
    st(wc + i, v);
    const int tt = flip ? taps - 1 - t : t;
    st(wt + ((size_t)ci * taps + tt) * cout + co, v);
  }
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// FP32 output x (batch, H, W, 2) of the input gradient (channels 0, 1)
template <typename T>
__global__ void k_unpack_grad(const T* __restrict__ g, float* __restrict__ out, long long P) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P * 2;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = ld(g + (i >> 1) * 32 + (i & 1));
}

inline int blocks_for(long long n, int threads = 256) {
  return (int)std::max<long long>(1, std::min<long long>((n + threads - 1) / threads, 152 * 32));
}
inline int pad32(int c) { return (c + 31) / 32 * 32; }

}  // namespace unet
}  // namespace pic

using namespace pic;
using namespace pic::unet;

namespace {

enum LayerKind { kLConv = 0, kLUp = 1, kLHead = 2 };

struct Layer {
  int kind;
  int cin, cout;        // real channels
  int cinp, coutp;      // padded channels (head: coutp = 1)
  int cu, cup;          // concatenated input: real / padded upsampled channels (0: none)
  int taps;             // 9, 4 or 1
  long long nw;         // padded weights
  float *w, *b, *gw, *gb, *mw, *vw, *mb, *vb;
  void *wc, *wt;        // compute copies
};

// index of a real input channel in the padded layout
int in_slot(const Layer& L, int ci) {
  if (L.cu > 0 && ci >= L.cu) return L.cup + (ci - L.cu);
  return ci;
}

}  // namespace

struct pic_unet {
  int c, H, W, B, prec;
  cudaStream_t stream;
  pic_allocator alloc;
  bool has_alloc;
  std::vector<void*> owned;
  std::vector<Layer> L;   // in the flat parameter order
  long long n_params;     // real parameters
  size_t es;              // activation element size
  int C[5];               // padded widths of levels 1..4 (C[0] unused)
  // activations (T) and gradient buffers
  void *x0, *e1a, *cat1, *p1, *e2a, *cat2, *p2, *e3a, *cat3, *p3, *e4a, *e4b;
  void *d3a, *d3b, *d2a, *d2b, *d1a, *d1b;
  void *g1b, *g1a, *gc1, *g2b, *g2a, *gc2, *g3b, *g3a, *gc3, *g4b, *g4a, *gp3, *gs3, *ge3a,
      *gp2, *gs2, *ge2a, *gp1, *gs1, *ge1a, *gx0;
  float *y, *gy, *loss;
  int* dev_err;           // set by a tensor-core GEMM whose bounded wait ran out
  int tc_mode = -1;       // 3 x 3 GEMMs on tcgen05: -1 where the grid fills the GPU, 0 never,
                          // 1 wherever the shape allows
  int sms;
};

namespace {

void* u_alloc(pic_unet* n, size_t bytes) {
  bytes = std::max<size_t>(bytes, 256);
  void* p = nullptr;
  if (n->has_alloc) p = n->alloc.alloc(bytes, (void*)n->stream, n->alloc.ctx);
  else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
  if (p) n->owned.push_back(p);
  return p;
}

// layer table: name order of the flat parameter vector
void make_layers(pic_unet* n) {
  const int c = n->c;
  auto conv = [&](int cin, int cout, int cu) {
    Layer l;
    std::memset(&l, 0, sizeof(l));
    l.kind = kLConv; l.cin = cin; l.cout = cout; l.taps = 9;
    l.cu = cu; l.cup = cu ? pad32(cu) : 0;
    l.cinp = cu ? 2 * pad32(cu) : pad32(cin);
    l.coutp = pad32(cout);
    return l;
  };
  auto up = [&](int cin, int cout) {
    Layer l;
    std::memset(&l, 0, sizeof(l));
    l.kind = kLUp; l.cin = cin; l.cout = cout; l.taps = 4;
    l.cinp = pad32(cin); l.coutp = pad32(cout);
    return l;
  };
  n->L = {conv(2, c, 0), conv(c, c, 0), conv(c, 2 * c, 0), conv(2 * c, 2 * c, 0),
          conv(2 * c, 4 * c, 0), conv(4 * c, 4 * c, 0), conv(4 * c, 8 * c, 0),
          conv(8 * c, 8 * c, 0),
          up(8 * c, 4 * c), conv(8 * c, 4 * c, 4 * c), conv(4 * c, 4 * c, 0),
          up(4 * c, 2 * c), conv(4 * c, 2 * c, 2 * c), conv(2 * c, 2 * c, 0),
          up(2 * c, c), conv(2 * c, c, c), conv(c, c, 0)};
  Layer h;
  std::memset(&h, 0, sizeof(h));
  h.kind = kLHead; h.cin = c; h.cout = 1; h.cinp = pad32(c); h.coutp = 1; h.taps = 1;
  n->L.push_back(h);
  n->n_params = 0;
  for (Layer& l : n->L) {
    l.nw = (long long)l.coutp * l.taps * l.cinp;
    n->n_params += (long long)l.cout * l.taps * l.cin + l.cout;
  }
}

enum {   // positions in the layer table
  E1A, E1B, E2A, E2B, E3A, E3B, E4A, E4B, UP3, D3A, D3B, UP2, D2A, D2B, UP1, D1A, D1B, HEAD
};

int derive_all(pic_unet* n) {
  for (Layer& l : n->L) {
    if (l.kind == kLHead) continue;
    const int nb = blocks_for(l.nw);
    const int flip = l.kind == kLConv ? 1 : 0;
    if (n->prec == 16)
      k_derive<bf16><<<nb, 256, 0, n->stream>>>(l.w, l.coutp, l.taps, l.cinp, flip, (bf16*)l.wc,
                                                (bf16*)l.wt);
    else
      k_derive<float><<<nb, 256, 0, n->stream>>>(l.w, l.coutp, l.taps, l.cinp, flip,
                                                 (float*)l.wc, (float*)l.wt);
  }
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

// dynamic shared memory of the tensor-core GEMMs (once per process)
int tc_prepare() {
  static int rc = -1;
  if (rc < 0) {
    auto set = [](auto kern, int bytes) {
      return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ==
             cudaSuccess;
    };
    const bool ok = set(k_conv3_tc<32, 1>, TcShape<32, 1>::kSmemBytes) &&
                    set(k_conv3_tc<64, 1>, TcShape<64, 1>::kSmemBytes) &&
                    set(k_conv3_tc<128, 1>, TcShape<128, 1>::kSmemBytes) &&
                    set(k_conv3_tc<256, 1>, TcShape<256, 1>::kSmemBytes) &&
                    set(k_conv3_tc<32, 2>, TcShape<32, 2>::kSmemBytes) &&
                    set(k_conv3_tc<64, 2>, TcShape<64, 2>::kSmemBytes) &&
                    set(k_conv3_tc<128, 2>, TcShape<128, 2>::kSmemBytes) &&
                    set(k_conv3_tc<256, 2>, TcShape<256, 2>::kSmemBytes);
    rc = ok ? PIC_OK : PIC_ECUDA;
  }
  return rc;
}

// a tensor-core GEMM's bounded wait that ran out (synchronises)
int tc_status(pic_unet* n) {
  int e = 0;
  if (cudaMemcpyAsync(&e, n->dev_err, sizeof(int), cudaMemcpyDeviceToHost, n->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(n->stream) != cudaSuccess)
    return PIC_ECUDA;
  return e ? PIC_ETIMEOUT : PIC_OK;
}

// out[p, n] (+ epilogue) = GEMM over the taps of `map`; weights `w` with
// row stride ldw (taps * K, or 4 * K for one sub-grid of a transposed layer)
void gemm_fwd(pic_unet* n, const void* X, int ldx, int K, const void* w, int ldw, int taps,
              int map, int tap0, Grid3 g, const float* bias, void* Y, int ldy, int N, int epi,
              const void* act, int lda, int mask_from) {
  const long long P = (long long)g.B * g.H * g.W;
  const long long tc_ctas = P / kTcM;
  if (n->prec == 16 && map == kConv3 && taps == 9 && tap0 == 0 && K % kTcK == 0 &&
      g.H % kTcTileH == 0 && g.W % kTcTileW == 0 &&
      (N == 32 || N == 64 || N == 128 || N == 256) && n->tc_mode != 0 &&
      (n->tc_mode == 1 || tc_ctas >= 2LL * n->sms)) {
    // tcgen05: one CTA per 8 x 16 pixel block computes every output channel
    // (grids of fewer than two CTAs per SM stay on the smaller mma.sync tiles)
    const unsigned grid = (unsigned)tc_ctas;
    auto run = [&](auto nn) {
      constexpr int NN = decltype(nn)::value;
      if (K == kTcK)
        k_conv3_tc<NN, 1><<<grid, kTcThreads, TcShape<NN, 1>::kSmemBytes, n->stream>>>(
            (const bf16*)X, ldx, K, (const bf16*)w, ldw, g, bias, (bf16*)Y, ldy, epi,
            (const bf16*)act, lda, mask_from, n->dev_err);
      else
        k_conv3_tc<NN, 2><<<grid, kTcThreads, TcShape<NN, 2>::kSmemBytes, n->stream>>>(
            (const bf16*)X, ldx, K, (const bf16*)w, ldw, g, bias, (bf16*)Y, ldy, epi,
            (const bf16*)act, lda, mask_from, n->dev_err);
    };
    if (N == 32) run(std::integral_constant<int, 32>());
    else if (N == 64) run(std::integral_constant<int, 64>());
    else if (N == 128) run(std::integral_constant<int, 128>());
    else run(std::integral_constant<int, 256>());
  } else if (n->prec == 16) {
    const dim3 grid((unsigned)((P + kBM - 1) / kBM), N % 64 == 0 ? N / 64 : N / 32);
    if (N % 64 == 0)
      k_gemm_fwd<64><<<grid, 128, 0, n->stream>>>((const bf16*)X, ldx, K, (const bf16*)w, ldw,
                                                   taps, map, tap0, g, bias, (bf16*)Y, ldy, epi,
                                                   (const bf16*)act, lda, mask_from);
    else
      k_gemm_fwd<32><<<grid, 128, 0, n->stream>>>((const bf16*)X, ldx, K, (const bf16*)w, ldw,
                                                   taps, map, tap0, g, bias, (bf16*)Y, ldy, epi,
                                                   (const bf16*)act, lda, mask_from);
  } else {
    k_gemm_fwd_ref<<<blocks_for(P * N), 256, 0, n->stream>>>(
        (const float*)X, ldx, K, (const float*)w, ldw, taps, map, tap0, g, bias, (float*)Y, ldy,
        epi, (const float*)act, lda, mask_from, N);
  }
}

void gemm_wgrad(pic_unet* n, const void* G, int ldg, const void* X, int ldx, int K, int N,
                int map, Grid3 g, float* dW, int taps) {
  const long long P = (long long)g.B * g.H * g.W;
  if (n->prec == 16 && (K == 32 || N == 32)) {
    // 32 x 32 tiles; pixels split so that the grid fills the machine about
    // four times
    const long long tiles = (long long)(K / 32) * (N / 32) * taps;
    long long splits = std::max<long long>(1, (4LL * n->sms + tiles - 1) / tiles);
    long long per = (P + splits - 1) / splits;
    per = std::max<long long>(kW2K * 4, (per + kW2K - 1) / kW2K * kW2K);
    splits = (P + per - 1) / per;
    const dim3 grid(K / 32, N / 32, (unsigned)(splits * taps));
    k_gemm_wgrad32<<<grid, 128, 0, n->stream>>>((const bf16*)G, ldg, (const bf16*)X, ldx, K, N,
                                                map, g, per, dW, taps);
  } else if (n->prec == 16) {
    // split the pixels so that the grid fills the machine about four times
    const long long tiles = (long long)((K + kWN - 1) / kWN) * ((N + kWM - 1) / kWM) * taps;
    long long splits = std::max<long long>(1, (4LL * n->sms + tiles - 1) / tiles);
    long long per = (P + splits - 1) / splits;
    per = std::max<long long>(kWK * 4, (per + kWK - 1) / kWK * kWK);
    splits = (P + per - 1) / per;
    const dim3 grid((K + kWN - 1) / kWN, (N + kWM - 1) / kWM, (unsigned)(splits * taps));
    k_gemm_wgrad<<<grid, 128, 0, n->stream>>>((const bf16*)G, ldg, (const bf16*)X, ldx, K, N, map,
                                              g, per, dW, taps);
  } else {
    k_gemm_wgrad_ref<<<blocks_for((long long)N * taps * K), 256, 0, n->stream>>>(
        (const float*)G, ldg, (const float*)X, ldx, K, N, map, g, dW, taps);
  }
}

void colsum(pic_unet* n, const void* G, int ldg, int N, float* gb, long long P) {
  const int lanes = std::max(1, 256 / N);
  const int blocks = (int)std::max<long long>(1, std::min<long long>((P + lanes * 64 - 1) / (lanes * 64),
                                                                     (long long)n->sms * 4));
  if (n->prec == 16) k_colsum<bf16><<<blocks, lanes * N, 0, n->stream>>>((const bf16*)G, ldg, N, gb, P);
  else k_colsum<float><<<blocks, lanes * N, 0, n->stream>>>((const float*)G, ldg, N, gb, P);
}

char* el(pic_unet* n, void* p, long long off) { return (char*)p + off * (long long)n->es; }

void conv_fwd(pic_unet* n, int li, const void* X, int ldx, Grid3 g, void* Y, int ldy) {
  const Layer& l = n->L[li];
  gemm_fwd(n, X, ldx, l.cinp, l.wc, 9 * l.cinp, 9, kConv3, 0, g, l.b, Y, ldy, l.coutp, kBiasRelu,
           nullptr, 0, 0);
}

// transposed 2 x 2 layer from the coarse grid g into the fine-grid buffer Y
void up_fwd(pic_unet* n, int li, const void* X, Grid3 g, void* Y, int ldy) {
  const Layer& l = n->L[li];
  for (int t = 0; t < 4; ++t)
    gemm_fwd(n, X, l.cinp, l.cinp, el(n, l.wc, (long long)t * l.cinp), 4 * l.cinp, 1, kUpFwd, t,
             g, l.b, Y, ldy, l.coutp, kBias, nullptr, 0, 0);
}

void pool_fwd(pic_unet* n, const void* x, int ldx, void* y, int C, Grid3 fine) {
  const long long total = (long long)fine.B * (fine.H / 2) * (fine.W / 2) * C;
  if (n->prec == 16) k_pool<bf16><<<blocks_for(total), 256, 0, n->stream>>>((const bf16*)x, ldx, (bf16*)y, C, fine.B, fine.H, fine.W);
  else k_pool<float><<<blocks_for(total), 256, 0, n->stream>>>((const float*)x, ldx, (float*)y, C, fine.B, fine.H, fine.W);
}

// backward of a 3 x 3 layer: weight and bias gradients from its input X
// and the pre-activation gradient G; the data gradient into GX with
// epilogue epi (kMask with act = X for a ReLU input, kPlain otherwise)
void conv_bwd(pic_unet* n, int li, const void* X, int ldx, const void* G, Grid3 g, void* GX,
              int epi) {
  const Layer& l = n->L[li];
  const long long P = (long long)g.B * g.H * g.W;
  gemm_wgrad(n, G, l.coutp, X, ldx, l.cinp, l.coutp, kConv3, g, l.gw, 9);
  colsum(n, G, l.coutp, l.coutp, l.gb, P);
  if (GX)
    gemm_fwd(n, G, l.coutp, l.coutp, l.wt, 9 * l.coutp, 9, kConv3, 0, g, nullptr, GX, l.cinp,
             l.cinp, epi, epi == kMask ? X : nullptr, ldx, 0);
}

// backward of a transposed layer: X its (coarse, post-ReLU) input, G the
// gradient of its output on the fine grid (stride ldg); writes the
// pre-activation gradient of the layer below (masked by relu'(X))
void up_bwd(pic_unet* n, int li, const void* X, const void* G, int ldg, Grid3 coarse, void* GX) {
  const Layer& l = n->L[li];
  const Grid3 fine{coarse.B, 2 * coarse.H, 2 * coarse.W};
  gemm_wgrad(n, G, ldg, X, l.cinp, l.cinp, l.coutp, kUpFwd, coarse, l.gw, 4);
  colsum(n, G, ldg, l.coutp, l.gb, (long long)fine.B * fine.H * fine.W);
  gemm_fwd(n, G, ldg, l.coutp, l.wt, 4 * l.coutp, 4, kUpBwd, 0, coarse, nullptr, GX, l.cinp,
           l.cinp, kMask, X, l.cinp, 0);
}

void pool_bwd(pic_unet* n, const void* gcat, int ldg, const void* gp, const void* s, int lds,
              void* out, int C, Grid3 fine) {
  const long long total = (long long)fine.B * fine.H * fine.W * C;
  if (n->prec == 16)
    k_pool_bwd_mask<bf16><<<blocks_for(total), 256, 0, n->stream>>>(
        (const bf16*)gcat, ldg, (const bf16*)gp, (const bf16*)s, lds, (bf16*)out, C, fine.B,
        fine.H, fine.W);
  else
    k_pool_bwd_mask<float><<<blocks_for(total), 256, 0, n->stream>>>(
        (const float*)gcat, ldg, (const float*)gp, (const float*)s, lds, (float*)out, C, fine.B,
        fine.H, fine.W);
}

int forward_impl(pic_unet* n, const float* x) {
  const int B = n->B, H = n->H, W = n->W;
  const int C1 = n->C[1], C2 = n->C[2], C3 = n->C[3], C4 = n->C[4];
  const Grid3 g1{B, H, W}, g2{B, H / 2, W / 2}, g3{B, H / 4, W / 4}, g4{B, H / 8, W / 8};
  const long long P1 = (long long)B * H * W;
  if (n->prec == 16) k_pack_input<bf16><<<blocks_for(P1 * 32), 256, 0, n->stream>>>(x, (bf16*)n->x0, P1);
  else k_pack_input<float><<<blocks_for(P1 * 32), 256, 0, n->stream>>>(x, (float*)n->x0, P1);
  conv_fwd(n, E1A, n->x0, 32, g1, n->e1a, C1);
  conv_fwd(n, E1B, n->e1a, C1, g1, el(n, n->cat1, C1), 2 * C1);
  pool_fwd(n, el(n, n->cat1, C1), 2 * C1, n->p1, C1, g1);
  conv_fwd(n, E2A, n->p1, C1, g2, n->e2a, C2);
  conv_fwd(n, E2B, n->e2a, C2, g2, el(n, n->cat2, C2), 2 * C2);
  pool_fwd(n, el(n, n->cat2, C2), 2 * C2, n->p2, C2, g2);
  conv_fwd(n, E3A, n->p2, C2, g3, n->e3a, C3);
  conv_fwd(n, E3B, n->e3a, C3, g3, el(n, n->cat3, C3), 2 * C3);
  pool_fwd(n, el(n, n->cat3, C3), 2 * C3, n->p3, C3, g3);
  conv_fwd(n, E4A, n->p3, C3, g4, n->e4a, C4);
  conv_fwd(n, E4B, n->e4a, C4, g4, n->e4b, C4);
  up_fwd(n, UP3, n->e4b, g4, n->cat3, 2 * C3);
  conv_fwd(n, D3A, n->cat3, 2 * C3, g3, n->d3a, C3);
  conv_fwd(n, D3B, n->d3a, C3, g3, n->d3b, C3);
  up_fwd(n, UP2, n->d3b, g3, n->cat2, 2 * C2);
  conv_fwd(n, D2A, n->cat2, 2 * C2, g2, n->d2a, C2);
  conv_fwd(n, D2B, n->d2a, C2, g2, n->d2b, C2);
  up_fwd(n, UP1, n->d2b, g2, n->cat1, 2 * C1);
  conv_fwd(n, D1A, n->cat1, 2 * C1, g1, n->d1a, C1);
  conv_fwd(n, D1B, n->d1a, C1, g1, n->d1b, C1);
  const Layer& h = n->L[HEAD];
  if (n->prec == 16) k_head_fwd<bf16><<<blocks_for(P1), 256, 0, n->stream>>>((const bf16*)n->d1b, C1, h.w, h.b, n->y, P1);
  else k_head_fwd<float><<<blocks_for(P1), 256, 0, n->stream>>>((const float*)n->d1b, C1, h.w, h.b, n->y, P1);
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

// backward from n->gy (gradient of the loss wrt the output); accumulates
// into the parameter gradients; input gradient into gx when not null
int backward_impl(pic_unet* n, float* gx) {
  const int B = n->B, H = n->H, W = n->W;
  const int C1 = n->C[1], C2 = n->C[2], C3 = n->C[3], C4 = n->C[4];
  const Grid3 g1{B, H, W}, g2{B, H / 2, W / 2}, g3{B, H / 4, W / 4}, g4{B, H / 8, W / 8};
  const long long P1 = (long long)B * H * W;
  Layer& h = n->L[HEAD];
  {
    const int lanes = std::max(1, 256 / C1);
    const int blocks = (int)std::max<long long>(1, std::min<long long>((P1 + lanes - 1) / lanes, (long long)n->sms * 8));
    if (n->prec == 16)
      k_head_bwd<bf16><<<blocks, lanes * C1, 0, n->stream>>>((const bf16*)n->d1b, C1, h.w, n->gy,
                                                            (bf16*)n->g1b, h.gw, h.gb, P1);
    else
      k_head_bwd<float><<<blocks, lanes * C1, 0, n->stream>>>((const float*)n->d1b, C1, h.w, n->gy,
                                                             (float*)n->g1b, h.gw, h.gb, P1);
  }
  conv_bwd(n, D1B, n->d1a, C1, n->g1b, g1, n->g1a, kMask);
  conv_bwd(n, D1A, n->cat1, 2 * C1, n->g1a, g1, n->gc1, kPlain);
  up_bwd(n, UP1, n->d2b, n->gc1, 2 * C1, g2, n->g2b);
  conv_bwd(n, D2B, n->d2a, C2, n->g2b, g2, n->g2a, kMask);
  conv_bwd(n, D2A, n->cat2, 2 * C2, n->g2a, g2, n->gc2, kPlain);
  up_bwd(n, UP2, n->d3b, n->gc2, 2 * C2, g3, n->g3b);
  conv_bwd(n, D3B, n->d3a, C3, n->g3b, g3, n->g3a, kMask);
  conv_bwd(n, D3A, n->cat3, 2 * C3, n->g3a, g3, n->gc3, kPlain);
  up_bwd(n, UP3, n->e4b, n->gc3, 2 * C3, g4, n->g4b);
  conv_bwd(n, E4B, n->e4a, C4, n->g4b, g4, n->g4a, kMask);
  conv_bwd(n, E4A, n->p3, C3, n->g4a, g4, n->gp3, kPlain);
  pool_bwd(n, el(n, n->gc3, C3), 2 * C3, n->gp3, el(n, n->cat3, C3), 2 * C3, n->gs3, C3, g3);
  conv_bwd(n, E3B, n->e3a, C3, n->gs3, g3, n->ge3a, kMask);
  conv_bwd(n, E3A, n->p2, C2, n->ge3a, g3, n->gp2, kPlain);
  pool_bwd(n, el(n, n->gc2, C2), 2 * C2, n->gp2, el(n, n->cat2, C2), 2 * C2, n->gs2, C2, g2);
  conv_bwd(n, E2B, n->e2a, C2, n->gs2, g2, n->ge2a, kMask);
  conv_bwd(n, E2A, n->p1, C1, n->ge2a, g2, n->gp1, kPlain);
  pool_bwd(n, el(n, n->gc1, C1), 2 * C1, n->gp1, el(n, n->cat1, C1), 2 * C1, n->gs1, C1, g1);
  conv_bwd(n, E1B, n->e1a, C1, n->gs1, g1, n->ge1a, kMask);
  conv_bwd(n, E1A, n->x0, 32, n->ge1a, g1, gx ? n->gx0 : nullptr, kPlain);
  if (gx) {
    if (n->prec == 16) k_unpack_grad<bf16><<<blocks_for(P1 * 2), 256, 0, n->stream>>>((const bf16*)n->gx0, gx, P1);
    else k_unpack_grad<float><<<blocks_for(P1 * 2), 256, 0, n->stream>>>((const float*)n->gx0, gx, P1);
  }
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

int zero_grads(pic_unet* n) {
  for (Layer& l : n->L) {
    if (cudaMemsetAsync(l.gw, 0, (size_t)l.nw * 4, n->stream) != cudaSuccess ||
        cudaMemsetAsync(l.gb, 0, (size_t)l.coutp * 4, n->stream) != cudaSuccess)
      return PIC_ECUDA;
  }
  return PIC_OK;
}

// real flat layout <-> padded device layout (host side)
void pack_layer(const Layer& l, const float* src, std::vector<float>& w, std::vector<float>& b) {
  w.assign((size_t)l.nw, 0.f);
  b.assign((size_t)l.coutp, 0.f);
  if (l.kind == kLHead) {
    for (int ci = 0; ci < l.cin; ++ci) w[ci] = src[ci];
    b[0] = src[l.cin];
    return;
  }
  const int kk = l.kind == kLConv ? 3 : 2;
  for (int ky = 0; ky < kk; ++ky)
    for (int kx = 0; kx < kk; ++kx)
      for (int ci = 0; ci < l.cin; ++ci)
        for (int co = 0; co < l.cout; ++co) {
          const int t = ky * kk + kx;
          w[((size_t)co * l.taps + t) * l.cinp + in_slot(l, ci)] =
              src[(((size_t)ky * kk + kx) * l.cin + ci) * l.cout + co];
        }
  const float* bs = src + (size_t)kk * kk * l.cin * l.cout;
  for (int co = 0; co < l.cout; ++co) b[co] = bs[co];
}

void unpack_layer(const Layer& l, const std::vector<float>& w, const std::vector<float>& b,
                  float* dst) {
  if (l.kind == kLHead) {
    for (int ci = 0; ci < l.cin; ++ci) dst[ci] = w[ci];
    dst[l.cin] = b[0];
    return;
  }
  const int kk = l.kind == kLConv ? 3 : 2;
  for (int ky = 0; ky < kk; ++ky)
    for (int kx = 0; kx < kk; ++kx)
      for (int ci = 0; ci < l.cin; ++ci)
        for (int co = 0; co < l.cout; ++co)
          dst[(((size_t)ky * kk + kx) * l.cin + ci) * l.cout + co] =
              w[((size_t)co * l.taps + ky * kk + kx) * l.cinp + in_slot(l, ci)];
  float* bd = dst + (size_t)kk * kk * l.cin * l.cout;
  for (int co = 0; co < l.cout; ++co) bd[co] = b[co];
}

long long layer_params(const Layer& l) { return (long long)l.cout * l.taps * l.cin + l.cout; }

int copy_out(pic_unet* n, bool grads, float* host) {
  if (const int st = tc_status(n)) return st;
  std::vector<float> w, b;
  long long o = 0;
  for (Layer& l : n->L) {
    w.resize((size_t)l.nw);
    b.resize((size_t)l.coutp);
    if (cudaMemcpyAsync(w.data(), grads ? l.gw : l.w, (size_t)l.nw * 4, cudaMemcpyDeviceToHost,
                        n->stream) != cudaSuccess ||
        cudaMemcpyAsync(b.data(), grads ? l.gb : l.b, (size_t)l.coutp * 4, cudaMemcpyDeviceToHost,
                        n->stream) != cudaSuccess ||
        cudaStreamSynchronize(n->stream) != cudaSuccess)
      return PIC_ECUDA;
    unpack_layer(l, w, b, host + o);
    o += layer_params(l);
  }
  return PIC_OK;
}

}  // namespace

// ------------------------------------------------------------------ ABI

extern "C" {

int pic_unet_create(int base_channels, int H, int W, int batch, int precision, void* cuda_stream,
                    const pic_allocator* alloc, pic_unet** out) {
  if (!out) return PIC_EINVAL;
  *out = nullptr;
  if (base_channels < 1 || base_channels > 32 || batch < 1 || H < 8 || W < 8 || H % 8 ||
      W % 8 || (precision != 16 && precision != 32))
    return PIC_EINVAL;
  if ((long long)batch * H * W > (1LL << 28)) return PIC_EINVAL;
  pic_unet* n = new (std::nothrow) pic_unet();
  if (!n) return PIC_ENOMEM;
  n->c = base_channels; n->H = H; n->W = W; n->B = batch; n->prec = precision;
  n->stream = (cudaStream_t)cuda_stream;
  n->has_alloc = alloc && alloc->alloc && alloc->free;
  if (n->has_alloc) n->alloc = *alloc;
  n->es = precision == 16 ? 2 : 4;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete n;
    return PIC_ECUDA;
  }
  make_layers(n);
  for (int k = 1; k <= 4; ++k) n->C[k] = pad32(base_channels << (k - 1));
  bool ok = true;
  for (Layer& l : n->L) {
    const size_t wb = (size_t)l.nw * 4, bb = (size_t)l.coutp * 4;
    l.w = (float*)u_alloc(n, wb); l.gw = (float*)u_alloc(n, wb);
    l.mw = (float*)u_alloc(n, wb); l.vw = (float*)u_alloc(n, wb);
    l.b = (float*)u_alloc(n, bb); l.gb = (float*)u_alloc(n, bb);
    l.mb = (float*)u_alloc(n, bb); l.vb = (float*)u_alloc(n, bb);
    l.wc = u_alloc(n, (size_t)l.nw * n->es);
    l.wt = u_alloc(n, (size_t)l.nw * n->es);
    ok = ok && l.w && l.gw && l.mw && l.vw && l.b && l.gb && l.mb && l.vb && l.wc && l.wt;
    if (ok) {
      for (float* p : {l.w, l.gw, l.mw, l.vw})
        ok = ok && cudaMemsetAsync(p, 0, wb, n->stream) == cudaSuccess;
      for (float* p : {l.b, l.gb, l.mb, l.vb})
        ok = ok && cudaMemsetAsync(p, 0, bb, n->stream) == cudaSuccess;
    }
  }
  const long long P1 = (long long)batch * H * W, P2 = P1 / 4, P3 = P1 / 16, P4 = P1 / 64;
  const int C1 = n->C[1], C2 = n->C[2], C3 = n->C[3], C4 = n->C[4];
  auto act = [&](long long elems) { return u_alloc(n, (size_t)elems * n->es); };
  n->x0 = act(P1 * 32);
  n->e1a = act(P1 * C1); n->cat1 = act(P1 * 2 * C1); n->p1 = act(P2 * C1);
  n->e2a = act(P2 * C2); n->cat2 = act(P2 * 2 * C2); n->p2 = act(P3 * C2);
  n->e3a = act(P3 * C3); n->cat3 = act(P3 * 2 * C3); n->p3 = act(P4 * C3);
  n->e4a = act(P4 * C4); n->e4b = act(P4 * C4);
  n->d3a = act(P3 * C3); n->d3b = act(P3 * C3); n->d2a = act(P2 * C2); n->d2b = act(P2 * C2);
  n->d1a = act(P1 * C1); n->d1b = act(P1 * C1);
  n->g1b = act(P1 * C1); n->g1a = act(P1 * C1); n->gc1 = act(P1 * 2 * C1);
  n->g2b = act(P2 * C2); n->g2a = act(P2 * C2); n->gc2 = act(P2 * 2 * C2);
  n->g3b = act(P3 * C3); n->g3a = act(P3 * C3); n->gc3 = act(P3 * 2 * C3);
  n->g4b = act(P4 * C4); n->g4a = act(P4 * C4); n->gp3 = act(P4 * C3);
  n->gs3 = act(P3 * C3); n->ge3a = act(P3 * C3); n->gp2 = act(P3 * C2);
  n->gs2 = act(P2 * C2); n->ge2a = act(P2 * C2); n->gp1 = act(P2 * C1);
  n->gs1 = act(P1 * C1); n->ge1a = act(P1 * C1); n->gx0 = act(P1 * 32);
  n->y = (float*)u_alloc(n, (size_t)P1 * 4);
  n->gy = (float*)u_alloc(n, (size_t)P1 * 4);
  n->loss = (float*)u_alloc(n, 16);
  n->dev_err = (int*)u_alloc(n, 16);
  for (void* p : {n->x0, n->e1a, n->cat1, n->p1, n->e2a, n->cat2, n->p2, n->e3a, n->cat3, n->p3,
                  n->e4a, n->e4b, n->d3a, n->d3b, n->d2a, n->d2b, n->d1a, n->d1b, n->g1b, n->g1a,
                  n->gc1, n->g2b, n->g2a, n->gc2, n->g3b, n->g3a, n->gc3, n->g4b, n->g4a, n->gp3,
                  n->gs3, n->ge3a, n->gp2, n->gs2, n->ge2a, n->gp1, n->gs1, n->ge1a, n->gx0,
                  (void*)n->y, (void*)n->gy, (void*)n->loss, (void*)n->dev_err})
    ok = ok && p;
  if (ok) ok = cudaMemsetAsync(n->dev_err, 0, 16, n->stream) == cudaSuccess;
  // the tensor-core GEMMs stage four operand tiles in dynamic shared memory
  if (ok) ok = tc_prepare() == PIC_OK;
  // the concatenation buffers' padded channels must read as zero
  if (ok) {
    ok = cudaMemsetAsync(n->cat1, 0, (size_t)P1 * 2 * C1 * n->es, n->stream) == cudaSuccess &&
         cudaMemsetAsync(n->cat2, 0, (size_t)P2 * 2 * C2 * n->es, n->stream) == cudaSuccess &&
         cudaMemsetAsync(n->cat3, 0, (size_t)P3 * 2 * C3 * n->es, n->stream) == cudaSuccess &&
         cudaStreamSynchronize(n->stream) == cudaSuccess;
  }
  if (!ok) {
    pic_unet_free(n);
    return PIC_ENOMEM;
  }
  *out = n;
  return PIC_OK;
}

void pic_unet_free(pic_unet* n) {
  if (!n) return;
  cudaStreamSynchronize(n->stream);
  for (void* p : n->owned) {
    if (n->has_alloc) n->alloc.free(p, (void*)n->stream, n->alloc.ctx);
    else cudaFree(p);
  }
  delete n;
}

int64_t pic_unet_param_count(const pic_unet* n) { return n ? n->n_params : -1; }

int pic_unet_set_params(pic_unet* n, const float* params) {
  if (!n || !params) return PIC_EINVAL;
  std::vector<float> w, b;
  long long o = 0;
  for (Layer& l : n->L) {
    pack_layer(l, params + o, w, b);
    o += layer_params(l);
    if (cudaMemcpyAsync(l.w, w.data(), (size_t)l.nw * 4, cudaMemcpyHostToDevice, n->stream) != cudaSuccess ||
        cudaMemcpyAsync(l.b, b.data(), (size_t)l.coutp * 4, cudaMemcpyHostToDevice, n->stream) != cudaSuccess ||
        cudaStreamSynchronize(n->stream) != cudaSuccess)
      return PIC_ECUDA;
    cudaMemsetAsync(l.mw, 0, (size_t)l.nw * 4, n->stream);
    cudaMemsetAsync(l.vw, 0, (size_t)l.nw * 4, n->stream);
    cudaMemsetAsync(l.mb, 0, (size_t)l.coutp * 4, n->stream);
    cudaMemsetAsync(l.vb, 0, (size_t)l.coutp * 4, n->stream);
  }
  const int rc = derive_all(n);
  return rc ? rc : (cudaStreamSynchronize(n->stream) == cudaSuccess ? PIC_OK : PIC_ECUDA);
}

int pic_unet_set_tensor_path(pic_unet* n, int mode) {
  if (!n || mode < -1 || mode > 1) return PIC_EINVAL;
  n->tc_mode = mode;
  return PIC_OK;
}

int pic_unet_get_params(pic_unet* n, float* params) {
  if (!n || !params) return PIC_EINVAL;
  return copy_out(n, false, params);
}

int pic_unet_get_grads(pic_unet* n, float* grads) {
  if (!n || !grads) return PIC_EINVAL;
  return copy_out(n, true, grads);
}

int pic_unet_forward(pic_unet* n, const float* x, float* y) {
  if (!n || !x) return PIC_EINVAL;
  int rc = forward_impl(n, x);
  if (!rc && y &&
      cudaMemcpyAsync(y, n->y, (size_t)n->B * n->H * n->W * 4, cudaMemcpyDeviceToDevice,
                      n->stream) != cudaSuccess)
    rc = PIC_ECUDA;
  return rc;
}

int pic_unet_backward(pic_unet* n, const float* gy, float* gx) {
  if (!n || !gy) return PIC_EINVAL;
  if (cudaMemcpyAsync(n->gy, gy, (size_t)n->B * n->H * n->W * 4, cudaMemcpyDeviceToDevice,
                      n->stream) != cudaSuccess)
    return PIC_ECUDA;
  int rc = zero_grads(n);
  return rc ? rc : backward_impl(n, gx);
}

int pic_unet_train_step(pic_unet* n, const float* x, const float* target, float lr, float beta1,
                        float beta2, float eps, int64_t t, float* loss) {
  if (!n || !x || !target || t < 1) return PIC_EINVAL;
  const long long P1 = (long long)n->B * n->H * n->W;
  int rc = forward_impl(n, x);
  if (rc) return rc;
  if (cudaMemsetAsync(n->loss, 0, 4, n->stream) != cudaSuccess) return PIC_ECUDA;
  k_loss<<<blocks_for(P1), 256, 0, n->stream>>>(n->y, target, n->gy, n->loss, P1);
  rc = zero_grads(n);
  if (!rc) rc = backward_impl(n, nullptr);
  if (rc) return rc;
  const float c1 = 1.f / (1.f - std::pow(beta1, (float)t));
  const float c2 = 1.f / (1.f - std::pow(beta2, (float)t));
  for (Layer& l : n->L) {
    k_adam<<<blocks_for(l.nw), 256, 0, n->stream>>>(l.w, l.gw, l.mw, l.vw, l.nw, lr, beta1, beta2,
                                                   eps, c1, c2);
    k_adam<<<1, 256, 0, n->stream>>>(l.b, l.gb, l.mb, l.vb, l.coutp, lr, beta1, beta2, eps, c1, c2);
  }
  rc = derive_all(n);
  if (!rc && loss &&
      cudaMemcpyAsync(loss, n->loss, 4, cudaMemcpyDeviceToDevice, n->stream) != cudaSuccess)
    rc = PIC_ECUDA;
  return rc;
}

}  // extern "C"

// ------------------------------------------- the simulation's warm start

namespace pic {
namespace {

// node (i, j) of simulation s <-> pixel (s, i - 1, j), i = 1..nr, j < nz

// network input of every simulation: channel 0 the last deposit's charge
// (C; fixed-point counts times the simulation's unit, or FP64 charges) over
// rho_scale, channel 1 phi_rho (V) over phi_scale
__global__ void k_ws_input(FieldTables T, const unsigned long long* __restrict__ cnt,
                           const double* __restrict__ units, const double* __restrict__ rhs,
                           float* __restrict__ x, float inv_rho, float inv_phi) {
  const int nr = T.nr, nz = T.nz, M1 = nz + 1;
  const long long per = (long long)nr * nz, total = per * T.nsim;
  const size_t nn = (size_t)(nr + 1) * M1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i / per);
    const long long q = i % per;
    const int y = (int)(q / nz), xx = (int)(q % nz);
    const size_t o = (size_t)s * nn + (size_t)(y + 1) * M1 + xx;
    const double b = cnt ? (double)cnt[o] * units[s] : rhs[o];
    const float2 ph = T.phir[o];
    x[2 * i] = (float)b * inv_rho;
    x[2 * i + 1] = (ph.x + ph.y) * inv_phi;
  }
}

// phi_rho += dphi_scale * y on the interior lines; node column nz takes the
// prediction of pixel column nz - 1
__global__ void k_ws_apply(FieldTables T, const float* __restrict__ y, float dphi) {
  const int nr = T.nr, nz = T.nz, M1 = nz + 1;
  const long long per = (long long)(nr - 1) * M1, total = per * T.nsim;
  const size_t nn = (size_t)(nr + 1) * M1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i / per);
    const long long q = i % per;
    const int ii = (int)(q / M1) + 1, j = (int)(q % M1);
    const size_t o = (size_t)s * nn + (size_t)ii * M1 + j;
    const float d = dphi * y[((long long)s * nr + (ii - 1)) * nz + (j < nz ? j : nz - 1)];
    float2 p = T.phir[o];
    // double-float p + d
    const float sum = p.x + d;
    const float v = sum - p.x;
    const float err = (p.x - (sum - v)) + (d - v);
    const float lo = p.y + err;
    const float hi = sum + lo;
    T.phir[o] = make_float2(hi, lo - (hi - sum));
  }
}

// images of the field state: rho (C) and phi_rho (V), pixel layout
__global__ void k_field_images(FieldTables T, const unsigned long long* __restrict__ cnt,
                               const double* __restrict__ units, const double* __restrict__ rhs,
                               float* __restrict__ rho, float* __restrict__ phi) {
  const int nr = T.nr, nz = T.nz, M1 = nz + 1;
  const long long per = (long long)nr * nz, total = per * T.nsim;
  const size_t nn = (size_t)(nr + 1) * M1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i / per);
    const long long q = i % per;
    const size_t o = (size_t)s * nn + (size_t)(q / nz + 1) * M1 + (q % nz);
    if (rho) rho[i] = (float)(cnt ? (double)cnt[o] * units[s] : rhs[o]);
    if (phi) phi[i] = T.phir[o].x + T.phir[o].y;
  }
}

}  // namespace

// the learned initial guess: input images, net forward, phi_rho update
int warm_start_learned(pic_unet* n, const FieldTables& T, const unsigned long long* cnt,
                       const double* units, const double* rhs, float* xbuf, float rho_scale,
                       float phi_scale, float dphi_scale, cudaStream_t stream) {
  const long long px = (long long)T.nsim * T.nr * T.nz;
  const int blocks = (int)std::min<long long>((px + 255) / 256, 152 * 16);
  k_ws_input<<<blocks, 256, 0, stream>>>(T, cnt, units, rhs, xbuf, 1.f / rho_scale,
                                         1.f / phi_scale);
  cudaStream_t keep = n->stream;
  n->stream = stream;
  const int rc = forward_impl(n, xbuf);
  n->stream = keep;
  if (rc) return rc;
  const long long nodes = (long long)T.nsim * (T.nr - 1) * (T.nz + 1);
  k_ws_apply<<<(int)std::min<long long>((nodes + 255) / 256, 152 * 16), 256, 0, stream>>>(
      T, n->y, dphi_scale);
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

int field_images(const FieldTables& T, const unsigned long long* cnt, const double* units,
                 const double* rhs, float* rho, float* phi, cudaStream_t stream) {
  const long long px = (long long)T.nsim * T.nr * T.nz;
  k_field_images<<<(int)std::min<long long>((px + 255) / 256, 152 * 16), 256, 0, stream>>>(
      T, cnt, units, rhs, rho, phi);
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

bool unet_fits(const pic_unet* n, int nsim, int nr, int nz) {
  return n->B == nsim && n->H == nr && n->W == nz;
}
int unet_kernels_per_forward(const pic_unet* n) {
  // pack, 14 convolutions, 3 x 4 transposed sub-grids, 3 pools, head
  (void)n;
  return 1 + 14 + 12 + 3 + 1;
}

}  // namespace pic
