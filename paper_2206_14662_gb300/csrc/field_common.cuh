// field_common.cuh -- device pieces of the field solve (field_solve.cu):
// double-float arithmetic, the charge pass of one node, the node field, the
// z-matrix products and row terms of the residual, one radix-2 butterfly
// and the DCT-I output of a line pair, the Thomas steps and the stopping
// test.  Internal to the library.
#pragma once

#include <type_traits>

#include "pic_internal.cuh"

namespace pic {

// ------------------------------------------------------- double-float
// Error-free transformations (Knuth's two-sum, Dekker's product via FMA)
// and the usual double-float add / multiply built on them.

__device__ __forceinline__ float2 qts(float a, float b) {   // |a| >= |b|
  const float s = a + b;
  return make_float2(s, b - (s - a));
}
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = a + b;
  const float v = s - a;
  return make_float2(s, (a - (s - v)) + (b - v));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float2 s = two_sum(a.x, b.x);
  return qts(s.x, s.y + a.y + b.y);
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  return qts(p, e);
}
__device__ __forceinline__ float df_diff(float2 a, float2 b) {   // a - b to float
  return (a.x - b.x) + (a.y - b.y);
}

// ---------------------------------------------------------------- prep

// the deposit's charge source of a solve
struct ChargeIn {
  const double* rhs;                  // FP64 charges (C), or
  const unsigned long long* cnt;      // fixed-point counts
  float2 unit2;                       // count -> b' (double-float), or
  const float2* units;                //   per simulation (batch)
  double unit64;                      // charge -> b'
  unsigned long long* clear;          // buffer zeroed on the way, or null
};

// b' per node in double-float, the sweep-0 input, and the norms of the
// interior right-hand side and of the lifted one; clears the next deposit
// buffer.  FIX: b' = count * unit2 (fixed-point counts); else b' = rhs *
// unit64 (FP64 charges).
// b' at node o (global index) of simulation sim, node (i, j): stored in T.b2
// on the interior lines, with the squares of it and of the lifted value
// added to nb, nl; the node of `clear` is zeroed
template <bool FIX>
__device__ __forceinline__ float2 prep_node(const ChargeIn& in, const FieldTables& T, int sim,
                                            size_t o, int i, int j, float& nb, float& nl) {
  const int nr = T.nr;
  float2 b;
  if (FIX) {
    const float2 unit2 = in.units ? in.units[sim] : in.unit2;
    const unsigned long long c = in.cnt[o];
    const float hi = __ull2float_rn(c);
    const long long rem = (long long)(c - __float2ull_rn(hi));
    b = df_mul(qts(hi, __ll2float_rn(rem)), unit2);
  } else {
    const double x = in.rhs[o] * in.unit64;
    const float hi = (float)x;
    b = make_float2(hi, (float)(x - (double)hi));
  }
  if (in.clear) in.clear[o] = 0ull;
  if (i > 0 && i < nr) {
    T.b2[o] = b;
    // the wall potentials moved to the right-hand side: -K_r(1,0) V_in
    // and -K_r(nr-1,nr) V_out times the row sum of M_z
    const float zsum = (j == 0 || j == T.M) ? 0.5f * T.hz32 : T.hz32;
    const double* vac = T.phi_vac + (size_t)sim * (nr + 1);
    float lift = 0.f;
    if (i == 1) lift -= T.kr_o[0].x * (float)vac[0] * zsum;
    if (i == nr - 1) lift -= T.kr_o[nr - 1].x * (float)vac[nr] * zsum;
    nb = b.x * b.x;
    nl = (b.x + lift) * (b.x + lift);
  }
  return b;
}

// ------------------------------------------------------ node field, residual

// E = E_vac - grad phi_rho at node (i, j), o = i (M + 1) + j in one
// simulation's grid: central differences, one-sided second order on the
// boundary lines (phi_rho is zero on the walls).  FP32 particle path: the
// differences of hi and lo pairs in float; FP64: of hi + lo in double.
template <typename Real>
__device__ __forceinline__ typename Vec2<Real>::type node_field(
    const FieldTables& T, const float2* ph, const float* evac32, const double* evac64, size_t o,
    int i, int j) {
  const int nr = T.nr, M = T.M, M1 = M + 1;
  typename Vec2<Real>::type e;
  if constexpr (std::is_same<Real, float>::value) {
    float dr, dz;
    const float inv2hr = T.inv2hr, inv2hz = T.inv2hz;
    if (i == 0) {
      const float2 a = ph[o], b = ph[o + M1], c = ph[o + 2 * M1];
      dr = (-3.f * a.x + 4.f * b.x - c.x + (-3.f * a.y + 4.f * b.y - c.y)) * inv2hr;
    } else if (i == nr) {
      const float2 a = ph[o], b = ph[o - M1], c = ph[o - 2 * M1];
      dr = (3.f * a.x - 4.f * b.x + c.x + (3.f * a.y - 4.f * b.y + c.y)) * inv2hr;
    } else {
      dr = df_diff(ph[o + M1], ph[o - M1]) * inv2hr;
    }
    if (j == 0) {
      const float2 a = ph[o], b = ph[o + 1], c = ph[o + 2];
      dz = (-3.f * a.x + 4.f * b.x - c.x + (-3.f * a.y + 4.f * b.y - c.y)) * inv2hz;
    } else if (j == M) {
      const float2 a = ph[o], b = ph[o - 1], c = ph[o - 2];
      dz = (3.f * a.x - 4.f * b.x + c.x + (3.f * a.y - 4.f * b.y + c.y)) * inv2hz;
    } else {
      dz = df_diff(ph[o + 1], ph[o - 1]) * inv2hz;
    }
    e.x = evac32[i] - dr;
    e.y = -dz;
  } else {
    auto p = [&](size_t q) {
      const float2 v = ph[q];
      return (double)v.x + (double)v.y;
    };
    const double i2r = T.inv2hr_d, i2z = T.inv2hz_d;
    double ddr, ddz;
    if (i == 0) ddr = (-3.0 * p(o) + 4.0 * p(o + M1) - p(o + 2 * M1)) * i2r;
    else if (i == nr) ddr = (3.0 * p(o) - 4.0 * p(o - M1) + p(o - 2 * M1)) * i2r;
    else ddr = (p(o + M1) - p(o - M1)) * i2r;
    if (j == 0) ddz = (-3.0 * p(o) + 4.0 * p(o + 1) - p(o + 2)) * i2z;
    else if (j == M) ddz = (3.0 * p(o) - 4.0 * p(o - 1) + p(o - 2)) * i2z;
    else ddz = (p(o + 1) - p(o - 1)) * i2z;
    e.x = evac64[i] - ddr;
    e.y = -ddz;
  }
  return e;
}

// M_z phi and K_z phi of the r-line holding node q (column j), double-float
__device__ __forceinline__ void node_mzkz(const FieldTables& T, const float2* ph, size_t q, int j,
                                          float2& mz, float2& kz) {
  const int M = T.M;
  const bool end = (j == 0 || j == M);
  const float2 mzd = end ? T.mzd_end : T.mzd_in, kzd = end ? T.kzd_end : T.kzd_in;
  const float2 c = ph[q];
  float2 nb = make_float2(0.f, 0.f);
  if (j > 0) nb = ph[q - 1];
  if (j < M) nb = df_add(nb, ph[q + 1]);
  mz = df_add(df_mul(mzd, c), df_mul(T.mzo, nb));
  kz = df_add(df_mul(kzd, c), df_mul(T.kzo, nb));
}

// the contribution of r-line i + di to (A' phi) at an interior node of line
// i: K_r(i, i+di) M_z phi + M_r(i, i+di) K_z phi
__device__ __forceinline__ float2 row_term(const FieldTables& T, int i, int di, float2 mz,
                                           float2 kz) {
  float2 kr, mr;
  if (di == 0) { kr = T.kr_d[i]; mr = T.mr_d[i]; }
  else if (di < 0) { kr = T.kr_o[i - 1]; mr = T.mr_o[i - 1]; }
  else { kr = T.kr_o[i]; mr = T.mr_o[i]; }
  return df_add(df_mul(kr, mz), df_mul(mr, kz));
}

// ---------------------------------------------------------------- DCT-I

// butterfly t (< N / 2) of stage s (1..log2 N) of an in-place radix-2 FFT
// on bit-reversed input; tw[m] = exp(-2 pi i m / N)
__device__ __forceinline__ void fft_butterfly(float2* sh, const float2* tw, int N, int s, int t) {
  const int half = 1 << (s - 1), stride = N >> s;
  const int pos = t & (half - 1);
  const int i0 = ((t >> (s - 1)) << s) + pos, i1 = i0 + half;
  const float2 w = tw[pos * stride];
  const float2 a = sh[i0], b = sh[i1];
  const float2 bw = make_float2(b.x * w.x - b.y * w.y, b.x * w.y + b.y * w.x);
  sh[i0] = make_float2(a.x + bw.x, a.y + bw.y);
  sh[i1] = make_float2(a.x - bw.x, a.y - bw.y);
}

// DCT-I outputs k of two lines x (real part) and y (imaginary part) from
// bin k of the FFT of their even extension and the lines' end values
__device__ __forceinline__ float2 dct_out(float2 C, int k, float x0, float xM, float y0,
                                          float yM) {
  const float sg = (k & 1) ? -1.f : 1.f;
  return make_float2(0.5f * (C.x + x0 + sg * xM), 0.5f * (C.y + y0 + sg * yM));
}

// ------------------------------------------------------------- tridiag

// one step of the pre-factored Thomas recurrence: forward (right-hand side
// b, sub-diagonal a, 1 / pivot d) and backward (super-diagonal / pivot c)
__device__ __forceinline__ float thomas_fwd(float b, float a, float d, float y) {
  return (b - a * y) * d;
}
__device__ __forceinline__ float thomas_bwd(float b, float c, float x) { return b - c * x; }

// ------------------------------------------------------------ stopping test

// ||r|| / ||b'_lifted|| (rel) and ||r|| / ||b'_I|| (strict) from the three
// squared norms
__device__ __forceinline__ void solve_norms(double r2, double b2, double bl2, double& rel,
                                            double& strict) {
  strict = b2 > 0.0 ? sqrt(r2 / b2) : (r2 > 0.0 ? 1.0 : 0.0);
  rel = bl2 > 0.0 ? sqrt(r2 / bl2) : strict;
}

// records the test of a residual pass (sweep -1: the warm start's initial
// residual) in st; returns whether the solve ends here, latching
// PIC_ENOCONV when the last sweep missed rtol
__device__ __forceinline__ bool solve_record(DevState* st, const FieldTables& T, double rel,
                                             double strict, int sweep, bool last) {
  st->relres_last = rel;
  st->relres_strict = strict;
  st->poisson_iters = sweep + 1;
  if (sweep < 0) st->relres_init = rel;
  else if (!T.warm) st->relres_init = -1.0;
  const bool done = rel <= T.rtol || last;
  if (done) {
    st->solve_done = 1;
    if (!(rel <= T.rtol)) atomicCAS(&st->err, 0, PIC_ENOCONV);
  }
  return done;
}

}  // namespace pic
