// particle_step.cu -- the fused particle kernel of one PIC step and the
// small kernels around it (load, export, child-uid assignment, kinetic
// energy).  Method: arXiv 2206.14662, Sec. II.A.
//
// One pass over the particle store per step; per particle:
//   gather   bilinear E from the node grid (FP32 or FP64 copy of -grad phi),
//            analytic B (uniform, or the mirror field of A_theta = r Bz / 2)
//   push     Boris half kick / rotation / half kick in the local (r,theta,z)
//            basis, straight move in the local Cartesian frame, rotation of
//            (vr, vtheta) into the basis at the new position
//   absorb   perfectly absorbing walls, first crossing of the (r,z) segment
//   collide  null-collision Monte Carlo: one Philox4x32-10 call per particle
//            (candidate, type, scattering angle, azimuth); ionisation takes
//            a second call (energy share, secondary angles) and appends a
//            child whose uid is fixed after the kernel by parent-uid rank
//   deposit  b_i += q w Lambda_i: the block's particles accumulate the hat
//            weights into a shared-memory tile spanning their node bounding
//            box, flushed to the FP64 grid with one atomic per touched node;
//            blocks whose particles are spread too wide deposit directly.
//
// Memory traffic per particle-step: 28 B read (cell, two offsets, three
// velocity components, uid) and 24 B written (all but the uid) in FP32.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <type_traits>

#include "pic_internal.cuh"

namespace pic {

constexpr int kThreads = 128;
constexpr int kPPT = 4;                 // particles per thread per chunk
constexpr int kChunk = kThreads * kPPT;

// Shared-memory deposit tile.  The FP32 path accumulates hat weights as
// unsigned fixed-point numbers (native integer shared atomics, sums that do
// not depend on the order of the adds): a chunk holds at most 1024 (>=
// kChunk) particles of weight <= 1 per node, so kFix = floor((2^32 - 1) /
// 1024) cannot overflow even when the private copies are added; the
// rounding is 2^-23 of a particle's charge per contribution.  The FP64 path accumulates
// doubles.  cap is the tile's size in words (FP32: four copies of 1024).
template <typename Real> struct TileT { using type = unsigned; static constexpr int cap = 4096; };
template <> struct TileT<double> { using type = double; static constexpr int cap = 2048; };
static_assert(kChunk <= 1024, "fixed-point tile sums");
constexpr float kFix = (float)(4294967295u / 1024);   // 4194303
static_assert((double)kFix == kFixUnit, "fixed-point unit shared with the field solve");

__device__ __forceinline__ float d_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double d_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float d_floor(float x) { return floorf(x); }
__device__ __forceinline__ double d_floor(double x) { return floor(x); }
__device__ __forceinline__ void d_sincospi(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void d_sincospi(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ float d_tan(float x) { return tanf(x); }
__device__ __forceinline__ double d_tan(double x) { return tan(x); }
__device__ __forceinline__ float d_atan(float x) { return atanf(x); }
__device__ __forceinline__ double d_atan(double x) { return atan(x); }

__device__ __forceinline__ void set_error(DevState* st, int code) {
  atomicCAS(&st->err, 0, code);
}

// Direction after scattering through chi about the unit vector (vr,vt,vz):
// mu = cos chi from the inverse CDF of the pdf ~ (1 - xi mu)^-2,
// mu = 1 - 2u(1 - xi)/(1 + xi(1 - 2u)); azimuth 2 pi u_phi measured from
// e1 = (v x zhat)/|v x zhat| (rhat instead of zhat within 1e-6 of the
// axis), e2 = v x e1.
template <typename Real>
__device__ __forceinline__ void scatter_dir(Real vr, Real vt, Real vz,
                                            Real u_chi, Real u_phi, Real xi,
                                            Real& dr, Real& dt, Real& dz) {
  const Real one = 1;
  const Real mu = one - 2 * u_chi * (one - xi) / (one + xi * (one - 2 * u_chi));
  const Real sn = d_sqrt(fmax(Real(0), one - mu * mu));
  Real sp, cp;
  d_sincospi(2 * u_phi, &sp, &cp);
  Real e1r = vt, e1t = -vr, e1z = 0;
  Real n1 = d_sqrt(vr * vr + vt * vt);
  if (n1 < Real(1e-6)) {
    e1r = 0; e1t = vz; e1z = -vt;
    n1 = d_sqrt(vz * vz + vt * vt);
  }
  const Real in1 = one / n1;
  e1r *= in1; e1t *= in1; e1z *= in1;
  const Real e2r = vt * e1z - vz * e1t;
  const Real e2t = vz * e1r - vr * e1z;
  const Real e2z = vr * e1t - vt * e1r;
  dr = mu * vr + sn * (cp * e1r + sp * e2r);
  dt = mu * vt + sn * (cp * e1t + sp * e2t);
  dz = mu * vz + sn * (cp * e1z + sp * e2z);
}

// per-block tallies in shared memory (raw: counts, weights in macro units,
// energies per macro-electron; scaled by the weight at the flush)
struct BlockTally {
  double v[kTallyCount];
};

template <typename Real>
struct Dep {
  int ir, iz;   // ir < 0: nothing to deposit
  Real fr, fz;
};

// Deposit grid: the FP32 path accumulates unsigned 64-bit fixed-point hat
// weights (kFix per particle charge; integer atomics, sums independent of
// the order of the adds; 3e8 particles on one node stay below 2^63); the
// FP64 path accumulates the charge q w Lambda in doubles.
struct DepGrid {
  double* rhs;                  // FP64 path
  unsigned long long* cnt;      // FP32 path
  int nzp;
  double qw;
};

// FP32: the fixed-point count of a corner is rn((w_r kFix) w_z), the same
// rounding sequence as the shared-tile path of deposit_chunk, so a node's
// sum does not depend on which path a particle takes
__device__ __forceinline__ void deposit_global(const DepGrid& g, int ir, int iz, float fr,
                                               float fz) {
  const int n00 = ir * g.nzp + iz;
  const float ra = (1.f - fr) * kFix, rb = fr * kFix, za = 1.f - fz;
  atomicAdd(g.cnt + n00, (unsigned long long)__float2uint_rn(ra * za));
  atomicAdd(g.cnt + n00 + g.nzp, (unsigned long long)__float2uint_rn(rb * za));
  atomicAdd(g.cnt + n00 + 1, (unsigned long long)__float2uint_rn(ra * fz));
  atomicAdd(g.cnt + n00 + g.nzp + 1, (unsigned long long)__float2uint_rn(rb * fz));
}
__device__ __forceinline__ void deposit_global(const DepGrid& g, int ir, int iz, double fr,
                                               double fz) {
  const int n00 = ir * g.nzp + iz;
  atomicAdd(g.rhs + n00, g.qw * ((1.0 - fr) * (1.0 - fz)));
  atomicAdd(g.rhs + n00 + g.nzp, g.qw * (fr * (1.0 - fz)));
  atomicAdd(g.rhs + n00 + 1, g.qw * ((1.0 - fr) * fz));
  atomicAdd(g.rhs + n00 + g.nzp + 1, g.qw * (fr * fz));
}

// quotient and reciprocal square root: hardware approximations (2 ulp) in
// the FP32 path, IEEE operations in the FP64 path
__device__ __forceinline__ float q_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double q_div(double a, double b) { return a / b; }
__device__ __forceinline__ float q_rsqrt(float a) { return rsqrtf(a); }
// a b + c with one rounding
__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double mad(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double q_rsqrt(double a) { return 1.0 / sqrt(a); }

// Weighted B-spline field of degree N (the step's spline mode): the span
// of a particle is its cell and the local coordinate its offset, so the N
// + 1 non-zero B-splines per direction come from the triangular Cox-de
// Boor scheme at the offset (distances in cells, denominators j).
template <typename Real, int N>
__device__ __forceinline__ void spl_span(Real u, Real* B) {
  B[0] = Real(1);
#pragma unroll
  for (int j = 1; j <= N; ++j) {
    Real saved = Real(0);
#pragma unroll
    for (int r = 0; r < j; ++r) {
      const Real tmp = B[r] * (Real(1) / Real(j));
      B[r] = saved + (Real(r + 1) - u) * tmp;
      saved = (u + Real(j - r - 1)) * tmp;
    }
    B[j] = saved;
  }
}

// values and derivatives per cell width (d/du) of the span's functions
template <typename Real, int N>
__device__ __forceinline__ void spl_span_d(Real u, Real* B, Real* dB) {
  Real M[N > 0 ? N : 1];
  spl_span<Real, N>(u, B);
  spl_span<Real, N - 1>(u, M);
#pragma unroll
  for (int r = 0; r <= N; ++r) dB[r] = (r >= 1 ? M[r - 1] : Real(0)) - (r <= N - 1 ? M[r] : Real(0));
}

// R-function conjunction x + y - sqrt(x^2 + y^2) and its gradient
template <typename Real>
__device__ __forceinline__ void r_conj(Real x, Real x0, Real x1, Real y, Real y0, Real y1, Real& v,
                                       Real& g0, Real& g1) {
  const Real q = d_sqrt(x * x + y * y), qs = q > Real(0) ? q : Real(1);
  v = x + y - q;
  g0 = x0 + y0 - (x * x0 + y * y0) / qs;
  g1 = x1 + y1 - (x * x1 + y * y1) / qs;
}

// weight w of the spline field and its gradient, and the gradient of the
// lift, at (r, z): the walls' w = (r - r_in)(r_out - r)/(r_out - r_in) and
// the linear lift; with the trap's ellipse the conjunction of that w and
// w_e = s (x^2 + y^2 - 1) (x, y the normalised offsets), and the lift
// V_in + dV t, t = (r - r_in)/(r - r_in + w_o), w_o the conjunction of
// (r_out - r) and w_e
template <typename Real>
__device__ __forceinline__ void spl_wl(const PushParams<Real>& P, Real r, Real z, Real& w, Real& wr,
                                       Real& wz, Real& pr, Real& pz) {
  const Real wc = (r - P.r_in) * (P.spl_r_out - r) * P.spl_inv_ab;
  const Real gc = (P.r_in + P.spl_r_out - Real(2) * r) * P.spl_inv_ab;
  if (!P.spl_ell) {
    w = wc;
    wr = gc;
    wz = Real(0);
    pr = P.spl_dphi;
    pz = Real(0);
    return;
  }
  const Real x = (r - P.e_r0) * P.e_idr, y = (z - P.e_z0) * P.e_idz;
  const Real we = P.e_s * (x * x + y * y - Real(1));
  const Real ger = P.e_s * Real(2) * x * P.e_idr, gez = P.e_s * Real(2) * y * P.e_idz;
  r_conj<Real>(wc, gc, Real(0), we, ger, gez, w, wr, wz);
  Real wo, go0, go1;
  r_conj<Real>(P.spl_r_out - r, Real(-1), Real(0), we, ger, gez, wo, go0, go1);
  const Real xa = r - P.r_in, den = xa + wo;
  pr = P.spl_dv * (den - xa * (Real(1) + go0)) / (den * den);
  pz = P.spl_dv * (-xa * go1) / (den * den);
}

// E at a particle from the spline coefficients: E = -grad(phi_D + w sum c
// b_i b_j)
template <typename Real, int N>
__device__ __forceinline__ void spline_gather(const PushParams<Real>& P, int ir, int iz, Real fr,
                                              Real fz, Real r, Real& Er, Real& Ez) {
  Real Br[N + 1], dBr[N + 1], Bz[N + 1], dBz[N + 1];
  spl_span_d<Real, N>(fr, Br, dBr);
  spl_span_d<Real, N>(fz, Bz, dBz);
  const Real z = mad((Real)iz + fz, P.hz, P.z_min);
  Real w, wr, wz, pr, pz;
  spl_wl<Real>(P, r, z, w, wr, wz, pr, pz);
  const Real ihr = P.dt_hr / P.dt, ihz = P.dt_hz / P.dt;   // 1 / h_r, 1 / h_z
  Real sr = 0, sz = 0;
#pragma unroll
  for (int k = 0; k <= N; ++k) {
    const Real* row = P.spl_c + (size_t)(ir + k) * P.spl_mz + iz;
    Real s0 = 0, s1 = 0;
#pragma unroll
    for (int l = 0; l <= N; ++l) {
      const Real c = __ldg(row + l);
      s0 = mad(c, Bz[l], s0);
      s1 = mad(c, dBz[l], s1);
    }
    sr = mad(mad(wr, Br[k], w * dBr[k] * ihr), s0, sr);
    sz = mad(wz * Br[k], s0, mad(w * Br[k] * ihz, s1, sz));
  }
  Er = -(pr + sr);
  Ez = -(pz + sz);
}

// load of one particle: f_ij += q w w(r) b_i b_j (FP64 atomics)
template <typename Real, int N>
__device__ __forceinline__ void spline_deposit(const PushParams<Real>& P, int ir, int iz, Real fr,
                                               Real fz) {
  Real Br[N + 1], Bz[N + 1];
  spl_span<Real, N>(fr, Br);
  spl_span<Real, N>(fz, Bz);
  const Real r = mad((Real)ir + fr, P.hr, P.r_in);
  const Real z = mad((Real)iz + fz, P.hz, P.z_min);
  Real w, wr, wz, pr, pz;
  spl_wl<Real>(P, r, z, w, wr, wz, pr, pz);
#pragma unroll
  for (int k = 0; k <= N; ++k) {
    const double wk = P.qw * (double)(w * Br[k]);
    double* row = P.spl_f + (size_t)(ir + k) * P.spl_mz + iz;
#pragma unroll
    for (int l = 0; l <= N; ++l) atomicAdd(row + l, wk * (double)Bz[l]);
  }
}

template <typename Real>
struct Part {
  int cell;
  Real fr, fz, vr, vt, vz;
};

// Collision of a particle that passed the null-collision candidate test
// (rare): type from u1 against the cumulative frequencies, then elastic
// scattering or ionisation with a child appended.  q holds the state after
// the move.  The draw-0 Philox block is recomputed here, so the common path
// carries only the candidate flag.
template <typename Real, bool TAB, int SPL>
__device__ __forceinline__ void collide(Part<Real>& q, unsigned uid, unsigned uid_hi,
                                        const Soa<Real>& s,
                                     const DepGrid& g, DevState* st, unsigned* spawn_parent,
                                     int n_slots, unsigned step, const PushParams<Real>& P,
                                     BlockTally& bt) {
  const uint4 xr = philox4x32_10_rk(make_uint4(uid, uid_hi, step, 0u), P.rk0, P.rk1);
  atomicAdd(&bt.v[kNCandidate], 1.0);
  Real ur = q.vr, ut = q.vt, uz = q.vz;
  const Real v2 = ur * ur + ut * ut + uz * uz;
  const Real speed = d_sqrt(v2);
  const Real Ek = P.half_m * v2;
  const Real nu_el0 = P.nsig_el * speed;
  Real sig_io = 0;
  if (Ek > P.e_th) {
    const Real qq = (Ek - P.e_th) * P.e_span_inv;
    sig_io = P.sig_pk * 2 * qq / (1 + qq * qq);
  }
  const Real nu_io0 = P.n_gas * sig_io * speed;
  // tabulated (TAB kernels with tables); ionisation needs more than the
  // binding energy.  The analytic kernels keep the expressions above.
  const bool tab = TAB && P.xs_n > 0;
  Xs3<Real> xt = {};
  if constexpr (TAB) {
    if (tab) xt = xs_eval<Real>(P.xs_n, P.xs_E, P.xs_nel, P.xs_nio, P.xs_xi, P.xi, Ek);
  }
  const Real nu_el = tab ? xt.nel * speed : nu_el0;
  const Real nu_io = tab ? (Ek > P.e_th ? xt.nio * speed : Real(0)) : nu_io0;
  if (nu_el + nu_io > P.nu_max) atomicAdd(&bt.v[kNOver], 1.0);
  const Real x1 = u01<Real>(xr.y) * P.nu_max;
  if (!(x1 < nu_el + nu_io)) return;   // null collision
  const Real inv_s = 1 / speed;
  const Real hr_ = ur * inv_s, ht_ = ut * inv_s, hz_ = uz * inv_s;
  if (x1 < nu_el) {
    Real dr, dt, dz;
    scatter_dir<Real>(hr_, ht_, hz_, u01<Real>(xr.z), u01<Real>(xr.w), tab ? xt.xi : P.xi, dr, dt, dz);
    Real E1 = Ek;
    if (P.recoil != 0) {
      const Real mu = dr * hr_ + dt * ht_ + dz * hz_;
      E1 = Ek * (1 - P.recoil * (1 - mu));
      atomicAdd(&bt.v[kRecoilLoss], (double)(Ek - E1));
    }
    const Real s1 = d_sqrt(P.two_over_m * E1);
    q.vr = s1 * dr; q.vt = s1 * dt; q.vz = s1 * dz;
    atomicAdd(&bt.v[kNElastic], 1.0);
    return;
  }
  const uint4 x2 = philox4x32_10_rk(make_uint4(uid, uid_hi, step, 1u), P.rk0, P.rk1);
  const Real E_rem = Ek - P.e_th;
  const Real E2 = P.opal_b * d_tan(u01<Real>(x2.x) * d_atan(E_rem / (2 * P.opal_b)));
  const Real E1 = E_rem - E2;
  Real d1r, d1t, d1z, d2r, d2t, d2z;
  scatter_dir<Real>(hr_, ht_, hz_, u01<Real>(xr.z), u01<Real>(xr.w), tab ? xt.xi : P.xi, d1r, d1t, d1z);
  scatter_dir<Real>(hr_, ht_, hz_, u01<Real>(x2.y), u01<Real>(x2.z), tab ? xt.xi : P.xi, d2r, d2t, d2z);
  const Real s1 = d_sqrt(P.two_over_m * E1), s2 = d_sqrt(P.two_over_m * E2);
  q.vr = s1 * d1r; q.vt = s1 * d1t; q.vz = s1 * d1z;
  atomicAdd(&bt.v[kIonLoss], (double)P.e_th);
  atomicAdd(&bt.v[kNIonise], 1.0);
  const long long k = (long long)atomicAdd((unsigned long long*)&st->n_spawn, 1ull);
  const long long slot = (long long)n_slots + k;
  if (k < P.spawn_cap && slot < P.capacity) {
    s.cell[slot] = q.cell;
    s.offr[slot] = q.fr;
    s.offz[slot] = q.fz;
    s.vr[slot] = s2 * d2r;
    s.vt[slot] = s2 * d2t;
    s.vz[slot] = s2 * d2z;
    s.uid[slot] = 0u;   // fixed by the child-uid kernel
    spawn_parent[k] = uid;
    if constexpr (SPL == 0)
      deposit_global(g, q.cell >> 16, q.cell & 0xFFFF, q.fr, q.fz);
    else
      spline_deposit<Real, SPL>(P, q.cell >> 16, q.cell & 0xFFFF, q.fr, q.fz);
  } else {
    set_error(st, PIC_ECAPACITY);
  }
}

// Gather, push, absorb and test for a collision one particle held in
// registers; the new state is returned in q (cell -1 when absorbed) and
// the deposit location in the result (ir < 0 when absorbed).  Every
// multiply-add is written out (mad), and the file is compiled without
// automatic contraction, so each particle is computed by the same sequence
// of roundings whichever slot of its thread it occupies (results do not
// depend on the particle order the sort leaves).
template <typename Real, bool TAB, int SPL>
__device__ __forceinline__ Dep<Real> advance(
    Part<Real>& q, unsigned uid, unsigned uid_hi, const typename Vec2<Real>::type* __restrict__ E,
    const Soa<Real>& s, const DepGrid& g, DevState* st, unsigned* spawn_parent, int n_slots,
    unsigned step, const PushParams<Real>& P, BlockTally& bt, Real& work) {
  using V2 = typename Vec2<Real>::type;
  Dep<Real> dep;
  const int nzp = P.nz + 1;
  const int ir = q.cell >> 16, iz = q.cell & 0xFFFF;
  const Real fr = q.fr, fz = q.fz, vr = q.vr, vt = q.vt, vz = q.vz;
  const Real r = mad((Real)ir + fr, P.hr, P.r_in);

  Real Er, Ez;
  if constexpr (SPL == 0) {
    // gather: bilinear interpolation of the cell's four nodes, as linear
    // interpolation along r on both z-edges, then along z
    const int n00 = ir * nzp + iz;
    const V2 e00 = __ldg(E + n00), e01 = __ldg(E + n00 + 1);
    const V2 e10 = __ldg(E + n00 + nzp), e11 = __ldg(E + n00 + nzp + 1);
    const Real ar0 = mad(fr, e10.x - e00.x, e00.x), ar1 = mad(fr, e11.x - e01.x, e01.x);
    const Real az0 = mad(fr, e10.y - e00.y, e00.y), az1 = mad(fr, e11.y - e01.y, e01.y);
    Er = mad(fz, ar1 - ar0, ar0);
    Ez = mad(fz, az1 - az0, az0);
  } else {
    spline_gather<Real, SPL>(P, ir, iz, fr, fz, r, Er, Ez);
  }
  // t = (q dt / 2m) B: mirror Bz = b0 (1 + 2 zeta^2 / L^2),
  // Br = -2 b0 r zeta / L^2 (constants folded on the host)
  Real tr = 0, tz = P.tz0;
  if (P.bkind == 1) {
    const Real zeta = mad((Real)iz + fz, P.hz, P.zoff);
    tz = mad(P.tzc * zeta, zeta, P.tz0);
    tr = P.trc * r * zeta;
  }

  // Boris: half kick, rotation about B, half kick (components r, theta, z)
  const Real vmr = mad(P.qmdt2, Er, vr), vmt = vt, vmz = mad(P.qmdt2, Ez, vz);
  const Real sf = q_div(Real(2), mad(tz, tz, mad(tr, tr, Real(1))));
  const Real sr = sf * tr, sz = sf * tz;
  const Real qr = mad(vmt, tz, vmr);
  const Real qt = vmt + mad(vmz, tr, -vmr * tz);
  const Real qz = mad(-vmt, tr, vmz);
  const Real vpr = mad(qt, sz, vmr);
  const Real vpt = vmt + mad(qz, sr, -qr * sz);
  const Real vpz = mad(-qt, sr, vmz);
  const Real vnr = mad(P.qmdt2, Er, vpr), vnt = vpt, vnz = mad(P.qmdt2, Ez, vpz);
  // work of the two half kicks, (q dt / 4) E . (v + v- + v+ + v_new)
  work = mad(Ez, (vz + vmz) + (vpz + vnz), mad(Er, (vr + vmr) + (vpr + vnr), work));

  // move in the local Cartesian frame; the radial step is formed without
  // cancellation: r1 - r = dt (2 r vr + (vr^2 + vt^2) dt) / (r + r1)
  const Real x = mad(vnr, P.dt, r), y = vnt * P.dt;
  const Real rr = mad(y, y, x * x);
  const Real inv_r1 = q_rsqrt(rr);
  const Real r1 = rr * inv_r1;
  const Real v2p = mad(vnt, vnt, vnr * vnr);
  const Real dr_cells = q_div(mad(v2p, P.dt, 2 * r * vnr), r + r1) * P.dt_hr;
  const Real dz_cells = vnz * P.dt_hz;
  Real fr1 = fr + dr_cells, fz1 = fz + dz_cells;
  // cell jumps beyond +-2^20 cells (non-physical speeds) are clamped before
  // the integer conversion; they end outside the grid and are absorbed
  const Real jmax = Real(1048576);
  const Real flr = fmin(fmax(d_floor(fr1), -jmax), jmax);
  const Real flz = fmin(fmax(d_floor(fz1), -jmax), jmax);
  const int ir1 = ir + (int)flr, iz1 = iz + (int)flz;
  // an offset that rounds up to 1 (a tiny negative sum) stays in its cell
  // at the largest offset below 1
  const Real below1 = std::is_same<Real, float>::value ? Real(0x1.fffffep-1f)
                                                       : Real(0x1.fffffffffffffp-1);
  fr1 = fmin(fr1 - flr, below1);
  fz1 = fmin(fz1 - flz, below1);

  // absorbing walls: r1 <= a, r1 >= b, z1 <= z_min, z1 >= z_max
  const bool out_in = ir1 < 0 || (ir1 == 0 && fr1 == 0);
  const bool out_out = ir1 >= P.nr;
  const bool out_zl = iz1 < 0 || (iz1 == 0 && fz1 == 0);
  const bool out_zh = iz1 >= P.nz;
  // the trap's ellipse: first entry of the straight (r, z) segment (the
  // smaller root of the quadratic along it; a start inside enters at 0)
  bool ell_hit = false;
  Real te = Real(3);
  if constexpr (SPL > 0) {
    if (P.spl_ell) {
      const Real z0a = mad((Real)iz + fz, P.hz, P.z_min), z1a = mad(vnz, P.dt, z0a);
      const Real x0 = (r - P.e_r0) * P.e_idr, y0 = (z0a - P.e_z0) * P.e_idz;
      const Real dx = (r1 - r) * P.e_idr, dy = (z1a - z0a) * P.e_idz;
      const Real qa = dx * dx + dy * dy, qb = Real(2) * (x0 * dx + y0 * dy);
      const Real qc = x0 * x0 + y0 * y0 - Real(1);
      if (qc <= Real(0)) {
        ell_hit = true;
        te = Real(0);
      } else if (qa > Real(0)) {
        const Real disc = qb * qb - Real(4) * qa * qc;
        if (disc >= Real(0)) {
          const Real t = (-qb - d_sqrt(disc)) / (Real(2) * qa);
          if (t >= Real(0) && t <= Real(1)) {
            ell_hit = true;
            te = t;
          }
        }
      }
    }
  }
  if (out_in || out_out || out_zl || out_zh || ell_hit) {
    // first crossing along the straight (r,z) segment, ties in the order
    // inner, outer, z_min, z_max
    const Real s0r = (Real)ir + fr, s0z = (Real)iz + fz;
    Real tb = 3;
    int wall = 0;
    if (out_in) { const Real t = -s0r / dr_cells; if (t < tb) { tb = t; wall = 0; } }
    if (out_out) { const Real t = ((Real)P.nr - s0r) / dr_cells; if (t < tb) { tb = t; wall = 1; } }
    if (out_zl) { const Real t = -s0z / dz_cells; if (t < tb) { tb = t; wall = 2; } }
    if (out_zh) { const Real t = ((Real)P.nz - s0z) / dz_cells; if (t < tb) { tb = t; wall = 3; } }
    if (ell_hit && te < tb) wall = 4;
    atomicAdd(&bt.v[wall == 4 ? (int)kAbsEllipse : kAbsInner + wall], 1.0);
    atomicAdd(&bt.v[kKeAbsorbed], (double)(P.half_m * mad(vnz, vnz, v2p)));
    atomicAdd(&bt.v[kNAbsorbed], 1.0);
    q.cell = -1;
    dep.ir = -1;
    return dep;
  }

  // rotate (vr, vtheta) into the basis at the new position
  const Real c = x * inv_r1, sn = y * inv_r1;
  q.cell = (ir1 << 16) | iz1;
  q.fr = fr1; q.fz = fz1;
  q.vr = mad(sn, vnt, c * vnr);
  q.vt = mad(c, vnt, -sn * vnr);
  q.vz = vnz;

  // null-collision candidate test: the integer form of u0 < P_null
  const uint4 xr = philox4x32_10_rk(make_uint4(uid, uid_hi, step, 0u), P.rk0, P.rk1);
  if ((xr.x >> 8) < P.thr_null)
    collide<Real, TAB, SPL>(q, uid, uid_hi, s, g, st, spawn_parent, n_slots, step, P, bt);
  dep.ir = ir1; dep.iz = iz1; dep.fr = fr1; dep.fz = fz1;
  return dep;
}

// Particles [p0, p0 + kPPT) of one thread.  In the FP32 path the thread's
// four slots are consecutive and move as 16-byte vectors with streaming
// cache hints (each array is read and written once per step); the FP64
// path and the ragged end of the store use scalar accesses.
template <typename Real>
__device__ __forceinline__ bool load_group(const Soa<Real>& s, int p0, int n, Part<Real>* q,
                                           unsigned* uid) {
  if constexpr (std::is_same<Real, float>::value) {
    if (p0 + kPPT <= n) {
      const int4 c = __ldcs(reinterpret_cast<const int4*>(s.cell + p0));
      const float4 a = __ldcs(reinterpret_cast<const float4*>(s.offr + p0));
      const float4 b = __ldcs(reinterpret_cast<const float4*>(s.offz + p0));
      const float4 d = __ldcs(reinterpret_cast<const float4*>(s.vr + p0));
      const float4 e = __ldcs(reinterpret_cast<const float4*>(s.vt + p0));
      const float4 f = __ldcs(reinterpret_cast<const float4*>(s.vz + p0));
      const uint4 u = __ldcs(reinterpret_cast<const uint4*>(s.uid + p0));
      q[0] = {c.x, a.x, b.x, d.x, e.x, f.x};
      q[1] = {c.y, a.y, b.y, d.y, e.y, f.y};
      q[2] = {c.z, a.z, b.z, d.z, e.z, f.z};
      q[3] = {c.w, a.w, b.w, d.w, e.w, f.w};
      uid[0] = u.x; uid[1] = u.y; uid[2] = u.z; uid[3] = u.w;
      return true;
    }
  }
#pragma unroll
  for (int k = 0; k < kPPT; ++k) {
    const int p = p0 + k;
    if (p < n) {
      q[k] = {s.cell[p], s.offr[p], s.offz[p], s.vr[p], s.vt[p], s.vz[p]};
      uid[k] = s.uid[p];
    } else {
      q[k].cell = -1;
      uid[k] = 0u;
    }
  }
  return false;
}

template <typename Real>
__device__ __forceinline__ void store_group(const Soa<Real>& s, int p0, int n, const Part<Real>* q,
                                            const bool* live, bool vec) {
  if constexpr (std::is_same<Real, float>::value) {
    if (vec) {
      __stcs(reinterpret_cast<int4*>(s.cell + p0), make_int4(q[0].cell, q[1].cell, q[2].cell, q[3].cell));
      __stcs(reinterpret_cast<float4*>(s.offr + p0), make_float4(q[0].fr, q[1].fr, q[2].fr, q[3].fr));
      __stcs(reinterpret_cast<float4*>(s.offz + p0), make_float4(q[0].fz, q[1].fz, q[2].fz, q[3].fz));
      __stcs(reinterpret_cast<float4*>(s.vr + p0), make_float4(q[0].vr, q[1].vr, q[2].vr, q[3].vr));
      __stcs(reinterpret_cast<float4*>(s.vt + p0), make_float4(q[0].vt, q[1].vt, q[2].vt, q[3].vt));
      __stcs(reinterpret_cast<float4*>(s.vz + p0), make_float4(q[0].vz, q[1].vz, q[2].vz, q[3].vz));
      return;
    }
  }
#pragma unroll
  for (int k = 0; k < kPPT; ++k) {
    const int p = p0 + k;
    if (p < n && live[k]) {   // holes stay untouched
      s.cell[p] = q[k].cell;
      s.offr[p] = q[k].fr;
      s.offz[p] = q[k].fz;
      s.vr[p] = q[k].vr;
      s.vt[p] = q[k].vt;
      s.vz[p] = q[k].vz;
    }
  }
}

// Deposit of one chunk: the chunk's node bounding box is reduced over the
// block; if it fits the shared tile the block accumulates there and flushes
// one global atomic per touched node, otherwise every particle deposits
// with global atomics.  The tile is all zero between chunks (zeroed once at
// kernel start, and the flush zeroes every word it reads), so a chunk needs
// two block barriers; every thread of the block must call it.
//
// FP32 tile: unsigned fixed-point weights, native integer shared atomics.
// Cell-sorted particles put whole warps on the same four nodes, and
// same-address atomics of one instruction serialise; so the tile is kept in
// kCopies private copies (lane & 3 picks the copy) and the m-th of a
// lane's four corner updates goes to corner m ^ ((lane >> 2) & 3).  Lanes
// of one cell then hit 16 different words per instruction.  The copies of a node
// are interleaved word by word (word 4 t + c), which spreads those 16 words
// over different banks and lets the flush read a node's copies as one
// 16-byte vector.
constexpr int kCopies = 4;
constexpr int kCapF = 1024;   // nodes per FP32 tile copy

template <typename Real, int kCap>
__device__ __forceinline__ void deposit_chunk(const Dep<Real>* dep, typename TileT<Real>::type* tile,
                                              int (*bbox)[4], int buf, const DepGrid& g, int tid,
                                              int lane) {
  using TT = typename TileT<Real>::type;
  constexpr bool f32 = std::is_same<Real, float>::value;
  constexpr int cap = f32 ? kCapF : kCap;
  int lo_r = INT_MAX, hi_r = INT_MIN, lo_z = INT_MAX, hi_z = INT_MIN;
#pragma unroll
  for (int k = 0; k < kPPT; ++k) {
    if (dep[k].ir >= 0) {
      lo_r = min(lo_r, dep[k].ir); hi_r = max(hi_r, dep[k].ir);
      lo_z = min(lo_z, dep[k].iz); hi_z = max(hi_z, dep[k].iz);
    }
  }
  lo_r = __reduce_min_sync(0xffffffffu, lo_r);
  hi_r = __reduce_max_sync(0xffffffffu, hi_r);
  lo_z = __reduce_min_sync(0xffffffffu, lo_z);
  hi_z = __reduce_max_sync(0xffffffffu, hi_z);
  if (lane == 0 && lo_r <= hi_r) {
    atomicMin(&bbox[buf][0], lo_r); atomicMax(&bbox[buf][1], hi_r);
    atomicMin(&bbox[buf][2], lo_z); atomicMax(&bbox[buf][3], hi_z);
  }
  __syncthreads();
  const int br0 = bbox[buf][0], br1 = bbox[buf][1];
  const int bz0 = bbox[buf][2], bz1 = bbox[buf][3];
  if (tid < 4) bbox[buf ^ 1][tid] = (tid & 1) ? INT_MIN : INT_MAX;
  const int rows = br1 - br0 + 2, cols = bz1 - bz0 + 2;
  const bool any = br0 <= br1;
  const bool use_tile = any && rows * cols <= cap;
  const int warp = tid >> 5;
  if (use_tile) {
    // FP32: the m-th update of a lane goes to corner m ^ rot (bit 0 along
    // r, bit 1 along z), rot = (lane >> 2) & 3; its weight and word offset
    // per corner parity are chosen once per chunk and particle
    const int rot = (lane >> 2) & 3;
    const int cr0 = kCopies * ((rot & 1) ? cols : 0), cr1 = kCopies * ((rot & 1) ? 0 : cols);
    const int cz0 = kCopies * (rot >> 1), cz1 = kCopies * ((rot >> 1) ^ 1);
#pragma unroll
    for (int k = 0; k < kPPT; ++k) {
      if (dep[k].ir < 0) continue;
      const int t = (dep[k].ir - br0) * cols + (dep[k].iz - bz0);
      if constexpr (f32) {
        const float a = dep[k].fr, c = dep[k].fz;
        unsigned* tc = tile + kCopies * t + (lane & 3);
        const float ra = ((rot & 1) ? a : 1.f - a) * kFix, rb = ((rot & 1) ? 1.f - a : a) * kFix;
        const float za = (rot & 2) ? c : 1.f - c, zb = (rot & 2) ? 1.f - c : c;
        atomicAdd(tc + cr0 + cz0, __float2uint_rn(ra * za));
        atomicAdd(tc + cr1 + cz0, __float2uint_rn(rb * za));
        atomicAdd(tc + cr0 + cz1, __float2uint_rn(ra * zb));
        atomicAdd(tc + cr1 + cz1, __float2uint_rn(rb * zb));
      } else {
        const TT a = (TT)dep[k].fr, c = (TT)dep[k].fz;
        atomicAdd(&tile[t], (TT(1) - a) * (TT(1) - c));
        atomicAdd(&tile[t + cols], a * (TT(1) - c));
        atomicAdd(&tile[t + 1], (TT(1) - a) * c);
        atomicAdd(&tile[t + cols + 1], a * c);
      }
    }
  } else if (any) {
#pragma unroll
    for (int k = 0; k < kPPT; ++k)
      if (dep[k].ir >= 0) deposit_global(g, dep[k].ir, dep[k].iz, dep[k].fr, dep[k].fz);
  }
  __syncthreads();
  if (use_tile) {
    // one warp per tile row, lanes along z: coalesced atomics, no division
    for (int rr = warp; rr < rows; rr += kThreads / 32) {
      for (int cc = lane; cc < cols; cc += 32) {
        const int t = rr * cols + cc;
        const int node = (br0 + rr) * g.nzp + (bz0 + cc);
        if constexpr (f32) {
          const uint4 q = reinterpret_cast<const uint4*>(tile)[t];
          const unsigned v = q.x + q.y + q.z + q.w;
          if (v) {
            atomicAdd(g.cnt + node, (unsigned long long)v);
            reinterpret_cast<uint4*>(tile)[t] = make_uint4(0u, 0u, 0u, 0u);
          }
        } else {
          const TT v = tile[t];
          if (v != TT(0)) {
            atomicAdd(g.rhs + node, g.qw * (double)v);
            tile[t] = TT(0);
          }
        }
      }
    }
  }
}

// FP32 spline-mode deposit of a chunk.  The block's box of the deposit
// cells, widened by the N further coefficient rows and columns of a
// particle's support, holds fixed-point counts of w b_k b_l / w_max (each
// in [0, 1], P.spl_inv_wmax) in kCopies interleaved copies, like the node
// tile.  A warp whose k-th particles share one cell (most warps of a
// cell-sorted store) adds their counts with one integer warp reduction per
// coefficient and one shared atomic; other warps add per lane to the
// lane's copy.  The flush adds each touched coefficient's count, times
// P.spl_unit, to the FP64 load grid with one atomic.  A box beyond the
// tile falls back to the per-particle FP64 atomics.
template <int N>
__device__ __forceinline__ void spline_deposit_chunk(const Dep<float>* dep, unsigned* tile,
                                                     int (*bbox)[4], int buf,
                                                     const PushParams<float>& P, int tid,
                                                     int lane) {
  int lo_r = INT_MAX, hi_r = INT_MIN, lo_z = INT_MAX, hi_z = INT_MIN;
#pragma unroll
  for (int k = 0; k < kPPT; ++k) {
    if (dep[k].ir >= 0) {
      lo_r = min(lo_r, dep[k].ir); hi_r = max(hi_r, dep[k].ir);
      lo_z = min(lo_z, dep[k].iz); hi_z = max(hi_z, dep[k].iz);
    }
  }
  lo_r = __reduce_min_sync(0xffffffffu, lo_r);
  hi_r = __reduce_max_sync(0xffffffffu, hi_r);
  lo_z = __reduce_min_sync(0xffffffffu, lo_z);
  hi_z = __reduce_max_sync(0xffffffffu, hi_z);
  if (lane == 0 && lo_r <= hi_r) {
    atomicMin(&bbox[buf][0], lo_r); atomicMax(&bbox[buf][1], hi_r);
    atomicMin(&bbox[buf][2], lo_z); atomicMax(&bbox[buf][3], hi_z);
  }
  __syncthreads();
  const int br0 = bbox[buf][0], br1 = bbox[buf][1];
  const int bz0 = bbox[buf][2], bz1 = bbox[buf][3];
  if (tid < 4) bbox[buf ^ 1][tid] = (tid & 1) ? INT_MIN : INT_MAX;
  const int rows = br1 - br0 + 1 + N, cols = bz1 - bz0 + 1 + N;
  const bool any = br0 <= br1;
  const bool use_tile = any && rows * cols <= kCapF;
  if (use_tile) {
#pragma unroll
    for (int k = 0; k < kPPT; ++k) {
      const bool has = dep[k].ir >= 0;
      const int cell = has ? (dep[k].ir << 16) | dep[k].iz : -1;
      const int c0 = __shfl_sync(0xffffffffu, cell, 0);
      const bool uniform = __all_sync(0xffffffffu, cell == c0) && c0 >= 0;
      unsigned cnt[N + 1][N + 1];
      int t = 0;
      if (has) {
        const int ir = dep[k].ir, iz = dep[k].iz;
        const float fr = dep[k].fr, fz = dep[k].fz;
        float Br[N + 1], Bz[N + 1];
        spl_span<float, N>(fr, Br);
        spl_span<float, N>(fz, Bz);
        const float r = mad((float)ir + fr, P.hr, P.r_in);
        const float z = mad((float)iz + fz, P.hz, P.z_min);
        float w, wr, wz, pr, pz;
        spl_wl<float>(P, r, z, w, wr, wz, pr, pz);
        const float v = fminf(fmaxf(w * P.spl_inv_wmax, 0.f), 1.f) * kFix;
#pragma unroll
        for (int a = 0; a <= N; ++a) {
          const float va = v * Br[a];
#pragma unroll
          for (int b = 0; b <= N; ++b) cnt[a][b] = __float2uint_rn(va * Bz[b]);
        }
        t = (ir - br0) * cols + (iz - bz0);
      } else {
#pragma unroll
        for (int a = 0; a <= N; ++a)
#pragma unroll
          for (int b = 0; b <= N; ++b) cnt[a][b] = 0u;
      }
      if (uniform) {
#pragma unroll
        for (int a = 0; a <= N; ++a)
#pragma unroll
          for (int b = 0; b <= N; ++b) {
            const unsigned sum = __reduce_add_sync(0xffffffffu, cnt[a][b]);
            if (lane == 0 && sum) atomicAdd(tile + kCopies * (t + a * cols + b), sum);
          }
      } else if (has) {
        unsigned* tc = tile + kCopies * t + (lane & 3);
#pragma unroll
        for (int a = 0; a <= N; ++a)
#pragma unroll
          for (int b = 0; b <= N; ++b)
            if (cnt[a][b]) atomicAdd(tc + kCopies * (a * cols + b), cnt[a][b]);
      }
    }
  } else if (any) {
#pragma unroll
    for (int k = 0; k < kPPT; ++k)
      if (dep[k].ir >= 0) spline_deposit<float, N>(P, dep[k].ir, dep[k].iz, dep[k].fr, dep[k].fz);
  }
  __syncthreads();
  if (use_tile) {
    // one warp per tile row, lanes along z
    const int warp = tid >> 5;
    for (int rr = warp; rr < rows; rr += kThreads / 32) {
      for (int cc = lane; cc < cols; cc += 32) {
        const int t = rr * cols + cc;
        const uint4 q = reinterpret_cast<const uint4*>(tile)[t];
        const unsigned v = q.x + q.y + q.z + q.w;
        if (v) {
          atomicAdd(P.spl_f + (size_t)(br0 + rr) * P.spl_mz + (bz0 + cc), (double)v * P.spl_unit);
          reinterpret_cast<uint4*>(tile)[t] = make_uint4(0u, 0u, 0u, 0u);
        }
      }
    }
  }
}

// block tallies: the work sum and particle count, then one global atomic
// per non-zero slot (weights and energies scaled by the macro weight)
template <typename Real>
__device__ __forceinline__ void flush_tallies(BlockTally& bt, Real work, int pushed, DevState* st,
                                              const PushParams<Real>& P, int tid, int lane) {
  Real w = work;   // warp sum in the particle precision, then one FP64 add
  const int np = __reduce_add_sync(0xffffffffu, pushed);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
  if (lane == 0 && w != Real(0)) atomicAdd(&bt.v[kWorkE], (double)w);
  if (lane == 0 && np != 0) atomicAdd(&bt.v[kNPushed], (double)np);
  __syncthreads();
  if (tid < kTallyCount) {
    double v = bt.v[tid];
    if (v != 0.0) {
      if (tid <= kAbsZmax || tid == kAbsEllipse) v *= P.weight;
      else if (tid == kWorkE) v *= (double)P.work_scale * P.weight;
      else if (tid <= kRecoilLoss) v *= P.weight;
      atomicAdd(&st->tally[tid], v);
    }
  }
}

// resident blocks per SM the FP32 kernel is compiled for (register cap)
#ifndef PIC_MIN_BLOCKS
#define PIC_MIN_BLOCKS 7
#endif
// the batch kernel keeps its simulation's view in shared memory and
// addresses it through registers; it is given a few more of them
#ifndef PIC_MIN_BLOCKS_BATCH
#define PIC_MIN_BLOCKS_BATCH 6
#endif

// Each thread loads its kPPT consecutive particles directly (16-byte vector
// loads with streaming hints in the FP32 path), advances them, stores them
// back and joins the block's tile deposit.  TAB: some simulation has
// tabulated cross sections.  SPL > 0: the weighted B-spline field of that
// degree (gather from its coefficients; deposit into its load grid through
// the fixed-point tile in FP32, with FP64 atomics per particle in FP64).
template <typename Real, bool TAB, int SPL>
__global__ void __launch_bounds__(kThreads, std::is_same<Real, float>::value && SPL == 0 ? PIC_MIN_BLOCKS : 4)
k_particle_step(Soa<Real> s, const typename Vec2<Real>::type* __restrict__ E, DepGrid g,
                DevState* st, unsigned* __restrict__ spawn_parent, PushParams<Real> P) {
  using TT = typename TileT<Real>::type;
  constexpr int kCap = TileT<Real>::cap;
  __shared__ __align__(16) TT tile[kCap];
  __shared__ int bbox[2][4];   // min ir, max ir, min iz, max iz
  __shared__ BlockTally bt;

  const int tid = threadIdx.x, lane = tid & 31;
  const int n_slots = (int)*(volatile long long*)&st->n_slots;
  const unsigned step = *(volatile unsigned*)&st->step;
  if (tid < kTallyCount) bt.v[tid] = 0.0;
  if (tid < 8) bbox[tid >> 2][tid & 3] = (tid & 1) ? INT_MIN : INT_MAX;
  for (int t = tid; t < kCap; t += kThreads) tile[t] = TT(0);
  __syncthreads();
  Real work = 0;
  int pushed = 0;
  int buf = 0;

  // Chunks are handed out in order by a global counter (st->chunk_next,
  // reset by the spawn finalisation after the step), the next index
  // fetched while the current chunk runs: blocks finish within a chunk of
  // each other, and the chunks in flight at any time are neighbours in
  // the cell-sorted store (their field rows and deposit nodes shared in
  // L2).  Measured against chunks dealt round-robin: 111.0 -> 102.6 us a
  // launch on 9.8e6 particles.
  __shared__ int s_chunk[2];
  const int nchunks = (n_slots + kChunk - 1) / kChunk;
  if (tid == 0) s_chunk[0] = atomicAdd(&st->chunk_next, 1);
  __syncthreads();
  int cb = 0;
  for (int c = s_chunk[0]; c < nchunks; c = s_chunk[cb]) {
    // s_chunk[cb ^ 1] is read after this chunk's last barrier and written
    // again only after the next chunk's first one
    if (tid == 0) s_chunk[cb ^ 1] = atomicAdd(&st->chunk_next, 1);
    cb ^= 1;
    // the chunk's particles: thread tid holds slots base + kPPT tid + k
    const int base = c * kChunk;
    const int p0 = base + kPPT * tid;
    Part<Real> q[kPPT];
    unsigned uid[kPPT];
    const bool vec = load_group<Real>(s, p0, n_slots, q, uid);
    Dep<Real> dep[kPPT];
    bool live[kPPT];
#pragma unroll
    for (int k = 0; k < kPPT; ++k) {
      dep[k].ir = -1;
      live[k] = q[k].cell >= 0;
      if (live[k]) {
        ++pushed;
        dep[k] = advance<Real, TAB, SPL>(q[k], uid[k], 0u, E, s, g, st, spawn_parent, n_slots, step,
                                         P, bt, work);
        if constexpr (SPL > 0 && !std::is_same<Real, float>::value) {
          if (dep[k].ir >= 0) spline_deposit<Real, SPL>(P, dep[k].ir, dep[k].iz, dep[k].fr, dep[k].fz);
        }
      }
    }
    store_group<Real>(s, p0, n_slots, q, live, vec);
    if constexpr (SPL == 0) {
      deposit_chunk<Real, kCap>(dep, tile, bbox, buf, g, tid, lane);
      buf ^= 1;
    } else if constexpr (std::is_same<Real, float>::value) {
      spline_deposit_chunk<SPL>(dep, tile, bbox, buf, P, tid, lane);
      buf ^= 1;
    } else {
      __syncthreads();   // no deposit barrier: the next index is read after this
    }
  }
  flush_tallies<Real>(bt, work, pushed, st, P, tid, lane);
}

template <typename Real>
void launch_particle_step(const Soa<Real>& s, const void* efield, double* rhs,
                          unsigned long long* cnt, DevState* st, unsigned* spawn_parent,
                          const PushParams<Real>& P, int grid, cudaStream_t stream) {
  DepGrid g{rhs, cnt, P.nz + 1, P.qw};
  const auto* E = (const typename Vec2<Real>::type*)efield;
  auto run = [&](auto tab, auto spl) {
    k_particle_step<Real, decltype(tab)::value, decltype(spl)::value>
        <<<grid, kThreads, 0, stream>>>(s, E, g, st, spawn_parent, P);
  };
  using T0 = std::false_type;
  using T1 = std::true_type;
  auto by_spl = [&](auto tab) {
    switch (P.spl_n) {
      case 1: run(tab, std::integral_constant<int, 1>()); break;
      case 2: run(tab, std::integral_constant<int, 2>()); break;
      case 3: run(tab, std::integral_constant<int, 3>()); break;
      default: run(tab, std::integral_constant<int, 0>()); break;
    }
  };
  if (P.xs_n > 0) by_spl(T1());
  else by_spl(T0());
}

// ----------------------------------------------------------------- batch

// The simulation a block is working on: its parameters and its views of
// the store, the grids, the state and the spawn records.  Kept in shared
// memory (the fields are read at a few points per chunk), so the per-
// particle code keeps the register budget of the single-run kernel.
template <typename Real>
struct SimView {
  PushParams<Real> P;
  Soa<Real> s;
  const typename Vec2<Real>::type* E;
  DepGrid g;
  DevState* st;
  unsigned* spawn;
  int n_slots;
  unsigned step;
};

// One persistent launch over the chunks of every simulation of a batch
// (chunk table: pic_internal.cuh).  A block takes global chunks
// blockIdx.x, blockIdx.x + gridDim.x, ...; chunks of one simulation are
// consecutive, so a block changes simulation rarely; when it does, it
// flushes the tallies of the previous one and loads the new view.  The
// per-particle work is that of k_particle_step.
template <typename Real, bool TAB>
__global__ void __launch_bounds__(kThreads, std::is_same<Real, float>::value ? PIC_MIN_BLOCKS_BATCH : 4)
k_particle_step_batch(Soa<Real> s_all, const typename Vec2<Real>::type* __restrict__ E_all,
                      double* rhs_all, unsigned long long* cnt_all, DevState* st_all,
                      unsigned* spawn_all, long long spawn_stride,
                      const PushParams<Real>* __restrict__ params, int nsim, int nnodes) {
  using TT = typename TileT<Real>::type;
  constexpr int kCap = TileT<Real>::cap;
  __shared__ __align__(16) TT tile[kCap];
  __shared__ int bbox[2][4];
  __shared__ BlockTally bt;
  __shared__ int first[kMaxSims + 1];
  __shared__ long long nslots[kMaxSims];
  __shared__ __align__(16) SimView<Real> V;

  const int tid = threadIdx.x, lane = tid & 31;
  if (tid < kTallyCount) bt.v[tid] = 0.0;
  if (tid < 8) bbox[tid >> 2][tid & 3] = (tid & 1) ? INT_MIN : INT_MAX;
  for (int t = tid; t < kCap; t += kThreads) tile[t] = TT(0);
  chunk_table(st_all, nsim, kChunk, first, nslots);   // ends with a barrier
  const int total = first[nsim];
  Real work = 0;
  int pushed = 0;
  int buf = 0;
  int cur = -1;

  // global chunks handed out in order by the first simulation's counter
  // (as in the single-run kernel; every simulation's counter is reset by
  // the spawn finalisation)
  __shared__ int s_chunk[2];
  if (tid == 0) s_chunk[0] = atomicAdd(&st_all[0].chunk_next, 1);
  __syncthreads();
  int cb = 0;
  for (int c = s_chunk[0]; c < total; c = s_chunk[cb]) {
    if (tid == 0) s_chunk[cb ^ 1] = atomicAdd(&st_all[0].chunk_next, 1);
    cb ^= 1;
    const int sim = chunk_owner(first, nsim, c);
    if (sim != cur) {
      if (cur >= 0) {
        flush_tallies<Real>(bt, work, pushed, V.st, V.P, tid, lane);
        work = 0;
        pushed = 0;
        __syncthreads();   // V and bt are read by the flush
      }
      constexpr int kWords = sizeof(PushParams<Real>) / sizeof(unsigned);
      static_assert(sizeof(PushParams<Real>) % sizeof(unsigned) == 0, "word copy");
      const unsigned* src = reinterpret_cast<const unsigned*>(params + sim);
      for (int w = tid; w < kWords; w += kThreads) reinterpret_cast<unsigned*>(&V.P)[w] = src[w];
      if (tid < kTallyCount) bt.v[tid] = 0.0;
      if (tid == 0) {
        const long long base = params[sim].base;
        const size_t go = (size_t)sim * nnodes;
        V.s = soa_offset(s_all, base);
        V.E = E_all + go;
        V.g = DepGrid{rhs_all ? rhs_all + go : nullptr, cnt_all ? cnt_all + go : nullptr,
                      params[sim].nz + 1, params[sim].qw};
        V.st = st_all + sim;
        V.spawn = spawn_all + (size_t)sim * spawn_stride;
        V.n_slots = (int)nslots[sim];
        V.step = *(volatile unsigned*)&st_all[sim].step;
      }
      __syncthreads();
      cur = sim;
    }
    const int n_slots = V.n_slots;
    const int p0 = (c - first[sim]) * kChunk + kPPT * tid;
    Part<Real> q[kPPT];
    unsigned uid[kPPT];
    const bool vec = load_group<Real>(V.s, p0, n_slots, q, uid);
    Dep<Real> dep[kPPT];
    bool live[kPPT];
#pragma unroll
    for (int k = 0; k < kPPT; ++k) {
      dep[k].ir = -1;
      live[k] = q[k].cell >= 0;
      if (live[k]) {
        ++pushed;
        dep[k] = advance<Real, TAB, 0>(q[k], uid[k], V.P.uid_hi, V.E, V.s, V.g, V.st, V.spawn, n_slots,
                               V.step, V.P, bt, work);
      }
    }
    store_group<Real>(V.s, p0, n_slots, q, live, vec);
    deposit_chunk<Real, kCap>(dep, tile, bbox, buf, V.g, tid, lane);
    buf ^= 1;
  }
  if (cur >= 0) flush_tallies<Real>(bt, work, pushed, V.st, V.P, tid, lane);
}

template <typename Real>
void launch_particle_step_batch(const Soa<Real>& s, const void* efield, double* rhs,
                                unsigned long long* cnt, DevState* st, unsigned* spawn_parent,
                                long long spawn_stride, const PushParams<Real>* params, int nsim,
                                int nnodes, bool tables, int grid, cudaStream_t stream) {
  if (tables)
    k_particle_step_batch<Real, true><<<grid, kThreads, 0, stream>>>(
        s, (const typename Vec2<Real>::type*)efield, rhs, cnt, st, spawn_parent, spawn_stride,
        params, nsim, nnodes);
  else
    k_particle_step_batch<Real, false><<<grid, kThreads, 0, stream>>>(
        s, (const typename Vec2<Real>::type*)efield, rhs, cnt, st, spawn_parent, spawn_stride,
        params, nsim, nnodes);
}

// ------------------------------------------------------------ child uids

// Children of this step get uid_next + k, k the rank of the parent's uid
// among this step's ionising parents; then the step counter advances.
// In a batch (seg not null) block k serves simulation k.
__global__ void k_spawn_finalize(DevState* st, unsigned* uid,
                                 const unsigned* __restrict__ parent,
                                 long long spawn_cap, long long capacity,
                                 const SegInfo* __restrict__ seg, long long spawn_stride) {
  if (seg) {
    const int sim = blockIdx.x;
    st += sim;
    uid += seg[sim].base;
    parent += (size_t)sim * spawn_stride;
    spawn_cap = seg[sim].spawn_cap;
    capacity = seg[sim].capacity;
  }
  const long long ns_raw = st->n_spawn;
  const long long base = st->n_slots;
  long long ns = ns_raw < spawn_cap ? ns_raw : spawn_cap;
  if (base + ns > capacity) ns = capacity - base;
  const unsigned long long next = st->uid_next;
  if (next + (unsigned long long)ns > 0xFFFFFFFFull) {
    if (threadIdx.x == 0) atomicCAS(&st->err, 0, PIC_ECAPACITY);
  }
  for (long long i = threadIdx.x; i < ns; i += blockDim.x) {
    const unsigned pu = parent[i];
    long long rank = 0;
    for (long long j = 0; j < ns; ++j) rank += parent[j] < pu;
    uid[base + i] = (unsigned)(next + (unsigned long long)rank);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st->n_slots = base + ns;
    st->uid_next = next + (unsigned long long)ns;
    st->n_spawn = 0;
    st->step = st->step + 1u;
    st->chunk_next = 0;   // the particle kernels' chunk counter
  }
}

void launch_spawn_finalize(DevState* st, unsigned* uid, const unsigned* parent,
                           long long spawn_cap, long long capacity,
                           cudaStream_t stream) {
  k_spawn_finalize<<<1, 1024, 0, stream>>>(st, uid, parent, spawn_cap, capacity, nullptr, 0);
}

void launch_spawn_finalize_batch(DevState* st, unsigned* uid, const unsigned* parent,
                                 long long spawn_stride, const SegInfo* seg, int nsim,
                                 cudaStream_t stream) {
  k_spawn_finalize<<<nsim, 1024, 0, stream>>>(st, uid, parent, 0, 0, seg, spawn_stride);
}

// ---------------------------------------------------------- seed source

// Volumetric seed source (Sec. II.A: electrons created uniformly in space
// with a Maxwellian velocity distribution), one block per simulation, after
// the child uids of step n: src_acc += src_per_step, k = floor(src_acc)
// whole particles are appended with uids uid_next .. uid_next + k - 1.
// Each draws from its own stream (uid, uid_hi, n, draw): draw 2 gives
// (u_r, u_z, u_a, u_b), draw 3 (u_c, u_d, ., .);
//   r = sqrt(a^2 + u_r (b^2 - a^2)), z = z_min + u_z L,
//   (vr, vt) = vth sqrt(-2 ln u_a) (cos 2 pi u_b, sin 2 pi u_b),
//   vz = vth sqrt(-2 ln u_c) cos 2 pi u_d,
// evaluated in FP64 (a handful of particles per step), stored in the
// particle precision and deposited in this step's charge.
template <typename Real>
__global__ void k_source(Soa<Real> s_all, DevState* st_all, const PushParams<Real>* params,
                         double* rhs_all, unsigned long long* cnt_all, int nnodes) {
  const int sim = blockIdx.x;
  const PushParams<Real>& P = params[sim];
  if (!(P.src_per_step > 0.0)) return;
  DevState* st = st_all + sim;
  __shared__ long long s_k, s_base;
  __shared__ unsigned s_uid0, s_step;
  __shared__ double s_ke[32];
  if (threadIdx.x == 0) {
    double acc = st->src_acc + P.src_per_step;
    long long k = (long long)floor(acc);
    acc -= (double)k;
    const long long n = st->n_slots;
    if (n + k > P.capacity || st->uid_next + (unsigned long long)k > 0xFFFFFFFFull) {
      atomicCAS(&st->err, 0, PIC_ECAPACITY);
      k = 0;
    }
    st->src_acc = acc;
    s_k = k;
    s_base = n;
    s_uid0 = (unsigned)st->uid_next;
    s_step = st->step - 1u;   // the step whose child uids were just fixed
    st->n_slots = n + k;
    st->uid_next += (unsigned long long)k;
    if (k > 0) st->tally[kNSource] += (double)k;
  }
  if (threadIdx.x < 32) s_ke[threadIdx.x] = 0.0;
  __syncthreads();
  const long long k = s_k;
  const Soa<Real> s = soa_offset(s_all, P.base);
  const size_t go = (size_t)sim * nnodes;
  const DepGrid g{rhs_all ? rhs_all + go : nullptr, cnt_all ? cnt_all + go : nullptr, P.nz + 1,
                  P.qw};
  const double a2 = P.r_in_d * P.r_in_d, b2 = P.r_out_d * P.r_out_d;
  double ke = 0.0;
  for (long long j = threadIdx.x; j < k; j += blockDim.x) {
    const unsigned uid = s_uid0 + (unsigned)j;
    const uint4 x = philox4x32_10_rk(make_uint4(uid, P.uid_hi, s_step, 2u), P.rk0, P.rk1);
    const uint4 w = philox4x32_10_rk(make_uint4(uid, P.uid_hi, s_step, 3u), P.rk0, P.rk1);
    const double r = sqrt(a2 + u01<double>(x.x) * (b2 - a2));
    const double z = P.z_min_d + u01<double>(x.y) * (P.z_max_d - P.z_min_d);
    const double m1 = P.vth_src * sqrt(-2.0 * log(u01<double>(x.z)));
    double sn, cs;
    sincospi(2.0 * u01<double>(x.w), &sn, &cs);
    const double vz = P.vth_src * sqrt(-2.0 * log(u01<double>(w.x))) * cospi(2.0 * u01<double>(w.y));
    const double sr = (r - P.r_in_d) / P.hr_d, sz = (z - P.z_min_d) / P.hz_d;
    int ir = (int)floor(sr), iz = (int)floor(sz);
    ir = min(max(ir, 0), P.nr - 1);
    iz = min(max(iz, 0), P.nz - 1);
    Real fr = (Real)(sr - ir), fz = (Real)(sz - iz);
    if (fr >= Real(1)) fr = nextafter(Real(1), Real(0));
    if (fz >= Real(1)) fz = nextafter(Real(1), Real(0));
    if (fr < Real(0)) fr = 0;
    if (fz < Real(0)) fz = 0;
    const long long slot = s_base + j;
    const Real vr = (Real)(m1 * cs), vt = (Real)(m1 * sn), vzr = (Real)vz;
    s.cell[slot] = (ir << 16) | iz;
    s.offr[slot] = fr;
    s.offz[slot] = fz;
    s.vr[slot] = vr;
    s.vt[slot] = vt;
    s.vz[slot] = vzr;
    s.uid[slot] = uid;
    deposit_global(g, ir, iz, fr, fz);
    ke += (double)vr * vr + (double)vt * vt + (double)vzr * vzr;
  }
  for (int o = 16; o > 0; o >>= 1) ke += __shfl_xor_sync(0xffffffffu, ke, o);
  if ((threadIdx.x & 31) == 0) s_ke[threadIdx.x >> 5] = ke;
  __syncthreads();
  if (threadIdx.x == 0 && k > 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s_ke[i];
    st->tally[kKeSource] += 0.5 * kMe * t * P.weight;
  }
}

template <typename Real>
void launch_source(const Soa<Real>& s, DevState* st, const PushParams<Real>* params, int nsim,
                   double* rhs, unsigned long long* cnt, int nnodes, cudaStream_t stream) {
  k_source<Real><<<nsim, 256, 0, stream>>>(s, st, params, rhs, cnt, nnodes);
}

// ------------------------------------------------------------------ load

template <typename Real>
__global__ void k_load(const double* __restrict__ r, const double* __restrict__ z,
                       const double* __restrict__ vr, const double* __restrict__ vt,
                       const double* __restrict__ vz, const uint64_t* __restrict__ uid,
                       long long n, Soa<Real> s, double r_in, double inv_hr,
                       double z_min, double inv_hz, int nr, int nz) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const double sr = (r[p] - r_in) * inv_hr, sz = (z[p] - z_min) * inv_hz;
    int ir = (int)floor(sr), iz = (int)floor(sz);
    ir = min(max(ir, 0), nr - 1);
    iz = min(max(iz, 0), nz - 1);
    Real fr = (Real)(sr - ir), fz = (Real)(sz - iz);
    if (fr >= Real(1)) fr = nextafter(Real(1), Real(0));
    if (fz >= Real(1)) fz = nextafter(Real(1), Real(0));
    if (fr < Real(0)) fr = 0;
    if (fz < Real(0)) fz = 0;
    s.cell[p] = (ir << 16) | iz;
    s.offr[p] = fr;
    s.offz[p] = fz;
    s.vr[p] = (Real)vr[p];
    s.vt[p] = (Real)vt[p];
    s.vz[p] = (Real)vz[p];
    s.uid[p] = (unsigned)uid[p];
  }
}

// deposit of the loaded particles at their positions (no push)
template <typename Real>
__global__ void k_deposit_only(Soa<Real> s, int n, DepGrid g) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int c = s.cell[p];
    if (c < 0) continue;
    deposit_global(g, c >> 16, c & 0xFFFF, s.offr[p], s.offz[p]);
  }
}

// spline load of the stored particles at their positions (no push)
template <typename Real, int N>
__global__ void k_spline_deposit_store(Soa<Real> s, const DevState* st, PushParams<Real> P) {
  const long long n = st->n_slots;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int c = s.cell[p];
    if (c >= 0) spline_deposit<Real, N>(P, c >> 16, c & 0xFFFF, s.offr[p], s.offz[p]);
  }
}

template <typename Real>
void launch_spline_deposit_store(const Soa<Real>& s, const DevState* st,
                                 const PushParams<Real>& P, long long max_slots,
                                 cudaStream_t stream) {
  const int grid = (int)std::max<long long>(1, std::min<long long>((max_slots + 255) / 256, 152 * 16));
  switch (P.spl_n) {
    case 1: k_spline_deposit_store<Real, 1><<<grid, 256, 0, stream>>>(s, st, P); break;
    case 2: k_spline_deposit_store<Real, 2><<<grid, 256, 0, stream>>>(s, st, P); break;
    case 3: k_spline_deposit_store<Real, 3><<<grid, 256, 0, stream>>>(s, st, P); break;
    default: break;
  }
}
template void launch_spline_deposit_store<float>(const Soa<float>&, const DevState*,
                                                 const PushParams<float>&, long long, cudaStream_t);
template void launch_spline_deposit_store<double>(const Soa<double>&, const DevState*,
                                                  const PushParams<double>&, long long,
                                                  cudaStream_t);

// spline coefficients in the particle precision (gather copy)
template <typename Real>
__global__ void k_spline_coef(const double* __restrict__ c, Real* __restrict__ out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = (Real)c[i];
}
template <typename Real>
void launch_spline_coef(const double* c, Real* out, int n, cudaStream_t stream) {
  k_spline_coef<Real><<<std::min(152 * 4, (n + 255) / 256), 256, 0, stream>>>(c, out, n);
}
template void launch_spline_coef<float>(const double*, float*, int, cudaStream_t);
template void launch_spline_coef<double>(const double*, double*, int, cudaStream_t);

template <typename Real>
void launch_load(const double* r, const double* z, const double* vr,
                 const double* vt, const double* vz, const uint64_t* uid,
                 long long n, Soa<Real> s, const PushParams<Real>& P,
                 DevState*, cudaStream_t stream) {
  if (n <= 0) return;
  const int grid = (int)std::min<long long>((n + 255) / 256, 152 * 16);
  k_load<Real><<<grid, 256, 0, stream>>>(r, z, vr, vt, vz, uid, n, s, P.r_in_d, 1.0 / P.hr_d,
                                         P.z_min_d, 1.0 / P.hz_d, P.nr, P.nz);
}

template <typename Real>
void launch_deposit_only(const Soa<Real>& s, long long n, double* rhs, unsigned long long* cnt,
                         int nz, double qw, cudaStream_t stream) {
  if (n <= 0) return;
  const int grid = (int)std::min<long long>((n + 255) / 256, 152 * 16);
  DepGrid g{rhs, cnt, nz + 1, qw};
  k_deposit_only<Real><<<grid, 256, 0, stream>>>(s, (int)n, g);
}

// ---------------------------------------------------------------- export

template <typename Real>
__global__ void k_export(Soa<Real> s, long long n, double r_in, double hr,
                         double z_min, double hz, double* r, double* z,
                         double* vr, double* vt, double* vz,
                         unsigned long long* uid, int* live) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int c = s.cell[p];
    live[p] = c >= 0;
    if (c < 0) continue;
    r[p] = r_in + ((double)(c >> 16) + (double)s.offr[p]) * hr;
    z[p] = z_min + ((double)(c & 0xFFFF) + (double)s.offz[p]) * hz;
    vr[p] = (double)s.vr[p];
    vt[p] = (double)s.vt[p];
    vz[p] = (double)s.vz[p];
    uid[p] = s.uid[p];
  }
}

template <typename Real>
void launch_export(const Soa<Real>& s, long long n_slots,
                   const PushParams<Real>& P, double* r, double* z,
                   double* vr, double* vt, double* vz, unsigned long long* uid,
                   int* live, cudaStream_t stream) {
  if (n_slots <= 0) return;
  const int grid = (int)std::min<long long>((n_slots + 255) / 256, 152 * 16);
  k_export<Real><<<grid, 256, 0, stream>>>(s, n_slots, P.r_in_d, P.hr_d, P.z_min_d, P.hz_d, r,
                                           z, vr, vt, vz, uid, live);
}

// ------------------------------------------------------- kinetic energy

template <typename Real>
__global__ void k_kinetic_energy(Soa<Real> s, const DevState* st, double* out2) {
  const long long n = st->n_slots;
  double ke = 0.0, cnt = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    if (s.cell[p] < 0) continue;
    const double a = s.vr[p], b = s.vt[p], c = s.vz[p];
    ke += a * a + b * b + c * c;
    cnt += 1.0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ke += __shfl_xor_sync(0xffffffffu, ke, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out2, ke);
    atomicAdd(out2 + 1, cnt);
  }
}

template <typename Real>
void launch_kinetic_energy(const Soa<Real>& s, DevState* st, double* out2,
                           cudaStream_t stream) {
  k_kinetic_energy<Real><<<152 * 4, 256, 0, stream>>>(s, st, out2);
}

// ------------------------------------------------------------- E access

template <typename Real>
__global__ void k_efield_set(const double* er, const double* ez,
                             typename Vec2<Real>::type* E, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    typename Vec2<Real>::type v;
    v.x = (Real)er[i];
    v.y = (Real)ez[i];
    E[i] = v;
  }
}

template <typename Real>
__global__ void k_efield_get(const typename Vec2<Real>::type* E, double* out,
                             int comp, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = comp == 0 ? (double)E[i].x : (double)E[i].y;
}

template <typename Real>
void launch_efield_set(const double* er, const double* ez, void* efield,
                       int nnodes, cudaStream_t stream) {
  k_efield_set<Real><<<(nnodes + 255) / 256, 256, 0, stream>>>(
      er, ez, (typename Vec2<Real>::type*)efield, nnodes);
}

template <typename Real>
void launch_efield_get(const void* efield, double* out, int component,
                       int nnodes, cudaStream_t stream) {
  k_efield_get<Real><<<(nnodes + 255) / 256, 256, 0, stream>>>(
      (const typename Vec2<Real>::type*)efield, out, component, nnodes);
}

// ---------------------------------------------------------- instantiate

#define PIC_INSTANTIATE(R)                                                              \
  template void launch_particle_step<R>(const Soa<R>&, const void*, double*,             \
                                        unsigned long long*, DevState*, unsigned*,      \
                                        const PushParams<R>&, int, cudaStream_t);       \
  template void launch_particle_step_batch<R>(const Soa<R>&, const void*, double*,       \
                                              unsigned long long*, DevState*, unsigned*, \
                                              long long, const PushParams<R>*, int, int, \
                                              bool, int, cudaStream_t);                 \
  template void launch_load<R>(const double*, const double*, const double*,             \
                               const double*, const double*, const uint64_t*,           \
                               long long, Soa<R>, const PushParams<R>&, DevState*,      \
                               cudaStream_t);                                           \
  template void launch_deposit_only<R>(const Soa<R>&, long long, double*,              \
                                       unsigned long long*, int, double, cudaStream_t); \
  template void launch_export<R>(const Soa<R>&, long long, const PushParams<R>&,        \
                                 double*, double*, double*, double*, double*,           \
                                 unsigned long long*, int*, cudaStream_t);              \
  template void launch_kinetic_energy<R>(const Soa<R>&, DevState*, double*,             \
                                         cudaStream_t);                                 \
  template void launch_efield_set<R>(const double*, const double*, void*, int,          \
                                     cudaStream_t);                                     \
  template void launch_efield_get<R>(const void*, double*, int, int, cudaStream_t);       \
  template void launch_source<R>(const Soa<R>&, DevState*, const PushParams<R>*, int,    \
                                 double*, unsigned long long*, int, cudaStream_t);

PIC_INSTANTIATE(float)
PIC_INSTANTIATE(double)

}  // namespace pic

namespace pic {
// resident blocks of the fused kernel per SM (sizes its persistent grid;
// the lesser of the analytic and the tabulated variant)
template <typename K>
static int blocks_of(K kernel) {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kThreads, 0);
  return b;
}
int particle_step_blocks_per_sm(int precision, bool batch) {
  if (batch) {
    if (precision == 32)
      return std::min(blocks_of(k_particle_step_batch<float, false>),
                      blocks_of(k_particle_step_batch<float, true>));
    return std::min(blocks_of(k_particle_step_batch<double, false>),
                    blocks_of(k_particle_step_batch<double, true>));
  }
  if (precision == 32)
    return std::min(blocks_of(k_particle_step<float, false, 0>),
                    blocks_of(k_particle_step<float, true, 0>));
  return std::min(blocks_of(k_particle_step<double, false, 0>),
                  blocks_of(k_particle_step<double, true, 0>));
}
// slots of the store are allocated in whole multiples of this (the sort
// kernels read 1024-slot chunks)
int particle_chunk() { return kChunk < 1024 ? 1024 : kChunk; }
}  // namespace pic
