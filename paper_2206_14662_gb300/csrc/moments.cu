// moments.cu -- fluid moments of the particle distribution on the nodes and
// the terms of the electron fluid's force balance (arXiv 2206.14662, Sec.
// IV.A: the forces acting on the electron fluid, evaluated from the
// moments of the distribution function; their sum is approximately zero).
//
// Moments.  For node i with hat function Lambda_i and volume V_i,
//   M_c(i) = (w / V_i) sum_p Lambda_i(r_p, z_p) g_c(v_p),
//   g = (1, v_r, v_theta, v_z, v_r v_r, v_r v_theta, v_r v_z,
//        v_theta v_theta, v_theta v_z, v_z v_z, nu_d(|v|), nu_io(|v|)),
// w the macro weight, nu_d = n_gas (sigma_el + sigma_io) |v| the
// electron-neutral momentum-exchange frequency and nu_io = n_gas sigma_io
// |v| the ionisation frequency (the collision path's cross sections:
// analytic or tabulated, ionisation only above its threshold).  So M_0 =
// n, M_1..3 = n u, M_4..9 = n <v v>, M_10 = n <nu_d>, M_11 = n <nu_io>.
// The weights Lambda_i are the deposit's bilinear ones.  Products and
// short sums are in the particles' precision, running sums and the grids
// in FP64 (global atomics, each already multiplied by w / V_i, so a call
// can add a scaled set into a running average).
//
// Force terms at each node (per unit volume, components r, theta, z), with
// u = M_1..3 / n, P = m (n <v v> - n u u), q = -e, m = m_e:
//   F_E = q n (E_r, 0, E_z)                    (the node field)
//   F_B = q n u x B                            (B analytic at the node)
//   F_i = -m n (u . grad) u                    (cylindrical, with the
//         -u_theta^2 / r and u_r u_theta / r terms)
//   F_p = -div P                               (cylindrical)
//   F_d = -m n <nu_d> u
//   F_a = m n (u - u_prev) / dt_prev           (0 without a previous state)
//   S   = F_i + F_E + F_B + F_p + F_d - F_a
// Derivatives: central differences, one-sided second order on the boundary
// lines (as the node field); where n = 0, u = 0 and P = 0.
//
// Fluid-Poisson model (Sec. V.A, pressure neglected), per node from the
// moments and the node field, with Omega_c = e B_z / m_e and
// omega_p^2 = e^2 n / (eps0 m_e):
//   u_theta = -E_r / B_z                               (Eq. uthet)
//   <nu_d>, <nu_io> = M_10 / n, M_11 / n
//   u_r = -(q <nu_d> / m) E_r / (omega_p^2 - Omega_c^2)   (Eq. ur)
//   omega_p,max^2 = Omega_c^2 <nu_io> / (<nu_io> + <nu_d>)   (Eq. omegape_pred)
//   n_max = eps0 m omega_p,max^2 / e^2
//   nu_d, nu_io at the E x B drift speed v = |E x B| / |B|^2 (Sec. V.B's
//   approximation of the collision frequencies)
//   j = -eps0 E_r <nu_io>   (I = 2 pi L r_+ j at the cloud edge, Eq. current)
// Zero where n = 0 (the moment ratios) or where a denominator vanishes.
#include <algorithm>
#include <climits>

#include "fluid.cuh"

namespace pic {


// elastic and ionisation frequencies at speed^2 v2, in arithmetic type T
template <typename Real, typename T>
__device__ __forceinline__ void nu_parts(const PushParams<Real>& P, T v2, T& nu_el, T& nu_io) {
  // FP32: speed from the hardware reciprocal square root (the collision
  // moments are diagnostics held to 1e-5)
  const T speed = sizeof(T) == 4 ? (v2 > T(0) ? (T)(v2 * rsqrtf((float)v2)) : T(0)) : (T)sqrt((double)v2);
  const T Ek = (T)(0.5 * kMe) * v2;
  if (P.xs_n > 0) {
    const Xs3<Real> x = xs_eval<Real>(P.xs_n, P.xs_E, P.xs_nel, P.xs_nio, P.xs_xi, P.xi, (Real)Ek);
    nu_el = (T)x.nel * speed;
    nu_io = Ek > (T)P.e_th ? (T)x.nio * speed : T(0);
    return;
  }
  T sio = T(0);
  if (Ek > (T)P.e_th) {
    const T qq = (Ek - (T)P.e_th) * (T)P.e_span_inv;
    const T num = (T)P.sig_pk * T(2) * qq, den = T(1) + qq * qq;
    sio = sizeof(T) == 4 ? (T)__fdividef((float)num, (float)den) : num / den;
  }
  nu_el = (T)P.nsig_el * speed;
  nu_io = (T)P.n_gas * sio * speed;
}

// hat-function volume of node (i, j): 2 pi R_i Z_j
__device__ __forceinline__ double node_volume(const ForceParams& F, int i, int j) {
  const double hr = F.hr, hz = F.hz;
  const double r_out = F.r_in + F.nr * hr;
  const double R = i == 0 ? hr * (F.r_in / 2 + hr / 6)
                          : (i == F.nr ? hr * (r_out / 2 - hr / 6) : (F.r_in + i * hr) * hr);
  const double Z = (j == 0 || j == F.nz) ? hz / 2 : hz;
  return 2.0 * kPi * R * Z;
}

// Moment pass.  A warp takes chunks of kMomIters x 32 consecutive slots,
// with the next 32-slot tile's loads issued before the current one is
// processed.  Each particle contributes the 48 products g_k Lambda_j
// (moment k, corner j: column 4 k + j).  The cross-lane sums go through a
// padded shared-memory row per lane: lane l < 24 owns the column pair
// (2 l, 2 l + 1) and sums it down the rows.
//  * FP32, a tile of one or two cells (in a cell-sorted store all tiles but
//    those where three cells meet): each lane adds its products into 48
//    registers, one cell after the other in ascending order; a run of
//    additions on one cell, kRegTiles at most, is folded once it ends (the
//    registers written to the rows and summed down them).
//  * Otherwise the tile is sorted by cell across the warp (bitonic, on a
//    32-bit key packing the cell and the lane, holes last), each lane writes
//    its products to the row of its rank, and the lanes sum their columns
//    down the runs of equal cells.
// Both add a column pair's sums to a running sum while the cell stays the
// same.  When the cell changes the running sum is parked in a per-warp
// cache of kMomSlots cells in shared memory (added to its cell's entry, or
// replacing the oldest entry, which is then flushed); the entries left at
// the end of a chunk are flushed too.  A flush adds the sum, times w / V of
// the node, to M with one FP64 atomic per column, so a chunk flushes about
// once per distinct cell whatever the order of its slots.  FP32 running
// sums are compensated (each addition's rounding error is collected in a
// second FP32 word, both words flushed), and the FP32 -> FP64 conversion
// at a flush runs on the integer pipe: no FP64 arithmetic is left in the
// FP32 pass (on this part FP64 instructions take about 64 times the issue
// slots of FP32 ones).
constexpr int kMomCols = 4 * kMoments;   // column 4 k + j
constexpr int kMomPairs = kMomCols / 2;  // lanes owning a column pair
constexpr int kMomIters = 32;
constexpr int kRegTiles = 32;  // additions summed in registers before a fold
constexpr int kMomSlots = 16;  // cells parked per warp
template <typename Real>
struct MomShape;
template <>
struct MomShape<float> {
  static constexpr int warps = 4;
  static constexpr int row = 52;   // 208 B: 16-byte stores of 8 lanes in distinct banks
  using Store = float4;            // 4 columns (one moment); a cache entry (2 sums + 2 errors)
  using Pair = float2;
};
template <>
struct MomShape<double> {
  static constexpr int warps = 2;
  static constexpr int row = 50;   // 400 B
  using Store = double2;           // 2 columns; a cache entry (2 sums)
  using Pair = double2;
};

// Running sum of a column: FP32 pairs (s, e) with s the rounded sum and e
// the accumulated rounding errors of the additions (Knuth's two-sum), so
// that s + e carries about twice FP32's precision; FP64 plain.
template <typename Real>
struct MomSum {
  Real s, e;
};
template <typename Real>
__device__ __forceinline__ void sum_add(MomSum<Real>& a, Real x) {
  if (sizeof(Real) == 8) {
    a.s += x;
    return;
  }
  const Real t = a.s + x;
  const Real xp = t - a.s;
  a.e += (a.s - (t - xp)) + (x - xp);
  a.s = t;
}

// exact FP32 -> FP64 conversion in integer arithmetic (IEEE 754 binary32
// to binary64: exponent rebiased by 1023 - 127, fraction widened by 29
// bits; a subnormal is renormalised, infinities and NaNs keep their class)
__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  const unsigned ex = (u >> 23) & 0xFFu, fr = u & 0x7FFFFFu;
  unsigned long long bits;
  if (ex == 0xFFu) {
    bits = (0x7FFULL << 52) | ((unsigned long long)fr << 29);
  } else if (ex != 0) {
    bits = ((unsigned long long)(ex + 896) << 52) | ((unsigned long long)fr << 29);
  } else if (fr == 0) {
    bits = 0;
  } else {
    // fr 2^-149 with its leading one at bit p: 2^(p - 149) (1 + fraction)
    const int p = 31 - __clz((int)fr);
    bits = ((unsigned long long)(p + 874) << 52) |
           (((unsigned long long)fr << (52 - p)) & 0xFFFFFFFFFFFFFULL);
  }
  return __longlong_as_double((long long)(sign | bits));
}
__device__ __forceinline__ double to_f64(float x) { return f32_to_f64(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }

// packed pair arithmetic: FP32 pairs in one instruction (Blackwell's
// paired FP32 pipe), FP64 pairs as two
__device__ __forceinline__ float2 pair_fma(float a, float2 b, float2 c) {
  return __ffma2_rn(make_float2(a, a), b, c);
}
__device__ __forceinline__ double2 pair_fma(double a, double2 b, double2 c) {
  return make_double2(fma(a, b.x, c.x), fma(a, b.y, c.y));
}
__device__ __forceinline__ float2 pair_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 pair_add(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}

// 32-bit sort key: ((ir << 12 | iz) << 5 | lane), iz < 4096 and ir < 32768;
// holes 0xFFFFFFE0 | lane, above every cell's key
__device__ __forceinline__ unsigned mom_key(int cell, int lane) {
  if (cell < 0) return 0xFFFFFFE0u | (unsigned)lane;
  return ((((unsigned)cell >> 16) << 12 | ((unsigned)cell & 0xFFFu)) << 5) | (unsigned)lane;
}
__device__ __forceinline__ int key_cell(unsigned key) {
  return (int)(((key >> 17) << 16) | ((key >> 5) & 0xFFFu));
}

// w / V of node (i, j) in the particles' precision (an FP64 division costs
// dozens of FP64 operations; FP32 simulations are held to 1e-5 anyway)
template <typename Real>
__device__ __forceinline__ Real weight_per_volume(const ForceParams& F, double ws, int i, int j) {
  if (sizeof(Real) == 8) return (Real)(ws / node_volume(F, i, j));
  const float hr = (float)F.hr, hz = (float)F.hz, r_in = (float)F.r_in;
  const float R = i == 0 ? hr * (0.5f * r_in + hr / 6.0f)
                         : (i == F.nr ? hr * (0.5f * (r_in + F.nr * hr) - hr / 6.0f)
                                      : (r_in + i * hr) * hr);
  const float Z = (j == 0 || j == F.nz) ? 0.5f * hz : hz;
  return (Real)((float)ws / ((float)(2.0 * kPi) * R * Z));
}

// adds column col's sum v over cell `cell`, times w / V of its node, to M
template <typename Real>
__device__ __forceinline__ void moment_flush(const ForceParams& F, double ws, int cell, int col,
                                             const MomSum<Real>& v, double* M, int nzp,
                                             int nnodes) {
  const int k = col >> 2, j = col & 3;
  const int i = (cell >> 16) + (j & 1), jz = (cell & 0xFFFF) + (j >> 1);
  const Real w = weight_per_volume<Real>(F, ws, i, jz);
  double* at = M + (size_t)k * nnodes + i * nzp + jz;
  const Real p = v.s * w;
  // an FP32 product beyond FP32's range is formed in FP64 instead
  atomicAdd(at, isfinite(p) || !isfinite(v.s) ? to_f64(p) : to_f64(v.s) * to_f64(w));
  if (sizeof(Real) == 4 && v.e != Real(0)) atomicAdd(at, to_f64(v.e * w));
}

template <typename Real>
__global__ void __launch_bounds__(MomShape<Real>::warps * 32)
k_moments(Soa<Real> s, const DevState* st, PushParams<Real> P, ForceParams F, double scale,
          double* M) {
  using Sh = MomShape<Real>;
  constexpr int W = Sh::warps, RW = Sh::row;
  constexpr int kPerStore = (int)(sizeof(typename Sh::Store) / sizeof(Real));
  __shared__ __align__(16) Real rows[W][32][RW];
  __shared__ int rrank[W][32];
  __shared__ typename Sh::Store cache[W][kMomSlots][kMomPairs];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long n = st->n_slots;
  const int nzp = F.nz + 1, nnodes = (F.nr + 1) * nzp;
  const double ws = scale * F.weight;
  const long long chunk = 32LL * kMomIters;
  const long long nchunks = (n + chunk - 1) / chunk;
  const bool owner = lane < kMomPairs;   // owns columns 2 lane, 2 lane + 1
  const int col0 = 2 * lane;
  Real(*row)[RW] = rows[wib];
  int* rk = rrank[wib];
  // cache entry of lane l < kMomPairs: its two columns' sums (and, FP32,
  // their errors); each lane touches only its own entries
  typename Sh::Store(*slot_data)[kMomPairs] = cache[wib];
  // register runs: FP32 only (48 FP64 registers a lane would halve the
  // resident warps; FP64 simulations are the small validation cases)
  constexpr bool kReg = sizeof(Real) == 4;
  for (long long ch = (long long)blockIdx.x * W + wib; ch < nchunks;
       ch += (long long)gridDim.x * W) {
    int run_cell = -1;
    MomSum<Real> run0{Real(0), Real(0)}, run1{Real(0), Real(0)};
    // lane t < kMomSlots holds the cell of cache slot t (-1: empty); the
    // slots are replaced oldest first
    int slot_cell = -1, next_slot = 0;
    auto entry_load = [&](int t, MomSum<Real>& a, MomSum<Real>& b) {
      const typename Sh::Store v = slot_data[t][lane];
      if (sizeof(Real) == 4) {
        const Real* e = reinterpret_cast<const Real*>(&v);
        a = {e[0], e[2 % kPerStore]};
        b = {e[1], e[3 % kPerStore]};
      } else {
        const Real* e = reinterpret_cast<const Real*>(&v);
        a = {e[0], Real(0)};
        b = {e[1], Real(0)};
      }
    };
    auto entry_store = [&](int t, const MomSum<Real>& a, const MomSum<Real>& b) {
      typename Sh::Store v;
      Real* e = reinterpret_cast<Real*>(&v);
      e[0] = a.s;
      e[1] = b.s;
      if (sizeof(Real) == 4) {
        e[2 % kPerStore] = a.e;
        e[3 % kPerStore] = b.e;
      }
      slot_data[t][lane] = v;
    };
    auto flush_pair = [&](int cell, const MomSum<Real>& a, const MomSum<Real>& b) {
      moment_flush<Real>(F, ws, cell, col0, a, M, nzp, nnodes);
      moment_flush<Real>(F, ws, cell, col0 + 1, b, M, nzp, nnodes);
    };
    // parks the running sums of run_cell in the cache
    auto park = [&]() {
      const unsigned hit = __ballot_sync(0xffffffffu, lane < kMomSlots && slot_cell == run_cell);
      if (hit) {
        const int t = __ffs(hit) - 1;
        if (owner) {
          MomSum<Real> a, b;
          entry_load(t, a, b);
          sum_add(a, run0.s);
          a.e += run0.e;
          sum_add(b, run1.s);
          b.e += run1.e;
          entry_store(t, a, b);
        }
        return;
      }
      const int t = next_slot;
      next_slot = next_slot + 1 == kMomSlots ? 0 : next_slot + 1;
      const int old = __shfl_sync(0xffffffffu, slot_cell, t);
      if (owner) {
        if (old >= 0) {
          MomSum<Real> a, b;
          entry_load(t, a, b);
          flush_pair(old, a, b);
        }
        entry_store(t, run0, run1);
      }
      if (lane == t) slot_cell = run_cell;
    };
    // adds a column pair's sums over cell cr to the running sums, parking
    // them first if the cell changes
    auto merge = [&](int cr, Real part0, Real part1) {
      if (cr != run_cell) {
        if (run_cell >= 0) park();
        run_cell = cr;
        run0 = run1 = MomSum<Real>{Real(0), Real(0)};
      }
      sum_add(run0, part0);
      sum_add(run1, part1);
    };
    // sums of the column pair down rows [r0, r1)
    auto column_sums = [&](int r0, int r1, Real& part0, Real& part1) {
      using Pr = typename Sh::Pair;
      Pr s0{Real(0), Real(0)}, s1{Real(0), Real(0)};
      if (owner) {
        int r = r0;
        for (; r + 1 < r1; r += 2) {
          s0 = pair_add(s0, *reinterpret_cast<const Pr*>(&row[r][col0]));
          s1 = pair_add(s1, *reinterpret_cast<const Pr*>(&row[r + 1][col0]));
        }
        if (r < r1) s0 = pair_add(s0, *reinterpret_cast<const Pr*>(&row[r][col0]));
        s0 = pair_add(s0, s1);
      }
      part0 = s0.x;
      part1 = s0.y;
    };
    typename Sh::Pair acc[kMomCols / 2];   // columns (2 q, 2 q + 1)
#pragma unroll
    for (int q = 0; q < kMomCols / 2; ++q) acc[q] = typename Sh::Pair{Real(0), Real(0)};
    int reg_cell = -1, reg_tiles = 0;
    // folds the register run into the running sums through the rows
    auto fold = [&]() {
#pragma unroll
      for (int q = 0; q < kMomCols; q += kPerStore) {
        typename Sh::Store v;
        Real* e = reinterpret_cast<Real*>(&v);
#pragma unroll
        for (int t = 0; t < kPerStore; ++t) {
          e[t] = reinterpret_cast<const Real*>(acc)[q + t];
          reinterpret_cast<Real*>(acc)[q + t] = Real(0);
        }
        *reinterpret_cast<typename Sh::Store*>(&row[lane][q]) = v;
      }
      __syncwarp();
      Real part0, part1;
      column_sums(0, 32, part0, part1);
      __syncwarp();   // the rows are rewritten next
      merge(reg_cell, part0, part1);
      reg_tiles = 0;
    };
    const long long base = ch * chunk + lane;
    int ncell = -1;
    Real nfr = Real(0), nfz = Real(0), nvr = Real(0), nvt = Real(0), nvz = Real(0);
    if (base < n) {
      ncell = s.cell[base];
      nfr = s.offr[base];
      nfz = s.offz[base];
      nvr = s.vr[base];
      nvt = s.vt[base];
      nvz = s.vz[base];
    }
    for (int it = 0; it < kMomIters; ++it) {
      const int cell = ncell;
      const Real fr = nfr, fz = nfz, vr = nvr, vt = nvt, vz = nvz;
      {
        const long long q = base + (long long)(it + 1) * 32;
        ncell = -1;
        if (it + 1 < kMomIters && q < n) {
          ncell = s.cell[q];
          nfr = s.offr[q];
          nfz = s.offz[q];
          nvr = s.vr[q];
          nvt = s.vt[q];
          nvz = s.vz[q];
        }
      }
      Real c[4] = {Real(0), Real(0), Real(0), Real(0)};
      Real g[kMoments];
#pragma unroll
      for (int k = 0; k < kMoments; ++k) g[k] = Real(0);
      if (cell >= 0) {
        c[0] = (Real(1) - fr) * (Real(1) - fz);
        c[1] = fr * (Real(1) - fz);
        c[2] = (Real(1) - fr) * fz;
        c[3] = fr * fz;
        Real nel, nio;
        nu_parts<Real, Real>(P, vr * vr + vt * vt + vz * vz, nel, nio);
        g[0] = Real(1);
        g[1] = vr;
        g[2] = vt;
        g[3] = vz;
        g[4] = vr * vr;
        g[5] = vr * vt;
        g[6] = vr * vz;
        g[7] = vt * vt;
        g[8] = vt * vz;
        g[9] = vz * vz;
        g[10] = nel + nio;
        g[11] = nio;
      }
      if (kReg) {
        // a tile of at most two cells is added to the registers cell by
        // cell, in ascending order; the warp's reductions are uniform
        const int cmin = __reduce_min_sync(0xffffffffu, cell >= 0 ? cell : INT_MAX);
        const int cmax = __reduce_max_sync(0xffffffffu, cell);
        if (cmin != INT_MAX && __all_sync(0xffffffffu, cell < 0 || cell == cmin || cell == cmax)) {
#pragma unroll
          for (int pass = 0; pass < 2; ++pass) {
            const int cc = pass == 0 ? cmin : cmax;
            if (pass == 1 && cmax == cmin) break;
            if (reg_tiles > 0 && (cc != reg_cell || reg_tiles == kRegTiles)) fold();
            reg_cell = cc;
            ++reg_tiles;
            const bool mine = cell == cc;
            Real cm[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) cm[j] = mine ? c[j] : Real(0);
            const typename Sh::Pair c01{cm[0], cm[1]}, c23{cm[2], cm[3]};
#pragma unroll
            for (int k = 0; k < kMoments; ++k) {
              acc[2 * k] = pair_fma(g[k], c01, acc[2 * k]);
              acc[2 * k + 1] = pair_fma(g[k], c23, acc[2 * k + 1]);
            }
          }
          continue;
        }
        if (reg_tiles > 0) fold();
      }
      // rank of each lane's particle in cell order: bitonic sort of the
      // packed keys across the warp, then the inverse permutation
      unsigned key = mom_key(cell, lane);
#pragma unroll
      for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
          const unsigned other = __shfl_xor_sync(0xffffffffu, key, j);
          const bool ascending = (lane & k) == 0, lower = (lane & j) == 0;
          key = lower == ascending ? min(key, other) : max(key, other);
        }
      }
      rk[key & 31u] = lane;
      __syncwarp();
      const int rank = rk[lane];
      if (cell >= 0) {
#pragma unroll
        for (int k = 0; k < kMoments; ++k) {
#pragma unroll
          for (int h = 0; h < 4; h += kPerStore) {
            typename Sh::Store v;
            Real* e = reinterpret_cast<Real*>(&v);
#pragma unroll
            for (int t = 0; t < kPerStore; ++t) e[t] = g[k] * c[h + t];
            *reinterpret_cast<typename Sh::Store*>(&row[rank][4 * k + h]) = v;
          }
        }
      }
      // runs of equal cells among the sorted rows (holes last): lane r
      // holds the r-th key
      const unsigned prev = __shfl_up_sync(0xffffffffu, key, 1);
      const bool valid = key < 0xFFFFFFE0u;
      const unsigned heads =
          __ballot_sync(0xffffffffu, valid && (lane == 0 || (prev >> 5) != (key >> 5)));
      const int nvalid = __popc(__ballot_sync(0xffffffffu, valid));
      __syncwarp();
      unsigned rest = heads;
      while (rest) {
        const int r0 = __ffs(rest) - 1;
        rest &= rest - 1;
        const int r1 = rest ? __ffs(rest) - 1 : nvalid;
        const int cr = key_cell(__shfl_sync(0xffffffffu, key, r0));
        Real part0, part1;
        column_sums(r0, r1, part0, part1);
        merge(cr, part0, part1);
      }
      __syncwarp();   // the rows and ranks are rewritten by the next tile
    }
    if (kReg && reg_tiles > 0) fold();
    if (run_cell >= 0) park();
    // flush the chunk's parked cells
#pragma unroll 1
    for (int t = 0; t < kMomSlots; ++t) {
      const int cell = __shfl_sync(0xffffffffu, slot_cell, t);
      if (cell >= 0 && owner) {
        MomSum<Real> a, b;
        entry_load(t, a, b);
        flush_pair(cell, a, b);
      }
    }
  }
}

// magnetic field (B_r, B_z) at node (i, j)
__device__ __forceinline__ void node_b(const ForceParams& F, int i, int j, double& Br,
                                       double& Bz) {
  Br = 0.0;
  Bz = F.b0;
  if (F.bkind == 1) {
    const double r = F.r_in + i * F.hr;
    const double zeta = F.z_min + j * F.hz - F.z_mid;
    Bz = F.b0 * (1.0 + 2.0 * zeta * zeta / (F.L * F.L));
    Br = -2.0 * F.b0 * r * zeta / (F.L * F.L);
  }
}

// fluid velocity and pressure tensor at node o from the moments
struct Fluid {
  double n, u[3], P[6];   // P: rr, rt, rz, tt, tz, zz
};
__device__ __forceinline__ Fluid fluid_at(const double* M, int nnodes, int o, double m) {
  Fluid f;
  f.n = M[o];
  const double inv = f.n > 0 ? 1.0 / f.n : 0.0;
  for (int a = 0; a < 3; ++a) f.u[a] = f.n > 0 ? M[(size_t)(1 + a) * nnodes + o] * inv : 0.0;
  const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
  for (int k = 0; k < 6; ++k)
    f.P[k] = f.n > 0 ? m * (M[(size_t)(4 + k) * nnodes + o] - f.n * f.u[ia[k]] * f.u[ib[k]])
                     : 0.0;
  return f;
}

// d/dx of f at index k of n+1 points spaced h: central, one-sided second
// order at the ends
__device__ __forceinline__ double ddx(double fm2, double fm1, double f0, double fp1, double fp2,
                                      int k, int n, double h) {
  if (k == 0) return (-3.0 * f0 + 4.0 * fp1 - fp2) / (2.0 * h);
  if (k == n) return (3.0 * f0 - 4.0 * fm1 + fm2) / (2.0 * h);
  return (fp1 - fm1) / (2.0 * h);
}

template <typename Real>
__global__ void k_force_terms(const double* __restrict__ M, const double* __restrict__ Mprev,
                              const typename Vec2<Real>::type* __restrict__ E, ForceParams F,
                              double* __restrict__ out) {
  const int nr = F.nr, nz = F.nz, nzp = nz + 1, nnodes = (nr + 1) * nzp;
  const double m = kMe, q = -kQe;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < nnodes; o += gridDim.x * blockDim.x) {
    const int i = o / nzp, j = o % nzp;
    const double r = F.r_in + i * F.hr;
    const Fluid c = fluid_at(M, nnodes, o, m);
    // neighbours along r (i-2..i+2) and z (j-2..j+2), clamped to the grid
    // (the difference formula reads only those it needs)
    auto at = [&](int ii, int jj) {
      ii = min(max(ii, 0), nr);
      jj = min(max(jj, 0), nz);
      return fluid_at(M, nnodes, ii * nzp + jj, m);
    };
    const Fluid rm2 = at(i - 2, j), rm1 = at(i - 1, j), rp1 = at(i + 1, j), rp2 = at(i + 2, j);
    const Fluid zm2 = at(i, j - 2), zm1 = at(i, j - 1), zp1 = at(i, j + 1), zp2 = at(i, j + 2);
    const double rr[5] = {F.r_in + (i - 2) * F.hr, F.r_in + (i - 1) * F.hr, r,
                          F.r_in + (i + 1) * F.hr, F.r_in + (i + 2) * F.hr};
    auto dr = [&](double a, double b, double cc, double d, double e) {
      return ddx(a, b, cc, d, e, i, nr, F.hr);
    };
    auto dz = [&](double a, double b, double cc, double d, double e) {
      return ddx(a, b, cc, d, e, j, nz, F.hz);
    };
    double du_r[3], du_z[3];
    for (int a = 0; a < 3; ++a) {
      du_r[a] = dr(rm2.u[a], rm1.u[a], c.u[a], rp1.u[a], rp2.u[a]);
      du_z[a] = dz(zm2.u[a], zm1.u[a], c.u[a], zp1.u[a], zp2.u[a]);
    }
    double Br, Bz;
    node_b(F, i, j, Br, Bz);
    const double n = c.n, ur = c.u[0], ut = c.u[1], uz = c.u[2];
    double T[7][3];
    T[0][0] = q * n * (double)E[o].x;
    T[0][1] = 0.0;
    T[0][2] = q * n * (double)E[o].y;
    T[1][0] = q * n * (ut * Bz);
    T[1][1] = q * n * (uz * Br - ur * Bz);
    T[1][2] = q * n * (-ut * Br);
    T[2][0] = -m * n * (ur * du_r[0] + uz * du_z[0] - ut * ut / r);
    T[2][1] = -m * n * (ur * du_r[1] + uz * du_z[1] + ur * ut / r);
    T[2][2] = -m * n * (ur * du_r[2] + uz * du_z[2]);
    // div P: (1/r) d(r P_rr)/dr + dP_rz/dz - P_tt / r ; (1/r^2) d(r^2 P_rt)/dr
    // + dP_tz/dz ; (1/r) d(r P_rz)/dr + dP_zz/dz
    const Fluid* R5[5] = {&rm2, &rm1, &c, &rp1, &rp2};
    double rPrr[5], r2Prt[5], rPrz[5];
    for (int k = 0; k < 5; ++k) {
      rPrr[k] = rr[k] * R5[k]->P[0];
      r2Prt[k] = rr[k] * rr[k] * R5[k]->P[1];
      rPrz[k] = rr[k] * R5[k]->P[2];
    }
    const double div_r = dr(rPrr[0], rPrr[1], rPrr[2], rPrr[3], rPrr[4]) / r +
                         dz(zm2.P[2], zm1.P[2], c.P[2], zp1.P[2], zp2.P[2]) - c.P[3] / r;
    const double div_t = dr(r2Prt[0], r2Prt[1], r2Prt[2], r2Prt[3], r2Prt[4]) / (r * r) +
                         dz(zm2.P[4], zm1.P[4], c.P[4], zp1.P[4], zp2.P[4]);
    const double div_z = dr(rPrz[0], rPrz[1], rPrz[2], rPrz[3], rPrz[4]) / r +
                         dz(zm2.P[5], zm1.P[5], c.P[5], zp1.P[5], zp2.P[5]);
    T[3][0] = -div_r;
    T[3][1] = -div_t;
    T[3][2] = -div_z;
    const double nud = M[(size_t)10 * nnodes + o];
    for (int a = 0; a < 3; ++a) T[4][a] = -m * nud * c.u[a];
    if (Mprev && F.dt_prev > 0) {
      const Fluid pv = fluid_at(Mprev, nnodes, o, m);
      for (int a = 0; a < 3; ++a) T[5][a] = m * n * (c.u[a] - pv.u[a]) / F.dt_prev;
    } else {
      for (int a = 0; a < 3; ++a) T[5][a] = 0.0;
    }
    for (int a = 0; a < 3; ++a) T[6][a] = T[2][a] + T[0][a] + T[1][a] + T[3][a] + T[4][a] - T[5][a];
    for (int t = 0; t < 7; ++t)
      for (int a = 0; a < 3; ++a) out[(size_t)(3 * t + a) * nnodes + o] = T[t][a];
  }
}

template <typename Real>
__global__ void k_fluid_model(const double* __restrict__ M,
                              const typename Vec2<Real>::type* __restrict__ E, ForceParams F,
                              PushParams<Real> P, double* __restrict__ out) {
  const int nzp = F.nz + 1, nnodes = (F.nr + 1) * nzp;
  const double m = kMe, q = -kQe;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < nnodes; o += gridDim.x * blockDim.x) {
    const int i = o / nzp, j = o % nzp;
    double Br, Bz;
    node_b(F, i, j, Br, Bz);
    const double Er = (double)E[o].x, Ez = (double)E[o].y;
    const double n = M[o];
    const double nud = n > 0 ? M[(size_t)10 * nnodes + o] / n : 0.0;
    const double nuio = n > 0 ? M[(size_t)11 * nnodes + o] / n : 0.0;
    const double Oc2 = (q * Bz / m) * (q * Bz / m);
    const double wp2 = q * q * n / (kEps0 * m);
    const double den = wp2 - Oc2;
    const double wmax2 = nuio + nud > 0 ? Oc2 * nuio / (nuio + nud) : 0.0;
    // E x B drift speed: |E x B| = |E_z B_r - E_r B_z| (E and B in the r-z plane)
    const double B2 = Br * Br + Bz * Bz;
    const double vd = B2 > 0 ? fabs(Ez * Br - Er * Bz) / B2 : 0.0;
    double dnel, dnio;
    nu_parts<Real, double>(P, vd * vd, dnel, dnio);
    double g[kFluidModel];
    g[0] = Bz != 0 ? -Er / Bz : 0.0;
    g[1] = nud;
    g[2] = nuio;
    g[3] = den != 0 ? -(q * nud / m) * Er / den : 0.0;
    g[4] = wmax2;
    g[5] = kEps0 * m * wmax2 / (q * q);
    g[6] = dnel + dnio;
    g[7] = dnio;
    g[8] = -kEps0 * Er * nuio;
    for (int k = 0; k < kFluidModel; ++k) out[(size_t)k * nnodes + o] = g[k];
  }
}

template <typename Real>
void launch_fluid_model(const double* M, const void* efield, const ForceParams& F,
                        const PushParams<Real>& P, double* out, cudaStream_t stream) {
  const int nnodes = (F.nr + 1) * (F.nz + 1);
  k_fluid_model<Real><<<std::min(152 * 4, (nnodes + 127) / 128), 128, 0, stream>>>(
      M, (const typename Vec2<Real>::type*)efield, F, P, out);
}

template <typename Real>
void launch_moments(const Soa<Real>& s, const DevState* st, const PushParams<Real>& P,
                    const ForceParams& F, double scale, double* M, long long max_slots,
                    cudaStream_t stream) {
  constexpr int W = MomShape<Real>::warps;
  const long long chunks = (max_slots + 32LL * kMomIters - 1) / (32LL * kMomIters);
  const long long blocks = std::min<long long>((chunks + W - 1) / W, 152 * 8);
  k_moments<Real><<<(int)std::max<long long>(blocks, 1), W * 32, 0, stream>>>(s, st, P, F, scale,
                                                                             M);
}

template <typename Real>
void launch_force_terms(const double* M, const double* Mprev, const void* efield,
                        const ForceParams& F, double* out, cudaStream_t stream) {
  const int nnodes = (F.nr + 1) * (F.nz + 1);
  k_force_terms<Real><<<std::min(152 * 4, (nnodes + 127) / 128), 128, 0, stream>>>(
      M, Mprev, (const typename Vec2<Real>::type*)efield, F, out);
}

template void launch_moments<float>(const Soa<float>&, const DevState*, const PushParams<float>&,
                                    const ForceParams&, double, double*, long long, cudaStream_t);
template void launch_moments<double>(const Soa<double>&, const DevState*,
                                     const PushParams<double>&, const ForceParams&, double,
                                     double*, long long, cudaStream_t);
template void launch_force_terms<float>(const double*, const double*, const void*,
                                        const ForceParams&, double*, cudaStream_t);
template void launch_force_terms<double>(const double*, const double*, const void*,
                                         const ForceParams&, double*, cudaStream_t);
template void launch_fluid_model<float>(const double*, const void*, const ForceParams&,
                                        const PushParams<float>&, double*, cudaStream_t);
template void launch_fluid_model<double>(const double*, const void*, const ForceParams&,
                                         const PushParams<double>&, double*, cudaStream_t);

}  // namespace pic
