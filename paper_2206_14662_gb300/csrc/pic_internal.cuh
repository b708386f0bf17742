// pic_internal.cuh -- device data layout, kernel parameter blocks and the
// Philox generator of libpic (sm_103a).  Internal to the library.
//
// Particle store (structure of arrays, one slot per macro-electron):
//   cell  : int32, (ir << 16) | iz of the cell holding the particle, or -1
//           for an empty slot (absorbed particle awaiting the next sort)
//   offr, offz : position inside the cell in cell units, [0, 1)
//   vr, vt, vz : velocity in the local (r, theta, z) basis, m/s
//   uid   : uint32, the particle's random-stream identity
// Offsets and velocities are float in the FP32 path and double in the FP64
// path.  Holding positions as cell + offset keeps 24 (53) bits of the
// position inside its cell, whatever the cell index.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pic.h"

namespace pic {

// CODATA 2018 / exact SI values.
constexpr double kQe = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kKb = 1.380649e-23;
constexpr double kAmu = 1.66053906660e-27;
constexpr double kPi = 3.14159265358979323846;

// cumulative tallies in DevState::tally
enum Tally {
  kAbsInner = 0, kAbsOuter, kAbsZmin, kAbsZmax,  // absorbed weight per wall
  kWorkE,          // work of E, J
  kKeAbsorbed,     // kinetic energy into walls, J
  kIonLoss,        // binding energy removed by ionisation, J
  kRecoilLoss,     // elastic recoil loss, J
  kNElastic, kNIonise, kNAbsorbed, kNOver, kNCandidate,
  kNPushed,        // particle-steps taken (live particles advanced)
  kNSource,        // particles created by the seed source
  kKeSource,       // their kinetic energy, J
  kAbsEllipse,     // absorbed weight on the trap's ellipse
  kTallyCount
};

// Device-resident scalars of one simulation.  Every kernel reads its
// counters from here, so a fixed launch sequence can be captured in a graph.
struct DevState {
  long long n_slots;          // slots [0, n_slots) hold particles or holes
  long long n_spawn;          // children appended during the current step
  unsigned long long uid_next;
  unsigned int step;          // global step counter (Philox counter word 2)
  int err;                    // sticky PIC_E* code, 0 = none
  double tally[kTallyCount];
  // field solve: squared norms of the (scaled) right-hand side, of the
  // right-hand side with the wall potentials moved into it, and of the
  // residual of the current sweep; reset when a solve ends
  double b2sum, bl2sum, r2sum;
  double relres_last;         // ||r|| / ||b_lifted|| of the last solve
  double relres_strict;       // ||r|| / ||b_interior|| of the last solve
  unsigned solve_blocks_done; // last-block counter of the residual kernel
  int poisson_iters;          // sweeps of the last solve
  int solve_done;             // set when the solve has converged
  int chunk_next;             // the particle kernel's next chunk (handed out
                              // by atomics; reset by the spawn finalisation)
  long long n_live;           // live count after the last sort / load
  double relres_init;         // ||r|| / ||b_lifted|| of the last solve's
                              // initial guess (warm start), -1 if cold
  double src_acc;             // fractional seed-source count carried over
};

template <typename Real>
struct Soa {
  int* cell;
  Real* offr;
  Real* offz;
  Real* vr;
  Real* vt;
  Real* vz;
  unsigned* uid;
};

template <typename Real> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// Parameters of the fused particle kernel, in the particle precision.
template <typename Real>
struct PushParams {
  Real r_in, hr;              // radial grid
  Real z_min, hz;             // axial grid
  int nr, nz, bkind;          // cells, field kind
  Real qmdt2;                 // q dt / (2 m)
  Real dt;
  Real dt_hr, dt_hz;          // dt / h_r, dt / h_z
  Real zoff;                  // z_min - z_mid
  // the Boris rotation vector t = (q dt / 2m) B: t_z = tz0 + tzc zeta^2,
  // t_r = trc r zeta (mirror field; uniform: t_z = tz0, t_r = 0)
  Real tz0, tzc, trc;
  unsigned thr_null;          // candidate iff (x0 >> 8) < thr_null
  Real nsig_el;               // n_gas sigma_el, 1/m
  Real n_gas;
  Real e_th, e_span_inv;      // ionisation threshold (J), 1 / (E_pk - E_th)
  Real sig_pk;
  Real opal_b;                // J
  Real xi;
  Real recoil;                // 2 m_e / M, or 0 when recoil is off
  Real nu_max;
  Real half_m;                // m_e / 2
  Real two_over_m;            // 2 / m_e
  Real work_scale;            // q dt / 4 (times weight at the end)
  double weight;              // electrons per macro-electron
  double qw;                  // q weight, C
  unsigned seed_lo, seed_hi;
  unsigned uid_hi;            // Philox counter word 1: the high word of the
                              // particles' 64-bit identity, the index of the
                              // simulation in a batch (0 for a single run)
  unsigned rk0[10], rk1[10];  // Philox round keys of the seed
  long long capacity;         // particle slots
  long long spawn_cap;        // children per step
  long long base;             // first slot of the simulation's segment of the
                              // store (0 for a single run)
  double src_per_step;        // seed source: macro-electrons per step
  double vth_src;             // sqrt(e T0 / m_e), m/s
  double r_out_d, z_max_d;
  // grid geometry in FP64 for converting absolute positions to and from
  // (cell, offset) at load and export
  double r_in_d, hr_d, z_min_d, hz_d;
  // tabulated cross sections (pic_set_cross_sections): xs_n points, 0 for
  // the analytic ones; energies in J, n_gas sigma in 1/m, anisotropy xi
  // (xs_xi null: the constant xi)
  int xs_n;
  const Real* xs_E;
  const Real* xs_nel;
  const Real* xs_nio;
  const Real* xs_xi;
  // weighted B-spline field of degree spl_n (0: the bilinear node field):
  // its coefficients in the particle precision (mr x mz, row i at i spl_mz)
  // for the gather, the FP64 load grid for the deposit, the walls' weight
  // w = (r - r_in)(r_out - r) spl_inv_ab and the lift's slope spl_dphi
  int spl_n, spl_mz;
  const Real* spl_c;
  double* spl_f;
  Real spl_r_out, spl_inv_ab, spl_dphi;
  // the trap's metal ellipse (spl_ell): centre, inverse semi-axes, the
  // weight's scale min(dr, dz)/2 and the wall potential difference; the
  // weight and lift become the web-spline field's and electrons entering
  // the ellipse are absorbed
  int spl_ell;
  Real e_r0, e_z0, e_idr, e_idz, e_s, spl_dv;
  // FP32 tile deposit of the spline load: w b_k b_l / w_max (in [0, 1]:
  // w <= w_max = (r_out - r_in) / 4, the B-splines a partition of unity)
  // as fixed-point counts (kFixUnit a unit), each count spl_unit = q weight
  // w_max / kFixUnit of load
  Real spl_inv_wmax;
  double spl_unit;
};

// ------------------------------------------------------------- batches
// A batch holds nsim simulations on one grid geometry.  Simulation k owns
// the slots [base_k, base_k + capacity_k) of the store (base_k a multiple
// of the fused kernel's chunk), its own DevState, node grids at offset
// k * nodes and spawn records at offset k * spawn_stride.  Kernels that walk
// the particles of all simulations in one launch number the chunks of all
// segments consecutively: chunk c belongs to the simulation k with
// first[k] <= c < first[k + 1], first[] the prefix sum of each segment's
// ceil(n_slots / chunk).
constexpr int kMaxSims = 256;

struct SegInfo {
  long long base, capacity, spawn_cap;
};

// first[0..nsim] of the chunk table, built by one warp from the
// device-resident slot counts (call from every thread of the block; ends
// with a block barrier)
__device__ __forceinline__ void chunk_table(const DevState* st, int nsim, int chunk,
                                            int* first, long long* nslots) {
  if (threadIdx.x < 32) {
    int carry = 0;
    for (int k0 = 0; k0 < nsim; k0 += 32) {
      const int k = k0 + (int)threadIdx.x;
      long long n = 0;
      if (k < nsim) n = *(volatile const long long*)&st[k].n_slots;
      int c = (int)((n + chunk - 1) / chunk);
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)threadIdx.x >= o) incl += v;
      }
      if (k < nsim) {
        first[k] = carry + incl - c;
        nslots[k] = n;
      }
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (threadIdx.x == 0) first[nsim] = carry;
  }
  __syncthreads();
}

// simulation owning global chunk c (first[k] <= c < first[k + 1]; segments
// with no chunk are skipped)
__device__ __forceinline__ int chunk_owner(const int* first, int nsim, int c) {
  int lo = 0, hi = nsim - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= c) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename Real>
__host__ __device__ inline Soa<Real> soa_offset(const Soa<Real>& s, long long base) {
  Soa<Real> o;
  o.cell = s.cell + base; o.offr = s.offr + base; o.offz = s.offz + base;
  o.vr = s.vr + base; o.vt = s.vt + base; o.vz = s.vz + base; o.uid = s.uid + base;
  return o;
}

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications by the round constants, the high halves mixed
// with the other two words and the round key, which is advanced by the
// Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, unsigned k0,
                                               unsigned k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const unsigned lo0 = 0xD2511F53u * c.x;
    const unsigned hi0 = __umulhi(0xD2511F53u, c.x);
    const unsigned lo1 = 0xCD9E8D57u * c.z;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// The same generator with the ten round keys precomputed (they depend only
// on the seed): each round is two 32x32->64 multiplications and two
// three-input XORs.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const unsigned* rk0,
                                                  const unsigned* rk1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    c = make_uint4((unsigned)(p1 >> 32) ^ c.y ^ rk0[round], (unsigned)p1,
                   (unsigned)(p0 >> 32) ^ c.w ^ rk1[round], (unsigned)p0);
  }
  return c;
}

// Uniform (k + 0.5) 2^-24 of k = x >> 8.  FP64: exact.  FP32: the value
// needs 25 significant bits once k >= 2^23, so it is rounded once (an FMA of
// the exact k) and held below 1: exact for k < 2^23, otherwise within
// 2^-25 of the exact value, and always strictly inside (0, 1).  The
// collision candidate test does not use it (it compares k itself).
template <typename Real>
__device__ __forceinline__ Real u01(unsigned x) {
  return fminf(__fmaf_rn((float)(x >> 8), 0x1p-24f, 0x1p-25f), 0x1.fffffep-1f);
}
template <>
__device__ __forceinline__ double u01<double>(unsigned x) {
  return ((double)(x >> 8) + 0.5) * (1.0 / 16777216.0);
}

// Tabulated n_gas sigma_el, n_gas sigma_io and xi at energy E (J): the
// point k with E_k <= E < E_{k+1} by bisection, f = f_k + w (f_{k+1} -
// f_k); the first (last) value at or below E_0 (at or above E_{n-1}); xi0
// when there is no xi table.  (The particle step compiles it only into the
// kernels launched while some simulation has tables.)
template <typename Real>
struct Xs3 {
  Real nel, nio, xi;
};
template <typename Real>
__device__ __forceinline__ Xs3<Real> xs_eval(int n, const Real* __restrict__ Et,
                                          const Real* __restrict__ el,
                                          const Real* __restrict__ io,
                                          const Real* __restrict__ xt, Real xi0, Real E) {
  int k;
  Real w;
  if (!(E > Et[0])) {
    k = 0;
    w = 0;
  } else if (!(E < Et[n - 1])) {
    k = n - 2;
    w = 1;
  } else {
    int lo = 0, hi = n - 1;   // Et[lo] <= E < Et[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (Et[mid] <= E) lo = mid;
      else hi = mid;
    }
    k = lo;
    w = (E - Et[k]) / (Et[k + 1] - Et[k]);
  }
  Xs3<Real> r;
  r.nel = fma(w, el[k + 1] - el[k], el[k]);
  r.nio = fma(w, io[k + 1] - io[k], io[k]);
  r.xi = xt ? fma(w, xt[k + 1] - xt[k], xt[k]) : xi0;
  return r;
}

// ------------------------------------------------------------ host side

// Tables and work arrays of the field solver (field_solve.cu), all in
// device memory.  The solver works on the system divided by 2 pi eps0 and
// on the space-charge part phi_rho = phi - phi_vac only (phi_vac, the exact
// discrete vacuum solution, is precomputed in FP64); phi_rho is refined in
// double-float (pairs of floats, hi + lo) with an FP32 separable
// preconditioner.
struct FieldTables {
  int nr, nz, M, NI;          // cells, M = nz, NI = nr - 1 interior r-lines
  int log2N;                  // FFT length N = 2M = 2^log2N, or -1 (direct)
  int maxit;                  // refinement sweeps at most
  int warm;                   // 1: refine from the previous phi_rho
  double hr, hz, rtol;
  float inv2hr, inv2hz;       // 1 / (2 h) for the node-field differences
  double inv2hr_d, inv2hz_d;
  float hz32;                 // h_z
  float2* tw32;               // exp(-2 pi i m / N), m < N/2
  float* cos32;               // cos(pi m / M), m < 2M (direct transform)
  float* scale32;             // 2 eps_k / M, k = 0..M
  float* tri_a;               // per (interior line, mode): sub-diagonal
  float* tri_inv;             //   1 / pivot
  float* tri_cp;              //   super-diagonal / pivot
  double* phi_vac;            // vacuum solution per r-line (FP64)
  float* evac32;              // its radial field per r-line
  double* evac64;
  float2* kr_d; float2* kr_o; // r-weighted stiffness: diagonal, (i, i+1)  [hi, lo]
  float2* mr_d; float2* mr_o; // r-weighted mass                            [hi, lo]
  float2 mzd_end, mzd_in, mzo, kzd_end, kzd_in, kzo;  // z matrices [hi, lo]
  // A batch of nsim simulations shares the geometry and so every table
  // above except the vacuum solution; phi_vac, evac32 and evac64 hold
  // nsim blocks of nr + 1 entries, the arrays below nsim blocks of one grid
  // (nodes, or NI x (M+1) for bhat / phihat).  The kernels take the
  // simulation from their last grid dimension.
  int nsim;
  float2* b2;                 // right-hand side / (2 pi eps0), per node [hi, lo]
  float2* phir;               // phi_rho per node [hi, lo]; zero on the walls
  float* res;                 // FP32 input of the next sweep per node
  float* bhat;                // transformed input, NI x (M+1)
  float* phihat;              // transformed correction, NI x (M+1)
};

// Host staging of the tables (caller-owned arrays; sizes: kd..tmp_y and
// kd2..mo2 nr + 1, ta/tinv/tcp (nr - 1)(nz + 1), scale nz + 1, tw and cos
// 2 nz, evac32 nr + 1).
struct HostTables {
  double *kd, *ko, *md, *mo, *vac, *evac64, *tmp_cp, *tmp_y;
  float *ta, *tinv, *tcp, *scale, *tw, *cos, *evac32;
  float2 *kd2, *ko2, *md2, *mo2;
};
// fills T's scalar fields (nsim = 1) and the host tables (FP64
// arithmetic, no allocation)
void field_tables_host(const pic_config& cfg, FieldTables& T, const HostTables& H);
// copies the host tables into T's device arrays (which must exist; the
// vacuum tables into the block of simulation 0) and clears the work arrays
// of all T.nsim simulations; queued on `stream`
int field_tables_upload(FieldTables& T, const HostTables& H, cudaStream_t stream);
// allocates T's device arrays for nsim simulations with `dev_alloc`,
// builds and uploads the tables (the shared ones from cfgs[0], the vacuum
// solution of each simulation from its own wall potentials).  Returns
// PIC_OK or an error code.
int field_tables_build(const pic_config* cfgs, int nsim, FieldTables& T,
                       void* (*dev_alloc)(size_t, void*), void* ctx,
                       cudaStream_t stream);
float2 df_from(double x);   // double -> double-float (hi, lo)
constexpr double kFixUnit = 4194303.0;   // fixed-point deposit counts per particle charge
// Solve for the node charge given either as FP64 charges (rhs) or as
// fixed-point counts (cnt, charge = count * cnt_unit, or cnt_units[k] for
// simulation k when cnt_units is a device array); `cnt_clear`, when not
// null, is zeroed on the way (the next step's deposit buffer).  Writes the
// node field E = E_vac - grad phi_rho in the particle precision and latches
// PIC_ENOCONV in st if ||r|| / ||b_lifted|| > rtol after the last sweep.
// All T.nsim simulations are solved (grids at k * nodes, st + k).
template <typename Real>
void launch_field_solve(const FieldTables& T, const double* rhs,
                        const unsigned long long* cnt, double cnt_unit,
                        const float2* cnt_units, unsigned long long* cnt_clear,
                        void* efield, DevState* st, cudaStream_t stream);
// phi = phi_vac + phi_rho of simulation `sim` on all nodes (FP64)
void launch_phi_out(const FieldTables& T, double* phi, cudaStream_t stream, int sim = 0);
int field_solve_kernels(const FieldTables& T);   // launches per solve

// kernels launched from capi.cu (defined in particle_step.cu / sort.cu)
// rhs: FP64 deposit grid (FP64 path); cnt: fixed-point deposit grid (FP32
// path, kFix counts per particle charge)
template <typename Real>
void launch_particle_step(const Soa<Real>& s, const void* efield,
                          double* rhs, unsigned long long* cnt, DevState* st,
                          unsigned* spawn_parent, const PushParams<Real>& P,
                          int grid, cudaStream_t stream);
// spline mode: load of every stored particle into P.spl_f, and the gather
// copy of the coefficients
template <typename Real>
void launch_spline_deposit_store(const Soa<Real>& s, const DevState* st,
                                 const PushParams<Real>& P, long long max_slots,
                                 cudaStream_t stream);
template <typename Real>
void launch_spline_coef(const double* c, Real* out, int n, cudaStream_t stream);
void launch_spawn_finalize(DevState* st, unsigned* uid, const unsigned* parent,
                           long long spawn_cap, long long capacity,
                           cudaStream_t stream);
// a batch: the fused kernel over all simulations' chunks (params: device
// array of nsim PushParams, each with its segment base; tables: some
// simulation has tabulated cross sections), child uids per
// simulation, and the counting sort of every segment
template <typename Real>
void launch_particle_step_batch(const Soa<Real>& s, const void* efield, double* rhs,
                                unsigned long long* cnt, DevState* st,
                                unsigned* spawn_parent, long long spawn_stride,
                                const PushParams<Real>* params, int nsim, int nnodes,
                                bool tables, int grid, cudaStream_t stream);
// seed source of every simulation with src_per_step > 0 (after the child
// uids, before the sort and the field solve)
template <typename Real>
void launch_source(const Soa<Real>& s, DevState* st, const PushParams<Real>* params, int nsim,
                   double* rhs, unsigned long long* cnt, int nnodes, cudaStream_t stream);
void launch_spawn_finalize_batch(DevState* st, unsigned* uid, const unsigned* parent,
                                 long long spawn_stride, const SegInfo* seg, int nsim,
                                 cudaStream_t stream);
template <typename Real>
void launch_sort_batch(const Soa<Real>& src, const Soa<Real>& dst, DevState* st,
                       const SegInfo* seg, int nsim, int* cell_count, int ncells,
                       int nz, int grid, cudaStream_t stream);
template <typename Real>
void launch_deposit_only(const Soa<Real>& s, long long n, double* rhs,
                         unsigned long long* cnt, int nz, double qw,
                         cudaStream_t stream);
template <typename Real>
void launch_load(const double* r, const double* z, const double* vr,
                 const double* vt, const double* vz, const uint64_t* uid,
                 long long n, Soa<Real> s, const PushParams<Real>& P,
                 DevState* st, cudaStream_t stream);
template <typename Real>
void launch_export(const Soa<Real>& s, long long n_slots,
                   const PushParams<Real>& P, double* r, double* z,
                   double* vr, double* vt, double* vz,
                   unsigned long long* uid, int* live, cudaStream_t stream);
template <typename Real>
void launch_kinetic_energy(const Soa<Real>& s, DevState* st, double* out2,
                           cudaStream_t stream);
template <typename Real>
void launch_sort(const Soa<Real>& src, const Soa<Real>& dst, DevState* st,
                 int* cell_count, int ncells, int nz, int grid,
                 cudaStream_t stream);
template <typename Real>
void launch_efield_set(const double* er, const double* ez, void* efield,
                       int nnodes, cudaStream_t stream);
template <typename Real>
void launch_efield_get(const void* efield, double* out, int component,
                       int nnodes, cudaStream_t stream);

// learned initial guess (unet.cu): network input from the deposit (cnt with
// per-simulation charge units, or FP64 charges rhs) and phi_rho, forward
// pass on `stream`, phi_rho += dphi_scale * output on the interior lines
int warm_start_learned(pic_unet* net, const FieldTables& T, const unsigned long long* cnt,
                       const double* units, const double* rhs, float* xbuf, float rho_scale,
                       float phi_scale, float dphi_scale, cudaStream_t stream);
// (nsim, nr, nz) FP32 images of the deposit's charge and of phi_rho
int field_images(const FieldTables& T, const unsigned long long* cnt, const double* units,
                 const double* rhs, float* rho, float* phi, cudaStream_t stream);
bool unet_fits(const pic_unet* net, int nsim, int nr, int nz);
int unet_kernels_per_forward(const pic_unet* net);

}  // namespace pic
