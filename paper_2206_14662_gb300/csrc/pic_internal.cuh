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
  double res_num, res_den;    // squared residual sums (reset per solve)
  double relres_last;         // relative residual of the last solve
  unsigned solve_blocks_done; // last-block counter of the residual kernel
  int poisson_iters;          // sweeps of the last solve
  long long n_live;           // live count after the last sort / load
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
  Real r_in, hr, inv_hr;      // radial grid
  Real z_min, hz, inv_hz;     // axial grid
  Real z_mid, inv_L2, b0;     // magnetic field: mirror centre, 1/L^2
  int nr, nz, bkind;          // cells, field kind
  Real qmdt2;                 // q dt / (2 m)
  Real dt;
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
  long long capacity;         // particle slots
  long long spawn_cap;        // children per step
  // grid geometry in FP64 for converting absolute positions to and from
  // (cell, offset) at load and export
  double r_in_d, hr_d, z_min_d, hz_d;
};

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

// ((x >> 8) + 0.5) 2^-24: exact in float and double, strictly in (0, 1)
template <typename Real>
__device__ __forceinline__ Real u01(unsigned x) {
  return (Real)((x >> 8) + 0.5f) * (Real)(1.0 / 16777216.0);
}
template <>
__device__ __forceinline__ double u01<double>(unsigned x) {
  return ((double)(x >> 8) + 0.5) * (1.0 / 16777216.0);
}

// ------------------------------------------------------------ host side

// Tables of the fast field solver (field_solve.cu), all in device memory.
struct FieldTables {
  int nr, nz, M, NI;          // cells, M = nz, NI = nr - 1 interior r-lines
  int log2N;                  // FFT length N = 2M = 2^log2N, or -1 (direct)
  double hr, hz, rtol;
  double2* twiddle;           // exp(-2 pi i m / N), m < N/2
  double* costab;             // cos(pi m / M), m < 2M (direct transform)
  double* fwd_scale;          // 2 eps_k / (M 2 pi eps0), k = 0..M
  double* tri_a;              // per (interior line, mode): sub-diagonal
  double* tri_invd;           //   1 / pivot
  double* tri_cp;             //   super-diagonal / pivot
  double* phi_vac;            // vacuum solution per r-line (z-independent)
  double* kr_d; double* kr_o; // r-weighted stiffness: diagonal, (i, i+1)
  double* mr_d; double* mr_o; // r-weighted mass
  double* bhat;               // transformed right-hand side, NI x (M+1)
  double* phihat;             // transformed solution, NI x (M+1)
};

// builds the tables on the host (FP64) and uploads them; `dev_alloc`
// allocates device memory.  Returns PIC_OK or an error code.
int field_tables_build(const pic_config& cfg, FieldTables& T,
                       void* (*dev_alloc)(size_t, void*), void* ctx,
                       cudaStream_t stream);
void field_tables_free(FieldTables& T, void (*dev_free)(void*, void*),
                       void* ctx);
// phi <- solution for the right-hand side rhs (all nodes; Dirichlet rows of
// phi must already hold the wall potentials); then, when efield != NULL,
// E = -grad phi in the particle precision, the residual check, and
// rho_last <- rhs, rhs <- 0 when zero_rhs.
template <typename Real>
void launch_field_solve(const FieldTables& T, double* rhs, double* phi,
                        void* efield, double* rho_last, DevState* st,
                        bool zero_rhs, cudaStream_t stream);

// kernels launched from capi.cu (defined in particle_step.cu / sort.cu)
template <typename Real>
void launch_particle_step(const Soa<Real>& s, const void* efield,
                          double* rhs, DevState* st, unsigned* spawn_parent,
                          const PushParams<Real>& P, int grid,
                          cudaStream_t stream);
void launch_spawn_finalize(DevState* st, unsigned* uid, const unsigned* parent,
                           long long spawn_cap, long long capacity,
                           cudaStream_t stream);
template <typename Real>
void launch_deposit_only(const Soa<Real>& s, long long n, double* rhs, int nz,
                         double qw, cudaStream_t stream);
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

}  // namespace pic
