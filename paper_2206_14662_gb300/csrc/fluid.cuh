// fluid.cuh -- declarations of the fluid moments, force-balance terms and
// fluid-model predictions (moments.cu), shared with the C ABI (capi.cu).
#pragma once

#include "pic_internal.cuh"

namespace pic {

constexpr int kMoments = 12;   // n, n u (3), n <v v> (6), n <nu_d>, n <nu_io>
constexpr int kFluidModel = 9;  // fluid-model grids (launch_fluid_model)
struct ForceParams {
  int nr, nz, bkind;
  double r_in, hr, z_min, hz;
  double b0, L, z_mid;          // field: uniform b0, or the mirror about z_mid
  double weight;                // electrons per macro-electron
  double dt_prev;               // time since the previous moments (F_a), 0: none
};
// adds scale x the moments of simulation `sim`'s particles (its views s,
// st, P) on the nodes, per volume, to the kMoments x nnodes FP64 grids at M
template <typename Real>
void launch_moments(const Soa<Real>& s, const DevState* st, const PushParams<Real>& P,
                    const ForceParams& F, double scale, double* M, long long max_slots,
                    cudaStream_t stream);
// the 7 x 3 force-term grids (F_E, F_B, F_i, F_p, F_d, F_a, sum; r, theta,
// z) from moments M (and Mprev for F_a, or null) and the node field
template <typename Real>
void launch_force_terms(const double* M, const double* Mprev, const void* efield,
                        const ForceParams& F, double* out, cudaStream_t stream);
// the kFluidModel grids of the fluid-Poisson model's predictions at every
// node, from moments M, the node field and simulation P's cross sections
template <typename Real>
void launch_fluid_model(const double* M, const void* efield, const ForceParams& F,
                        const PushParams<Real>& P, double* out, cudaStream_t stream);

}  // namespace pic
