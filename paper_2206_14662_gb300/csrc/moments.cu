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
// The weights Lambda_i are the deposit's bilinear ones; accumulation is in
// FP64 global atomics, a warp whose particles share one cell adding its
// sums once.
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

#include "fluid.cuh"

namespace pic {

constexpr int kMomThreads = 256;

// elastic and ionisation frequencies at speed^2 v2
template <typename Real>
__device__ __forceinline__ void nu_parts(const PushParams<Real>& P, double v2, double& nu_el,
                                         double& nu_io) {
  const double speed = sqrt(v2);
  const double Ek = 0.5 * kMe * v2;
  if (P.xs_n > 0) {
    const Xs3<Real> x = xs_eval<Real>(P.xs_n, P.xs_E, P.xs_nel, P.xs_nio, P.xs_xi, P.xi, (Real)Ek);
    nu_el = (double)x.nel * speed;
    nu_io = Ek > (double)P.e_th ? (double)x.nio * speed : 0.0;
    return;
  }
  double sio = 0.0;
  if (Ek > (double)P.e_th) {
    const double qq = (Ek - (double)P.e_th) * (double)P.e_span_inv;
    sio = (double)P.sig_pk * 2.0 * qq / (1.0 + qq * qq);
  }
  nu_el = (double)P.nsig_el * speed;
  nu_io = (double)P.n_gas * sio * speed;
}

template <typename Real>
__global__ void __launch_bounds__(kMomThreads)
k_moments(Soa<Real> s, const DevState* st, PushParams<Real> P, double* M, int nnodes) {
  const long long n = st->n_slots;
  const int lane = threadIdx.x & 31, nzp = P.nz + 1;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n;
       base += (long long)gridDim.x * blockDim.x) {
    const long long p = base + threadIdx.x;
    const int cell = p < n ? s.cell[p] : -1;
    double c[4] = {0.0, 0.0, 0.0, 0.0};
    double g[kMoments];
    int n00 = 0;
    if (cell >= 0) {
      const int ir = cell >> 16, iz = cell & 0xFFFF;
      n00 = ir * nzp + iz;
      const double fr = (double)s.offr[p], fz = (double)s.offz[p];
      c[0] = (1.0 - fr) * (1.0 - fz);
      c[1] = fr * (1.0 - fz);
      c[2] = (1.0 - fr) * fz;
      c[3] = fr * fz;
      const double vr = (double)s.vr[p], vt = (double)s.vt[p], vz = (double)s.vz[p];
      g[0] = 1.0; g[1] = vr; g[2] = vt; g[3] = vz;
      g[4] = vr * vr; g[5] = vr * vt; g[6] = vr * vz;
      g[7] = vt * vt; g[8] = vt * vz; g[9] = vz * vz;
      double nel, nio;
      nu_parts<Real>(P, vr * vr + vt * vt + vz * vz, nel, nio);
      g[10] = nel + nio;
      g[11] = nio;
    } else {
#pragma unroll
      for (int k = 0; k < kMoments; ++k) g[k] = 0.0;
    }
    const int off[4] = {0, nzp, 1, nzp + 1};
    // one cell for the whole warp (sorted stores): sum in the warp first
    int same = 0;
    __match_all_sync(0xffffffffu, cell, &same);
    if (same && cell >= 0) {
#pragma unroll
      for (int k = 0; k < kMoments; ++k) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          double v = g[k] * c[j];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) atomicAdd(M + (size_t)k * nnodes + n00 + off[j], v);
        }
      }
    } else if (cell >= 0) {
#pragma unroll
      for (int k = 0; k < kMoments; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) atomicAdd(M + (size_t)k * nnodes + n00 + off[j], g[k] * c[j]);
    }
  }
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

__global__ void k_moment_scale(double* M, ForceParams F) {
  const int nnodes = (F.nr + 1) * (F.nz + 1);
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < nnodes; o += gridDim.x * blockDim.x) {
    const double s = F.weight / node_volume(F, o / (F.nz + 1), o % (F.nz + 1));
    for (int k = 0; k < kMoments; ++k) M[(size_t)k * nnodes + o] *= s;
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
    nu_parts<Real>(P, vd * vd, dnel, dnio);
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
                    const ForceParams& F, double* M, long long max_slots, cudaStream_t stream) {
  const int nnodes = (F.nr + 1) * (F.nz + 1);
  cudaMemsetAsync(M, 0, (size_t)kMoments * nnodes * sizeof(double), stream);
  const long long blocks = std::min<long long>((max_slots + kMomThreads - 1) / kMomThreads, 152 * 16);
  k_moments<Real><<<(int)std::max<long long>(blocks, 1), kMomThreads, 0, stream>>>(s, st, P, M,
                                                                                    nnodes);
  k_moment_scale<<<std::min(152 * 4, (nnodes + 255) / 256), 256, 0, stream>>>(M, F);
}

template <typename Real>
void launch_force_terms(const double* M, const double* Mprev, const void* efield,
                        const ForceParams& F, double* out, cudaStream_t stream) {
  const int nnodes = (F.nr + 1) * (F.nz + 1);
  k_force_terms<Real><<<std::min(152 * 4, (nnodes + 127) / 128), 128, 0, stream>>>(
      M, Mprev, (const typename Vec2<Real>::type*)efield, F, out);
}

template void launch_moments<float>(const Soa<float>&, const DevState*, const PushParams<float>&,
                                    const ForceParams&, double*, long long, cudaStream_t);
template void launch_moments<double>(const Soa<double>&, const DevState*,
                                     const PushParams<double>&, const ForceParams&, double*,
                                     long long, cudaStream_t);
template void launch_force_terms<float>(const double*, const double*, const void*,
                                        const ForceParams&, double*, cudaStream_t);
template void launch_force_terms<double>(const double*, const double*, const void*,
                                         const ForceParams&, double*, cudaStream_t);
template void launch_fluid_model<float>(const double*, const void*, const ForceParams&,
                                        const PushParams<float>&, double*, cudaStream_t);
template void launch_fluid_model<double>(const double*, const void*, const ForceParams&,
                                         const PushParams<double>&, double*, cudaStream_t);

}  // namespace pic
