/*
 * pic_oracle.c -- plain, slow, FP64 CPU oracle for one particle step of the
 * axisymmetric (r,z) 2D3V electrostatic PIC with Monte-Carlo electron-neutral
 * collisions of Le Bars et al., "trapped electron clouds with a neutral gas
 * background" (arXiv 2206.14662), Sec. II.A.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA path; it follows
 * the method's steps in the order the paper states them, one particle at a
 * time, in double precision, with no blocking, fusion or reordering.  (With
 * OpenMP the particles' own steps run on several threads; every sum and the
 * list of children are still formed one particle after another in particle
 * order, so the results are bitwise those of one thread.)
 *
 * Steps of one particle step (leapfrog: position at n, velocity at n-1/2):
 *   1. gather  : bilinear interpolation of node E (Sec. II.A, standard PIC);
 *                analytic B (uniform, or a mirror field derived from
 *                A_theta = r Bz(z) / 2).
 *   2. push    : Boris kick-rotate-kick (Sec. II.A, cites Birdsall), then the
 *                straight move in the local Cartesian frame and the rotation
 *                of (vr, vtheta) back to the new local basis.
 *   3. absorb  : perfectly absorbing walls (Sec. II.A); the first wall the
 *                straight (r,z) segment crosses takes the charge.
 *   4. collide : null-collision Monte Carlo (Sec. II.A, Birdsall 1991 cited
 *                there): elastic scattering with a screened-Coulomb angle law
 *                (Okhrimovskyy family) and ionisation with binding-energy
 *                loss, Opal-type energy sharing, both electrons scattered and
 *                the ion dropped.
 *   5. deposit : finite-element weak-form right-hand side b_i = sum q w L_i.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written
 * here from that paper's definition; counter (uid_lo, uid_hi, step, draw),
 * key (seed_lo, seed_hi); uniforms ((x >> 8) + 0.5) * 2^-24.
 *
 * Pins (tests/test_oracle_pins.py): Philox known-answer vectors, the Boris
 * gyration closed form, ExB drift, canonical angular momentum, the mirror loss
 * cone, binomial collision counts, the angle-law mean and CDF, the ionisation
 * energy split and its CDF, charge conservation of the deposit, and the global
 * energy ledger.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA 2018 / exact SI values. */
#define OR_E    1.602176634e-19  /* elementary charge, C */
#define OR_ME   9.1093837015e-31 /* electron mass, kg */
#define OR_PI   3.14159265358979323846

typedef struct {
  double r_in, r_out, z_min, z_max; /* coaxial gap and axial extent, m */
  int32_t nr, nz;                   /* cells */
  int32_t bfield_kind;              /* 0 uniform Bz = b0; 1 mirror */
  int32_t elastic_recoil;           /* 1: elastic energy loss 2m/M(1-cos chi) */
  double b0;                        /* T */
  double n_gas;                     /* neutral density, m^-3 */
  double sigma_el;                  /* constant elastic cross-section, m^2 */
  double ion_E_th_eV, ion_sigma_pk, ion_E_pk_eV; /* ionisation fit */
  double opal_B_eV;                 /* energy-sharing width, eV */
  double xi;                        /* angle-law anisotropy, 0 = isotropic */
  double gas_mass_kg;
  double weight;                    /* physical electrons per macro-electron */
  double dt;                        /* s */
  double nu_max;                    /* null-collision majorant, s^-1 */
  uint64_t seed;
  double T0_eV;                     /* temperature of the seed source, eV */
  /* tabulated cross sections (Sec. II.A: momentum-transfer elastic and
   * total ionisation cross sections from tabulated data, and the angle
   * law's anisotropy): xs_n points (0: the analytic ones above) */
  int32_t xs_n;
  const double* xs_E_eV;            /* strictly increasing */
  const double* xs_sigma_el;        /* m^2 */
  const double* xs_sigma_io;        /* m^2 */
  const double* xs_xi;              /* NULL: the constant xi */
  /* 1: or_step's er/ez hold E at each particle (length n, e.g. the exact
   * gradient of a B-spline field) instead of node grids */
  int32_t e_per_particle;
  /* optional filled ellipse ((r - e_r0)/e_dr)^2 + ((z - e_z0)/e_dz)^2 <= 1
   * of metal (Sec. II.B's trap): particles entering it are absorbed */
  int32_t has_ellipse;
  double e_r0, e_z0, e_dr, e_dz;
} or_params;

/* tally slots (accumulated, doubles) */
enum {
  T_ABS_INNER = 0, T_ABS_OUTER, T_ABS_ZMIN, T_ABS_ZMAX, /* absorbed weight */
  T_WORK_E,          /* work of E on the particles, J (macro-weighted) */
  T_KE_ABSORBED,     /* kinetic energy carried into the walls, J */
  T_ION_LOSS,        /* binding energy removed by ionisation, J */
  T_RECOIL_LOSS,     /* elastic recoil loss, J */
  T_N_ELASTIC, T_N_IONISE, T_N_ABSORBED, T_N_OVER, T_N_CANDIDATE,
  T_ABS_ELLIPSE,     /* weight absorbed by the ellipse */
  T_COUNT
};

/* per-particle event codes */
enum { EV_NONE = 0, EV_ELASTIC = 1, EV_IONISE = 2, EV_NULL = 3,
       EV_WALL_INNER = 10, EV_WALL_OUTER = 11, EV_WALL_ZMIN = 12,
       EV_WALL_ZMAX = 13, EV_WALL_ELLIPSE = 14 };

/* ---------------------------------------------------------------- Philox */

/* Philox4x32 with 10 rounds: each round multiplies words 0 and 2 by the two
 * round constants into 64-bit products, mixes their high halves with words
 * 1 and 3 and the round key, and bumps the key by the Weyl constants. */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                      uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static double or_uniform(uint32_t x) {
  return ((double)(x >> 8) + 0.5) * (1.0 / 16777216.0);
}

/* four uniforms of the stream (uid, step, draw) */
static void or_draw4(const or_params* P, uint64_t uid, uint32_t step,
                     uint32_t draw, double u[4]) {
  uint32_t ctr[4] = {(uint32_t)uid, (uint32_t)(uid >> 32), step, draw};
  uint32_t key[2] = {(uint32_t)P->seed, (uint32_t)(P->seed >> 32)};
  uint32_t x[4];
  or_philox4x32_10(ctr, key, x);
  for (int k = 0; k < 4; ++k) u[k] = or_uniform(x[k]);
}

/* ------------------------------------------------------- cross sections */

/* ionisation fit: zero at threshold, sigma_pk at E_pk, ~1/E above */
double or_sigma_ion(const or_params* P, double E_eV) {
  if (E_eV <= P->ion_E_th_eV) return 0.0;
  double s = (E_eV - P->ion_E_th_eV) / (P->ion_E_pk_eV - P->ion_E_th_eV);
  return P->ion_sigma_pk * 2.0 * s / (1.0 + s * s);
}

/* Tabulated values at energy E (eV): the table point k with E_k <= E <
 * E_{k+1} found by bisection and f = f_k + w (f_{k+1} - f_k), w = (E -
 * E_k) / (E_{k+1} - E_k); at or below E_0 the first value (w = 0 on the
 * first segment), at or above E_{n-1} the last (w = 1 on the last). */
void or_xs_lookup(const or_params* P, double E_eV, double* sig_el, double* sig_io,
                  double* xi) {
  const int n = P->xs_n;
  const double* E = P->xs_E_eV;
  int k;
  double w;
  if (!(E_eV > E[0])) {
    k = 0;
    w = 0.0;
  } else if (!(E_eV < E[n - 1])) {
    k = n - 2;
    w = 1.0;
  } else {
    int lo = 0, hi = n - 1;   /* E[lo] <= E_eV < E[hi] */
    while (hi - lo > 1) {
      const int mid = (lo + hi) / 2;
      if (E[mid] <= E_eV) lo = mid;
      else hi = mid;
    }
    k = lo;
    w = (E_eV - E[k]) / (E[k + 1] - E[k]);
  }
  *sig_el = P->xs_sigma_el[k] + w * (P->xs_sigma_el[k + 1] - P->xs_sigma_el[k]);
  *sig_io = P->xs_sigma_io[k] + w * (P->xs_sigma_io[k + 1] - P->xs_sigma_io[k]);
  *xi = P->xs_xi ? P->xs_xi[k] + w * (P->xs_xi[k + 1] - P->xs_xi[k]) : P->xi;
}

/* collision frequencies at speed v, and the angle law's anisotropy there;
 * ionisation needs more energy than the binding energy whatever a table
 * says */
static void or_nu_xi(const or_params* P, double v, double* nu_el, double* nu_io, double* xi) {
  double E_eV = 0.5 * OR_ME * v * v / OR_E;
  if (P->xs_n > 0) {
    double se, si;
    or_xs_lookup(P, E_eV, &se, &si, xi);
    *nu_el = P->n_gas * se * v;
    *nu_io = E_eV > P->ion_E_th_eV ? P->n_gas * si * v : 0.0;
  } else {
    *nu_el = P->n_gas * P->sigma_el * v;
    *nu_io = P->n_gas * or_sigma_ion(P, E_eV) * v;
    *xi = P->xi;
  }
}
static void or_nu(const or_params* P, double v, double* nu_el, double* nu_io) {
  double xi;
  or_nu_xi(P, v, nu_el, nu_io, &xi);
}

/* elastic and ionisation frequencies at speed v; their sum is the
 * electron-neutral momentum-exchange frequency nu_d of the fluid force
 * balance (Sec. IV.A) */
void or_nu_parts(const or_params* P, double v, double* nu_el, double* nu_io) {
  or_nu(P, v, nu_el, nu_io);
}

/* Majorant: (1 + 1e-6) * max of nu_el + nu_io over E_k = E_cap k / 1e5,
 * k = 0..1e5, with E_cap in eV. */
double or_nu_max(const or_params* P, double E_cap_eV) {
  double best = 0.0;
  for (int k = 0; k <= 100000; ++k) {
    double E_eV = E_cap_eV * (double)k / 100000.0;
    double v = sqrt(2.0 * E_eV * OR_E / OR_ME);
    double a, b;
    or_nu(P, v, &a, &b);
    if (a + b > best) best = a + b;
  }
  return best * (1.0 + 1e-6);
}

/* ----------------------------------------------------------- scattering */

/* New direction after scattering through chi, with the pdf of mu = cos chi
 * proportional to (1 - xi mu)^-2 on [-1, 1]; its inverse CDF is
 * mu = 1 - 2u(1 - xi) / (1 + xi(1 - 2u)).  The azimuth is 2 pi u_phi about
 * the incident direction, measured from e1 = (vhat x zhat)/|vhat x zhat|
 * (rhat replaces zhat when vhat is within 1e-6 of the axis), e2 = vhat x e1.
 * Components are in the local (r, theta, z) basis. */
void or_scatter_dir(const double vhat[3], double u_chi, double u_phi,
                    double xi, double out[3]) {
  double mu = 1.0 - 2.0 * u_chi * (1.0 - xi) / (1.0 + xi * (1.0 - 2.0 * u_chi));
  double sn = sqrt(fmax(0.0, 1.0 - mu * mu));
  double phi = 2.0 * OR_PI * u_phi;
  double vr = vhat[0], vt = vhat[1], vz = vhat[2];
  /* vhat x zhat = (vt, -vr, 0) */
  double e1[3] = {vt, -vr, 0.0};
  double n1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  if (n1 < 1e-6) {
    /* vhat x rhat = (0, vz, -vt) */
    e1[0] = 0.0; e1[1] = vz; e1[2] = -vt;
    n1 = sqrt(e1[1] * e1[1] + e1[2] * e1[2]);
  }
  e1[0] /= n1; e1[1] /= n1; e1[2] /= n1;
  /* e2 = vhat x e1 */
  double e2[3] = {vt * e1[2] - vz * e1[1],
                  vz * e1[0] - vr * e1[2],
                  vr * e1[1] - vt * e1[0]};
  double cp = cos(phi), sp = sin(phi);
  for (int k = 0; k < 3; ++k)
    out[k] = mu * vhat[k] + sn * (cp * e1[k] + sp * e2[k]);
}

/* Secondary energy for ionisation: inverse CDF of the Lorentzian
 * 1/(1 + (E2/B)^2) on [0, E_rem/2]. */
double or_opal_secondary(double E_rem, double B, double u) {
  return B * tan(u * atan(E_rem / (2.0 * B)));
}

/* --------------------------------------------------------------- fields */

static void or_bfield(const or_params* P, double r, double z, double* br,
                      double* bz) {
  if (P->bfield_kind == 1) {
    double L = P->z_max - P->z_min;
    double zc = z - 0.5 * (P->z_min + P->z_max);
    double q = 2.0 * zc / L;
    *bz = P->b0 * (1.0 + 0.5 * q * q);
    *br = -2.0 * P->b0 * r * zc / (L * L); /* -(r/2) dBz/dz */
  } else {
    *bz = P->b0;
    *br = 0.0;
  }
}

/* bilinear cell location; the cell index is clamped to the grid */
static void or_locate(const or_params* P, double r, double z, int* i, int* j,
                      double* fr, double* fz) {
  double hr = (P->r_out - P->r_in) / P->nr;
  double hz = (P->z_max - P->z_min) / P->nz;
  double sr = (r - P->r_in) / hr, sz = (z - P->z_min) / hz;
  int ii = (int)floor(sr), jj = (int)floor(sz);
  if (ii < 0) ii = 0;
  if (ii > P->nr - 1) ii = P->nr - 1;
  if (jj < 0) jj = 0;
  if (jj > P->nz - 1) jj = P->nz - 1;
  *i = ii; *j = jj;
  *fr = sr - ii; *fz = sz - jj;
}

static void or_gather(const or_params* P, const double* er, const double* ez,
                      double r, double z, double* Er, double* Ez) {
  int i, j; double fr, fz;
  or_locate(P, r, z, &i, &j, &fr, &fz);
  int nzp = P->nz + 1;
  int n00 = i * nzp + j, n10 = (i + 1) * nzp + j;
  double w00 = (1 - fr) * (1 - fz), w10 = fr * (1 - fz);
  double w01 = (1 - fr) * fz, w11 = fr * fz;
  *Er = w00 * er[n00] + w10 * er[n10] + w01 * er[n00 + 1] + w11 * er[n10 + 1];
  *Ez = w00 * ez[n00] + w10 * ez[n10] + w01 * ez[n00 + 1] + w11 * ez[n10 + 1];
}

/* b_i += q w Lambda_i(r, z) on the four nodes of the particle's cell */
void or_deposit(const or_params* P, int64_t n, const double* r,
                const double* z, double* b) {
  double qw = -OR_E * P->weight;
  int nzp = P->nz + 1;
  for (int64_t p = 0; p < n; ++p) {
    int i, j; double fr, fz;
    or_locate(P, r[p], z[p], &i, &j, &fr, &fz);
    int n00 = i * nzp + j, n10 = (i + 1) * nzp + j;
    b[n00] += qw * (1 - fr) * (1 - fz);
    b[n10] += qw * fr * (1 - fz);
    b[n00 + 1] += qw * (1 - fr) * fz;
    b[n10 + 1] += qw * fr * fz;
  }
}

/* First entry of the straight (r,z) segment (r0,z0) -> (r1,z1) into the
 * filled ellipse: f(t) = X(t)^2 + Y(t)^2 - 1 with X, Y the normalised
 * offsets is a quadratic a t^2 + b t + c; a start inside (c <= 0) enters
 * at t = 0, otherwise at the smaller root if it lies in [0, 1].  Returns 1
 * and *t on entry; *f_least is the least f on the segment (the decision's
 * distance from its threshold). */
static int or_ellipse_entry(const or_params* P, double r0, double z0, double r1, double z1,
                            double* t, double* f_least) {
  double x0 = (r0 - P->e_r0) / P->e_dr, y0 = (z0 - P->e_z0) / P->e_dz;
  double dx = (r1 - r0) / P->e_dr, dy = (z1 - z0) / P->e_dz;
  double a = dx * dx + dy * dy, b = 2.0 * (x0 * dx + y0 * dy), c = x0 * x0 + y0 * y0 - 1.0;
  double tm = a > 0 ? fmin(fmax(-b / (2.0 * a), 0.0), 1.0) : 0.0;
  *f_least = (a * tm + b) * tm + c;
  if (c <= 0.0) { *t = 0.0; return 1; }
  if (*f_least > 0.0) return 0;
  double disc = b * b - 4.0 * a * c;
  *t = (-b - sqrt(fmax(disc, 0.0))) / (2.0 * a);
  return *t >= 0.0 && *t <= 1.0;
}

/* ----------------------------------------------------------------- step */

/* What one particle's step contributes to the step's sums and lists, kept
 * so that the sums can be formed afterwards in particle order. */
typedef struct {
  double work;       /* W_E of the two half kicks (macro-weighted), J */
  double ke_abs;     /* kinetic energy carried into a wall, J */
  double recoil;     /* elastic recoil loss, J */
  int wall;          /* -1, or 0..3 the walls, 4 the ellipse */
  int candidate;     /* passed the null-collision candidate test */
  int over;          /* nu_el + nu_io above the majorant */
  int kind;          /* EV_ELASTIC, EV_IONISE or 0 */
  double child[5];   /* r, z, vr, vt, vz of an ionisation's secondary */
} or_rec;

/* Gather, push, absorb and collide particle p: its new state, event and
 * margin are written in place, its contributions to the sums into *rec. */
static void or_advance(const or_params* P, int64_t p, double* r, double* z, double* vr,
                       double* vt, double* vz, const uint64_t* uid, int8_t* event,
                       double* margin, const double* er, const double* ez, uint32_t step,
                       or_rec* rec) {
  const double q = -OR_E, m = OR_ME;
  const double qmdt2 = q * P->dt / (2.0 * m);
  const double hr = (P->r_out - P->r_in) / P->nr;
  const double hz = (P->z_max - P->z_min) / P->nz;
  const double p_null = 1.0 - exp(-P->nu_max * P->dt);
  const double E_ion = P->ion_E_th_eV * OR_E;
  const double B_share = P->opal_B_eV * OR_E;
  rec->wall = -1;
  rec->candidate = rec->over = rec->kind = 0;
  double r0 = r[p], z0 = z[p];
  double v0[3] = {vr[p], vt[p], vz[p]};
  double Er, Ez, Br, Bz;
  if (P->e_per_particle) {
    Er = er[p];
    Ez = ez[p];
  } else {
    or_gather(P, er, ez, r0, z0, &Er, &Ez);
  }
  or_bfield(P, r0, z0, &Br, &Bz);
  /* Boris: half kick, rotation about B, half kick; components (r,theta,z) */
  double vm[3] = {v0[0] + qmdt2 * Er, v0[1], v0[2] + qmdt2 * Ez};
  double t[3] = {qmdt2 * Br, 0.0, qmdt2 * Bz};
  double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  double s[3] = {2 * t[0] / (1 + t2), 2 * t[1] / (1 + t2), 2 * t[2] / (1 + t2)};
  double vpr[3] = {vm[0] + (vm[1] * t[2] - vm[2] * t[1]),
                   vm[1] + (vm[2] * t[0] - vm[0] * t[2]),
                   vm[2] + (vm[0] * t[1] - vm[1] * t[0])};
  double vp[3] = {vm[0] + (vpr[1] * s[2] - vpr[2] * s[1]),
                  vm[1] + (vpr[2] * s[0] - vpr[0] * s[2]),
                  vm[2] + (vpr[0] * s[1] - vpr[1] * s[0])};
  double vn[3] = {vp[0] + qmdt2 * Er, vp[1], vp[2] + qmdt2 * Ez};
  /* exact work of the two half kicks: (q dt / 4) E . (v0 + vm + vp + vn) */
  rec->work = P->weight * (q * P->dt / 4.0) *
              (Er * (v0[0] + vm[0] + vp[0] + vn[0]) + Ez * (v0[2] + vm[2] + vp[2] + vn[2]));
  /* move in the local Cartesian frame (x along rhat, y along thetahat) */
  double x = r0 + vn[0] * P->dt, y = vn[1] * P->dt;
  double r1 = sqrt(x * x + y * y);
  double z1 = z0 + vn[2] * P->dt;
  /* absorbing walls: first crossing along the straight (r,z) segment */
  double mg = fmin(fmin(fabs(r1 - P->r_in), fabs(r1 - P->r_out)) / hr,
                   fmin(fabs(z1 - P->z_min), fabs(z1 - P->z_max)) / hz);
  int wall = -1;
  double tbest = 2.0;
  double tw[4] = {3.0, 3.0, 3.0, 3.0};
  if (r1 <= P->r_in) tw[0] = (P->r_in - r0) / (r1 - r0);
  if (r1 >= P->r_out) tw[1] = (P->r_out - r0) / (r1 - r0);
  if (z1 <= P->z_min) tw[2] = (P->z_min - z0) / (z1 - z0);
  if (z1 >= P->z_max) tw[3] = (P->z_max - z0) / (z1 - z0);
  for (int w = 0; w < 4; ++w)
    if (tw[w] < 3.0 && tw[w] < tbest) { tbest = tw[w]; wall = w; }
  if (P->has_ellipse) {
    double te, fm;
    int hit = or_ellipse_entry(P, r0, z0, r1, z1, &te, &fm);
    mg = fmin(mg, fabs(fm) * 0.5 * fmin(P->e_dr, P->e_dz) / fmin(hr, hz));
    if (hit && te < tbest) { tbest = te; wall = 4; }
  }
  if (wall >= 0) {
    double v2 = vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2];
    rec->wall = wall;
    rec->ke_abs = P->weight * 0.5 * m * v2;
    event[p] = (int8_t)(EV_WALL_INNER + wall);
    margin[p] = mg;
    r[p] = r1; z[p] = z1;
    vr[p] = vn[0]; vt[p] = vn[1]; vz[p] = vn[2];
    return;
  }
  /* rotate (vr, vtheta) into the basis at the new position */
  double c = x / r1, sn = y / r1;
  double v[3] = {c * vn[0] + sn * vn[1], -sn * vn[0] + c * vn[1], vn[2]};
  r[p] = r1; z[p] = z1;
  event[p] = EV_NONE;
  /* null-collision Monte Carlo */
  double u[4];
  or_draw4(P, uid[p], step, 0u, u);
  if (u[0] < p_null) {
    rec->candidate = 1;
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    double speed = sqrt(v2);
    double E = 0.5 * m * v2;
    double nu_el, nu_io, xi;
    or_nu_xi(P, speed, &nu_el, &nu_io, &xi);
    if (nu_el + nu_io > P->nu_max) rec->over = 1;
    double x1 = u[1] * P->nu_max;
    mg = fmin(mg, fmin(fabs(x1 - nu_el), fabs(x1 - nu_el - nu_io)) / P->nu_max);
    double vhat[3] = {v[0] / speed, v[1] / speed, v[2] / speed};
    if (x1 < nu_el) {
      double d[3];
      or_scatter_dir(vhat, u[2], u[3], xi, d);
      double E1 = E;
      if (P->elastic_recoil) {
        double mu = d[0] * vhat[0] + d[1] * vhat[1] + d[2] * vhat[2];
        E1 = E * (1.0 - (2.0 * m / P->gas_mass_kg) * (1.0 - mu));
        rec->recoil = P->weight * (E - E1);
      }
      double s1 = sqrt(2.0 * E1 / m);
      for (int k = 0; k < 3; ++k) v[k] = s1 * d[k];
      rec->kind = EV_ELASTIC;
      event[p] = EV_ELASTIC;
    } else if (x1 < nu_el + nu_io) {
      double u2[4];
      or_draw4(P, uid[p], step, 1u, u2);
      double E_rem = E - E_ion;
      double E2 = or_opal_secondary(E_rem, B_share, u2[0]);
      double E1 = E_rem - E2;
      double d1[3], d2[3];
      or_scatter_dir(vhat, u[2], u[3], xi, d1);
      or_scatter_dir(vhat, u2[1], u2[2], xi, d2);
      double s1 = sqrt(2.0 * E1 / m), s2 = sqrt(2.0 * E2 / m);
      for (int k = 0; k < 3; ++k) v[k] = s1 * d1[k];
      rec->child[0] = r1; rec->child[1] = z1;
      rec->child[2] = s2 * d2[0]; rec->child[3] = s2 * d2[1]; rec->child[4] = s2 * d2[2];
      rec->kind = EV_IONISE;
      event[p] = EV_IONISE;
    } else {
      event[p] = EV_NULL;
    }
  }
  margin[p] = mg;
  vr[p] = v[0]; vt[p] = v[1]; vz[p] = v[2];
}

/* Threads or_step may use (OpenMP builds; 1 otherwise).  The particles'
 * own work runs in parallel, every sum and list is formed afterwards in
 * particle order, so the results do not depend on the thread count. */
void or_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}
int or_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* One step for particles sorted by ascending uid.  Arrays are updated in
 * place; event[p] >= 10 marks an absorbed particle (the caller removes it).
 * Children are written to the c* arrays and get uids uid_next + k, k the
 * rank of the parent among this step's ionising parents (array order is uid
 * order).  margin[p] is the smallest distance of a discrete decision from
 * its threshold: walls in cells, collision-type tests relative to nu_max.
 * The surviving particles and the children are deposited into b.  er, ez
 * are node grids, or E at each particle when P->e_per_particle is set.
 * Each particle is advanced on its own (or_advance); its contributions to
 * the tallies and its child are then added in particle order, as a loop
 * over the particles one after another would add them.
 * Returns the number of children, or -1 if child_cap was too small (or
 * the record buffer could not be allocated). */
int64_t or_step(const or_params* P, int64_t n, double* r, double* z,
                double* vr, double* vt, double* vz, const uint64_t* uid,
                int8_t* event, double* margin, const double* er,
                const double* ez, uint32_t step, uint64_t uid_next,
                int64_t child_cap, double* cr, double* cz, double* cvr,
                double* cvt, double* cvz, uint64_t* cuid, double* b,
                double* tally) {
  const double q = -OR_E;
  const double E_ion = P->ion_E_th_eV * OR_E;
  const int64_t block = 32768;
  or_rec* rec = (or_rec*)malloc((size_t)(n < block ? (n > 0 ? n : 1) : block) * sizeof(or_rec));
  if (!rec) return -1;
  int64_t nchild = 0;
  for (int64_t p0 = 0; p0 < n; p0 += block) {
    const int64_t m = n - p0 < block ? n - p0 : block;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t k = 0; k < m; ++k)
      or_advance(P, p0 + k, r, z, vr, vt, vz, uid, event, margin, er, ez, step, &rec[k]);
    for (int64_t k = 0; k < m; ++k) {
      const or_rec* e = &rec[k];
      tally[T_WORK_E] += e->work;
      if (e->wall >= 0) {
        tally[e->wall == 4 ? T_ABS_ELLIPSE : T_ABS_INNER + e->wall] += P->weight;
        tally[T_KE_ABSORBED] += e->ke_abs;
        tally[T_N_ABSORBED] += 1.0;
        continue;
      }
      if (!e->candidate) continue;
      tally[T_N_CANDIDATE] += 1.0;
      if (e->over) tally[T_N_OVER] += 1.0;
      if (e->kind == EV_ELASTIC) {
        if (P->elastic_recoil) tally[T_RECOIL_LOSS] += e->recoil;
        tally[T_N_ELASTIC] += 1.0;
      } else if (e->kind == EV_IONISE) {
        if (nchild >= child_cap) {
          free(rec);
          return -1;
        }
        cr[nchild] = e->child[0]; cz[nchild] = e->child[1];
        cvr[nchild] = e->child[2]; cvt[nchild] = e->child[3]; cvz[nchild] = e->child[4];
        cuid[nchild] = uid_next + (uint64_t)nchild;
        ++nchild;
        tally[T_ION_LOSS] += P->weight * E_ion;
        tally[T_N_IONISE] += 1.0;
      }
    }
  }
  free(rec);
  /* deposit survivors and children at their new positions */
  double qw = q * P->weight;
  int nzp = P->nz + 1;
  for (int64_t p = 0; p < n + nchild; ++p) {
    double rp, zp;
    if (p < n) {
      if (event[p] >= EV_WALL_INNER) continue;
      rp = r[p]; zp = z[p];
    } else {
      rp = cr[p - n]; zp = cz[p - n];
    }
    int i, j; double fr, fz;
    or_locate(P, rp, zp, &i, &j, &fr, &fz);
    int n00 = i * nzp + j, n10 = (i + 1) * nzp + j;
    b[n00] += qw * (1 - fr) * (1 - fz);
    b[n10] += qw * fr * (1 - fz);
    b[n00 + 1] += qw * (1 - fr) * fz;
    b[n10 + 1] += qw * fr * fz;
  }
  return nchild;
}

/* Volumetric seed source (Sec. II.A: electrons created uniformly in space
 * with a Maxwellian velocity distribution): k new electrons with uids
 * uid0 .. uid0 + k - 1, born in step `step`.  Each draws from its own
 * stream: draw 2 gives (u_r, u_z, u_a, u_b), draw 3 gives (u_c, u_d, ., .);
 *   r = sqrt(a^2 + u_r (b^2 - a^2))      (uniform in the annulus' volume)
 *   z = z_min + u_z (z_max - z_min)
 *   vr, vt = vth sqrt(-2 ln u_a) (cos 2 pi u_b, sin 2 pi u_b)
 *   vz     = vth sqrt(-2 ln u_c) cos 2 pi u_d        (Box-Muller)
 * with vth = sqrt(e T0 / m_e).  The velocity is that of half step n + 1/2:
 * the particles first move in step n + 1. */
void or_source(const or_params* P, int64_t k, uint64_t uid0, uint32_t step,
               double* r, double* z, double* vr, double* vt, double* vz) {
  const double a2 = P->r_in * P->r_in, b2 = P->r_out * P->r_out;
  const double vth = sqrt(OR_E * P->T0_eV / OR_ME);
  for (int64_t j = 0; j < k; ++j) {
    double u[4], w[4];
    or_draw4(P, uid0 + (uint64_t)j, step, 2u, u);
    or_draw4(P, uid0 + (uint64_t)j, step, 3u, w);
    r[j] = sqrt(a2 + u[0] * (b2 - a2));
    z[j] = P->z_min + u[1] * (P->z_max - P->z_min);
    const double m1 = vth * sqrt(-2.0 * log(u[2]));
    vr[j] = m1 * cos(2.0 * OR_PI * u[3]);
    vt[j] = m1 * sin(2.0 * OR_PI * u[3]);
    vz[j] = vth * sqrt(-2.0 * log(w[0])) * cos(2.0 * OR_PI * w[1]);
  }
}

/* total kinetic energy of n macro-electrons, J */
double or_kinetic_energy(const or_params* P, int64_t n, const double* vr,
                         const double* vt, const double* vz) {
  double s = 0.0;
  for (int64_t p = 0; p < n; ++p)
    s += 0.5 * OR_ME * (vr[p] * vr[p] + vt[p] * vt[p] + vz[p] * vz[p]);
  return s * P->weight;
}
