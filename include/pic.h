/*
 * pic.h -- C ABI of libpic, a GB300 (sm_103a) implementation of one time
 * step of the axisymmetric (r,z) 2D3V electrostatic particle-in-cell method
 * with Monte-Carlo electron-neutral collisions of Le Bars et al.,
 * arXiv 2206.14662, Sec. II.A ("Numerical model"):
 *
 *   gather E at each macro-electron -> Boris push in cylindrical form ->
 *   perfectly absorbing walls -> null-collision elastic and ionisation
 *   collisions with a uniform neutral gas at rest -> charge deposit onto the
 *   (r,z) grid -> finite-element Poisson solve with Dirichlet metal walls and
 *   Neumann open ends -> node field E = -grad phi.
 *
 * Conventions for every call:
 *   - Units are SI.  Host arrays are FP64 unless stated; node arrays have
 *     (nr + 1) * (nz + 1) entries, node (i, j) at i * (nz + 1) + j, i along r
 *     (r_i = r_in + i h_r) and j along z (z_j = z_min + j h_z).
 *   - Return value: PIC_OK (0) or a negative PIC_E* code; pic_strerror()
 *     names it.  Errors found on the device (capacity, non-finite values,
 *     unconverged field solve) are sticky: they are latched in device memory
 *     and reported by the next synchronising call (pic_diagnostics,
 *     pic_export_particles, pic_get_grid); pic_step then returns the same
 *     code until particles are loaded again.
 *   - Ownership: the handle owns its device memory; the caller owns every
 *     host array it passes and the CUDA stream.  All device work is queued
 *     on that stream.  pic_step never synchronises; the calls that move data
 *     to or from the host (load, export, diagnostics, grids, field, solve,
 *     checkpoint, restore, profile stop) do.
 *   - Calls on one handle are not thread-safe.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PIC_OK = 0,
  PIC_EINVAL = -1,      /* bad argument or configuration */
  PIC_ENOMEM = -2,      /* device or host allocation failed */
  PIC_ECAPACITY = -3,   /* particle or spawn capacity exceeded */
  PIC_ENOCONV = -4,     /* field solve above poisson_rtol after poisson_maxit */
  PIC_ETIMEOUT = -5,    /* a bounded device wait ran out */
  PIC_ENONFINITE = -6,  /* a non-finite particle value was loaded or produced */
  PIC_ECUDA = -7        /* a CUDA runtime call failed */
};

/* Problem statement (Sec. II.A and II.B): geometry and electrode bias, the
 * applied magnetic field, the neutral gas (species mass, pressure and
 * temperature, uniform and constant), the seed load (n0, T0 of Sec. III.A),
 * the time step and the collision model parameters. */
typedef struct pic_config {
  double r_in, r_out;      /* inner / outer electrode radius a < b, m */
  double z_min, z_max;     /* open (Neumann) ends of the gap, m */
  int32_t nr, nz;          /* cells along r and z (2 <= nr <= 401,
                              2 <= nz <= 4096) */
  double v_inner, v_outer; /* Dirichlet potentials of the two walls, V */
  int32_t bfield_kind;     /* 0: uniform Bz = b0; 1: mirror
                              Bz = b0 (1 + 0.5 (2 zeta / L)^2),
                              Br = -2 b0 r zeta / L^2, zeta = z - z_mid */
  double b0;               /* T */
  double p_mbar, t_gas_K;  /* neutral density p / (k T) */
  double sigma_el;         /* elastic cross-section, constant, m^2 */
  double ion_E_th_eV;      /* ionisation threshold = binding energy, eV */
  double ion_sigma_pk;     /* peak ionisation cross-section, m^2 */
  double ion_E_pk_eV;      /* energy of the peak, eV; the fit is
                              sigma_pk 2 s / (1 + s^2),
                              s = (E - E_th) / (E_pk - E_th) */
  double opal_B_eV;        /* width of the secondary-energy law, eV */
  double xi_param;         /* angle-law anisotropy in [0, 1), 0 isotropic */
  int32_t elastic_recoil;  /* 1: elastic loss E (2 m_e / M)(1 - cos chi) */
  double gas_mass_amu;     /* neutral mass M, u */
  int64_t n_init;          /* macro-electrons of the seed load */
  double n0;               /* seed density, m^-3 (macro weight source) */
  double T0_eV;            /* temperature of the seed source, eV */
  double weight;           /* electrons per macro-electron; 0 derives
                              n0 pi (b^2 - a^2) L / n_init */
  double dt;               /* s */
  int32_t sort_every;      /* counting sort by cell every this many steps;
                              0 never */
  double poisson_rtol;     /* ||b - A phi|| / ||b_lifted|| bound */
  int32_t poisson_maxit;   /* refinement sweeps of the field solve */
  int64_t capacity;        /* particle slots; 0 derives 1.25 n_init + 4096 */
  uint64_t seed;           /* Philox key */
  int32_t precision;       /* particle path: 32 (FP32) or 64 (FP64) */
  double nu_max;           /* collision majorant, s^-1; 0 derives
                              (1 + 1e-6) max_E n (sigma_el + sigma_io(E)) v
                              over E = E_cap k / 1e5, k = 0..1e5,
                              E_cap = 2 |v_inner - v_outer| eV (with the
                              tables of pic_set_cross_sections once set) */
  int32_t fixed_efield;    /* 1: skip the field solve; E stays as set by
                              pic_set_efield (particle-only stepping) */
  int32_t warm_start;      /* initial guess of each field solve's
                              refinement: 0 zero, 1 the previous solve's
                              space-charge potential, 2 the learned guess
                              of an attached net (pic_attach_unet; the
                              previous potential until one is attached) */
  double source_rate;      /* volumetric seed source (Sec. II.A): macro-
                              electrons created per second, uniform in the
                              gap's volume, Maxwellian at T0_eV; 0 off */
  int32_t bspline_degree;  /* 0: bilinear node field; 1..3: the weighted
                              B-spline field of that degree (pic_spline_*)
                              with particle shapes from its basis: deposit
                              w(r) b_i(r) b_j(z), gather the exact -grad
                              phi.  Single simulations without a seed
                              source or a fixed field */
  int32_t has_ellipse;     /* 1: a filled metal ellipse at the outer
                              wall's potential (Sec. II.B's trap), needs
                              bspline_degree > 0: the field is the
                              web-spline field (pic_web_*, direct solve)
                              and electrons entering it are absorbed */
  double ellipse[4];       /* r centre, z centre, r semi-axis, z semi-axis, m */
} pic_config;

/* Diagnostics of one simulation (Sec. III.A: peak density and boundary
 * currents; the energy ledger and event counts are this library's). */
typedef struct pic_diag {
  int64_t step;                  /* steps taken */
  double t;                      /* step * dt, s */
  int64_t n_particles;           /* live macro-electrons */
  double I_inner, I_outer;       /* electron current into each wall, A,      */
  double I_zmin, I_zmax;         /*   averaged since the previous call       */
  double absorbed_weight[4];     /* cumulative electrons absorbed per wall:
                                    inner, outer, z_min, z_max */
  int64_t n_elastic, n_ionise, n_absorbed, n_candidates, n_over;
  int64_t n_pushed;              /* cumulative particle-steps (live
                                    particles advanced, summed over steps) */
  int64_t kernels_launched;      /* cumulative kernels run by pic_step */
  double ke_total_J;             /* kinetic energy of the live particles */
  double work_E_J;               /* cumulative work of E on the particles */
  double ke_absorbed_J;          /* cumulative kinetic energy into walls */
  double ion_loss_J;             /* cumulative binding energy removed */
  double recoil_loss_J;          /* cumulative elastic recoil loss */
  double ke_initial_J;           /* kinetic energy after the load */
  double ledger_residual_J;      /* ke_total - ke_initial - (work_E -
                                    ke_absorbed - ion_loss - recoil_loss) */
  double n_peak;                 /* largest node density, m^-3 */
  int32_t poisson_iters;         /* sweeps of the last field solve */
  double poisson_relres;         /* its residual relative to the right-hand
                                    side with the wall potentials moved into
                                    it (the convergence contract) */
  double poisson_relres_charge;  /* its residual relative to the charge
                                    alone (reported beside the contract) */
  double nu_max;                 /* collision majorant in use, s^-1 */
  double weight;                 /* macro weight in use */
  int32_t error;                 /* sticky error code (0 none) */
  double poisson_relres_init;    /* residual of the last solve's initial
                                    guess (warm starts), measured as
                                    poisson_relres; -1 after a cold start */
  int64_t n_source;              /* cumulative seed-source particles */
  double ke_source_J;            /* cumulative kinetic energy they brought
                                    (in the ledger: ledger_residual_J =
                                    ke_total - ke_initial - (work_E -
                                    ke_absorbed - ion_loss - recoil_loss +
                                    ke_source)) */
  double I_ellipse;              /* electron current into the ellipse, A
                                    (averaged as the wall currents) */
  double absorbed_ellipse;       /* cumulative electrons absorbed by it */
} pic_diag;

typedef struct pic_handle pic_handle;

/* Optional device allocator (for example a framework's caching allocator).
 * alloc returns a device pointer of at least `bytes` bytes, 256-byte
 * aligned, usable on `stream`, or NULL; free releases it. */
typedef struct pic_allocator {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, void* stream, void* ctx);
  void* ctx;
} pic_allocator;

/* Create a simulation, or a batch of n_sims simulations stepped together
 * (Sec. II.A: the PIC cycle; Sec. II.B: geometry and numerical parameters;
 * Sec. III: the parametric scans over pressure, voltage and magnetic field).
 * cfg points to n_sims configurations (1 <= n_sims <= 256).  The
 * simulations of a batch must agree in r_in, r_out, z_min, z_max, nr, nz,
 * dt, sort_every, poisson_rtol, poisson_maxit, precision, seed and
 * fixed_efield; everything else (wall potentials, field, gas, collision
 * parameters, particle count, weight, capacity) is per simulation.  The
 * random streams of simulation k use Philox counter word 1 = k (the high
 * word of its particles' 64-bit identity), so simulation 0 of a batch draws
 * exactly what a single run draws.  Validates cfg, derives the neutral
 * density, the macro weight and the collision majorant in FP64 on the host,
 * builds the field-solver tables and allocates all device memory (through
 * `alloc`, or cudaMalloc when alloc is NULL).  `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream).  No particles are loaded.
 * Returns PIC_EINVAL for an invalid configuration, PIC_ENOMEM, PIC_ECUDA. */
int pic_init(const pic_config* cfg, int n_sims, void* cuda_stream,
             const pic_allocator* alloc, pic_handle** out);

/* Load n macro-electrons into simulation `sim` (0 <= sim < n_sims) from
 * host FP64 arrays (structure of arrays): positions r, z (strictly inside
 * the gap), velocity components vr, vtheta, vz (the velocity at half step
 * -1/2 of the leapfrog) and unique uids (< 2^32 - 1, so that the uid
 * counter, max uid + 1, fits in 32 bits).  Replaces the
 * simulation's particles, resets its tallies and uid counter (max uid + 1),
 * deposits the charge and, unless fixed_efield, solves the field (Sec. II.A
 * seed load and first field; in a batch every simulation is solved again
 * from its last deposit, which leaves the others' fields as they were).  A
 * single simulation restarts at step 0 (with sort_every > 0 its store is
 * put in cell order right away, as the step's sort would); a simulation of
 * a batch joins at the batch's current step.  The arrays are checked on the
 * device after their copy; synchronises (page-locked host arrays make the
 * copies faster).  PIC_EINVAL for out-of-domain positions, uids at
 * or above 2^32 - 1, or n above the simulation's capacity; PIC_ENONFINITE
 * for a non-finite velocity (the first failing particle's code); a refused
 * load changes nothing.  The handle keeps the load's staging buffers (48 B
 * per particle of its largest load) until pic_free. */
int pic_load_particles(pic_handle* h, int sim, const double* r,
                       const double* z, const double* vr, const double* vt,
                       const double* vz, const uint64_t* uid, int64_t n);

/* Advance nsteps time steps (Sec. II.A): per step the fused particle kernel
 * (gather, Boris, absorb, null-collision MCC, spawn, deposit), child uid
 * assignment, the field solve and E = -grad phi; every sort_every steps a
 * counting sort by cell that also drops absorbed particles.  The Philox
 * stream of a particle is keyed by (seed) with counter (uid, step, draw).
 * Whole blocks of steps run as CUDA graphs (captured once, on a private
 * stream, the first time a block is reached; so the first call should come
 * before any capture of the caller's stream); while profiling (pic_profile)
 * every kernel is launched directly.  Asynchronous; never synchronises. */
int pic_step(pic_handle* h, int64_t nsteps);

/* Synchronise and fill *out; if density is not NULL, also write the node
 * density (b_i / q) / V_i of the last deposit ((nr + 1) * (nz + 1) FP64,
 * V_i the volume of the hat function).  Currents are averaged since the
 * previous call.  Returns the sticky error; a non-finite velocity among the
 * live particles, or a non-finite tally (a particle with non-finite values
 * reached a wall), latches PIC_ENONFINITE. */
int pic_diagnostics(pic_handle* h, int sim, pic_diag* out, double* density);

/* Synchronise and copy the live particles, sorted by uid, to host FP64
 * arrays of length cap.  *n receives the live count; PIC_ECAPACITY (and
 * nothing written) if cap is smaller. */
int pic_export_particles(pic_handle* h, int sim, double* r, double* z,
                         double* vr, double* vt, double* vz, uint64_t* uid,
                         int64_t cap, int64_t* n);

/* Replace the node field (E_r, E_z) used by the next step's gather.  Used
 * with fixed_efield = 1 for particle-only stepping in a given field.
 * Synchronises. */
int pic_set_efield(pic_handle* h, int sim, const double* er,
                   const double* ez);

/* Tabulated cross sections of simulation `sim` (Sec. II.A takes the
 * elastic momentum-transfer and the total ionisation cross sections from
 * tabulated data, and the scattering angle from an analytic law whose
 * anisotropy depends on the energy).  E_eV: n strictly increasing energies
 * >= 0 (eV), 2 <= n <= PIC_XS_MAX_POINTS; sigma_el_m2, sigma_io_m2: n
 * values >= 0 (m^2); xi: n anisotropies in [0, 1) of the angle law, or
 * NULL to keep the config's constant xi_param.  At energy E the values are
 * f_k + w (f_{k+1} - f_k), E_k <= E < E_{k+1}, w = (E - E_k) / (E_{k+1} -
 * E_k); the first (last) value holds at or below E_0 (at or above
 * E_{n-1}); sigma_io counts as 0 at or below ion_E_th_eV whatever the
 * table says.  The collision majorant is derived again from the tables as
 * at pic_init (unless the config set nu_max) and the step graphs are
 * rebuilt.  n = 0 (arrays ignored) returns to the config's analytic cross
 * sections.  The arrays are copied; the caller keeps them.  PIC_EINVAL on
 * a bad argument. */
#define PIC_XS_MAX_POINTS 1024

/* Fluid moments of simulation `sim`'s particles on the nodes (Sec. IV.A
 * evaluates the electron fluid's forces from moments of the distribution
 * function).  out: host array of PIC_MOMENTS grids of (nr + 1) (nz + 1)
 * FP64 (node i * (nz + 1) + j), in the order n, n u_r, n u_theta, n u_z,
 * n <v_r v_r>, n <v_r v_theta>, n <v_r v_z>, n <v_theta v_theta>,
 * n <v_theta v_z>, n <v_z v_z>, n <nu_d>, n <nu_io>, each
 * (w / V_i) sum_p Lambda_i(r_p, z_p) g(v_p) with the hat functions and
 * volumes of the density diagnostic, the particles' stored velocities (the
 * leapfrog's v^{n-1/2}), nu_d = n_gas (sigma_el + sigma_io) |v| (momentum
 * exchange) and nu_io = n_gas sigma_io |v| (ionisation), with the
 * collision path's cross sections (ionisation above its threshold).  Uses
 * a temporary device buffer; synchronises.  PIC_EINVAL on a bad handle,
 * index or NULL out; PIC_ENOMEM, PIC_ECUDA. */
#define PIC_MOMENTS 12
int pic_moments(pic_handle* h, int sim, double* out);

/* Adds scale x the moments of pic_moments (same layout and definitions) to
 * acc, a caller-owned DEVICE array of PIC_MOMENTS x (nr + 1) (nz + 1) FP64
 * (zeroed by the caller before the first call): the average over several
 * steps (Sec. IV.A averages over several cyclotron periods) accumulates on
 * the GPU with scale = 1 / (number of snapshots).  Asynchronous on the
 * handle's stream, no allocation, no host copy; acc must not be in use by
 * other work meanwhile.  PIC_EINVAL on a bad handle or index, NULL acc or a
 * non-finite scale; launch errors as PIC_ECUDA. */
int pic_moments_accumulate(pic_handle* h, int sim, double* acc, double scale);

/* The terms of the electron fluid's force balance (Sec. IV.A) at every
 * node from moments in the layout of pic_moments (host arrays, read only:
 * one call's moments, or averages over several steps): out (host) holds
 * PIC_FORCE_TERMS x 3 grids (components r, theta, z) of FP64 in N m^-3, in
 * the order F_E = q n E (the simulation's current node field), F_B =
 * q n u x B (B analytic), F_i = -m n (u . grad) u, F_p = -div P with
 * P = m (n <v v> - n u u), F_d = -m n <nu_d> u, F_a = m n (u - u_prev) /
 * dt_prev (zero when moments_prev is NULL), and the sum
 * F_i + F_E + F_B + F_p + F_d - F_a (q = -e, m = m_e).  Cylindrical
 * operators; derivatives by central differences, one-sided second order on
 * the boundary lines; u = 0 and P = 0 where n = 0.  Synchronises.
 * PIC_EINVAL on a bad handle or index, NULL moments or out, or
 * moments_prev with dt_prev <= 0; PIC_ENOMEM, PIC_ECUDA. */
#define PIC_FORCE_TERMS 7
int pic_force_balance(pic_handle* h, int sim, const double* moments,
                      const double* moments_prev, double dt_prev, double* out);

/* Predictions of the fluid-Poisson model (Sec. V.A: the force balance
 * without pressure, the continuity equation and Gauss's law) at every node
 * from moments in the layout of pic_moments (host, read only) and the
 * simulation's current node field.  out (host): PIC_FLUID_MODEL grids of
 * FP64, in the order
 *   u_theta = -E_r / B_z (m/s),
 *   <nu_d> = M_10 / n, <nu_io> = M_11 / n (1/s),
 *   u_r = -(q <nu_d> / m) E_r / (omega_p^2 - Omega_c^2) (m/s),
 *   omega_p,max^2 = Omega_c^2 <nu_io> / (<nu_io> + <nu_d>) (1/s^2),
 *   n_max = eps0 m omega_p,max^2 / e^2 (m^-3),
 *   nu_d and nu_io at the E x B drift speed |E x B| / |B|^2 (1/s, Sec. V.B's
 *   approximation),
 *   j = -eps0 E_r <nu_io> (A/m^2; the peak current is 2 pi L r_+ j at the
 *   cloud edge r_+),
 * with q = -e, m = m_e, Omega_c = e B_z / m, omega_p^2 = e^2 n / (eps0 m);
 * a value whose moment ratio has n = 0, or whose denominator is 0, is 0.
 * Averaging over time (the paper's <>_T) is the caller's: average the
 * moments, or the outputs.  Synchronises.  PIC_EINVAL on a bad handle or
 * index or NULL pointers; PIC_ENOMEM, PIC_ECUDA. */
#define PIC_FLUID_MODEL 9
int pic_fluid_model(pic_handle* h, int sim, const double* moments, double* out);

int pic_set_cross_sections(pic_handle* h, int sim, int n, const double* E_eV,
                           const double* sigma_el_m2, const double* sigma_io_m2,
                           const double* xi);

enum {
  PIC_GRID_PHI = 0,   /* potential phi, V */
  PIC_GRID_RHS = 1,   /* last deposit b_i = sum q w Lambda_i, C */
  PIC_GRID_ER = 2,    /* node field E_r in the particle precision, V/m */
  PIC_GRID_EZ = 3     /* node field E_z, V/m */
};

/* Synchronise and copy one node grid (see PIC_GRID_*) to host FP64. */
int pic_get_grid(pic_handle* h, int sim, int which, double* out);

/* Solve the field for a host right-hand side b (node array, C) and write
 * phi (host FP64): the same solver pic_step uses (Sec. II.A, finite
 * elements with Dirichlet walls and Neumann ends), with the wall potentials
 * of simulation 0.  Synchronises.  Leaves the simulations' own fields
 * untouched. */
int pic_solve_field(pic_handle* h, const double* b, double* phi,
                    double* relres);

/* Largest grid, in nodes (nr + 1) * (nz + 1), that pic_solve_field_static
 * accepts; the 128 x 512 benchmark grid has 66 177 nodes. */
#define PIC_STATIC_MAX_NODES 70000

/* The field solve of pic_solve_field for callers that cannot allocate
 * device memory (a framework that owns all device memory through its own
 * pool, a plug-in restricted to the buffers it is given, a service that must
 * not grow its footprint per call).  The paper has no counterpart: this is
 * a deployment variant of the same solve, with no handle.
 *   cfg     geometry, wall potentials and poisson_rtol (other fields unused)
 *   b       DEVICE pointer, right-hand side on all nodes (C), read only
 *   phi     DEVICE pointer, receives the potential on all nodes (V)
 *   relres  host pointer or NULL.  Non-NULL: the call synchronises the
 *           stream, stores the relative residual and returns PIC_ENOCONV if
 *           it exceeds poisson_rtol.  NULL: the work is only queued,
 *           and a solve that misses poisson_rtol is not reported.
 *   cuda_stream  cudaStream_t of the caller (NULL = legacy default stream)
 * Allocates nothing: its working memory is one fixed device array of about
 * 4 MB inside the library, which every GPU that loads the library keeps
 * until the process exits.  Grids above PIC_STATIC_MAX_NODES nodes, or with
 * nz > 4096 or nr > 401, return PIC_EINVAL before any device work.  All calls share that
 * array: calls whose GPU work overlaps (other streams, other host threads)
 * race and must be serialised by the caller.  The first call on each device
 * looks up the array's address with that device current; make it before
 * any stream capture. */
int pic_solve_field_static(const pic_config* cfg, const double* b, double* phi,
                           double* relres, void* cuda_stream);

/* Write the full state (particles, field, counters, tallies) to `path`;
 * pic_restore reads it into a handle made with the same configuration.
 * Stepping on after a restore gives the same particles as never stopping
 * (the random streams depend only on seed, uid and step).  Single
 * simulations only (PIC_EINVAL for a batch). */
int pic_checkpoint(pic_handle* h, const char* path);
int pic_restore(pic_handle* h, const char* path);

/* Device time of the step's kernels, measured with CUDA events recorded on
 * the handle's stream around each stage of every pic_step call made while
 * profiling is on.  enable = 1 starts (and clears) the record; enable = 0
 * stops it, synchronises and fills *out (out may be NULL when starting). */
typedef struct pic_kernel_times {
  double particle_ms;          /* fused particle kernel, total */
  int64_t particle_launches;
  double finalize_ms;          /* child-uid assignment, total */
  double field_ms;             /* field solve + E + residual check, total */
  int64_t field_solves;
  double sort_ms;              /* counting sorts, total */
  int64_t sorts;
  int64_t kernels_launched;    /* all kernels pic_step launched meanwhile */
} pic_kernel_times;
int pic_profile(pic_handle* h, int enable, pic_kernel_times* out);

/* Release the handle and its device memory (after the stream is idle). */
void pic_free(pic_handle* h);

/* Static string for a PIC_* code. */
const char* pic_strerror(int code);

/* ------------------------------------------------------------------------
 * Learned initial guess of the field solve.  The paper has no counterpart:
 * a four-level convolutional U-Net maps (charge, previous space-charge
 * potential) on the H x W node grid to a guess of the new space-charge
 * potential; the field solve then refines that guess to the same residual
 * bound (poisson_rtol), so the solver still decides convergence.
 *
 * Architecture (base width c, 1 <= c <= 32; H, W multiples of 8): per
 * level k = 1..4 at width c 2^(k-1) two 3 x 3 convolutions with bias and
 * ReLU, 2 x 2 average pooling between levels; back up through 2 x 2
 * transposed convolutions (stride 2, with bias, no activation) whose output
 * is concatenated before the level's skip activation and followed by two
 * 3 x 3 convolutions with ReLU; a 1 x 1 head to one channel.  The 3 x 3
 * layers are cross-correlations with zero padding:
 * out[y][x] = b + sum in[y + ky - 1][x + kx - 1] W[ky][kx].
 *
 * Flat parameter layout (FP32, host): for the layers enc1a, enc1b, enc2a,
 * enc2b, enc3a, enc3b, enc4a, enc4b, up3, dec3a, dec3b, up2, dec2a, dec2b,
 * up1, dec1a, dec1b, head in this order, the weights then the bias:
 * 3 x 3 layers W[ky][kx][in][out], transposed layers U[dy][dx][in][out]
 * (out[2y + dy][2x + dx] += in[y][x] U[dy][dx]), the head w[c] and one
 * bias.  Input channels of dec*a: the upsampled channels first, then the
 * skip channels.
 *
 * Arrays passed to the net are DEVICE pointers, FP32, (batch, H, W,
 * channels) with 2 input channels and 1 output channel.  Work is queued on
 * the net's stream; calls synchronise only where stated.
 * ---------------------------------------------------------------------- */
typedef struct pic_unet pic_unet;

/* Create a net for `batch` images of H x W.  precision 16: BF16
 * activations and weight copies, convolutions on the tensor cores with FP32
 * accumulation, FP32 master weights and Adam moments; precision 32: FP32
 * throughout (test mode).  Parameters start at zero; set them with
 * pic_unet_set_params.  PIC_EINVAL for unsupported sizes. */
int pic_unet_create(int base_channels, int H, int W, int batch, int precision,
                    void* cuda_stream, const pic_allocator* alloc,
                    pic_unet** out);
void pic_unet_free(pic_unet* net);
/* number of FP32 values of the flat parameter vector */
int64_t pic_unet_param_count(const pic_unet* net);
/* Which kernels the BF16 3 x 3 convolution GEMMs use: -1 (default) the
 * tcgen05 tensor-core kernel where its grid fills the GPU (at least two
 * CTAs of 8 x 16 pixels per SM), else the mma.sync kernel; 0 always
 * mma.sync; 1 tcgen05 wherever the shape allows (image height and width
 * multiples of 8 and 16, 32 to 256 output channels).  Results agree to
 * FP32 summation order.  This library's addition; the paper has no
 * counterpart.  PIC_EINVAL for another mode. */
int pic_unet_set_tensor_path(pic_unet* net, int mode);
/* host flat vector in / out (synchronise); set also clears the Adam
 * moments */
int pic_unet_set_params(pic_unet* net, const float* params);
int pic_unet_get_params(pic_unet* net, float* params);
/* y = net(x): x (batch, H, W, 2), y (batch, H, W) or NULL */
int pic_unet_forward(pic_unet* net, const float* x, float* y);
/* after pic_unet_forward: parameter gradients of sum(gy * y) (replacing
 * the previous ones), and the input gradient into gx (batch, H, W, 2) when
 * gx is not NULL */
int pic_unet_backward(pic_unet* net, const float* gy, float* gx);
/* host flat vector of the parameter gradients (synchronises) */
int pic_unet_get_grads(pic_unet* net, float* grads);
/* one Adam step (step number t >= 1) on the loss
 * sum (y - target)^2 / (2 batch H W); *loss (device, may be NULL) receives
 * the loss before the update */
int pic_unet_train_step(pic_unet* net, const float* x, const float* target,
                        float lr, float beta1, float beta2, float eps,
                        int64_t t, float* loss);

/* Use `net` (batch = n_sims, H = nr, W = nz) for the initial guess of the
 * field solves of a handle made with warm_start = 2 (NULL detaches): before
 * each solve the net reads, per simulation, the node charge of the step's
 * deposit over rho_scale (C) and the previous space-charge potential
 * phi_rho over phi_scale (V), node (i, j) as pixel (i - 1, j) for
 * i = 1..nr, j < nz, and the interior potential becomes
 * phi_rho + dphi_scale * output (node column nz takes pixel column
 * nz - 1).  The solve then refines that guess to poisson_rtol as usual.
 * The handle does not own the net; keep it alive while attached.
 * Synchronises.  PIC_EINVAL for a net of other dimensions. */
int pic_attach_unet(pic_handle* h, pic_unet* net, double rho_scale,
                    double phi_scale, double dphi_scale);

/* Schedule autotuner: tries sort periods {5, 10, 20, 40, 80} x fused-
 * kernel grids {1 .. resident blocks per SM} x SMs on the running
 * simulation, each over steps_per_trial steps (rounded up to a multiple of
 * 80) after an untimed graph block, times them with CUDA events on the
 * handle's stream and keeps the fastest (it replaces cfg.sort_every).  The
 * trials are ordinary steps: the simulation advances by all of them, and
 * its particles do not depend on the schedule (bit for bit in the FP32
 * path; in the FP64 path up to the order of the FP64 deposit sums).
 * Synchronises.  This library's addition; the paper has no counterpart. */
typedef struct pic_tune_result {
  int32_t sort_every;            /* chosen sort period, steps */
  int32_t particle_blocks;       /* chosen persistent grid of the fused
                                    kernel, blocks */
  double ms_per_step;            /* its measured time per step */
  int32_t trials;                /* candidates timed */
} pic_tune_result;
int pic_autotune(pic_handle* h, int64_t steps_per_trial, pic_tune_result* out);
/* The same with the caller's candidate sort periods (n_periods of them,
 * 1 .. 64, each 1 .. 100000): for instance only the periods that divide a
 * planned run's step count, so that the run holds whole sort periods.
 * Trials last a multiple of every candidate's graph block.  PIC_EINVAL on
 * a bad list.  This library's addition; the paper has no counterpart. */
int pic_autotune_periods(pic_handle* h, int64_t steps_per_trial, const int32_t* periods,
                         int n_periods, pic_tune_result* out);

/* Images of the current field state of every simulation, FP32 DEVICE
 * arrays of n_sims x nr x nz pixels in the net's layout (pixel (s, y, x) =
 * node (y + 1, x) of simulation s): the last deposit's node charge (C) and
 * the space-charge potential phi_rho = phi - phi_vac (V) of the last solve.
 * Either pointer may be NULL.  Queued on the handle's stream; checks the
 * sticky error (synchronises). */
int pic_field_images(pic_handle* h, float* rho, float* phi_rho);

/* ------------------------------------------------------------------
 * Weighted B-spline field of degree n (Sec. II.A: finite elements on
 * weighted B-splines of arbitrary degree, with the Dirichlet electrodes carried
 * by a weight function on a rectangular grid), with particle shapes from
 * the same basis.  Uniform B-splines b_i of degree n on knots extending n
 * cells past each end: mr = nr + n functions in r, mz = nz + n in z; the
 * coaxial walls carry the weight w(r) = (r - a)(b - r) / (b - a) and the
 * lift phi_D(r) = V_in + (V_out - V_in)(r - a) / (b - a):
 *   phi(r, z) = phi_D(r) + sum_ij c_ij w(r) b_i(r) b_j(z),
 * coefficient c_ij at i * mz + j.  Galerkin system (volume 2 pi r dr dz):
 *   (K_r (x) M_z + M_r (x) K_z) c = f / (2 pi eps0) - g_r (x) m_z
 * with K_r = int (w b_i)'(w b_k)' r dr, M_r = int w^2 b_i b_k r dr,
 * g_r = int phi_D' (w b_i)' r dr, K_z = int b_j' b_l' dz, M_z = int b_j b_l
 * dz, m_z = int b_j dz over [a, b] and [z_min, z_max]; the z ends are
 * natural (Neumann).  Geometry, grid and wall voltages come from a
 * pic_config (the other fields are ignored); 1 <= degree <=
 * PIC_SPLINE_MAX_DEGREE, nr + degree <= 1024 (the host eigen solve at
 * creation grows as (nr + degree)^3: under a second at 256 cells, about a
 * minute at 1024).
 * ------------------------------------------------------------------ */
#define PIC_SPLINE_MAX_DEGREE 5
typedef struct pic_spline pic_spline;

/* The 1D matrices (host only, no GPU): dense row-major K_r, M_r (mr x mr),
 * g_r (mr), K_z, M_z (mz x mz), m_z (mz); any pointer may be NULL.
 * PIC_EINVAL on a bad config or degree. */
int pic_spline_matrices(const pic_config* cfg, int degree, double* K_r, double* M_r,
                        double* g_r, double* K_z, double* M_z, double* m_z);

/* The generalised eigenpairs of (K_r, M_r) the solver uses (host only):
 * V (mr x mr, row-major, column k the k-th eigenvector) with V^T M_r V = I
 * and V^T K_r V = diag(lambda), lambda ascending.  PIC_ENOCONV if the
 * eigen solver did not converge. */
int pic_spline_eigen(const pic_config* cfg, int degree, double* V, double* lambda);

/* A solver on the current CUDA device: builds the tables on the host
 * (eigenpairs of (K_r, M_r), band Cholesky factors of lambda_k M_z + K_z
 * for every r-mode k) and copies them to device memory it owns (cudaMalloc,
 * freed by pic_spline_free).  Work is queued on cuda_stream (NULL: the
 * default stream).  PIC_EINVAL, PIC_ENOCONV, PIC_ENOMEM. */
int pic_spline_create(const pic_config* cfg, int degree, void* cuda_stream, pic_spline** out);
/* Frees the solver and its device memory (NULL is ignored); waits for
 * nothing: the caller makes sure no queued work still uses it. */
void pic_spline_free(pic_spline* s);
/* mr = nr + degree and mz = nz + degree (either pointer may be NULL).
 * PIC_EINVAL on a NULL solver. */
int pic_spline_sizes(const pic_spline* s, int* mr, int* mz);
/* The stream later calls queue on (NULL: the default stream). */
int pic_spline_set_stream(pic_spline* s, void* cuda_stream);

/* c = the Galerkin solution for the load f (DEVICE arrays of mr x mz
 * FP64; f is the charge term sum_p q w_p w(r_p) b_i(r_p) b_j(z_p), in C);
 * dirichlet = 0 solves with both walls at 0 V.  A direct solve: per
 * r-mode band solves (FP64, along z in segments) between two dense
 * transforms in double-float (FP32 pairs, about 2^-48 relative).
 * Asynchronous on the solver's stream.  PIC_EINVAL if f and c are the same
 * array. */
int pic_spline_solve(pic_spline* s, const double* f, double* c, int dirichlet);

/* f += qw w(r_p) b_i(r_p) b_j(z_p) for n particles at (r_p, z_p) (DEVICE
 * FP64 arrays; positions inside the gap are expected, others are charged
 * to the nearest cell's functions); FP64 atomics, asynchronous. */
int pic_spline_deposit(pic_spline* s, const double* r, const double* z, int64_t n, double qw,
                       double* f);

/* phi, E_r = -d phi/dr, E_z = -d phi/dz of coefficients c at n points
 * (DEVICE FP64 arrays; any of phi, er, ez may be NULL); dirichlet = 0
 * leaves out the lift phi_D.  Asynchronous. */
int pic_spline_eval(pic_spline* s, const double* c, const double* r, const double* z, int64_t n,
                    int dirichlet, double* phi, double* er, double* ez);

/* ------------------------------------------------------------------
 * Web-spline system for curved electrodes (Sec. II.A: weighted extended
 * B-splines carry curved Dirichlet surfaces on a rectangular grid; Sec.
 * II.B: the coaxial gap with a filled ellipse on the outer cylinder).
 * Host assembly, no GPU.  Domain: r_in < r < r_out, z_min < z < z_max of
 * cfg, minus the filled ellipse ((r - e0)/e2)^2 + ((z - e1)/e3)^2 <= 1 of
 * ellipse = {e0 (r centre), e1 (z centre), e2 (r semi-axis), e3 (z
 * semi-axis)} (NULL: none); V = v_inner on r_in, v_outer on r_out and on
 * the ellipse; natural ends in z.  B-spline grid: nr cells on [r_lo, r_hi]
 * (r_lo <= r_in, r_hi >= r_out: walls may lie between grid lines) and
 * cfg->nz cells on [z_min, z_max]; degree 1..PIC_SPLINE_MAX_DEGREE.
 * Weight: the R-function conjunction x + y - sqrt(x^2 + y^2) of
 * (r - r_in)(r_out - r)/(r_out - r_in) and min(e2, e3)/2 times the
 * ellipse's quadratic minus 1; lift V_in + dV (r - r_in)/(r - r_in + w_o),
 * w_o the conjunction of (r_out - r) and the ellipse weight.  Inner
 * B-splines (a whole grid cell of the support in the domain) carry the
 * outer ones (support meeting the domain only in cut cells) through
 * Lagrange coefficients on the nearest (n+1)^2 array of inner indices.
 * Output: A (n_inner x n_inner, CSR with sorted columns, row pointers of
 * n_inner + 1 ints) = T^T A_full T with A_full = eps0 int grad(w b_k) .
 * grad(w b_l) 2 pi r dr dz over the domain; g = T^T eps0 int grad(w b_k) .
 * grad(phi_D) dV (the load of the lift: solve A u = f_inner - g); the
 * full index (i * mz + j, mz = nz + degree) of each inner function; the
 * extension T (rows: mr * mz full functions, CSR).  Full coefficients of
 * phi - phi_D are c = T u.  PIC_EINVAL on bad arguments or a grid too
 * coarse for the geometry (an outer B-spline without an inner array). */
typedef struct pic_web pic_web;
int pic_web_create(const pic_config* cfg, const double* ellipse, double r_lo, double r_hi,
                   int nr, int degree, pic_web** out);
/* Frees the system and any device memory of pic_web_device (NULL is
 * ignored); the caller makes sure no queued work still uses it. */
void pic_web_free(pic_web* w);
/* The sizes of the exported arrays: inner functions, entries of A and of
 * T, and mr = nr + degree, mz = nz + degree (any pointer may be NULL).
 * PIC_EINVAL on a NULL system. */
int pic_web_sizes(const pic_web* w, int* n_inner, int64_t* nnz, int64_t* t_nnz, int* mr,
                  int* mz);
/* Copies out the arrays sized by pic_web_sizes; any pointer may be NULL. */
int pic_web_export(const pic_web* w, int* a_ptr, int* a_col, double* a_val, double* g,
                   int* inner_full, int* t_ptr, int* t_col, double* t_val);

/* A^-1 of the web-spline system (host only; n_inner^2 FP64, row-major,
 * by dense Cholesky: O(n_inner^3), seconds for a few thousand inner
 * functions).  PIC_ENOCONV if A is not positive definite. */
int pic_web_inverse(const pic_web* w, double* out);

/* Device side of a web-spline system on the current CUDA device: copies
 * the system, its extension and T^T to device memory owned by w (freed by
 * pic_web_free), and builds the preconditioner, the weighted B-spline
 * solver of the grid's box (pic_spline_create with walls at the grid's
 * ends).  Work is queued on cuda_stream.  PIC_ENOMEM, PIC_ENOCONV. */
int pic_web_device(pic_web* w, void* cuda_stream);

/* Solves A u = T^T f - [dirichlet] g by conjugate gradients preconditioned
 * with D P^T S^-1 P D (P: inner functions into the full basis, S: the box
 * solver, D = sqrt(diag(P^T S P) / diag A): the web functions near a
 * curved electrode carry a small weight), from u = 0, until ||r|| <= rtol ||b|| or maxit iterations; then
 * c = T u.  f (the particle load in the full basis, pic_web_deposit) and
 * c are DEVICE arrays of mr * mz FP64.  *iters, *relres (may be NULL) get
 * the count and the final relative residual.  Synchronises each
 * iteration.  PIC_ENOCONV if rtol was not met. */
int pic_web_solve(pic_web* w, const double* f, double* c, int dirichlet, double rtol, int maxit,
                  int* iters, double* relres);

/* Direct solve for time stepping: pic_web_direct (after pic_web_device)
 * makes A^-1 on the host and keeps it in device memory (n_inner^2 FP64:
 * 85 MB for 3260 inner functions, inside the L2); pic_web_solve_direct
 * then queues b = T^T f - [dirichlet] g, u = A^-1 b, c = T u with no host
 * synchronisation, so the solve can be captured in a CUDA graph. */
int pic_web_direct(pic_web* w);
/* The stream later device calls queue on (after pic_web_device). */
int pic_web_set_stream(pic_web* w, void* cuda_stream);
int pic_web_solve_direct(pic_web* w, const double* f, double* c, int dirichlet);

/* f_k += qw w(r_p, z_p) b_k(r_p, z_p) with the web weight (DEVICE arrays;
 * FP64 atomics), and phi, E = -grad phi of full coefficients c at points
 * (any output may be NULL; dirichlet = 0 leaves out the lift).
 * Asynchronous. */
int pic_web_deposit(pic_web* w, const double* r, const double* z, int64_t n, double qw,
                    double* f);
int pic_web_eval(pic_web* w, const double* c, const double* r, const double* z, int64_t n,
                 int dirichlet, double* phi, double* er, double* ez);

/* Potential-well depth (Sec. II.B: a well is a local maximum U_max of the
 * potential energy along a magnetic field line; its depth is U_max minus
 * the higher of the lowest values on either side) on the field lines
 * through (r_start[i], z1), i < lines (host array): each line is sampled
 * at `samples` equally spaced z over [z_min, z_max] with r^2 B_z(z) kept
 * (B_z = b0, or b0 (1 + 2 (z - z_mid)^2 / L^2) for bfield_kind 1), cut to
 * the stretch around z1 inside the domain, U = e phi in eV from the full
 * coefficients c (DEVICE, mr * mz FP64, with the lift).  depth[i] (eV)
 * and z_at[i] (z of the deepest well's maximum, NaN if none) are host
 * arrays.  Synchronises.  PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA. */
int pic_web_well_depth(pic_web* w, const double* c, const double* r_start, int lines, double z1,
                       int samples, int bfield_kind, double b0, double z_mid, double L,
                       double* depth, double* z_at);

#ifdef __cplusplus
}
#endif

#endif /* PIC_H */
