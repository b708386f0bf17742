// capi.cu -- the C ABI of libpic (include/pic.h): handle life cycle, the
// per-step launch sequence, diagnostics, particle exchange and
// checkpointing.  Method: arXiv 2206.14662, Sec. II.A.
//
// Per step (pic_step), all on the caller's stream:
//   1. k_particle_step     gather, push, absorb, collide, spawn, deposit
//   2. k_spawn_finalize    child uids by parent rank; slot and step counters
//   3. every sort_every steps: counting sort into the other buffer set
//   4. field solve         DCT-I (z) / Thomas (r) / inverse DCT-I, then
//                          E = -grad phi and the residual check
// Counters live in device memory, so the host never waits inside pic_step.
//
// A handle holds nsim >= 1 simulations on one grid geometry (a parametric
// scan: pressure, wall potentials, field strength, particle count per
// simulation).  Simulation k owns a segment of the particle store, its own
// device state, grids and spawn records; a batch runs each stage above as
// one launch over all simulations (the fused kernel walks a prefix-sum table
// of every segment's chunks).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <type_traits>
#include <vector>

#include "pic_internal.cuh"
#include "fluid.cuh"

using namespace pic;

namespace pic {
int particle_step_blocks_per_sm(int precision, bool batch);
int particle_chunk();
}

// per-simulation quantities derived on the host in FP64, and host
// bookkeeping
struct SimHost {
  double n_gas, weight, nu_max, p_null, gas_mass;
  unsigned thr_null;
  long long capacity, spawn_cap, base;
  double ke_initial;
  double last_abs[4];
  double last_abs_ell = 0.0;
  long long last_diag_step;
};

// tabulated cross sections of one simulation (pic_set_cross_sections):
// the caller's tables and their device copy in the particle precision
// (energies in J, n_gas sigma in 1/m, xi), 4 x PIC_XS_MAX_POINTS values
struct XsHost {
  int n = 0;
  std::vector<double> E_eV, sigma_el, sigma_io, xi;
  void* dev = nullptr;
};

struct pic_handle {
  pic_config cfg;                 // simulation 0 (the shared geometry)
  std::vector<pic_config> cfgs;   // every simulation
  int nsim;
  int prec;
  cudaStream_t stream;
  pic_allocator alloc;
  bool has_alloc;
  std::vector<void*> owned;

  std::vector<SimHost> sims;
  std::vector<XsHost> xs;         // per simulation
  bool any_xs;                    // some simulation has tables
  double hr, hz;
  long long capacity;             // slots of all segments
  long long spawn_stride;         // spawn records per simulation
  int nnodes, ncells, grid_particle, grid_sort;
  int sms, blocks_per_sm;         // device SMs, resident fused-kernel blocks
  bool any_source;                // some simulation has a seed source

  // device memory
  DevState* st;                   // nsim entries
  SegInfo* seg;                   // nsim entries (batch kernels)
  float2* cnt_units;              // nsim fixed-point charge units / (2 pi eps0)
  PushParams<float>* Pf_dev;      // nsim entries (batch kernel)
  PushParams<double>* Pd_dev;
  double* q_units;                // nsim: charge (C) per fixed-point count

  // learned initial guess of the field solve (warm_start 2)
  pic_unet* net;
  float ws_scale[3];              // rho, phi_rho, correction scales
  float* ws_x;                    // network input, nsim x nr x nz x 2
  Soa<float> sf[2];
  Soa<double> sd[2];
  int cur;
  unsigned* spawn_parent;
  int* cell_count;
  double* rhs;                  // FP64 path: this step's deposit
  unsigned long long* cnt[2];   // FP32 path: fixed-point deposit grids
  int dep_buf, last_buf;        // FP32: buffer of the next / last deposit
  double* phi;
  void* efield;
  double* scratch2;   // two doubles for reductions
  // the load's staging buffers (five FP64 arrays and the uids), kept
  // between loads and grown to the largest one: a load allocates nothing
  // after the first (a fresh device allocation of a few hundred MB took
  // 30-40 ms on the GPU machine, against 4.5 ms for the whole load)
  void* stage[6] = {};
  size_t stage_n = 0;
  FieldTables T;

  // host bookkeeping
  long long step;
  int sticky;
  long long kernels;

  // CUDA graphs of whole blocks of steps, keyed by the buffer set holding
  // the particles (cur) and the FP32 deposit buffer (dep_buf) at the start
  // of the block; captured on a private stream, replayed on the caller's
  cudaStream_t cap_stream;
  int graph_len;                        // steps per graph
  // The child-uid kernel and the sort run on a second stream beside the
  // field solve (forked after the particle kernel, joined at the end of
  // the step) unless a seed source needs the child uids before the solve
  // or the stages are being timed; null: everything on one stream.
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;
  cudaGraphExec_t graph[2][2];
  long long graph_kernels[2][2];
  bool graph_failed;

  // profiling
  bool profiling;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_marks;   // (event index, stage tag)
  int ev_used;
  long long prof_kernels0;
  long long prof_counts[4];

  std::vector<PushParams<float>> Pf;   // per simulation
  std::vector<PushParams<double>> Pd;

  // weighted B-spline field (bspline_degree > 0, single simulation): the
  // solver, the FP64 load grid and coefficients (mr x mz), and the
  // coefficients in the particle precision for the gather
  pic_spline* spl = nullptr;
  pic_web* web = nullptr;           // has_ellipse: the web-spline field instead
  double* spl_f = nullptr;
  double* spl_c = nullptr;
  void* spl_cr = nullptr;
  int spl_cells = 0;
};

namespace {

void* default_alloc(size_t bytes, void*, void*) {
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  return p;
}
void default_free(void* p, void*, void*) { cudaFree(p); }

struct AllocCtx {
  pic_handle* h;
};

void* h_alloc(size_t bytes, void* ctx) {
  pic_handle* h = (pic_handle*)ctx;
  void* p = h->has_alloc ? h->alloc.alloc(bytes, (void*)h->stream, h->alloc.ctx)
                         : default_alloc(bytes, nullptr, nullptr);
  if (p) h->owned.push_back(p);
  return p;
}
void h_free_one(void* p, void* ctx) {
  pic_handle* h = (pic_handle*)ctx;
  if (h->has_alloc) h->alloc.free(p, (void*)h->stream, h->alloc.ctx);
  else default_free(p, nullptr, nullptr);
}

#define CK(call)                                  \
  do {                                            \
    if ((call) != cudaSuccess) return PIC_ECUDA;  \
  } while (0)

double sigma_ion_host(const pic_config& c, double E_eV) {
  if (E_eV <= c.ion_E_th_eV) return 0.0;
  const double s = (E_eV - c.ion_E_th_eV) / (c.ion_E_pk_eV - c.ion_E_th_eV);
  return c.ion_sigma_pk * 2.0 * s / (1.0 + s * s);
}

// sigma_el, sigma_io at E (eV): the config's analytic cross sections, or
// the tables by the rule of pic_set_cross_sections
void sigmas_host(const pic_config& c, const XsHost& X, double E_eV, double& sel, double& sio) {
  if (X.n == 0) {
    sel = c.sigma_el;
    sio = sigma_ion_host(c, E_eV);
    return;
  }
  const int n = X.n;
  const double* E = X.E_eV.data();
  int k = 0;
  double w = 0.0;
  if (!(E_eV > E[0])) {
    k = 0;
    w = 0.0;
  } else if (!(E_eV < E[n - 1])) {
    k = n - 2;
    w = 1.0;
  } else {
    k = (int)(std::upper_bound(E, E + n, E_eV) - E) - 1;
    w = (E_eV - E[k]) / (E[k + 1] - E[k]);
  }
  sel = X.sigma_el[k] + w * (X.sigma_el[k + 1] - X.sigma_el[k]);
  sio = E_eV > c.ion_E_th_eV ? X.sigma_io[k] + w * (X.sigma_io[k + 1] - X.sigma_io[k]) : 0.0;
}

// the collision majorant of simulation k and its null-collision threshold
void derive_nu_max(const pic_config& ck, const XsHost& X, SimHost& m) {
  if (ck.nu_max > 0) {
    m.nu_max = ck.nu_max;
  } else {
    const double E_cap = 2.0 * std::fabs(ck.v_inner - ck.v_outer);
    double best = 0.0;
    for (int q = 0; q <= 100000; ++q) {
      const double E_eV = E_cap * (double)q / 100000.0;
      const double v = std::sqrt(2.0 * E_eV * kQe / kMe);
      double sel, sio;
      sigmas_host(ck, X, E_eV, sel, sio);
      const double nu = m.n_gas * sel * v + m.n_gas * sio * v;
      if (nu > best) best = nu;
    }
    m.nu_max = best * (1.0 + 1e-6);
  }
  m.p_null = 1.0 - std::exp(-m.nu_max * ck.dt);
  const double cthr = m.p_null * 16777216.0 - 0.5;
  m.thr_null = cthr <= 0 ? 0u : (unsigned)std::min(16777216.0, std::ceil(cthr));
}

int validate(const pic_config& c) {
  if (!(c.r_in > 0 && c.r_out > c.r_in && c.z_max > c.z_min)) return PIC_EINVAL;
  // nz + 1 doubles of one z-line must fit the direct transform's 48 KB of
  // shared memory; cell indices are packed in 16 bits
  if (c.nr < 2 || c.nz < 2 || c.nr > 32767 || c.nz > 4096) return PIC_EINVAL;
  if (!(c.dt > 0) || !std::isfinite(c.dt)) return PIC_EINVAL;
  if (c.bfield_kind != 0 && c.bfield_kind != 1) return PIC_EINVAL;
  if (c.precision != 32 && c.precision != 64) return PIC_EINVAL;
  if (!(c.p_mbar >= 0) || !(c.t_gas_K > 0) || !(c.sigma_el >= 0)) return PIC_EINVAL;
  if (!(c.ion_E_pk_eV > c.ion_E_th_eV) || !(c.ion_E_th_eV > 0)) return PIC_EINVAL;
  if (!(c.opal_B_eV > 0) || !(c.xi_param >= 0 && c.xi_param < 1)) return PIC_EINVAL;
  if (!(c.gas_mass_amu > 0)) return PIC_EINVAL;
  if (c.weight <= 0 && (c.n_init <= 0 || !(c.n0 > 0))) return PIC_EINVAL;
  if (c.sort_every < 0 || c.capacity < 0) return PIC_EINVAL;
  if (!(c.poisson_rtol > 0) || c.poisson_maxit < 0 || c.poisson_maxit > 64) return PIC_EINVAL;
  if (c.warm_start < 0 || c.warm_start > 2) return PIC_EINVAL;
  if (!(c.source_rate >= 0) || !std::isfinite(c.source_rate)) return PIC_EINVAL;
  if (c.bspline_degree < 0 || c.bspline_degree > 3) return PIC_EINVAL;
  if (c.bspline_degree > 0 && (c.source_rate > 0 || c.fixed_efield)) return PIC_EINVAL;
  if (c.has_ellipse && (c.bspline_degree <= 0 || !(c.ellipse[2] > 0) || !(c.ellipse[3] > 0)))
    return PIC_EINVAL;
  if (c.source_rate > 0 && !(c.T0_eV > 0)) return PIC_EINVAL;
  // the Thomas sweep keeps four (nr - 1) x 32 float columns in shared memory
  if ((long long)4 * (c.nr - 1) * 32 * 4 > 200 * 1024) return PIC_EINVAL;
  if ((long long)(c.nr + 1) * (c.nz + 1) > (1ll << 30)) return PIC_EINVAL;
  return PIC_OK;
}

// simulations of one handle share the grid geometry, the time step, the
// sort and field-solve settings, the precision and the seed (each
// simulation's particles draw from the counter block of its index)
int validate_batch(const pic_config* c, int n) {
  const pic_config& a = c[0];
  for (int k = 1; k < n; ++k) {
    const pic_config& b = c[k];
    if (b.r_in != a.r_in || b.r_out != a.r_out || b.z_min != a.z_min || b.z_max != a.z_max ||
        b.nr != a.nr || b.nz != a.nz || b.dt != a.dt || b.sort_every != a.sort_every ||
        b.poisson_rtol != a.poisson_rtol || b.poisson_maxit != a.poisson_maxit ||
        b.precision != a.precision || b.seed != a.seed || b.fixed_efield != a.fixed_efield ||
        b.warm_start != a.warm_start)
      return PIC_EINVAL;
  }
  return PIC_OK;
}

template <typename Real>
void fill_params(pic_handle* h, int k, PushParams<Real>& P) {
  const pic_config& c = h->cfgs[k];
  const SimHost& m = h->sims[k];
  const double L = c.z_max - c.z_min;
  P.r_in = (Real)c.r_in; P.hr = (Real)h->hr;
  P.z_min = (Real)c.z_min; P.hz = (Real)h->hz;
  P.nr = c.nr; P.nz = c.nz; P.bkind = c.bfield_kind;
  P.qmdt2 = (Real)(-kQe * c.dt / (2.0 * kMe));
  P.dt = (Real)c.dt;
  P.dt_hr = (Real)(c.dt / h->hr);
  P.dt_hz = (Real)(c.dt / h->hz);
  P.zoff = (Real)(c.z_min - 0.5 * (c.z_min + c.z_max));
  {
    const double q = -kQe * c.dt / (2.0 * kMe), il2 = 1.0 / (L * L);
    P.tz0 = (Real)(q * c.b0);
    P.tzc = (Real)(c.bfield_kind == 1 ? 2.0 * q * c.b0 * il2 : 0.0);
    P.trc = (Real)(c.bfield_kind == 1 ? -2.0 * q * c.b0 * il2 : 0.0);
  }
  P.thr_null = m.thr_null;
  P.nsig_el = (Real)(m.n_gas * c.sigma_el);
  P.n_gas = (Real)m.n_gas;
  P.e_th = (Real)(c.ion_E_th_eV * kQe);
  P.e_span_inv = (Real)(1.0 / ((c.ion_E_pk_eV - c.ion_E_th_eV) * kQe));
  P.sig_pk = (Real)c.ion_sigma_pk;
  P.opal_b = (Real)(c.opal_B_eV * kQe);
  P.xi = (Real)c.xi_param;
  P.recoil = c.elastic_recoil ? (Real)(2.0 * kMe / m.gas_mass) : (Real)0;
  P.nu_max = (Real)m.nu_max;
  P.half_m = (Real)(0.5 * kMe);
  const XsHost& X = h->xs[k];
  const bool tab = X.n > 0 && X.dev && h->prec == (int)(8 * sizeof(Real));
  const Real* xd = (const Real*)X.dev;
  P.xs_n = tab ? X.n : 0;
  P.xs_E = tab ? xd : nullptr;
  P.xs_nel = tab ? xd + PIC_XS_MAX_POINTS : nullptr;
  P.xs_nio = tab ? xd + 2 * PIC_XS_MAX_POINTS : nullptr;
  P.xs_xi = tab && !X.xi.empty() ? xd + 3 * PIC_XS_MAX_POINTS : nullptr;
  P.two_over_m = (Real)(2.0 / kMe);
  P.work_scale = (Real)(-kQe * c.dt / 4.0);
  P.weight = m.weight;
  P.qw = -kQe * m.weight;
  P.seed_lo = (unsigned)(c.seed & 0xFFFFFFFFull);
  P.seed_hi = (unsigned)(c.seed >> 32);
  P.uid_hi = (unsigned)k;
  for (int r = 0; r < 10; ++r) {
    P.rk0[r] = P.seed_lo + (unsigned)r * 0x9E3779B9u;
    P.rk1[r] = P.seed_hi + (unsigned)r * 0xBB67AE85u;
  }
  P.capacity = m.capacity;
  P.spawn_cap = m.spawn_cap;
  P.base = m.base;
  P.src_per_step = c.source_rate > 0 ? c.source_rate * c.dt : 0.0;
  P.vth_src = std::sqrt(kQe * c.T0_eV / kMe);
  P.r_out_d = c.r_out;
  P.z_max_d = c.z_max;
  P.r_in_d = c.r_in;
  P.hr_d = h->hr;
  P.z_min_d = c.z_min;
  P.hz_d = h->hz;
  const bool spl = (h->spl || h->web) && h->prec == (int)(8 * sizeof(Real));
  P.spl_n = spl ? c.bspline_degree : 0;
  P.spl_mz = c.nz + c.bspline_degree;
  P.spl_c = spl ? (const Real*)h->spl_cr : nullptr;
  P.spl_f = spl ? h->spl_f : nullptr;
  P.spl_r_out = (Real)c.r_out;
  P.spl_inv_ab = (Real)(1.0 / (c.r_out - c.r_in));
  P.spl_dphi = (Real)((c.v_outer - c.v_inner) / (c.r_out - c.r_in));
  P.spl_ell = spl && h->web ? 1 : 0;
  P.e_r0 = (Real)c.ellipse[0];
  P.e_z0 = (Real)c.ellipse[1];
  P.e_idr = (Real)(c.ellipse[2] > 0 ? 1.0 / c.ellipse[2] : 0.0);
  P.e_idz = (Real)(c.ellipse[3] > 0 ? 1.0 / c.ellipse[3] : 0.0);
  P.e_s = (Real)(0.5 * std::min(c.ellipse[2], c.ellipse[3]));
  P.spl_dv = (Real)(c.v_outer - c.v_inner);
  P.spl_inv_wmax = (Real)(4.0 / (c.r_out - c.r_in));
  P.spl_unit = P.qw * (0.25 * (c.r_out - c.r_in)) / kFixUnit;
}

// spline mode: the solver on the handle's geometry and its grids
int spline_setup(pic_handle* h) {
  const pic_config& c = h->cfg;
  int mr = 0, mz = 0;
  if (c.has_ellipse) {
    // the trap: web-spline system on the gap's grid, solved through its
    // dense inverse kept on the device (graph-capturable)
    int rc = pic_web_create(&c, c.ellipse, c.r_in, c.r_out, c.nr, c.bspline_degree, &h->web);
    if (!rc) rc = pic_web_device(h->web, h->stream);
    if (!rc) rc = pic_web_direct(h->web);
    if (rc) return rc;
    pic_web_sizes(h->web, nullptr, nullptr, nullptr, &mr, &mz);
  } else {
    const int rc = pic_spline_create(&c, c.bspline_degree, h->stream, &h->spl);
    if (rc) return rc;
    pic_spline_sizes(h->spl, &mr, &mz);
  }
  h->spl_cells = mr * mz;
  const size_t cells = (size_t)h->spl_cells;
  h->spl_f = (double*)h_alloc(cells * sizeof(double), h);
  h->spl_c = (double*)h_alloc(cells * sizeof(double), h);
  h->spl_cr = h_alloc(cells * (h->prec == 32 ? sizeof(float) : sizeof(double)), h);
  if (!h->spl_f || !h->spl_c || !h->spl_cr) return PIC_ENOMEM;
  return cudaMemsetAsync(h->spl_f, 0, cells * sizeof(double), h->stream) == cudaSuccess
             ? PIC_OK
             : PIC_ECUDA;
}

// spline mode: coefficients of the load in spl_f (solve on the handle's
// current stream) and their copy in the particle precision
int spline_solve_into(pic_handle* h) {
  int rc;
  if (h->web) {
    pic_web_set_stream(h->web, h->stream);
    rc = pic_web_solve_direct(h->web, h->spl_f, h->spl_c, 1);
  } else {
    pic_spline_set_stream(h->spl, h->stream);
    rc = pic_spline_solve(h->spl, h->spl_f, h->spl_c, 1);
  }
  if (rc) return rc;
  if (h->prec == 32)
    launch_spline_coef<float>(h->spl_c, (float*)h->spl_cr, h->spl_cells, h->stream);
  else
    launch_spline_coef<double>(h->spl_c, (double*)h->spl_cr, h->spl_cells, h->stream);
  return PIC_OK;
}

template <typename Real>
int alloc_soa(pic_handle* h, Soa<Real>& s) {
  // whole chunks of the fused kernel: its bulk copies read full chunks
  const size_t ch = (size_t)particle_chunk();
  const size_t n = ((size_t)h->capacity + ch - 1) / ch * ch;
  auto al = [&](size_t bytes) { return h_alloc(std::max<size_t>(bytes, 256), h); };
  s.cell = (int*)al(n * sizeof(int));
  s.offr = (Real*)al(n * sizeof(Real));
  s.offz = (Real*)al(n * sizeof(Real));
  s.vr = (Real*)al(n * sizeof(Real));
  s.vt = (Real*)al(n * sizeof(Real));
  s.vz = (Real*)al(n * sizeof(Real));
  s.uid = (unsigned*)al(n * sizeof(unsigned));
  if (!s.cell || !s.offr || !s.offz || !s.vr || !s.vt || !s.vz || !s.uid) return PIC_ENOMEM;
  return PIC_OK;
}

// A graph block returns the alternating buffers (sort ping-pong, FP32
// deposit buffers) to a fixed pattern: lcm(sort_every, 2) steps, at least 8.
int graph_len_of(int se) {
  int len = se > 0 ? (se % 2 == 0 ? se : 2 * se) : 2;
  while (len < 8) len *= 2;
  return len;
}

void set_graph_len(pic_handle* h) { h->graph_len = graph_len_of(h->cfg.sort_every); }

void drop_graphs(pic_handle* h) {
  for (auto& row : h->graph)
    for (auto& x : row)
      if (x) {
        cudaGraphExecDestroy(x);
        x = nullptr;
      }
}

// profiling: an event on the stream tagged with the stage that just ended
void mark(pic_handle* h, int tag) {
  if (!h->profiling) return;
  if (h->ev_used == (int)h->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    h->ev_pool.push_back(e);
  }
  cudaEventRecord(h->ev_pool[h->ev_used], h->stream);
  h->ev_marks.push_back({h->ev_used, tag});
  ++h->ev_used;
}

enum { kTagStart = -1, kTagParticle = 0, kTagFinalize = 1, kTagSort = 2, kTagField = 3 };

template <typename Real>
Soa<Real>& soa(pic_handle* h, int which);
template <>
Soa<float>& soa<float>(pic_handle* h, int which) { return h->sf[which]; }
template <>
Soa<double>& soa<double>(pic_handle* h, int which) { return h->sd[which]; }
template <typename Real>
const PushParams<Real>& params(pic_handle* h, int k = 0);
template <>
const PushParams<float>& params<float>(pic_handle* h, int k) { return h->Pf[k]; }
template <>
const PushParams<double>& params<double>(pic_handle* h, int k) { return h->Pd[k]; }
template <typename Real>
const PushParams<Real>* params_dev(pic_handle* h);
template <>
const PushParams<float>* params_dev<float>(pic_handle* h) { return h->Pf_dev; }
template <>
const PushParams<double>* params_dev<double>(pic_handle* h) { return h->Pd_dev; }

template <typename Real>
int step_impl(pic_handle* h, long long nsteps) {
  const PushParams<Real>& P = params<Real>(h);
  const bool solve = h->cfg.fixed_efield == 0;
  const bool batch = h->nsim > 1;
  const size_t grid_nodes = (size_t)h->nsim * h->nnodes;
  // child uids and the sort beside the field solve (neither reads the
  // other's data; the source, when on, needs the uids before the solve)
  const bool fork = solve && h->side && !h->any_source && !h->profiling;
  for (long long s = 0; s < nsteps; ++s) {
    mark(h, kTagStart);
    const bool fp32 = std::is_same<Real, float>::value;
    if (fp32 && !solve) {
      CK(cudaMemsetAsync(h->cnt[h->dep_buf], 0, grid_nodes * sizeof(unsigned long long),
                         h->stream));
    }
    if (!fp32) {
      CK(cudaMemsetAsync(h->rhs, 0, grid_nodes * sizeof(double), h->stream));
    }
    if (h->spl || h->web)
      CK(cudaMemsetAsync(h->spl_f, 0, (size_t)h->spl_cells * sizeof(double), h->stream));
    if (batch)
      launch_particle_step_batch<Real>(soa<Real>(h, h->cur), h->efield, fp32 ? nullptr : h->rhs,
                                       fp32 ? h->cnt[h->dep_buf] : nullptr, h->st,
                                       h->spawn_parent, h->spawn_stride, params_dev<Real>(h),
                                       h->nsim, h->nnodes, h->any_xs, h->grid_particle,
                                       h->stream);
    else
      launch_particle_step<Real>(soa<Real>(h, h->cur), h->efield, h->rhs,
                                 fp32 ? h->cnt[h->dep_buf] : nullptr, h->st, h->spawn_parent, P,
                                 h->grid_particle, h->stream);
    mark(h, kTagParticle);
    cudaStream_t aux = h->stream;
    if (fork) {
      CK(cudaEventRecord(h->ev_fork, h->stream));
      CK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
      aux = h->side;
    }
    if (batch)
      launch_spawn_finalize_batch(h->st, soa<Real>(h, h->cur).uid, h->spawn_parent,
                                  h->spawn_stride, h->seg, h->nsim, aux);
    else
      launch_spawn_finalize(h->st, soa<Real>(h, h->cur).uid, h->spawn_parent,
                            h->sims[0].spawn_cap, h->sims[0].capacity, aux);
    h->kernels += 2;
    if (h->any_source) {
      launch_source<Real>(soa<Real>(h, h->cur), h->st, params_dev<Real>(h), h->nsim,
                          fp32 ? nullptr : h->rhs, fp32 ? h->cnt[h->dep_buf] : nullptr,
                          h->nnodes, h->stream);
      h->kernels += 1;
    }
    mark(h, kTagFinalize);
    ++h->step;
    if (h->cfg.sort_every > 0 && h->step % h->cfg.sort_every == 0) {
      if (batch)
        launch_sort_batch<Real>(soa<Real>(h, h->cur), soa<Real>(h, h->cur ^ 1), h->st, h->seg,
                                h->nsim, h->cell_count, h->ncells, h->cfg.nz, h->grid_sort, aux);
      else
        launch_sort<Real>(soa<Real>(h, h->cur), soa<Real>(h, h->cur ^ 1), h->st, h->cell_count,
                          h->ncells, h->cfg.nz, h->grid_sort, aux);
      h->cur ^= 1;
      h->kernels += 4;
      mark(h, kTagSort);
    }
    if (fp32) h->last_buf = h->dep_buf;
    if (solve && h->net && h->cfg.warm_start == 2) {
      const int rc = warm_start_learned(h->net, h->T, fp32 ? h->cnt[h->dep_buf] : nullptr,
                                        h->q_units, fp32 ? nullptr : h->rhs, h->ws_x,
                                        h->ws_scale[0], h->ws_scale[1], h->ws_scale[2],
                                        h->stream);
      if (rc) return rc;
      h->kernels += unet_kernels_per_forward(h->net) + 2;
    }
    if (solve && (h->spl || h->web)) {
      const int rc = spline_solve_into(h);
      if (rc) return rc;
      // spline: lift, two transforms, band solves; web: T^T f - g, A^-1 b,
      // T u; and the precision copy
      h->kernels += h->web ? 4 : 5;
      mark(h, kTagField);
    } else if (solve) {
      if (fp32)
        launch_field_solve<Real>(h->T, nullptr, h->cnt[h->dep_buf],
                                 -kQe * h->sims[0].weight / kFixUnit,
                                 batch ? h->cnt_units : nullptr, h->cnt[h->dep_buf ^ 1],
                                 h->efield, h->st, h->stream);
      else
        launch_field_solve<Real>(h->T, h->rhs, nullptr, 0.0, nullptr, nullptr, h->efield, h->st,
                                 h->stream);
      if (fp32) h->dep_buf ^= 1;
      h->kernels += field_solve_kernels(h->T);
      mark(h, kTagField);
    }
    if (fork) {
      CK(cudaEventRecord(h->ev_join, h->side));
      CK(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    }
  }
  CK(cudaGetLastError());
  return PIC_OK;
}

// node charge b_i of the last deposit (C) copied to the host: the FP32
// path keeps fixed-point counts, the FP64 path charges
int read_rho(pic_handle* h, int sim, double* out) {
  const size_t go = (size_t)sim * h->nnodes;
  if (h->prec == 32) {
    std::vector<unsigned long long> c(h->nnodes);
    CK(cudaMemcpyAsync(c.data(), h->cnt[h->last_buf] + go,
                       (size_t)h->nnodes * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const double unit = -kQe * h->sims[sim].weight / kFixUnit;
    for (int i = 0; i < h->nnodes; ++i) out[i] = (double)c[i] * unit;
  } else {
    CK(cudaMemcpyAsync(out, h->rhs + go, (size_t)h->nnodes * sizeof(double),
                       cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return PIC_OK;
}

int check_sticky(pic_handle* h) {
  if (h->sticky) return h->sticky;
  std::vector<DevState> s(h->nsim);
  if (cudaMemcpyAsync(s.data(), h->st, s.size() * sizeof(DevState), cudaMemcpyDeviceToHost,
                      h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return h->sticky = PIC_ECUDA;
  for (const DevState& x : s)
    if (x.err && !h->sticky) h->sticky = x.err;
  return h->sticky;
}

// the store of the current buffer set as seen by simulation `sim`
template <typename Real>
Soa<Real> sim_soa(pic_handle* h, int sim, int which) {
  return soa_offset(soa<Real>(h, which), h->sims[sim].base);
}

}  // namespace

// ------------------------------------------------------------------ ABI

extern "C" {

const char* pic_strerror(int code) {
  switch (code) {
    case PIC_OK: return "ok";
    case PIC_EINVAL: return "invalid argument or configuration";
    case PIC_ENOMEM: return "out of memory";
    case PIC_ECAPACITY: return "particle or spawn capacity exceeded";
    case PIC_ENOCONV: return "field solve did not reach poisson_rtol";
    case PIC_ETIMEOUT: return "bounded device wait timed out";
    case PIC_ENONFINITE: return "non-finite particle value";
    case PIC_ECUDA: return "CUDA runtime error";
    default: return "unknown error";
  }
}

namespace {
// spline mode: load the stored particles (deposit = true) or none, solve,
// and wait
int spline_refresh(pic_handle* h, bool deposit) {
  const size_t cells = (size_t)h->spl_cells;
  if (cudaMemsetAsync(h->spl_f, 0, cells * sizeof(double), h->stream) != cudaSuccess)
    return PIC_ECUDA;
  if (deposit) {
    if (h->prec == 32)
      launch_spline_deposit_store<float>(sim_soa<float>(h, 0, h->cur), h->st, h->Pf[0],
                                         h->sims[0].capacity, h->stream);
    else
      launch_spline_deposit_store<double>(sim_soa<double>(h, 0, h->cur), h->st, h->Pd[0],
                                          h->sims[0].capacity, h->stream);
  }
  const int rc = spline_solve_into(h);
  if (rc) return rc;
  return cudaStreamSynchronize(h->stream) == cudaSuccess && cudaGetLastError() == cudaSuccess
             ? PIC_OK
             : PIC_ECUDA;
}
}  // namespace

int pic_init(const pic_config* cfg, int n_sims, void* cuda_stream,
             const pic_allocator* alloc, pic_handle** out) {
  if (!cfg || !out) return PIC_EINVAL;
  *out = nullptr;
  if (n_sims < 1 || n_sims > kMaxSims) return PIC_EINVAL;
  for (int k = 0; k < n_sims; ++k) {
    const int rc = validate(cfg[k]);
    if (rc) return rc;
  }
  int rc = validate_batch(cfg, n_sims);
  if (rc) return rc;
  if (cfg[0].bspline_degree > 0 && n_sims > 1) return PIC_EINVAL;
  pic_handle* h = new (std::nothrow) pic_handle();
  if (!h) return PIC_ENOMEM;
  h->cfg = cfg[0];
  h->cfgs.assign(cfg, cfg + n_sims);
  h->nsim = n_sims;
  h->prec = cfg->precision;
  h->stream = (cudaStream_t)cuda_stream;
  h->has_alloc = alloc && alloc->alloc && alloc->free;
  if (h->has_alloc) h->alloc = *alloc;
  const pic_config& c = h->cfg;

  // derived quantities (FP64, host), per simulation; segments of the store
  // start on whole chunks of the fused kernel
  const double L = c.z_max - c.z_min;
  h->hr = (c.r_out - c.r_in) / c.nr;
  h->hz = L / c.nz;
  const long long ch = particle_chunk();
  h->sims.resize(n_sims);
  h->xs.resize(n_sims);
  long long base = 0, spawn_stride = 0;
  for (int k = 0; k < n_sims; ++k) {
    const pic_config& ck = h->cfgs[k];
    SimHost& m = h->sims[k];
    std::memset(&m, 0, sizeof(m));
    m.n_gas = ck.p_mbar * 100.0 / (kKb * ck.t_gas_K);
    m.weight = ck.weight > 0 ? ck.weight
                             : ck.n0 * kPi * (ck.r_out * ck.r_out - ck.r_in * ck.r_in) * L /
                                   (double)ck.n_init;
    m.gas_mass = ck.gas_mass_amu * kAmu;
    derive_nu_max(ck, h->xs[k], m);
    m.capacity = ck.capacity > 0 ? ck.capacity
                                 : (long long)(1.25 * (double)std::max<int64_t>(ck.n_init, 0)) + 4096;
    m.spawn_cap = std::min<long long>(m.capacity, 1 << 20);
    m.base = base;
    base += (m.capacity + ch - 1) / ch * ch;
    spawn_stride = std::max(spawn_stride, m.spawn_cap);
  }
  h->capacity = base;
  h->spawn_stride = spawn_stride;
  h->any_source = false;
  for (const pic_config& ck : h->cfgs) h->any_source = h->any_source || ck.source_rate > 0;
  if (h->capacity > (1ll << 31) - 1) { delete h; return PIC_EINVAL; }
  h->nnodes = (c.nr + 1) * (c.nz + 1);
  h->ncells = c.nr * c.nz;
  const size_t S = (size_t)n_sims;

  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete h;
    return PIC_ECUDA;
  }
  const bool batch = n_sims > 1;
  const int bps = std::max(1, particle_step_blocks_per_sm(h->prec, batch));
  h->sms = sms;
  h->blocks_per_sm = bps;
  const long long chunks = (h->capacity + 1023) / 1024;
  h->grid_particle = (int)std::max<long long>(1, std::min<long long>((long long)sms * bps, chunks));
  h->grid_sort = (int)std::max<long long>(1, std::min<long long>((long long)sms * 8,
                                                                 (h->capacity + 255) / 256));

  // device memory
  h->st = (DevState*)h_alloc(S * sizeof(DevState), h);
  h->seg = (SegInfo*)h_alloc(S * sizeof(SegInfo), h);
  h->cnt_units = (float2*)h_alloc(S * sizeof(float2), h);
  h->Pf_dev = (PushParams<float>*)h_alloc(S * sizeof(PushParams<float>), h);
  h->Pd_dev = (PushParams<double>*)h_alloc(S * sizeof(PushParams<double>), h);
  h->q_units = (double*)h_alloc(S * sizeof(double), h);
  if (h->prec == 32) {
    rc = alloc_soa(h, h->sf[0]);
    if (!rc) rc = alloc_soa(h, h->sf[1]);
  } else {
    rc = alloc_soa(h, h->sd[0]);
    if (!rc) rc = alloc_soa(h, h->sd[1]);
  }
  const size_t gn = S * (size_t)h->nnodes;
  h->spawn_parent = (unsigned*)h_alloc(S * (size_t)h->spawn_stride * sizeof(unsigned), h);
  // whole multiples of 4096 counts per simulation: the scan reads them as
  // int4 vectors
  h->cell_count = (int*)h_alloc(S * ((size_t)(h->ncells + 4095) / 4096 * 4096) * sizeof(int), h);
  h->rhs = (double*)h_alloc(gn * sizeof(double), h);
  h->cnt[0] = (unsigned long long*)h_alloc(gn * sizeof(unsigned long long), h);
  h->cnt[1] = (unsigned long long*)h_alloc(gn * sizeof(unsigned long long), h);
  h->phi = (double*)h_alloc((size_t)h->nnodes * sizeof(double), h);
  h->efield = h_alloc(gn * (h->prec == 32 ? sizeof(float2) : sizeof(double2)), h);
  h->scratch2 = (double*)h_alloc(2 * sizeof(double), h);
  if (!rc && (!h->st || !h->seg || !h->cnt_units || !h->Pf_dev || !h->Pd_dev || !h->q_units ||
              !h->spawn_parent || !h->cell_count || !h->rhs || !h->cnt[0] || !h->cnt[1] ||
              !h->phi || !h->efield || !h->scratch2))
    rc = PIC_ENOMEM;
  if (!rc) rc = field_tables_build(h->cfgs.data(), n_sims, h->T, h_alloc, h, h->stream);
  if (!rc && c.bspline_degree > 0) rc = spline_setup(h);
  if (!rc) {
    h->Pf.resize(n_sims);
    h->Pd.resize(n_sims);
    std::vector<SegInfo> seg(n_sims);
    std::vector<float2> units(n_sims);
    std::vector<double> qunits(n_sims);
    const double s0 = 1.0 / (2.0 * kPi * kEps0);
    for (int k = 0; k < n_sims; ++k) {
      fill_params<float>(h, k, h->Pf[k]);
      fill_params<double>(h, k, h->Pd[k]);
      seg[k] = SegInfo{h->sims[k].base, h->sims[k].capacity, h->sims[k].spawn_cap};
      units[k] = df_from(-kQe * h->sims[k].weight / kFixUnit * s0);
      qunits[k] = -kQe * h->sims[k].weight / kFixUnit;
    }
    std::vector<DevState> s0v(n_sims);
    std::memset(s0v.data(), 0, S * sizeof(DevState));
    if (cudaMemcpyAsync(h->st, s0v.data(), S * sizeof(DevState), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->seg, seg.data(), S * sizeof(SegInfo), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->cnt_units, units.data(), S * sizeof(float2), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->q_units, qunits.data(), S * sizeof(double), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->Pf_dev, h->Pf.data(), S * sizeof(PushParams<float>),
                        cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->Pd_dev, h->Pd.data(), S * sizeof(PushParams<double>),
                        cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->rhs, 0, gn * sizeof(double), h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->cnt[0], 0, gn * sizeof(unsigned long long), h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->cnt[1], 0, gn * sizeof(unsigned long long), h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      rc = PIC_ECUDA;
  }
  if (!rc) {
    // vacuum field until particles are loaded
    if (h->prec == 32)
      launch_field_solve<float>(h->T, nullptr, h->cnt[0], 1.0, nullptr, nullptr, h->efield,
                                h->st, h->stream);
    else
      launch_field_solve<double>(h->T, h->rhs, nullptr, 0.0, nullptr, nullptr, h->efield, h->st,
                                 h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = PIC_ECUDA;
  }
  if (!rc && (h->spl || h->web)) rc = spline_refresh(h, false);   // vacuum spline field
  if (rc) {
    pic_free(h);
    return rc;
  }
  // the last deposit is in cnt[last_buf], the next goes to cnt[dep_buf]
  h->last_buf = 0;
  h->dep_buf = c.fixed_efield ? 0 : 1;
  set_graph_len(h);
  if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    h->side = nullptr;
    h->ev_fork = h->ev_join = nullptr;
  }
  *out = h;
  return PIC_OK;
}

void pic_free(pic_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  for (auto& row : h->graph)
    for (auto& x : row)
      if (x) cudaGraphExecDestroy(x);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->side) {
    cudaStreamSynchronize(h->side);
    cudaStreamDestroy(h->side);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  pic_spline_free(h->spl);
  pic_web_free(h->web);
  for (void* p : h->owned) h_free_one(p, h);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  delete h;
}

// The load's argument checks on the staged arrays: out[0] = min over the
// failing particles of 8 p + code (a position outside the open gap or a
// uid of 2^32 - 1 or more: PIC_EINVAL; a non-finite velocity, tested on
// the exponent bits: PIC_ENONFINITE; the position test first), out[1] =
// the largest uid.  out[0] starts at ~0, out[1] at 0.
__global__ void k_load_check(const double* __restrict__ r, const double* __restrict__ z,
                             const double* __restrict__ vr, const double* __restrict__ vt,
                             const double* __restrict__ vz, const uint64_t* __restrict__ uid,
                             long long n, double r_in, double r_out, double z_min, double z_max,
                             unsigned long long* out) {
  auto finite = [](double x) {
    return ((__double_as_longlong(x) >> 52) & 0x7FF) != 0x7FF;
  };
  unsigned long long first = ~0ull, um = 0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const double rp = r[p], zp = z[p];
    int e = 0;
    if (!(rp > r_in && rp < r_out && zp > z_min && zp < z_max)) e = PIC_EINVAL;
    else if (!finite(vr[p]) || !finite(vt[p]) || !finite(vz[p])) e = PIC_ENONFINITE;
    else if (uid[p] >= 0xFFFFFFFFull) e = PIC_EINVAL;
    if (e) first = min(first, 8ull * (unsigned long long)p + (unsigned long long)(-e));
    else um = max(um, (unsigned long long)uid[p]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
    um = max(um, __shfl_xor_sync(0xffffffffu, um, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (first != ~0ull) atomicMin(out, first);
    if (um) atomicMax(out + 1, um);
  }
}

int pic_load_particles(pic_handle* h, int sim, const double* r, const double* z,
                       const double* vr, const double* vt, const double* vz,
                       const uint64_t* uid, int64_t n) {
  if (!h || sim < 0 || sim >= h->nsim || n < 0 || n > h->sims[sim].capacity) return PIC_EINVAL;
  if (n > 0 && (!r || !z || !vr || !vt || !vz || !uid)) return PIC_EINVAL;
  const pic_config& c = h->cfgs[sim];
  SimHost& m = h->sims[sim];
  // staging buffers for the FP64 host arrays (checked there, on the
  // device, before anything of the simulation changes)
  const size_t want = std::max<size_t>((size_t)n, 1);
  if (want > h->stage_n) {
    for (void*& q : h->stage) {
      if (!q) continue;
      auto it = std::find(h->owned.begin(), h->owned.end(), q);
      if (it != h->owned.end()) h->owned.erase(it);
      h_free_one(q, h);
      q = nullptr;
    }
    h->stage_n = 0;
    for (void*& q : h->stage) {
      q = h_alloc(want * sizeof(double), h);   // owned: freed with the handle
      if (!q) return PIC_ENOMEM;
    }
    h->stage_n = want;
  }
  double* d[5];
  for (int k = 0; k < 5; ++k) d[k] = (double*)h->stage[k];
  uint64_t* du = (uint64_t*)h->stage[5];
  const double* src[5] = {r, z, vr, vt, vz};
  int rc = PIC_OK;
  for (int k = 0; k < 5 && n > 0; ++k)
    if (cudaMemcpyAsync(d[k], src[k], (size_t)n * sizeof(double), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess)
      rc = PIC_ECUDA;
  if (n > 0 && cudaMemcpyAsync(du, uid, (size_t)n * sizeof(uint64_t), cudaMemcpyHostToDevice,
                               h->stream) != cudaSuccess)
    rc = PIC_ECUDA;
  // the checks, on the staged arrays (nothing of the simulation has
  // changed yet): the first failing particle's code and the largest uid
  uint64_t chk[2] = {~0ull, 0ull};
  if (!rc && n > 0) {
    unsigned long long* out = (unsigned long long*)h->scratch2;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 8);
    if (cudaMemsetAsync(out, 0xFF, sizeof(unsigned long long), h->stream) != cudaSuccess ||
        cudaMemsetAsync(out + 1, 0, sizeof(unsigned long long), h->stream) != cudaSuccess)
      rc = PIC_ECUDA;
    if (!rc) {
      k_load_check<<<blocks, 256, 0, h->stream>>>(d[0], d[1], d[2], d[3], d[4], du, (long long)n,
                                                  c.r_in, c.r_out, c.z_min, c.z_max, out);
      if (cudaMemcpyAsync(chk, out, sizeof(chk), cudaMemcpyDeviceToHost, h->stream) !=
              cudaSuccess ||
          cudaStreamSynchronize(h->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        rc = PIC_ECUDA;
    }
  }
  if (rc || chk[0] != ~0ull) {
    cudaStreamSynchronize(h->stream);   // the staging copies end before the call returns
    return rc ? rc : -(int)(chk[0] & 7);
  }
  const uint64_t umax = chk[1];
  h->sticky = 0;
  // a single simulation restarts from step 0 in buffer set 0; a simulation
  // of a batch is loaded into the current buffer set at the batch's step
  const bool batch = h->nsim > 1;
  if (!batch) {
    h->cur = 0;
    h->step = 0;
    h->last_buf = 0;
  }
  if (!rc) {
    if (h->prec == 32)
      launch_load<float>(d[0], d[1], d[2], d[3], d[4], du, n, sim_soa<float>(h, sim, h->cur),
                         h->Pf[sim], h->st + sim, h->stream);
    else
      launch_load<double>(d[0], d[1], d[2], d[3], d[4], du, n, sim_soa<double>(h, sim, h->cur),
                          h->Pd[sim], h->st + sim, h->stream);
  }
  DevState s0;
  std::memset(&s0, 0, sizeof(s0));
  s0.n_slots = n;
  s0.n_live = n;
  s0.uid_next = n > 0 ? umax + 1 : 0;
  s0.step = (unsigned)h->step;
  const size_t go = (size_t)sim * h->nnodes, gb = (size_t)h->nnodes;
  const int ld = h->last_buf;   // the load's deposit becomes the last deposit
  if (!rc && (cudaMemcpyAsync(h->st + sim, &s0, sizeof(s0), cudaMemcpyHostToDevice, h->stream) !=
                  cudaSuccess ||
              cudaMemsetAsync(h->rhs + go, 0, gb * sizeof(double), h->stream) != cudaSuccess ||
              cudaMemsetAsync(h->cnt[0] + go, 0, gb * sizeof(unsigned long long), h->stream) !=
                  cudaSuccess ||
              cudaMemsetAsync(h->cnt[1] + go, 0, gb * sizeof(unsigned long long), h->stream) !=
                  cudaSuccess ||
              cudaMemsetAsync(h->T.phir + go, 0, gb * sizeof(float2), h->stream) != cudaSuccess))
    rc = PIC_ECUDA;
  // a single simulation that sorts starts in cell order (the same
  // particles, in the order the step's sort leaves: the first steps then
  // run at the sorted store's speed instead of the load order's)
  if (!rc && !batch && c.sort_every > 0 && n > 0) {
    if (h->prec == 32)
      launch_sort<float>(soa<float>(h, h->cur), soa<float>(h, h->cur ^ 1), h->st, h->cell_count,
                         h->ncells, c.nz, h->grid_sort, h->stream);
    else
      launch_sort<double>(soa<double>(h, h->cur), soa<double>(h, h->cur ^ 1), h->st,
                          h->cell_count, h->ncells, c.nz, h->grid_sort, h->stream);
    h->cur ^= 1;
  }
  if (!rc) {
    const double qw = -kQe * m.weight;
    if (h->prec == 32)
      launch_deposit_only<float>(sim_soa<float>(h, sim, h->cur), n, nullptr, h->cnt[ld] + go,
                                 c.nz, qw, h->stream);
    else
      launch_deposit_only<double>(sim_soa<double>(h, sim, h->cur), n, h->rhs + go, nullptr, c.nz,
                                  qw, h->stream);
    if (c.fixed_efield == 0) {
      // every simulation is solved again from its last deposit (the others'
      // fields come out as they were)
      if (h->prec == 32)
        launch_field_solve<float>(h->T, nullptr, h->cnt[ld], qw / kFixUnit,
                                  batch ? h->cnt_units : nullptr, h->cnt[ld ^ 1], h->efield,
                                  h->st, h->stream);
      else
        launch_field_solve<double>(h->T, h->rhs, nullptr, 0.0, nullptr, nullptr, h->efield,
                                   h->st, h->stream);
      h->dep_buf = ld ^ 1;
    } else {
      h->dep_buf = ld;
    }
    // initial kinetic energy
    cudaMemsetAsync(h->scratch2, 0, 2 * sizeof(double), h->stream);
    if (h->prec == 32)
      launch_kinetic_energy<float>(sim_soa<float>(h, sim, h->cur), h->st + sim, h->scratch2,
                                   h->stream);
    else
      launch_kinetic_energy<double>(sim_soa<double>(h, sim, h->cur), h->st + sim, h->scratch2,
                                    h->stream);
    double ke[2] = {0, 0};
    if (cudaMemcpyAsync(ke, h->scratch2, sizeof(ke), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
      rc = PIC_ECUDA;
    m.ke_initial = 0.5 * kMe * ke[0] * m.weight;
    if (!rc && (h->spl || h->web)) rc = spline_refresh(h, true);
  } else {
    cudaStreamSynchronize(h->stream);
  }
  m.last_diag_step = h->step;
  for (double& a : m.last_abs) a = 0.0;
  m.last_abs_ell = 0.0;
  return rc;
}

namespace {

int step_direct(pic_handle* h, long long n) {
  return h->prec == 32 ? step_impl<float>(h, n) : step_impl<double>(h, n);
}

// Capture graph_len steps starting from the current host state into
// h->graph[cur][dep]; the host state is restored afterwards (capture
// executes nothing).
int build_graph(pic_handle* h) {
  const int cur = h->cur, dep = h->dep_buf;
  const long long step0 = h->step, kern0 = h->kernels;
  const int last0 = h->last_buf;
  cudaStream_t user = h->stream;
  if (!h->cap_stream &&
      cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return PIC_ECUDA;
  if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return PIC_ECUDA;
  h->stream = h->cap_stream;
  const int rc = step_direct(h, h->graph_len);
  h->stream = user;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  const long long nk = h->kernels - kern0;
  h->cur = cur; h->dep_buf = dep; h->last_buf = last0;
  h->step = step0; h->kernels = kern0;
  if (rc != PIC_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return PIC_ECUDA;
  }
  cudaGraphExec_t x = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&x, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    cudaGetLastError();
    return PIC_ECUDA;
  }
  h->graph[cur][dep] = x;
  h->graph_kernels[cur][dep] = nk;
  return PIC_OK;
}

}  // namespace

int pic_step(pic_handle* h, int64_t nsteps) {
  if (!h || nsteps < 0) return PIC_EINVAL;
  if (h->sticky) return h->sticky;
  long long n = nsteps;
  if (h->profiling || h->graph_failed || h->graph_len <= 0) return step_direct(h, n);
  // direct steps up to a block boundary, whole blocks as graph replays, the
  // remainder direct again
  while (n > 0 && h->step % h->graph_len != 0) {
    const int rc = step_direct(h, 1);
    if (rc) return rc;
    --n;
  }
  while (n >= h->graph_len) {
    const int cur = h->cur, dep = h->dep_buf;
    if (!h->graph[cur][dep] && build_graph(h) != PIC_OK) {
      h->graph_failed = true;   // stay on direct launches
      return step_direct(h, n);
    }
    if (cudaGraphLaunch(h->graph[cur][dep], h->stream) != cudaSuccess) return PIC_ECUDA;
    // the host-side view of the block: the same bookkeeping as direct steps
    h->step += h->graph_len;
    h->kernels += h->graph_kernels[cur][dep];
    const bool solve = h->cfg.fixed_efield == 0;
    if (h->prec == 32) {
      h->last_buf = solve ? (dep ^ ((h->graph_len - 1) & 1)) : dep;
      if (solve) h->dep_buf = dep ^ (h->graph_len & 1);
    }
    if (h->cfg.sort_every > 0) h->cur = cur ^ ((h->graph_len / h->cfg.sort_every) & 1);
    n -= h->graph_len;
  }
  return n > 0 ? step_direct(h, n) : PIC_OK;
}

int pic_diagnostics(pic_handle* h, int sim, pic_diag* out, double* density) {
  if (!h || sim < 0 || sim >= h->nsim || !out) return PIC_EINVAL;
  if (density && (h->spl || h->web)) return PIC_EINVAL;   // no node deposit in spline mode
  const pic_config& c = h->cfgs[sim];
  SimHost& m = h->sims[sim];
  DevState s;
  CK(cudaMemsetAsync(h->scratch2, 0, 2 * sizeof(double), h->stream));
  if (h->prec == 32)
    launch_kinetic_energy<float>(sim_soa<float>(h, sim, h->cur), h->st + sim, h->scratch2,
                                 h->stream);
  else
    launch_kinetic_energy<double>(sim_soa<double>(h, sim, h->cur), h->st + sim, h->scratch2,
                                  h->stream);
  double ke[2];
  CK(cudaMemcpyAsync(&s, h->st + sim, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(ke, h->scratch2, sizeof(ke), cudaMemcpyDeviceToHost, h->stream));
  std::vector<double> grid;
  CK(cudaStreamSynchronize(h->stream));
  if (density) {
    grid.resize(h->nnodes);
    int rr = read_rho(h, sim, grid.data());
    if (rr) return rr;
  }
  CK(cudaGetLastError());
  if (s.err && !h->sticky) h->sticky = s.err;
  if (!h->sticky) {
    // a non-finite velocity among the live particles, or one that reached a
    // tally before its particle was removed (an unphysical field, say)
    bool finite = std::isfinite(ke[0]);
    for (double v : s.tally) finite = finite && std::isfinite(v);
    if (!finite) h->sticky = PIC_ENONFINITE;
  }
  std::memset(out, 0, sizeof(*out));
  out->step = h->step;
  out->t = (double)h->step * c.dt;
  out->n_particles = (int64_t)ke[1];
  const double dtw = (double)(h->step - m.last_diag_step) * c.dt;
  double* I[4] = {&out->I_inner, &out->I_outer, &out->I_zmin, &out->I_zmax};
  for (int w = 0; w < 4; ++w) {
    out->absorbed_weight[w] = s.tally[kAbsInner + w];
    *I[w] = dtw > 0 ? (s.tally[kAbsInner + w] - m.last_abs[w]) * kQe / dtw : 0.0;
    m.last_abs[w] = s.tally[kAbsInner + w];
  }
  out->absorbed_ellipse = s.tally[kAbsEllipse];
  out->I_ellipse = dtw > 0 ? (s.tally[kAbsEllipse] - m.last_abs_ell) * kQe / dtw : 0.0;
  m.last_abs_ell = s.tally[kAbsEllipse];
  m.last_diag_step = h->step;
  out->n_elastic = (int64_t)s.tally[kNElastic];
  out->n_ionise = (int64_t)s.tally[kNIonise];
  out->n_absorbed = (int64_t)s.tally[kNAbsorbed];
  out->n_candidates = (int64_t)s.tally[kNCandidate];
  out->n_over = (int64_t)s.tally[kNOver];
  out->n_pushed = (int64_t)s.tally[kNPushed];
  out->kernels_launched = h->kernels;
  out->ke_total_J = 0.5 * kMe * ke[0] * m.weight;
  out->work_E_J = s.tally[kWorkE];
  out->ke_absorbed_J = s.tally[kKeAbsorbed];
  out->ion_loss_J = s.tally[kIonLoss];
  out->recoil_loss_J = s.tally[kRecoilLoss];
  out->ke_initial_J = m.ke_initial;
  out->n_source = (int64_t)s.tally[kNSource];
  out->ke_source_J = s.tally[kKeSource];
  out->ledger_residual_J = (out->ke_total_J - m.ke_initial) -
                           (out->work_E_J - out->ke_absorbed_J - out->ion_loss_J -
                            out->recoil_loss_J + out->ke_source_J);
  out->poisson_iters = s.poisson_iters;
  out->poisson_relres = s.relres_last;
  out->poisson_relres_charge = s.relres_strict;
  out->nu_max = m.nu_max;
  out->weight = m.weight;
  out->error = h->sticky;
  out->poisson_relres_init = s.relres_init;
  if (density) {
    // node volume of each hat function: 2 pi R_i Z_j
    const double hr = h->hr, hz = h->hz;
    double peak = 0.0;
    for (int i = 0; i <= c.nr; ++i) {
      const double ri = c.r_in + i * hr;
      const double R = i == 0 ? hr * (c.r_in / 2 + hr / 6)
                              : (i == c.nr ? hr * (c.r_out / 2 - hr / 6) : ri * hr);
      for (int j = 0; j <= c.nz; ++j) {
        const double Z = (j == 0 || j == c.nz) ? hz / 2 : hz;
        const size_t o = (size_t)i * (c.nz + 1) + j;
        density[o] = grid[o] / (-kQe) / (2.0 * kPi * R * Z);
        peak = std::max(peak, density[o]);
      }
    }
    out->n_peak = peak;
  }
  return h->sticky;
}

int pic_export_particles(pic_handle* h, int sim, double* r, double* z, double* vr,
                         double* vt, double* vz, uint64_t* uid, int64_t cap, int64_t* n) {
  if (!h || sim < 0 || sim >= h->nsim || !n) return PIC_EINVAL;
  DevState s;
  CK(cudaMemcpyAsync(&s, h->st + sim, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (s.err && !h->sticky) h->sticky = s.err;
  const long long ns = s.n_slots;
  std::vector<double> a[5];
  std::vector<unsigned long long> u(ns);
  std::vector<int> live(ns);
  for (auto& v : a) v.resize(ns);
  if (ns > 0) {
    const size_t bytes = (size_t)ns * sizeof(double);
    void* d[7];
    for (int k = 0; k < 7; ++k) {
      d[k] = h_alloc(bytes, h);
      if (!d[k]) return PIC_ENOMEM;
    }
    if (h->prec == 32)
      launch_export<float>(sim_soa<float>(h, sim, h->cur), ns, h->Pf[sim], (double*)d[0],
                           (double*)d[1], (double*)d[2], (double*)d[3], (double*)d[4],
                           (unsigned long long*)d[5], (int*)d[6], h->stream);
    else
      launch_export<double>(sim_soa<double>(h, sim, h->cur), ns, h->Pd[sim], (double*)d[0],
                            (double*)d[1], (double*)d[2], (double*)d[3], (double*)d[4],
                            (unsigned long long*)d[5], (int*)d[6], h->stream);
    int rc = PIC_OK;
    for (int k = 0; k < 5; ++k)
      if (cudaMemcpyAsync(a[k].data(), d[k], bytes, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        rc = PIC_ECUDA;
    if (cudaMemcpyAsync(u.data(), d[5], bytes, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(live.data(), d[6], (size_t)ns * sizeof(int), cudaMemcpyDeviceToHost,
                        h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      rc = PIC_ECUDA;
    for (int k = 0; k < 7; ++k) {
      auto it = std::find(h->owned.begin(), h->owned.end(), d[k]);
      if (it != h->owned.end()) h->owned.erase(it);
      h_free_one(d[k], h);
    }
    if (rc) return rc;
  }
  std::vector<long long> idx;
  idx.reserve(ns);
  for (long long p = 0; p < ns; ++p)
    if (live[p]) idx.push_back(p);
  *n = (int64_t)idx.size();
  if ((int64_t)idx.size() > cap) return PIC_ECAPACITY;
  std::sort(idx.begin(), idx.end(), [&](long long x, long long y) { return u[x] < u[y]; });
  double* dst[5] = {r, z, vr, vt, vz};
  for (size_t q = 0; q < idx.size(); ++q) {
    for (int k = 0; k < 5; ++k)
      if (dst[k]) dst[k][q] = a[k][idx[q]];
    if (uid) uid[q] = u[idx[q]];
  }
  return h->sticky;
}

int pic_set_efield(pic_handle* h, int sim, const double* er, const double* ez) {
  if (!h || sim < 0 || sim >= h->nsim || !er || !ez) return PIC_EINVAL;
  const size_t eo = (size_t)sim * h->nnodes * (h->prec == 32 ? sizeof(float2) : sizeof(double2));
  void* efield = (char*)h->efield + eo;
  const size_t bytes = (size_t)h->nnodes * sizeof(double);
  double* d0 = (double*)h_alloc(bytes, h);
  double* d1 = (double*)h_alloc(bytes, h);
  if (!d0 || !d1) return PIC_ENOMEM;
  int rc = PIC_OK;
  if (cudaMemcpyAsync(d0, er, bytes, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(d1, ez, bytes, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    rc = PIC_ECUDA;
  if (!rc) {
    if (h->prec == 32) launch_efield_set<float>(d0, d1, efield, h->nnodes, h->stream);
    else launch_efield_set<double>(d0, d1, efield, h->nnodes, h->stream);
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = PIC_ECUDA;
  for (double* p : {d0, d1}) {
    auto it = std::find(h->owned.begin(), h->owned.end(), (void*)p);
    if (it != h->owned.end()) h->owned.erase(it);
    h_free_one(p, h);
  }
  return rc;
}

int pic_set_cross_sections(pic_handle* h, int sim, int n, const double* E_eV,
                           const double* sigma_el_m2, const double* sigma_io_m2,
                           const double* xi) {
  if (!h || sim < 0 || sim >= h->nsim || n < 0 || n == 1 || n > PIC_XS_MAX_POINTS)
    return PIC_EINVAL;
  if (n > 0) {
    if (!E_eV || !sigma_el_m2 || !sigma_io_m2) return PIC_EINVAL;
    for (int k = 0; k < n; ++k) {
      if (!std::isfinite(E_eV[k]) || !(E_eV[k] >= 0) || (k > 0 && !(E_eV[k] > E_eV[k - 1])))
        return PIC_EINVAL;
      if (!std::isfinite(sigma_el_m2[k]) || !(sigma_el_m2[k] >= 0) ||
          !std::isfinite(sigma_io_m2[k]) || !(sigma_io_m2[k] >= 0))
        return PIC_EINVAL;
      if (xi && !(xi[k] >= 0 && xi[k] < 1)) return PIC_EINVAL;
    }
  }
  if (h->sticky) return h->sticky;
  // kernels in flight may read the current tables
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return PIC_ECUDA;
  XsHost& X = h->xs[sim];
  SimHost& m = h->sims[sim];
  X.n = n;
  X.E_eV.clear();
  X.sigma_el.clear();
  X.sigma_io.clear();
  X.xi.clear();
  if (n > 0) {
    X.E_eV.assign(E_eV, E_eV + n);
    X.sigma_el.assign(sigma_el_m2, sigma_el_m2 + n);
    X.sigma_io.assign(sigma_io_m2, sigma_io_m2 + n);
    if (xi) X.xi.assign(xi, xi + n);
  }
  if (n > 0) {
    const size_t rs = h->prec == 32 ? sizeof(float) : sizeof(double);
    if (!X.dev) {
      X.dev = h_alloc(4 * (size_t)PIC_XS_MAX_POINTS * rs, h);
      if (!X.dev) {
        X.n = 0;
        return PIC_ENOMEM;
      }
    }
    // device copy in the particle precision: E in J, n_gas sigma in 1/m
    std::vector<double> v(4 * (size_t)PIC_XS_MAX_POINTS, 0.0);
    for (int k = 0; k < n; ++k) {
      v[k] = E_eV[k] * kQe;
      v[PIC_XS_MAX_POINTS + k] = m.n_gas * sigma_el_m2[k];
      v[2 * PIC_XS_MAX_POINTS + k] = m.n_gas * sigma_io_m2[k];
      v[3 * PIC_XS_MAX_POINTS + k] = xi ? xi[k] : 0.0;
    }
    cudaError_t e;
    if (h->prec == 32) {
      std::vector<float> f(v.begin(), v.end());
      e = cudaMemcpy(X.dev, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice);
    } else {
      e = cudaMemcpy(X.dev, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return PIC_ECUDA;
  }
  derive_nu_max(h->cfgs[sim], X, m);
  fill_params<float>(h, sim, h->Pf[sim]);
  fill_params<double>(h, sim, h->Pd[sim]);
  if (cudaMemcpy(h->Pf_dev + sim, &h->Pf[sim], sizeof(PushParams<float>), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(h->Pd_dev + sim, &h->Pd[sim], sizeof(PushParams<double>), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return PIC_ECUDA;
  h->any_xs = false;
  for (const XsHost& x : h->xs) h->any_xs = h->any_xs || x.n > 0;
  // the captured steps hold the old parameters (and kernel variant)
  drop_graphs(h);
  return PIC_OK;
}

namespace {
ForceParams force_params(const pic_handle* h, int sim, double dt_prev) {
  const pic_config& c = h->cfgs[sim];
  ForceParams F;
  F.nr = c.nr;
  F.nz = c.nz;
  F.bkind = c.bfield_kind;
  F.r_in = c.r_in;
  F.hr = h->hr;
  F.z_min = c.z_min;
  F.hz = h->hz;
  F.b0 = c.b0;
  F.L = c.z_max - c.z_min;
  F.z_mid = 0.5 * (c.z_min + c.z_max);
  F.weight = h->sims[sim].weight;
  F.dt_prev = dt_prev;
  return F;
}

// device buffer of `bytes` owned by this call (freed by drop_tmp)
void* tmp_alloc(pic_handle* h, size_t bytes) { return h_alloc(bytes, h); }
void drop_tmp(pic_handle* h, void* p) {
  if (!p) return;
  auto it = std::find(h->owned.begin(), h->owned.end(), p);
  if (it != h->owned.end()) h->owned.erase(it);
  h_free_one(p, h);
}
}  // namespace

static_assert(kMoments == PIC_MOMENTS, "moment count of the ABI");
static_assert(kFluidModel == PIC_FLUID_MODEL, "fluid-model grid count of the ABI");

namespace {
void moments_into(pic_handle* h, int sim, double scale, double* M) {
  const ForceParams F = force_params(h, sim, 0.0);
  if (h->prec == 32)
    launch_moments<float>(sim_soa<float>(h, sim, h->cur), h->st + sim, h->Pf[sim], F, scale, M,
                          h->sims[sim].capacity, h->stream);
  else
    launch_moments<double>(sim_soa<double>(h, sim, h->cur), h->st + sim, h->Pd[sim], F, scale,
                           M, h->sims[sim].capacity, h->stream);
}
}  // namespace

int pic_moments(pic_handle* h, int sim, double* out) {
  if (!h || sim < 0 || sim >= h->nsim || !out) return PIC_EINVAL;
  if (h->sticky) return h->sticky;
  const size_t bytes = (size_t)kMoments * h->nnodes * sizeof(double);
  double* M = (double*)tmp_alloc(h, bytes);
  if (!M) return PIC_ENOMEM;
  int rc = PIC_OK;
  if (cudaMemsetAsync(M, 0, bytes, h->stream) != cudaSuccess) rc = PIC_ECUDA;
  if (!rc) moments_into(h, sim, 1.0, M);
  if (!rc && (cudaMemcpyAsync(out, M, bytes, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
              cudaStreamSynchronize(h->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess))
    rc = PIC_ECUDA;
  drop_tmp(h, M);
  return rc;
}

int pic_moments_accumulate(pic_handle* h, int sim, double* acc, double scale) {
  if (!h || sim < 0 || sim >= h->nsim || !acc || !std::isfinite(scale)) return PIC_EINVAL;
  if (h->sticky) return h->sticky;
  moments_into(h, sim, scale, acc);
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

int pic_force_balance(pic_handle* h, int sim, const double* moments, const double* moments_prev,
                      double dt_prev, double* out) {
  if (!h || sim < 0 || sim >= h->nsim || !moments || !out) return PIC_EINVAL;
  if (moments_prev && !(dt_prev > 0)) return PIC_EINVAL;
  if (h->sticky) return h->sticky;
  const size_t nn = (size_t)h->nnodes;
  const size_t mb = (size_t)kMoments * nn * sizeof(double);
  const size_t ob = (size_t)PIC_FORCE_TERMS * 3 * nn * sizeof(double);
  double* M = (double*)tmp_alloc(h, mb);
  double* Mp = moments_prev ? (double*)tmp_alloc(h, mb) : nullptr;
  double* O = (double*)tmp_alloc(h, ob);
  int rc = (!M || !O || (moments_prev && !Mp)) ? PIC_ENOMEM : PIC_OK;
  if (!rc && (cudaMemcpyAsync(M, moments, mb, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
              (Mp && cudaMemcpyAsync(Mp, moments_prev, mb, cudaMemcpyHostToDevice, h->stream) !=
                         cudaSuccess)))
    rc = PIC_ECUDA;
  if (!rc) {
    const ForceParams F = force_params(h, sim, moments_prev ? dt_prev : 0.0);
    const size_t eo = (size_t)sim * nn * (h->prec == 32 ? sizeof(float2) : sizeof(double2));
    const void* E = (const char*)h->efield + eo;
    if (h->prec == 32) launch_force_terms<float>(M, Mp, E, F, O, h->stream);
    else launch_force_terms<double>(M, Mp, E, F, O, h->stream);
    if (cudaMemcpyAsync(out, O, ob, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
      rc = PIC_ECUDA;
  }
  drop_tmp(h, M);
  drop_tmp(h, Mp);
  drop_tmp(h, O);
  return rc;
}

int pic_fluid_model(pic_handle* h, int sim, const double* moments, double* out) {
  if (!h || sim < 0 || sim >= h->nsim || !moments || !out) return PIC_EINVAL;
  if (h->sticky) return h->sticky;
  const size_t nn = (size_t)h->nnodes;
  const size_t mb = (size_t)kMoments * nn * sizeof(double);
  const size_t ob = (size_t)kFluidModel * nn * sizeof(double);
  double* M = (double*)tmp_alloc(h, mb);
  double* O = (double*)tmp_alloc(h, ob);
  int rc = (!M || !O) ? PIC_ENOMEM : PIC_OK;
  if (!rc && cudaMemcpyAsync(M, moments, mb, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    rc = PIC_ECUDA;
  if (!rc) {
    const ForceParams F = force_params(h, sim, 0.0);
    const size_t eo = (size_t)sim * nn * (h->prec == 32 ? sizeof(float2) : sizeof(double2));
    const void* E = (const char*)h->efield + eo;
    if (h->prec == 32) launch_fluid_model<float>(M, E, F, h->Pf[sim], O, h->stream);
    else launch_fluid_model<double>(M, E, F, h->Pd[sim], O, h->stream);
    if (cudaMemcpyAsync(out, O, ob, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
      rc = PIC_ECUDA;
  }
  drop_tmp(h, M);
  drop_tmp(h, O);
  return rc;
}

int pic_get_grid(pic_handle* h, int sim, int which, double* out) {
  if (!h || sim < 0 || sim >= h->nsim || !out) return PIC_EINVAL;
  const size_t bytes = (size_t)h->nnodes * sizeof(double);
  const size_t eo = (size_t)sim * h->nnodes * (h->prec == 32 ? sizeof(float2) : sizeof(double2));
  const void* efield = (const char*)h->efield + eo;
  if (h->spl || h->web) {
    // spline mode: phi or E at the nodes from the coefficients
    if (which != PIC_GRID_PHI && which != PIC_GRID_ER && which != PIC_GRID_EZ) return PIC_EINVAL;
    double* d = (double*)h_alloc(3 * bytes, h);
    if (!d) return PIC_ENOMEM;
    std::vector<double> nr_(h->nnodes), nz_(h->nnodes);
    for (int i = 0; i <= h->cfg.nr; ++i)
      for (int j = 0; j <= h->cfg.nz; ++j) {
        nr_[(size_t)i * (h->cfg.nz + 1) + j] = std::min(h->cfg.r_in + i * h->hr, h->cfg.r_out);
        nz_[(size_t)i * (h->cfg.nz + 1) + j] = std::min(h->cfg.z_min + j * h->hz, h->cfg.z_max);
      }
    double* dr = d + h->nnodes;
    double* dz = d + 2 * (size_t)h->nnodes;
    int rc = PIC_OK;
    if (h->web) pic_web_set_stream(h->web, h->stream);
    else pic_spline_set_stream(h->spl, h->stream);
    if (cudaMemcpyAsync(dr, nr_.data(), bytes, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(dz, nz_.data(), bytes, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
      rc = PIC_ECUDA;
    double* o_phi = which == PIC_GRID_PHI ? d : nullptr;
    double* o_er = which == PIC_GRID_ER ? d : nullptr;
    double* o_ez = which == PIC_GRID_EZ ? d : nullptr;
    if (!rc)
      rc = h->web ? pic_web_eval(h->web, h->spl_c, dr, dz, h->nnodes, 1, o_phi, o_er, o_ez)
                  : pic_spline_eval(h->spl, h->spl_c, dr, dz, h->nnodes, 1, o_phi, o_er, o_ez);
    if (!rc && (cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
                cudaStreamSynchronize(h->stream) != cudaSuccess))
      rc = PIC_ECUDA;
    auto it = std::find(h->owned.begin(), h->owned.end(), (void*)d);
    if (it != h->owned.end()) h->owned.erase(it);
    h_free_one(d, h);
    return rc ? rc : check_sticky(h);
  }
  if (which == PIC_GRID_RHS) {
    const int rr = read_rho(h, sim, out);
    return rr ? rr : check_sticky(h);
  }
  if (which == PIC_GRID_PHI) {
    launch_phi_out(h->T, h->phi, h->stream, sim);
    CK(cudaMemcpyAsync(out, h->phi, bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return check_sticky(h);
  }
  if (which != PIC_GRID_ER && which != PIC_GRID_EZ) return PIC_EINVAL;
  double* d = (double*)h_alloc(bytes, h);
  if (!d) return PIC_ENOMEM;
  if (h->prec == 32) launch_efield_get<float>(efield, d, which == PIC_GRID_ER ? 0 : 1, h->nnodes, h->stream);
  else launch_efield_get<double>(efield, d, which == PIC_GRID_ER ? 0 : 1, h->nnodes, h->stream);
  int rc = PIC_OK;
  if (cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    rc = PIC_ECUDA;
  auto it = std::find(h->owned.begin(), h->owned.end(), (void*)d);
  if (it != h->owned.end()) h->owned.erase(it);
  h_free_one(d, h);
  return rc ? rc : check_sticky(h);
}

int pic_solve_field(pic_handle* h, const double* b, double* phi, double* relres) {
  if (!h || !b || !phi) return PIC_EINVAL;
  const size_t nn = (size_t)h->nnodes;
  const size_t tri = (size_t)h->T.NI * (h->T.M + 1);
  // the tables are shared; the work arrays are this call's own, so the
  // simulation's field is untouched
  FieldTables T = h->T;
  T.nsim = 1;   // the first simulation's wall potentials
  double* d_b = (double*)h_alloc(nn * sizeof(double), h);
  double* d_phi = (double*)h_alloc(nn * sizeof(double), h);
  void* d_e = h_alloc(nn * sizeof(double2), h);
  DevState* d_st = (DevState*)h_alloc(sizeof(DevState), h);
  T.b2 = (float2*)h_alloc(nn * sizeof(float2), h);
  T.phir = (float2*)h_alloc(nn * sizeof(float2), h);
  T.res = (float*)h_alloc(nn * sizeof(float), h);
  T.bhat = (float*)h_alloc(tri * sizeof(float), h);
  T.phihat = (float*)h_alloc(tri * sizeof(float), h);
  void* tmp[] = {d_b, d_phi, d_e, d_st, T.b2, T.phir, T.res, T.bhat, T.phihat};
  int rc = PIC_OK;
  for (void* p : tmp)
    if (!p) rc = PIC_ENOMEM;
  DevState s0;
  std::memset(&s0, 0, sizeof(s0));
  if (!rc && (cudaMemcpyAsync(d_b, b, nn * sizeof(double), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
              cudaMemcpyAsync(d_st, &s0, sizeof(s0), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
              cudaMemsetAsync(T.phir, 0, nn * sizeof(float2), h->stream) != cudaSuccess))
    rc = PIC_ECUDA;
  if (!rc) {
    launch_field_solve<double>(T, d_b, nullptr, 0.0, nullptr, nullptr, d_e, d_st, h->stream);
    launch_phi_out(T, d_phi, h->stream);
    if (cudaMemcpyAsync(phi, d_phi, nn * sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(&s0, d_st, sizeof(s0), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
      rc = PIC_ECUDA;
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = PIC_ECUDA;
  if (!rc && relres) *relres = s0.relres_last;
  if (!rc && s0.err) rc = s0.err;
  for (void* p : tmp) {
    if (!p) continue;
    auto it = std::find(h->owned.begin(), h->owned.end(), p);
    if (it != h->owned.end()) h->owned.erase(it);
    h_free_one(p, h);
  }
  return rc;
}

// checkpoint layout: magic, version, precision, nr, nz, capacity, seed, host
// step, ke_initial, last_abs[4], last_diag_step, DevState, n_slots, the
// seven SoA arrays of the current buffer set (n_slots entries), phi, the
// space-charge potential (double-float pairs), node field, FP64 deposit and
// the FP32 path's last fixed-point deposit
static const char kMagic[8] = {'P', 'I', 'C', 'C', 'K', 'P', 'T', '2'};

int pic_checkpoint(pic_handle* h, const char* path) {
  if (!h || !path || h->nsim != 1) return PIC_EINVAL;
  DevState s;
  CK(cudaMemcpyAsync(&s, h->st, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  FILE* f = std::fopen(path, "wb");
  if (!f) return PIC_EINVAL;
  const size_t rs = h->prec == 32 ? sizeof(float) : sizeof(double);
  const long long ns = s.n_slots;
  int64_t hdr[6] = {h->prec, h->cfg.nr, h->cfg.nz, h->capacity, (int64_t)h->cfg.seed, h->step};
  bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
            std::fwrite(&h->sims[0].ke_initial, sizeof(double), 1, f) == 1 &&
            std::fwrite(h->sims[0].last_abs, sizeof(double), 4, f) == 4 &&
            std::fwrite(&h->sims[0].last_diag_step, sizeof(long long), 1, f) == 1 &&
            std::fwrite(&s, sizeof(s), 1, f) == 1;
  std::vector<char> buf;
  void* arrays[7];
  size_t sizes[7];
  if (h->prec == 32) {
    Soa<float>& q = h->sf[h->cur];
    void* a[7] = {q.cell, q.offr, q.offz, q.vr, q.vt, q.vz, q.uid};
    std::copy(a, a + 7, arrays);
  } else {
    Soa<double>& q = h->sd[h->cur];
    void* a[7] = {q.cell, q.offr, q.offz, q.vr, q.vt, q.vz, q.uid};
    std::copy(a, a + 7, arrays);
  }
  for (int k = 0; k < 7; ++k) sizes[k] = (k == 0 || k == 6) ? 4 : rs;
  for (int k = 0; k < 7 && ok; ++k) {
    buf.resize(std::max<size_t>(1, (size_t)ns * sizes[k]));
    if (ns > 0 && cudaMemcpy(buf.data(), arrays[k], (size_t)ns * sizes[k], cudaMemcpyDeviceToHost) != cudaSuccess) { ok = false; break; }
    ok = std::fwrite(buf.data(), 1, (size_t)ns * sizes[k], f) == (size_t)ns * sizes[k];
  }
  const size_t gbytes = (size_t)h->nnodes * sizeof(double);
  const size_t ebytes = (size_t)h->nnodes * 2 * rs;
  const void* grids[4] = {h->T.phir, h->efield, h->rhs, h->cnt[h->last_buf]};
  const size_t gsz[4] = {(size_t)h->nnodes * sizeof(float2), ebytes, gbytes,
                         (size_t)h->nnodes * sizeof(unsigned long long)};
  for (int k = 0; k < 4 && ok; ++k) {
    buf.resize(gsz[k]);
    if (cudaMemcpy(buf.data(), grids[k], gsz[k], cudaMemcpyDeviceToHost) != cudaSuccess) { ok = false; break; }
    ok = std::fwrite(buf.data(), 1, gsz[k], f) == gsz[k];
  }
  std::fclose(f);
  return ok ? check_sticky(h) : PIC_EINVAL;
}

int pic_restore(pic_handle* h, const char* path) {
  if (!h || !path || h->nsim != 1) return PIC_EINVAL;
  FILE* f = std::fopen(path, "rb");
  if (!f) return PIC_EINVAL;
  char magic[8];
  int64_t hdr[6];
  DevState s;
  double ke0, labs[4];
  long long lds;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
            std::fread(hdr, sizeof(hdr), 1, f) == 1 && std::fread(&ke0, sizeof(double), 1, f) == 1 &&
            std::fread(labs, sizeof(double), 4, f) == 4 &&
            std::fread(&lds, sizeof(long long), 1, f) == 1 && std::fread(&s, sizeof(s), 1, f) == 1;
  ok = ok && hdr[0] == h->prec && hdr[1] == h->cfg.nr && hdr[2] == h->cfg.nz &&
       hdr[3] == h->capacity && (uint64_t)hdr[4] == h->cfg.seed && s.n_slots <= h->capacity;
  if (!ok) { std::fclose(f); return PIC_EINVAL; }
  const size_t rs = h->prec == 32 ? sizeof(float) : sizeof(double);
  const long long ns = s.n_slots;
  h->cur = 0;
  void* arrays[7];
  if (h->prec == 32) {
    Soa<float>& q = h->sf[0];
    void* a[7] = {q.cell, q.offr, q.offz, q.vr, q.vt, q.vz, q.uid};
    std::copy(a, a + 7, arrays);
  } else {
    Soa<double>& q = h->sd[0];
    void* a[7] = {q.cell, q.offr, q.offz, q.vr, q.vt, q.vz, q.uid};
    std::copy(a, a + 7, arrays);
  }
  std::vector<char> buf;
  for (int k = 0; k < 7 && ok; ++k) {
    const size_t sz = (k == 0 || k == 6) ? 4 : rs;
    buf.resize(std::max<size_t>(1, (size_t)ns * sz));
    ok = std::fread(buf.data(), 1, (size_t)ns * sz, f) == (size_t)ns * sz;
    if (ok && ns > 0 && cudaMemcpy(arrays[k], buf.data(), (size_t)ns * sz, cudaMemcpyHostToDevice) != cudaSuccess) ok = false;
  }
  const size_t gbytes = (size_t)h->nnodes * sizeof(double);
  const size_t ebytes = (size_t)h->nnodes * 2 * rs;
  void* grids[4] = {h->T.phir, h->efield, h->rhs, h->cnt[0]};
  const size_t gsz[4] = {(size_t)h->nnodes * sizeof(float2), ebytes, gbytes,
                         (size_t)h->nnodes * sizeof(unsigned long long)};
  for (int k = 0; k < 4 && ok; ++k) {
    buf.resize(gsz[k]);
    ok = std::fread(buf.data(), 1, gsz[k], f) == gsz[k];
    if (ok && cudaMemcpy(grids[k], buf.data(), gsz[k], cudaMemcpyHostToDevice) != cudaSuccess) ok = false;
  }
  std::fclose(f);
  if (!ok) return PIC_EINVAL;
  CK(cudaMemcpy(h->st, &s, sizeof(s), cudaMemcpyHostToDevice));
  CK(cudaMemset(h->cnt[1], 0, (size_t)h->nnodes * sizeof(unsigned long long)));
  h->last_buf = 0;
  h->dep_buf = h->cfg.fixed_efield ? 0 : 1;
  h->step = hdr[5];
  h->sims[0].ke_initial = ke0;
  std::copy(labs, labs + 4, h->sims[0].last_abs);
  h->sims[0].last_diag_step = lds;
  h->sticky = s.err;
  // spline mode: the field of the restored particles (the checkpoint holds
  // the node grids only)
  if (h->spl || h->web) return spline_refresh(h, true);
  return PIC_OK;
}

int pic_attach_unet(pic_handle* h, pic_unet* net, double rho_scale, double phi_scale,
                    double dphi_scale) {
  if (!h) return PIC_EINVAL;
  if (net && (!unet_fits(net, h->nsim, h->cfg.nr, h->cfg.nz) || !(rho_scale > 0) ||
              !(phi_scale > 0) || !(dphi_scale > 0)))
    return PIC_EINVAL;
  CK(cudaStreamSynchronize(h->stream));
  if (net && !h->ws_x) {
    h->ws_x = (float*)h_alloc((size_t)h->nsim * h->cfg.nr * h->cfg.nz * 2 * sizeof(float), h);
    if (!h->ws_x) return PIC_ENOMEM;
  }
  h->net = net;
  h->ws_scale[0] = (float)rho_scale;
  h->ws_scale[1] = (float)phi_scale;
  h->ws_scale[2] = (float)dphi_scale;
  // captured step blocks do not contain the net's launches: capture again
  drop_graphs(h);
  return PIC_OK;
}

// Schedule autotuner: the sort period and the fused kernel's persistent
// grid are tried on the running simulation (particle states do not depend
// on either: every particle's arithmetic is fixed, the FP32 deposit is an
// integer sum, child uids go by parent rank), each candidate timed with
// events over whole graph blocks; the fastest is kept.
int pic_autotune(pic_handle* h, int64_t steps_per_trial, pic_tune_result* out) {
  const int32_t sort_cand[] = {5, 10, 20, 40, 80};
  return pic_autotune_periods(h, steps_per_trial, sort_cand, 5, out);
}

int pic_autotune_periods(pic_handle* h, int64_t steps_per_trial, const int32_t* periods,
                         int n_periods, pic_tune_result* out) {
  if (!h || !out || steps_per_trial < 1 || !periods || n_periods < 1 || n_periods > 64)
    return PIC_EINVAL;
  for (int k = 0; k < n_periods; ++k)
    if (periods[k] < 1 || periods[k] > 100000) return PIC_EINVAL;
  if (h->sticky) return h->sticky;
  std::memset(out, 0, sizeof(*out));
  const std::vector<int> sort_cand(periods, periods + n_periods);
  std::vector<int> grid_cand;
  for (int b = 1; b <= h->blocks_per_sm; ++b) grid_cand.push_back(h->sms * b);
  // whole graph blocks of every candidate: a multiple of the lcm of their
  // block lengths
  long long unit = 1;
  for (int se : sort_cand) {
    const long long g = graph_len_of(se);
    unit = unit / std::gcd(unit, g) * g;
    if (unit > 1000000) return PIC_EINVAL;
  }
  const long long trial = (steps_per_trial + unit - 1) / unit * unit;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best = 1e300;
  int best_se = h->cfg.sort_every, best_grid = h->grid_particle;
  int rc = PIC_OK;
  for (int se : sort_cand) {
    for (int grid : grid_cand) {
      h->cfg.sort_every = se;
      for (pic_config& c : h->cfgs) c.sort_every = se;
      h->grid_particle = grid;
      set_graph_len(h);
      drop_graphs(h);
      // align to a graph block and capture, untimed
      rc = pic_step(h, h->graph_len + (h->graph_len - h->step % h->graph_len) % h->graph_len);
      if (rc) break;
      if (cudaEventRecord(e0, h->stream) != cudaSuccess) { rc = PIC_ECUDA; break; }
      rc = pic_step(h, trial);
      if (rc) break;
      float ms = 0.f;
      if (cudaEventRecord(e1, h->stream) != cudaSuccess ||
          cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = PIC_ECUDA;
        break;
      }
      ++out->trials;
      const double per = ms / (double)trial;
      if (per < best) { best = per; best_se = se; best_grid = grid; }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->cfg.sort_every = best_se;
  for (pic_config& c : h->cfgs) c.sort_every = best_se;
  h->grid_particle = best_grid;
  set_graph_len(h);
  drop_graphs(h);
  out->sort_every = best_se;
  out->particle_blocks = best_grid;
  out->ms_per_step = best;
  return rc ? rc : check_sticky(h);
}

int pic_field_images(pic_handle* h, float* rho, float* phi_rho) {
  if (!h) return PIC_EINVAL;
  const bool fp32 = h->prec == 32;
  const int rc = field_images(h->T, fp32 ? h->cnt[h->last_buf] : nullptr, h->q_units,
                              fp32 ? nullptr : h->rhs, rho, phi_rho, h->stream);
  return rc ? rc : check_sticky(h);
}

int pic_profile(pic_handle* h, int enable, pic_kernel_times* out) {
  if (!h) return PIC_EINVAL;
  if (enable) {
    h->profiling = true;
    h->ev_used = 0;
    h->ev_marks.clear();
    h->prof_kernels0 = h->kernels;
    return PIC_OK;
  }
  if (!out) return PIC_EINVAL;
  std::memset(out, 0, sizeof(*out));
  h->profiling = false;
  CK(cudaStreamSynchronize(h->stream));
  for (size_t k = 1; k < h->ev_marks.size(); ++k) {
    const int tag = h->ev_marks[k].second;
    if (tag == kTagStart) continue;
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev_pool[h->ev_marks[k - 1].first], h->ev_pool[h->ev_marks[k].first]));
    switch (tag) {
      case kTagParticle: out->particle_ms += ms; ++out->particle_launches; break;
      case kTagFinalize: out->finalize_ms += ms; break;
      case kTagSort: out->sort_ms += ms; ++out->sorts; break;
      case kTagField: out->field_ms += ms; ++out->field_solves; break;
    }
  }
  out->kernels_launched = h->kernels - h->prof_kernels0;
  h->ev_marks.clear();
  h->ev_used = 0;
  return PIC_OK;
}

}  // extern "C"
