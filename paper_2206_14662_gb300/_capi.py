"""ctypes binding of libpic (include/pic.h): the same entry points, argument
marshalling only.  Every step of the method runs in the library's CUDA
kernels; there is no CPU path.  Importing works without a GPU, but loading
the library requires it to have been built (``build.build()``), and any call
that reaches the device requires a CUDA GPU.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpic.so")

PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_ECAPACITY = 0, -1, -2, -3
PIC_ENOCONV, PIC_ETIMEOUT, PIC_ENONFINITE, PIC_ECUDA = -4, -5, -6, -7
PIC_GRID_PHI, PIC_GRID_RHS, PIC_GRID_ER, PIC_GRID_EZ = 0, 1, 2, 3
MOMENTS, FORCE_TERMS, FLUID_MODEL = 12, 7, 9   # PIC_MOMENTS, PIC_FORCE_TERMS, PIC_FLUID_MODEL

c_d, c_i32, c_i64, c_u64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64


class PicConfig(ctypes.Structure):
    _fields_ = [
        ("r_in", c_d), ("r_out", c_d), ("z_min", c_d), ("z_max", c_d),
        ("nr", c_i32), ("nz", c_i32), ("v_inner", c_d), ("v_outer", c_d),
        ("bfield_kind", c_i32), ("b0", c_d), ("p_mbar", c_d), ("t_gas_K", c_d),
        ("sigma_el", c_d), ("ion_E_th_eV", c_d), ("ion_sigma_pk", c_d),
        ("ion_E_pk_eV", c_d), ("opal_B_eV", c_d), ("xi_param", c_d),
        ("elastic_recoil", c_i32), ("gas_mass_amu", c_d), ("n_init", c_i64),
        ("n0", c_d), ("T0_eV", c_d), ("weight", c_d), ("dt", c_d),
        ("sort_every", c_i32), ("poisson_rtol", c_d), ("poisson_maxit", c_i32),
        ("capacity", c_i64), ("seed", c_u64), ("precision", c_i32),
        ("nu_max", c_d), ("fixed_efield", c_i32), ("warm_start", c_i32), ("source_rate", c_d),
        ("bspline_degree", c_i32), ("has_ellipse", c_i32), ("ellipse", c_d * 4),
    ]


class PicDiag(ctypes.Structure):
    _fields_ = [
        ("step", c_i64), ("t", c_d), ("n_particles", c_i64),
        ("I_inner", c_d), ("I_outer", c_d), ("I_zmin", c_d), ("I_zmax", c_d),
        ("absorbed_weight", c_d * 4),
        ("n_elastic", c_i64), ("n_ionise", c_i64), ("n_absorbed", c_i64),
        ("n_candidates", c_i64), ("n_over", c_i64), ("n_pushed", c_i64),
        ("kernels_launched", c_i64),
        ("ke_total_J", c_d), ("work_E_J", c_d), ("ke_absorbed_J", c_d),
        ("ion_loss_J", c_d), ("recoil_loss_J", c_d), ("ke_initial_J", c_d),
        ("ledger_residual_J", c_d), ("n_peak", c_d), ("poisson_iters", c_i32),
        ("poisson_relres", c_d), ("poisson_relres_charge", c_d), ("nu_max", c_d),
        ("weight", c_d), ("error", c_i32), ("poisson_relres_init", c_d),
        ("n_source", c_i64), ("ke_source_J", c_d), ("I_ellipse", c_d),
        ("absorbed_ellipse", c_d),
    ]


class PicKernelTimes(ctypes.Structure):
    _fields_ = [
        ("particle_ms", c_d), ("particle_launches", c_i64), ("finalize_ms", c_d),
        ("field_ms", c_d), ("field_solves", c_i64), ("sort_ms", c_d), ("sorts", c_i64),
        ("kernels_launched", c_i64),
    ]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class PicAllocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class PicError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {lib().pic_strerror(code).decode()} ({code})")


_lib = None


def lib() -> ctypes.CDLL:
    """Load libpic.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpic.so is not built ({LIB_PATH}); run "
                               "paper_2206_14662_gb300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        vp, P = ctypes.c_void_p, ctypes.POINTER
        L.pic_strerror.argtypes = [ctypes.c_int]
        L.pic_strerror.restype = ctypes.c_char_p
        L.pic_init.argtypes = [P(PicConfig), ctypes.c_int, vp, P(PicAllocator), P(vp)]
        L.pic_load_particles.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, vp, vp, c_i64]
        L.pic_step.argtypes = [vp, c_i64]
        L.pic_diagnostics.argtypes = [vp, ctypes.c_int, P(PicDiag), vp]
        L.pic_export_particles.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, vp, vp, c_i64, P(c_i64)]
        L.pic_set_efield.argtypes = [vp, ctypes.c_int, vp, vp]
        L.pic_set_cross_sections.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp]
        L.pic_moments.argtypes = [vp, ctypes.c_int, vp]
        L.pic_moments_accumulate.argtypes = [vp, ctypes.c_int, vp, c_d]
        L.pic_force_balance.argtypes = [vp, ctypes.c_int, vp, vp, c_d, vp]
        L.pic_fluid_model.argtypes = [vp, ctypes.c_int, vp, vp]
        L.pic_get_grid.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp]
        L.pic_solve_field.argtypes = [vp, vp, vp, P(c_d)]
        L.pic_checkpoint.argtypes = [vp, ctypes.c_char_p]
        L.pic_restore.argtypes = [vp, ctypes.c_char_p]
        L.pic_profile.argtypes = [vp, ctypes.c_int, P(PicKernelTimes)]
        L.pic_free.argtypes = [vp]
        L.pic_free.restype = None
        L.pic_spline_matrices.argtypes = [P(PicConfig), ctypes.c_int, vp, vp, vp, vp, vp, vp]
        L.pic_spline_eigen.argtypes = [P(PicConfig), ctypes.c_int, vp, vp]
        L.pic_spline_create.argtypes = [P(PicConfig), ctypes.c_int, vp, P(vp)]
        L.pic_spline_free.argtypes = [vp]
        L.pic_spline_free.restype = None
        L.pic_spline_sizes.argtypes = [vp, P(ctypes.c_int), P(ctypes.c_int)]
        L.pic_spline_set_stream.argtypes = [vp, vp]
        L.pic_spline_solve.argtypes = [vp, vp, vp, ctypes.c_int]
        L.pic_spline_deposit.argtypes = [vp, vp, vp, c_i64, c_d, vp]
        L.pic_spline_eval.argtypes = [vp, vp, vp, vp, c_i64, ctypes.c_int, vp, vp, vp]
        L.pic_web_create.argtypes = [P(PicConfig), vp, c_d, c_d, ctypes.c_int, ctypes.c_int, P(vp)]
        L.pic_web_free.argtypes = [vp]
        L.pic_web_free.restype = None
        L.pic_web_sizes.argtypes = [vp, P(ctypes.c_int), P(c_i64), P(c_i64), P(ctypes.c_int),
                                    P(ctypes.c_int)]
        L.pic_web_export.argtypes = [vp] * 9
        L.pic_web_device.argtypes = [vp, vp]
        L.pic_web_solve.argtypes = [vp, vp, vp, ctypes.c_int, c_d, ctypes.c_int,
                                    P(ctypes.c_int), P(c_d)]
        L.pic_web_deposit.argtypes = [vp, vp, vp, c_i64, c_d, vp]
        L.pic_web_eval.argtypes = [vp, vp, vp, vp, c_i64, ctypes.c_int, vp, vp, vp]
        L.pic_web_well_depth.argtypes = [vp, vp, vp, ctypes.c_int, c_d, ctypes.c_int,
                                         ctypes.c_int, c_d, c_d, c_d, vp, vp]
        L.pic_web_inverse.argtypes = [vp, vp]
        L.pic_web_direct.argtypes = [vp]
        L.pic_web_set_stream.argtypes = [vp, vp]
        L.pic_web_solve_direct.argtypes = [vp, vp, vp, ctypes.c_int]
        for name in ("pic_web_create", "pic_web_sizes", "pic_web_export", "pic_web_device",
                     "pic_web_solve", "pic_web_deposit", "pic_web_eval", "pic_web_well_depth",
                     "pic_web_inverse", "pic_web_direct", "pic_web_solve_direct",
                     "pic_web_set_stream"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("pic_spline_matrices", "pic_spline_eigen", "pic_spline_create",
                     "pic_spline_sizes", "pic_spline_solve", "pic_spline_deposit",
                     "pic_spline_eval", "pic_spline_set_stream"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("pic_init", "pic_load_particles", "pic_step", "pic_diagnostics",
                     "pic_export_particles", "pic_set_efield", "pic_set_cross_sections",
                     "pic_moments", "pic_moments_accumulate", "pic_force_balance", "pic_fluid_model",
                     "pic_get_grid", "pic_solve_field",
                     "pic_checkpoint", "pic_restore", "pic_profile"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != PIC_OK:
        raise PicError(rc, where)


def make_config(cfg: dict) -> PicConfig:
    """pic_config from a workload dict (keys are the struct's field names;
    other keys are ignored)."""
    c = PicConfig()
    if cfg.get("ellipse") is not None:   # (r0, z0, dr, dz) of the trap's ellipse
        c.has_ellipse = 1
        c.ellipse = (c_d * 4)(*[float(v) for v in cfg["ellipse"]])
    for name, ctype in PicConfig._fields_:
        if name in ("ellipse", "has_ellipse"):
            continue
        if name in cfg:
            setattr(c, name, ctype(cfg[name]).value if ctype in (c_i32, c_i64, c_u64) else float(cfg[name]))
    return c


def _f64(a):
    """(pointer, keep-alive) of a contiguous float64 host array or tensor."""
    if hasattr(a, "data_ptr"):
        assert a.dtype.__str__() == "torch.float64" and a.is_contiguous() and not a.is_cuda
        return ctypes.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(a, dtype=np.float64)
    return arr.ctypes.data_as(ctypes.c_void_p), arr


def _u64(a):
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(a, dtype=np.uint64)
    return arr.ctypes.data_as(ctypes.c_void_p), arr


def _torch_allocator():
    """A pic_allocator backed by PyTorch's CUDA caching allocator."""
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      stream or 0)
        except Exception:   # out of memory: the library reports PIC_ENOMEM
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    fa, ff = ALLOC_FN(_alloc), FREE_FN(_free)
    return PicAllocator(fa, ff, None), (fa, ff)


class Simulation:
    """One handle (pic_init ... pic_free): a single simulation (cfg a dict)
    or a batch stepped together (cfg a list of dicts, one per simulation;
    the per-simulation calls take ``sim``)."""

    def __init__(self, cfg, stream=None, torch_allocator: bool = True):
        L = lib()
        cfgs = [dict(c) for c in cfg] if isinstance(cfg, (list, tuple)) else [dict(cfg)]
        self.cfgs = cfgs
        self.cfg = cfgs[0]
        self.n_sims = len(cfgs)
        self._c = (PicConfig * len(cfgs))(*[make_config(c) for c in cfgs])
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = int(stream)
        self._keep = None
        alloc_p = None
        if torch_allocator:
            al, self._keep = _torch_allocator()
            self._alloc = al
            alloc_p = ctypes.byref(self._alloc)
        h = ctypes.c_void_p()
        _check(L.pic_init(self._c, len(cfgs), ctypes.c_void_p(self.stream), alloc_p,
                          ctypes.byref(h)), "pic_init")
        self.h = h
        self.nnodes = (self.cfg["nr"] + 1) * (self.cfg["nz"] + 1)

    def close(self):
        if getattr(self, "h", None):
            lib().pic_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def load_particles(self, r, z, vr, vt, vz, uid, sim: int = 0):
        ptrs = [_f64(a) for a in (r, z, vr, vt, vz)]
        pu = _u64(uid)
        n = len(r)
        _check(lib().pic_load_particles(self.h, sim, *[p for p, _ in ptrs], pu[0], n),
               "pic_load_particles")

    def step(self, nsteps: int = 1):
        _check(lib().pic_step(self.h, int(nsteps)), "pic_step")

    def diagnostics(self, density: bool = False, raise_on_error: bool = True,
                    sim: int = 0) -> dict:
        d = PicDiag()
        dens = np.zeros(self.nnodes) if density else None
        rc = lib().pic_diagnostics(self.h, sim, ctypes.byref(d),
                                   dens.ctypes.data_as(ctypes.c_void_p) if density else None)
        if raise_on_error:
            _check(rc, "pic_diagnostics")
        out = {name: (list(getattr(d, name)) if name == "absorbed_weight" else getattr(d, name))
               for name, _ in PicDiag._fields_}
        if density:
            out["density"] = dens
        return out

    def export_particles(self, sim: int = 0) -> dict:
        cap = int(self.diagnostics(raise_on_error=False, sim=sim)["n_particles"])
        arrs = [np.zeros(cap) for _ in range(5)]
        uid = np.zeros(cap, dtype=np.uint64)
        n = c_i64()
        _check(lib().pic_export_particles(self.h, sim, *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs],
                                          uid.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(n)),
               "pic_export_particles")
        k = n.value
        return dict(r=arrs[0][:k], z=arrs[1][:k], vr=arrs[2][:k], vt=arrs[3][:k], vz=arrs[4][:k],
                    uid=uid[:k])

    def set_efield(self, er, ez, sim: int = 0):
        pe, pz = _f64(er), _f64(ez)
        _check(lib().pic_set_efield(self.h, sim, pe[0], pz[0]), "pic_set_efield")

    def set_cross_sections(self, E_eV=None, sigma_el=None, sigma_io=None, xi=None, sim: int = 0):
        """Tabulated cross sections of simulation `sim` (pic_set_cross_sections);
        no arguments return to the config's analytic ones."""
        if E_eV is None:
            _check(lib().pic_set_cross_sections(self.h, sim, 0, None, None, None, None),
                   "pic_set_cross_sections")
            return
        pe, ps, pi = _f64(E_eV), _f64(sigma_el), _f64(sigma_io)
        px = _f64(xi) if xi is not None else (None, None)
        n = len(pe[1])
        assert len(ps[1]) == n and len(pi[1]) == n and (xi is None or len(px[1]) == n)
        _check(lib().pic_set_cross_sections(self.h, sim, n, pe[0], ps[0], pi[0], px[0]),
               "pic_set_cross_sections")

    def moments(self, sim: int = 0) -> np.ndarray:
        """Fluid moments on the nodes (pic_moments): shape (11, nr + 1, nz + 1)."""
        out = np.zeros((MOMENTS, self.cfg["nr"] + 1, self.cfg["nz"] + 1))
        _check(lib().pic_moments(self.h, sim, out.ctypes.data_as(ctypes.c_void_p)), "pic_moments")
        return out

    def moments_accumulate(self, acc, scale: float = 1.0, sim: int = 0):
        """Add scale x the moments to acc (pic_moments_accumulate), a CUDA
        float64 tensor of shape (12, nr + 1, nz + 1), asynchronously on the
        simulation's stream."""
        shape = (MOMENTS, self.cfg["nr"] + 1, self.cfg["nz"] + 1)
        if not (getattr(acc, "is_cuda", False) and str(acc.dtype) == "torch.float64"
                and acc.is_contiguous() and tuple(acc.shape) == shape):
            raise ValueError(f"acc must be a contiguous CUDA float64 tensor of shape {shape}")
        _check(lib().pic_moments_accumulate(self.h, sim, ctypes.c_void_p(acc.data_ptr()),
                                            float(scale)), "pic_moments_accumulate")

    def force_balance(self, moments, moments_prev=None, dt_prev: float = 0.0, sim: int = 0):
        """Force-balance terms (pic_force_balance) from moments of shape
        (11, nr + 1, nz + 1): shape (7, 3, nr + 1, nz + 1), terms F_E, F_B,
        F_i, F_p, F_d, F_a and their sum; components r, theta, z."""
        shape = (MOMENTS, self.cfg["nr"] + 1, self.cfg["nz"] + 1)
        for m in (moments, moments_prev):
            if m is not None and np.shape(m) != shape:
                raise ValueError(f"moments must have shape {shape}, got {np.shape(m)}")
        pm = _f64(np.ascontiguousarray(moments).ravel())
        pp = _f64(np.ascontiguousarray(moments_prev).ravel()) if moments_prev is not None else (None, None)
        out = np.zeros((FORCE_TERMS, 3, self.cfg["nr"] + 1, self.cfg["nz"] + 1))
        _check(lib().pic_force_balance(self.h, sim, pm[0], pp[0], float(dt_prev),
                                       out.ctypes.data_as(ctypes.c_void_p)), "pic_force_balance")
        return out

    def fluid_model(self, moments, sim: int = 0) -> np.ndarray:
        """Fluid-Poisson model predictions (pic_fluid_model) from moments of
        shape (12, nr + 1, nz + 1): shape (9, nr + 1, nz + 1), in the order
        u_theta, <nu_d>, <nu_io>, u_r, omega_p,max^2, n_max, nu_d and nu_io
        at the E x B drift speed, j."""
        shape = (MOMENTS, self.cfg["nr"] + 1, self.cfg["nz"] + 1)
        if np.shape(moments) != shape:
            raise ValueError(f"moments must have shape {shape}, got {np.shape(moments)}")
        pm = _f64(np.ascontiguousarray(moments).ravel())
        out = np.zeros((FLUID_MODEL, self.cfg["nr"] + 1, self.cfg["nz"] + 1))
        _check(lib().pic_fluid_model(self.h, sim, pm[0], out.ctypes.data_as(ctypes.c_void_p)),
               "pic_fluid_model")
        return out

    def get_grid(self, which: int, sim: int = 0) -> np.ndarray:
        out = np.zeros(self.nnodes)
        _check(lib().pic_get_grid(self.h, sim, which, out.ctypes.data_as(ctypes.c_void_p)),
               "pic_get_grid")
        return out

    def solve_field(self, b):
        pb = _f64(b)
        phi = np.zeros(self.nnodes)
        rel = c_d()
        _check(lib().pic_solve_field(self.h, pb[0], phi.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.byref(rel)), "pic_solve_field")
        return phi, rel.value

    def checkpoint(self, path: str):
        _check(lib().pic_checkpoint(self.h, path.encode()), "pic_checkpoint")

    def restore(self, path: str):
        _check(lib().pic_restore(self.h, path.encode()), "pic_restore")

    def attach_unet(self, net, rho_scale: float, phi_scale: float, dphi_scale: float):
        """Learned initial guess of the field solves (warm_start = 2)."""
        L = lib()
        L.pic_attach_unet.argtypes = [ctypes.c_void_p, ctypes.c_void_p, c_d, c_d, c_d]
        _check(L.pic_attach_unet(self.h, net.h if net is not None else None, rho_scale,
                                 phi_scale, dphi_scale), "pic_attach_unet")
        self._net = net

    def field_images(self, rho=None, phi_rho=None):
        """Charge and space-charge potential images (n_sims, nr, nz) into
        float32 CUDA tensors (either may be None)."""
        L = lib()
        L.pic_field_images.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        p = [ctypes.c_void_p(t.data_ptr()) if t is not None else None for t in (rho, phi_rho)]
        _check(L.pic_field_images(self.h, *p), "pic_field_images")

    def autotune(self, steps_per_trial: int = 80, periods=None) -> dict:
        """pic_autotune: time sort periods and fused-kernel grids on the
        running simulation (which advances) and keep the fastest.  periods:
        the candidate sort periods (pic_autotune_periods), default {5, 10,
        20, 40, 80}."""
        class R(ctypes.Structure):
            _fields_ = [("sort_every", c_i32), ("particle_blocks", c_i32),
                        ("ms_per_step", c_d), ("trials", c_i32)]
        L = lib()
        r = R()
        if periods is None:
            L.pic_autotune.argtypes = [ctypes.c_void_p, c_i64, ctypes.c_void_p]
            _check(L.pic_autotune(self.h, int(steps_per_trial), ctypes.byref(r)), "pic_autotune")
        else:
            arr = (c_i32 * len(periods))(*[int(p) for p in periods])
            L.pic_autotune_periods.argtypes = [ctypes.c_void_p, c_i64, ctypes.c_void_p,
                                               ctypes.c_int, ctypes.c_void_p]
            _check(L.pic_autotune_periods(self.h, int(steps_per_trial), arr, len(periods),
                                          ctypes.byref(r)), "pic_autotune_periods")
        return {name: getattr(r, name) for name, _ in R._fields_}

    def profile_start(self):
        _check(lib().pic_profile(self.h, 1, None), "pic_profile")

    def profile_stop(self) -> dict:
        t = PicKernelTimes()
        _check(lib().pic_profile(self.h, 0, ctypes.byref(t)), "pic_profile")
        return {name: getattr(t, name) for name, _ in PicKernelTimes._fields_}


def solve_field_static(cfg: dict, b_dev_ptr: int, phi_dev_ptr: int, stream: int = 0,
                       check: bool = True):
    """pic_solve_field_static: the field solve with no device allocation.
    ``b_dev_ptr`` and ``phi_dev_ptr`` are device addresses of (nr+1)*(nz+1)
    doubles owned by the caller.  Returns the relative residual when
    ``check`` (the call then synchronises the stream), else None."""
    L = lib()
    fn = L.pic_solve_field_static
    fn.argtypes = [ctypes.POINTER(PicConfig), ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.POINTER(c_d), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    c = make_config(cfg)
    rel = c_d()
    rc = fn(ctypes.byref(c), ctypes.c_void_p(b_dev_ptr), ctypes.c_void_p(phi_dev_ptr),
            ctypes.byref(rel) if check else None, ctypes.c_void_p(stream))
    _check(rc, "pic_solve_field_static")
    return rel.value if check else None


# ------------------------------------------------------- weighted B-splines

def _ptr_np(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def spline_matrices(cfg: dict, degree: int) -> dict:
    """The weighted B-spline field's 1D matrices (pic_spline_matrices,
    host only): K_r, M_r (mr x mr), g_r (mr), K_z, M_z (mz x mz), m_z (mz)."""
    mr, mz = cfg["nr"] + degree, cfg["nz"] + degree
    out = dict(K_r=np.zeros((mr, mr)), M_r=np.zeros((mr, mr)), g_r=np.zeros(mr),
               K_z=np.zeros((mz, mz)), M_z=np.zeros((mz, mz)), m_z=np.zeros(mz))
    c = make_config(cfg)
    _check(lib().pic_spline_matrices(ctypes.byref(c), int(degree),
                                     *[_ptr_np(out[k]) for k in ("K_r", "M_r", "g_r", "K_z",
                                                                "M_z", "m_z")]),
           "pic_spline_matrices")
    return out


def spline_eigen(cfg: dict, degree: int):
    """(V, lambda) of pic_spline_eigen (host only)."""
    mr = cfg["nr"] + degree
    V, lam = np.zeros((mr, mr)), np.zeros(mr)
    c = make_config(cfg)
    _check(lib().pic_spline_eigen(ctypes.byref(c), int(degree), _ptr_np(V), _ptr_np(lam)),
           "pic_spline_eigen")
    return V, lam


def _dev_f64(t, n=None, name="array"):
    if not (getattr(t, "is_cuda", False) and str(t.dtype) == "torch.float64" and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA float64 tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


class SplineSolver:
    """pic_spline_create ... pic_spline_free: the degree-n weighted B-spline
    field on the current CUDA device; arrays are torch CUDA float64
    tensors, coefficients of shape (mr, mz)."""

    def __init__(self, cfg: dict, degree: int, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.cfg, self.degree = dict(cfg), int(degree)
        h = ctypes.c_void_p()
        c = make_config(cfg)
        _check(lib().pic_spline_create(ctypes.byref(c), self.degree, ctypes.c_void_p(int(stream)),
                                       ctypes.byref(h)), "pic_spline_create")
        self.h = h
        mr, mz = ctypes.c_int(), ctypes.c_int()
        _check(lib().pic_spline_sizes(self.h, ctypes.byref(mr), ctypes.byref(mz)), "pic_spline_sizes")
        self.mr, self.mz = mr.value, mz.value

    def close(self):
        if self.h:
            lib().pic_spline_free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, f, dirichlet: bool = True):
        import torch
        c = torch.empty((self.mr, self.mz), dtype=torch.float64, device=f.device)
        _check(lib().pic_spline_solve(self.h, _dev_f64(f, self.mr * self.mz, "f"),
                                      _dev_f64(c), int(bool(dirichlet))), "pic_spline_solve")
        return c

    def deposit(self, r, z, qw: float, f=None):
        import torch
        if f is None:
            f = torch.zeros((self.mr, self.mz), dtype=torch.float64, device=r.device)
        n = r.numel()
        _check(lib().pic_spline_deposit(self.h, _dev_f64(r, n, "r"), _dev_f64(z, n, "z"), n,
                                        float(qw), _dev_f64(f, self.mr * self.mz, "f")),
               "pic_spline_deposit")
        return f

    def eval(self, c, r, z, dirichlet: bool = True):
        """(phi, E_r, E_z) at the points."""
        import torch
        n = r.numel()
        out = [torch.empty(n, dtype=torch.float64, device=r.device) for _ in range(3)]
        _check(lib().pic_spline_eval(self.h, _dev_f64(c, self.mr * self.mz, "c"),
                                     _dev_f64(r, n, "r"), _dev_f64(z, n, "z"), n,
                                     int(bool(dirichlet)), *[_dev_f64(o) for o in out]),
               "pic_spline_eval")
        return tuple(out)


def web_inverse(cfg: dict, ellipse, r_lo: float, r_hi: float, nr: int, degree: int) -> np.ndarray:
    """A^-1 of the web-spline system (pic_web_inverse, host only)."""
    c = make_config(cfg)
    e = None if ellipse is None else np.ascontiguousarray(ellipse, dtype=np.float64)
    h = ctypes.c_void_p()
    L = lib()
    _check(L.pic_web_create(ctypes.byref(c), _ptr_np(e), float(r_lo), float(r_hi), int(nr),
                            int(degree), ctypes.byref(h)), "pic_web_create")
    try:
        ni = ctypes.c_int()
        _check(L.pic_web_sizes(h, ctypes.byref(ni), None, None, None, None), "pic_web_sizes")
        out = np.zeros((ni.value, ni.value))
        _check(L.pic_web_inverse(h, _ptr_np(out)), "pic_web_inverse")
        return out
    finally:
        L.pic_web_free(h)


def web_system(cfg: dict, ellipse, r_lo: float, r_hi: float, nr: int, degree: int) -> dict:
    """The web-spline system of pic_web_create (host only): CSR arrays
    a_ptr, a_col, a_val (n_inner x n_inner), the lift load g, the full
    index of each inner function, and the extension T (t_ptr, t_col,
    t_val; mr * mz rows)."""
    c = make_config(cfg)
    e = None if ellipse is None else np.ascontiguousarray(ellipse, dtype=np.float64)
    h = ctypes.c_void_p()
    L = lib()
    _check(L.pic_web_create(ctypes.byref(c), _ptr_np(e), float(r_lo), float(r_hi), int(nr),
                            int(degree), ctypes.byref(h)), "pic_web_create")
    try:
        ni, nnz, tn = ctypes.c_int(), c_i64(), c_i64()
        mr, mz = ctypes.c_int(), ctypes.c_int()
        _check(L.pic_web_sizes(h, ctypes.byref(ni), ctypes.byref(nnz), ctypes.byref(tn),
                               ctypes.byref(mr), ctypes.byref(mz)), "pic_web_sizes")
        out = dict(a_ptr=np.zeros(ni.value + 1, np.int32), a_col=np.zeros(nnz.value, np.int32),
                   a_val=np.zeros(nnz.value), g=np.zeros(ni.value),
                   inner_full=np.zeros(ni.value, np.int32),
                   t_ptr=np.zeros(mr.value * mz.value + 1, np.int32),
                   t_col=np.zeros(tn.value, np.int32), t_val=np.zeros(tn.value))
        _check(L.pic_web_export(h, *[_ptr_np(out[k]) for k in ("a_ptr", "a_col", "a_val", "g",
                                                               "inner_full", "t_ptr", "t_col",
                                                               "t_val")]), "pic_web_export")
        out["mr"], out["mz"] = mr.value, mz.value
        return out
    finally:
        L.pic_web_free(h)


class WebSolver:
    """pic_web_create + pic_web_device ... pic_web_free: the web-spline
    field on the current CUDA device; arrays are torch CUDA float64
    tensors, full coefficients of shape (mr, mz)."""

    def __init__(self, cfg: dict, ellipse, r_lo: float, r_hi: float, nr: int, degree: int,
                 stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        c = make_config(cfg)
        e = None if ellipse is None else np.ascontiguousarray(ellipse, dtype=np.float64)
        h = ctypes.c_void_p()
        L = lib()
        _check(L.pic_web_create(ctypes.byref(c), _ptr_np(e), float(r_lo), float(r_hi), int(nr),
                                int(degree), ctypes.byref(h)), "pic_web_create")
        self.h = h
        mr, mz = ctypes.c_int(), ctypes.c_int()
        _check(L.pic_web_sizes(h, None, None, None, ctypes.byref(mr), ctypes.byref(mz)),
               "pic_web_sizes")
        self.mr, self.mz = mr.value, mz.value
        _check(L.pic_web_device(h, ctypes.c_void_p(int(stream))), "pic_web_device")

    def close(self):
        if self.h:
            lib().pic_web_free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def deposit(self, r, z, qw: float, f=None):
        import torch
        if f is None:
            f = torch.zeros((self.mr, self.mz), dtype=torch.float64, device=r.device)
        n = r.numel()
        _check(lib().pic_web_deposit(self.h, _dev_f64(r, n, "r"), _dev_f64(z, n, "z"), n,
                                     float(qw), _dev_f64(f, self.mr * self.mz, "f")),
               "pic_web_deposit")
        return f

    def solve_direct(self, f, dirichlet: bool = True):
        """c by the dense inverse (pic_web_direct once, then
        pic_web_solve_direct; asynchronous)."""
        import torch
        _check(lib().pic_web_direct(self.h), "pic_web_direct")
        c = torch.empty((self.mr, self.mz), dtype=torch.float64, device=f.device)
        _check(lib().pic_web_solve_direct(self.h, _dev_f64(f, self.mr * self.mz, "f"),
                                          _dev_f64(c), int(bool(dirichlet))),
               "pic_web_solve_direct")
        return c

    def solve(self, f, dirichlet: bool = True, rtol: float = 1e-12, maxit: int = 500):
        """(c, iterations, relative residual)."""
        import torch
        c = torch.empty((self.mr, self.mz), dtype=torch.float64, device=f.device)
        it, rel = ctypes.c_int(), c_d()
        _check(lib().pic_web_solve(self.h, _dev_f64(f, self.mr * self.mz, "f"), _dev_f64(c),
                                   int(bool(dirichlet)), float(rtol), int(maxit),
                                   ctypes.byref(it), ctypes.byref(rel)), "pic_web_solve")
        return c, it.value, rel.value

    def well_depth(self, c, r_start, z1: float, samples: int = 2001, bfield_kind: int = 0,
                   b0: float = 0.28, z_mid: float = 0.0, L: float = 1.0):
        """(U_d in eV, z of the well's maximum) on the field lines through
        (r, z1), r in r_start (pic_web_well_depth)."""
        rs = np.ascontiguousarray(r_start, dtype=np.float64)
        depth, z_at = np.zeros(len(rs)), np.zeros(len(rs))
        _check(lib().pic_web_well_depth(self.h, _dev_f64(c, self.mr * self.mz, "c"), _ptr_np(rs),
                                        len(rs), float(z1), int(samples), int(bfield_kind),
                                        float(b0), float(z_mid), float(L), _ptr_np(depth),
                                        _ptr_np(z_at)), "pic_web_well_depth")
        return depth, z_at

    def eval(self, c, r, z, dirichlet: bool = True):
        import torch
        n = r.numel()
        out = [torch.empty(n, dtype=torch.float64, device=r.device) for _ in range(3)]
        _check(lib().pic_web_eval(self.h, _dev_f64(c, self.mr * self.mz, "c"), _dev_f64(r, n, "r"),
                                  _dev_f64(z, n, "z"), n, int(bool(dirichlet)),
                                  *[_dev_f64(o) for o in out]), "pic_web_eval")
        return tuple(out)
