"""CPU FP64 oracle for the axisymmetric (r,z) 2D3V electrostatic PIC step with
null-collision Monte Carlo collisions (arXiv 2206.14662, Sec. II.A).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
cpu_baseline / reference legs of ``bench.py`` may use this package; the
product path never does.  It shares no code with the CUDA library and
imports nothing from it.

* The particle step (gather, Boris push, absorption, collisions, deposit) is
  plain C in ``pic_oracle.c``, one particle at a time, in double precision.
* The field solve is the finite-element system of Sec. II.A written out:
  the weak form of -div(eps0 grad phi) = rho with the axisymmetric volume
  element 2 pi r dr dz on bilinear elements, i.e. the global matrix
  2 pi eps0 (K_r (x) M_z + M_r (x) K_z), Dirichlet rows at the two metal
  walls and natural (Neumann) rows at the open z ends, solved by a sparse
  direct factorisation (a library primitive).
* The node field is E = -grad phi by central differences, one-sided
  second-order differences on the boundary rows (a reading: the paper does
  not state its field interpolation).

Functions whose results have no independent pin are marked "parity
unpinned" in their docstrings (none at present).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

# CODATA 2018 / exact SI values, written out for the oracle.
QE = 1.602176634e-19
ME = 9.1093837015e-31
EPS0 = 8.8541878128e-12
KB = 1.380649e-23
AMU = 1.66053906660e-27

T_ABS_INNER, T_ABS_OUTER, T_ABS_ZMIN, T_ABS_ZMAX = 0, 1, 2, 3
T_WORK_E, T_KE_ABSORBED, T_ION_LOSS, T_RECOIL_LOSS = 4, 5, 6, 7
T_N_ELASTIC, T_N_IONISE, T_N_ABSORBED, T_N_OVER, T_N_CANDIDATE = 8, 9, 10, 11, 12
T_ABS_ELLIPSE = 13
T_COUNT = 14

EV_NONE, EV_ELASTIC, EV_IONISE, EV_NULL = 0, 1, 2, 3
EV_WALL = 10  # 10 inner, 11 outer, 12 z_min, 13 z_max, 14 ellipse


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with the host compiler."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-fno-fast-math", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("r_in", ctypes.c_double), ("r_out", ctypes.c_double),
        ("z_min", ctypes.c_double), ("z_max", ctypes.c_double),
        ("nr", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("bfield_kind", ctypes.c_int32), ("elastic_recoil", ctypes.c_int32),
        ("b0", ctypes.c_double), ("n_gas", ctypes.c_double),
        ("sigma_el", ctypes.c_double), ("ion_E_th_eV", ctypes.c_double),
        ("ion_sigma_pk", ctypes.c_double), ("ion_E_pk_eV", ctypes.c_double),
        ("opal_B_eV", ctypes.c_double), ("xi", ctypes.c_double),
        ("gas_mass_kg", ctypes.c_double), ("weight", ctypes.c_double),
        ("dt", ctypes.c_double), ("nu_max", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("T0_eV", ctypes.c_double),
        ("xs_n", ctypes.c_int32), ("xs_E_eV", ctypes.c_void_p),
        ("xs_sigma_el", ctypes.c_void_p), ("xs_sigma_io", ctypes.c_void_p),
        ("xs_xi", ctypes.c_void_p), ("e_per_particle", ctypes.c_int32),
        ("has_ellipse", ctypes.c_int32), ("e_r0", ctypes.c_double), ("e_z0", ctypes.c_double),
        ("e_dr", ctypes.c_double), ("e_dz", ctypes.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        d, i64, u32, u64, vp = (ctypes.c_double, ctypes.c_int64, ctypes.c_uint32,
                                ctypes.c_uint64, ctypes.c_void_p)
        P = ctypes.POINTER(_Params)
        L.or_philox4x32_10.argtypes = [vp, vp, vp]
        L.or_philox4x32_10.restype = None
        L.or_nu_max.argtypes = [P, d]
        L.or_nu_max.restype = d
        L.or_sigma_ion.argtypes = [P, d]
        L.or_sigma_ion.restype = d
        L.or_xs_lookup.argtypes = [P, d, vp, vp, vp]
        L.or_xs_lookup.restype = None
        L.or_nu_parts.argtypes = [P, d, vp, vp]
        L.or_nu_parts.restype = None
        L.or_scatter_dir.argtypes = [vp, d, d, d, vp]
        L.or_scatter_dir.restype = None
        L.or_opal_secondary.argtypes = [d, d, d]
        L.or_opal_secondary.restype = d
        L.or_deposit.argtypes = [P, i64, vp, vp, vp]
        L.or_deposit.restype = None
        L.or_step.argtypes = [P, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                              u32, u64, i64, vp, vp, vp, vp, vp, vp, vp, vp]
        L.or_step.restype = i64
        L.or_kinetic_energy.argtypes = [P, i64, vp, vp, vp]
        L.or_kinetic_energy.restype = d
        L.or_source.argtypes = [P, i64, u64, u32, vp, vp, vp, vp, vp]
        L.or_source.restype = None
        L.or_set_threads.argtypes = [ctypes.c_int]
        L.or_set_threads.restype = None
        L.or_get_threads.argtypes = []
        L.or_get_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> None:
    """Threads of the particle loop of a step (OpenMP); the results do not
    depend on it."""
    lib().or_set_threads(int(n))


def threads() -> int:
    return int(lib().or_get_threads())


# ----------------------------------------------------------------- params

def derived(cfg: dict) -> dict:
    """Quantities the oracle derives from a workload description:
    neutral density n = p / (k T) with p in Pa; macro weight
    w = n0 pi (b^2 - a^2) L / N_init (unless given); gas mass; the energy
    cap 2 |V_in - V_out| eV of the collision majorant."""
    a, b = cfg["r_in"], cfg["r_out"]
    L = cfg["z_max"] - cfg["z_min"]
    n_gas = cfg["p_mbar"] * 100.0 / (KB * cfg["t_gas_K"])
    w = cfg["weight"] if cfg.get("weight", 0.0) > 0 else (
        cfg["n0"] * np.pi * (b * b - a * a) * L / cfg["n_init"])
    return dict(n_gas=n_gas, weight=w, gas_mass_kg=cfg["gas_mass_amu"] * AMU,
                E_cap_eV=2.0 * abs(cfg["v_inner"] - cfg["v_outer"]))


def params(cfg: dict) -> _Params:
    d = derived(cfg)
    p = _Params(
        r_in=cfg["r_in"], r_out=cfg["r_out"], z_min=cfg["z_min"], z_max=cfg["z_max"],
        nr=cfg["nr"], nz=cfg["nz"], bfield_kind=cfg["bfield_kind"],
        elastic_recoil=cfg["elastic_recoil"], b0=cfg["b0"], n_gas=d["n_gas"],
        sigma_el=cfg["sigma_el"], ion_E_th_eV=cfg["ion_E_th_eV"],
        ion_sigma_pk=cfg["ion_sigma_pk"], ion_E_pk_eV=cfg["ion_E_pk_eV"],
        opal_B_eV=cfg["opal_B_eV"], xi=cfg["xi_param"],
        gas_mass_kg=d["gas_mass_kg"], weight=d["weight"], dt=cfg["dt"],
        nu_max=0.0, seed=cfg["seed"], T0_eV=cfg.get("T0_eV", 1.0))
    xs = cfg.get("xs")
    if xs is not None:
        # tabulated cross sections: cfg["xs"] = dict(E_eV, sigma_el, sigma_io,
        # xi or None), kept alive on the structure
        arrs = [np.ascontiguousarray(xs[k], dtype=np.float64) for k in ("E_eV", "sigma_el", "sigma_io")]
        xi = xs.get("xi")
        arrs.append(None if xi is None else np.ascontiguousarray(xi, dtype=np.float64))
        p._xs_keep = arrs
        p.xs_n = len(arrs[0])
        p.xs_E_eV, p.xs_sigma_el, p.xs_sigma_io = (_ptr(a) for a in arrs[:3])
        p.xs_xi = None if arrs[3] is None else _ptr(arrs[3])
    ell = cfg.get("ellipse")
    if ell is not None:   # (r0, z0, dr, dz) of a filled metal ellipse
        p.has_ellipse = 1
        p.e_r0, p.e_z0, p.e_dr, p.e_dz = (float(v) for v in ell)
    if cfg.get("nu_max", 0.0) > 0:
        p.nu_max = cfg["nu_max"]
    else:
        p.nu_max = lib().or_nu_max(ctypes.byref(p), d["E_cap_eV"])
    return p


def source(cfg: dict, k: int, uid0: int, step: int):
    """k electrons of the volumetric seed source (Sec. II.A) born in step
    `step` with uids uid0.. (see or_source): arrays r, z, vr, vt, vz."""
    P = params(cfg)
    out = [np.zeros(max(k, 1)) for _ in range(5)]
    lib().or_source(ctypes.byref(P), k, uid0, step & 0xFFFFFFFF, *[_ptr(a) for a in out])
    return [a[:k] for a in out]


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def scatter_dir(vhat, u_chi, u_phi, xi) -> np.ndarray:
    v = np.ascontiguousarray(vhat, dtype=np.float64)
    out = np.zeros(3)
    lib().or_scatter_dir(_ptr(v), float(u_chi), float(u_phi), float(xi), _ptr(out))
    return out


def opal_secondary(E_rem, B, u) -> float:
    return lib().or_opal_secondary(float(E_rem), float(B), float(u))


def sigma_ion(cfg: dict, E_eV: float) -> float:
    p = params(dict(cfg, nu_max=1.0))   # (the majorant is not needed here)
    return lib().or_sigma_ion(ctypes.byref(p), float(E_eV))


def xs_lookup(cfg: dict, E_eV: float):
    """(sigma_el, sigma_io, xi) of cfg["xs"] at energy E_eV (see
    or_xs_lookup)."""
    p = params(dict(cfg, nu_max=1.0))   # (the majorant is not needed here)
    out = [ctypes.c_double() for _ in range(3)]
    lib().or_xs_lookup(ctypes.byref(p), float(E_eV), *[ctypes.byref(o) for o in out])
    return tuple(o.value for o in out)


def nu_parts(cfg: dict, speed):
    """(nu_el, nu_io) at each speed (m/s): elastic and ionisation
    frequencies of the collision path."""
    p = params(dict(cfg, nu_max=1.0))   # (the majorant is not needed here)
    L = lib()
    speed = np.ravel(np.asarray(speed, dtype=float))
    el, io = np.zeros(speed.size), np.zeros(speed.size)
    a, b = ctypes.c_double(), ctypes.c_double()
    for k, v in enumerate(speed):
        L.or_nu_parts(ctypes.byref(p), float(v), ctypes.byref(a), ctypes.byref(b))
        el[k], io[k] = a.value, b.value
    return el, io


def nu_drag(cfg: dict, speed) -> np.ndarray:
    """Electron-neutral momentum-exchange frequency nu_el + nu_io at each
    speed (m/s)."""
    el, io = nu_parts(cfg, speed)
    return el + io


def nu_max(cfg: dict) -> float:
    """The collision majorant the oracle derives for cfg (or cfg's own)."""
    return params(cfg).nu_max


# ------------------------------------------------------------------ grid

def grid(cfg: dict):
    """Node coordinates r_i (i = 0..nr) and z_j (j = 0..nz); node (i, j) is
    stored at i * (nz + 1) + j."""
    r = cfg["r_in"] + (cfg["r_out"] - cfg["r_in"]) * np.arange(cfg["nr"] + 1) / cfg["nr"]
    z = cfg["z_min"] + (cfg["z_max"] - cfg["z_min"]) * np.arange(cfg["nz"] + 1) / cfg["nz"]
    return r, z


def fem_1d(cfg: dict):
    """1D element matrices assembled on the node lines (dense, small):
    K_r, M_r are r-weighted (int r dr), K_z, M_z are plain; elements of
    length h with ends r0, r1:
      K_r^e = (r0 + r1)/(2h) [[1,-1],[-1,1]]
      M_r^e = h/12 [[3 r0 + r1, r0 + r1], [r0 + r1, r0 + 3 r1]]
      K_z^e = 1/h [[1,-1],[-1,1]],  M_z^e = h/6 [[2,1],[1,2]]."""
    r, z = grid(cfg)
    nr, nz = cfg["nr"], cfg["nz"]
    Kr = np.zeros((nr + 1, nr + 1)); Mr = np.zeros((nr + 1, nr + 1))
    for e in range(nr):
        r0, r1 = r[e], r[e + 1]
        h = r1 - r0
        Kr[e:e + 2, e:e + 2] += (r0 + r1) / (2 * h) * np.array([[1, -1], [-1, 1]])
        Mr[e:e + 2, e:e + 2] += h / 12 * np.array([[3 * r0 + r1, r0 + r1], [r0 + r1, r0 + 3 * r1]])
    Kz = np.zeros((nz + 1, nz + 1)); Mz = np.zeros((nz + 1, nz + 1))
    for e in range(nz):
        h = z[e + 1] - z[e]
        Kz[e:e + 2, e:e + 2] += 1 / h * np.array([[1, -1], [-1, 1]])
        Mz[e:e + 2, e:e + 2] += h / 6 * np.array([[2, 1], [1, 2]])
    return Kr, Mr, Kz, Mz


_factor_cache: dict = {}


def _system(cfg: dict):
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    key = (cfg["r_in"], cfg["r_out"], cfg["z_min"], cfg["z_max"], cfg["nr"], cfg["nz"])
    if key not in _factor_cache:
        Kr, Mr, Kz, Mz = fem_1d(cfg)
        A = 2 * np.pi * EPS0 * (sp.kron(sp.csr_matrix(Kr), sp.csr_matrix(Mz)) +
                                sp.kron(sp.csr_matrix(Mr), sp.csr_matrix(Kz)))
        A = A.tocsr()
        nr, nz = cfg["nr"], cfg["nz"]
        nzp = nz + 1
        interior = np.arange(nzp, nr * nzp)           # r-node rows 1..nr-1
        dirichlet = np.concatenate([np.arange(nzp), np.arange(nr * nzp, (nr + 1) * nzp)])
        A_II = A[interior][:, interior].tocsc()
        A_ID = A[interior][:, dirichlet].tocsr()
        _factor_cache.clear()
        _factor_cache[key] = (A, A_II, A_ID, interior, dirichlet, spla.splu(A_II))
    return _factor_cache[key]


def fem_matrix(cfg: dict):
    """The global sparse matrix 2 pi eps0 (K_r (x) M_z + M_r (x) K_z)."""
    return _system(cfg)[0]


def dirichlet_values(cfg: dict) -> np.ndarray:
    nzp = cfg["nz"] + 1
    return np.concatenate([np.full(nzp, cfg["v_inner"]), np.full(nzp, cfg["v_outer"])])


def poisson_solve(cfg: dict, b: np.ndarray) -> np.ndarray:
    """phi on all nodes: phi = V_in on r = a, V_out on r = b, and
    A_II phi_I = b_I - A_ID phi_D on the other nodes."""
    A, A_II, A_ID, interior, dirichlet, lu = _system(cfg)
    phi_D = dirichlet_values(cfg)
    phi = np.zeros((cfg["nr"] + 1) * (cfg["nz"] + 1))
    phi[dirichlet] = phi_D
    phi[interior] = lu.solve(b[interior] - A_ID @ phi_D)
    return phi


def poisson_relres(cfg: dict, b: np.ndarray, phi: np.ndarray) -> float:
    """||b_I - A_II phi_I - A_ID phi_D|| / ||b_I - A_ID phi_D||."""
    A, A_II, A_ID, interior, dirichlet, lu = _system(cfg)
    rhs = b[interior] - A_ID @ phi[dirichlet]
    res = rhs - A_II @ phi[interior]
    nb = np.linalg.norm(rhs)
    return float(np.linalg.norm(res) / nb) if nb > 0 else 0.0


def efield(cfg: dict, phi: np.ndarray):
    """Node field E = -grad phi: central differences inside, one-sided
    second-order differences on the first and last node lines."""
    nr, nz = cfg["nr"], cfg["nz"]
    hr = (cfg["r_out"] - cfg["r_in"]) / nr
    hz = (cfg["z_max"] - cfg["z_min"]) / nz
    f = phi.reshape(nr + 1, nz + 1)
    dr = np.empty_like(f); dz = np.empty_like(f)
    dr[1:-1] = (f[2:] - f[:-2]) / (2 * hr)
    dr[0] = (-3 * f[0] + 4 * f[1] - f[2]) / (2 * hr)
    dr[-1] = (3 * f[-1] - 4 * f[-2] + f[-3]) / (2 * hr)
    dz[:, 1:-1] = (f[:, 2:] - f[:, :-2]) / (2 * hz)
    dz[:, 0] = (-3 * f[:, 0] + 4 * f[:, 1] - f[:, 2]) / (2 * hz)
    dz[:, -1] = (3 * f[:, -1] - 4 * f[:, -2] + f[:, -3]) / (2 * hz)
    return (-dr).ravel(), (-dz).ravel()


def node_volumes(cfg: dict) -> np.ndarray:
    """V_ij = integral of the hat function Lambda_ij over the volume:
    2 pi R_i Z_j with R_i = r_i h_r inside, h_r (a/2 + h_r/6) at r = a,
    h_r (b/2 - h_r/6) at r = b, and Z_j = h_z inside, h_z / 2 at the ends."""
    nr, nz = cfg["nr"], cfg["nz"]
    a, b = cfg["r_in"], cfg["r_out"]
    hr = (b - a) / nr
    hz = (cfg["z_max"] - cfg["z_min"]) / nz
    r, _ = grid(cfg)
    R = r * hr
    R[0] = hr * (a / 2 + hr / 6)
    R[-1] = hr * (b / 2 - hr / 6)
    Z = np.full(nz + 1, hz)
    Z[0] = Z[-1] = hz / 2
    return (2 * np.pi * np.outer(R, Z)).ravel()


def deposit(cfg: dict, r: np.ndarray, z: np.ndarray) -> np.ndarray:
    p = params(cfg)
    b = np.zeros((cfg["nr"] + 1) * (cfg["nz"] + 1))
    r = np.ascontiguousarray(r, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    lib().or_deposit(ctypes.byref(p), len(r), _ptr(r), _ptr(z), _ptr(b))
    return b


def density(cfg: dict, b: np.ndarray) -> np.ndarray:
    """Electron density per node: (b_i / q) / V_i with q = -e."""
    return (b / -QE) / node_volumes(cfg)


# ------------------------------------------------------------- simulation

@dataclass
class StepResult:
    n_children: int
    event: np.ndarray      # per input particle
    margin: np.ndarray     # per input particle
    b: np.ndarray          # deposit of this step
    tally: np.ndarray      # this step only


class OracleSim:
    """One simulation advanced one step at a time.

    Particles are kept sorted by uid; children are appended (their uids are
    above every existing uid, so the order is kept).  Step n: particle step
    with E^n, removal of absorbed particles, then field solve for E^{n+1}.

    With cfg["bspline_degree"] = n >= 1 the field is the weighted B-spline
    field of degree n (oracle.bspline), or with cfg["ellipse"] = (r0, z0,
    dr, dz) as well the web-spline field of the gap minus that metal
    ellipse (oracle.webspline; particles entering the ellipse are absorbed
    and tallied in T_ABS_ELLIPSE): particles deposit with its basis and
    are pushed with its exact gradient at their position; self.coef holds
    its coefficients (self.phi, self.er, self.ez are then None).
    """

    def __init__(self, cfg: dict, r, z, vr, vt, vz, uid, efield_nodes=None,
                 solve_field: bool = True, step0: int = 0, uid_next: int | None = None):
        self.cfg = dict(cfg)
        self.P = params(self.cfg)
        order = np.argsort(np.asarray(uid, dtype=np.uint64), kind="stable")
        self.r = np.array(r, dtype=np.float64)[order]
        self.z = np.array(z, dtype=np.float64)[order]
        self.vr = np.array(vr, dtype=np.float64)[order]
        self.vt = np.array(vt, dtype=np.float64)[order]
        self.vz = np.array(vz, dtype=np.float64)[order]
        self.uid = np.array(uid, dtype=np.uint64)[order]
        self.step_index = step0
        self.uid_next = int(self.uid.max()) + 1 if uid_next is None and len(self.uid) else (uid_next or 0)
        self.tally = np.zeros(T_COUNT)
        self.n_source = 0
        self.ke_source = 0.0  # kinetic energy brought in by the seed source, J
        self.src_acc = 0.0    # fractional seed-source count carried between steps
        self.solve_field = solve_field
        self.spline = None
        if self.cfg.get("bspline_degree", 0) > 0:
            if self.cfg.get("ellipse") is not None:
                from .webspline import Geometry, WebSplineField
                c = self.cfg
                geo = Geometry(c["r_in"], c["r_out"], c["z_min"], c["z_max"], c["v_inner"],
                               c["v_outer"], ellipse=tuple(c["ellipse"]))
                self.spline = WebSplineField(geo, int(c["bspline_degree"]), c["r_in"],
                                             c["r_out"], c["nr"], c["nz"])
            else:
                from .bspline import SplineField
                self.spline = SplineField(self.cfg)
            self.P.e_per_particle = 1
            self.qw = -QE * derived(self.cfg)["weight"]
            self.b = self.spline.deposit(self.r, self.z, self.qw)
            self.coef = self.spline.solve(self.b)
            self.phi = self.er = self.ez = None
            self.ke0 = self.kinetic_energy()
            return
        self.b = deposit(self.cfg, self.r, self.z)
        if efield_nodes is not None:
            self.er, self.ez = (np.array(efield_nodes[0], dtype=np.float64),
                                np.array(efield_nodes[1], dtype=np.float64))
            self.phi = None
        else:
            self.phi = poisson_solve(self.cfg, self.b)
            self.er, self.ez = efield(self.cfg, self.phi)
        self.ke0 = self.kinetic_energy()

    @property
    def n(self) -> int:
        return len(self.r)

    def kinetic_energy(self) -> float:
        return lib().or_kinetic_energy(ctypes.byref(self.P), self.n, _ptr(self.vr),
                                       _ptr(self.vt), _ptr(self.vz))

    def set_efield(self, er, ez):
        self.er = np.array(er, dtype=np.float64)
        self.ez = np.array(ez, dtype=np.float64)

    def step(self) -> StepResult:
        n = self.n
        cap = max(16, n)
        event = np.zeros(n, dtype=np.int8)
        margin = np.zeros(n)
        ch = [np.zeros(cap) for _ in range(5)]
        cu = np.zeros(cap, dtype=np.uint64)
        b = np.zeros((self.cfg["nr"] + 1) * (self.cfg["nz"] + 1))
        tally = np.zeros(T_COUNT)
        if self.spline is not None:   # E at each particle from the spline field
            er, ez = self.spline.efield(self.coef, self.r, self.z)
            er, ez = np.ascontiguousarray(er), np.ascontiguousarray(ez)
        else:
            er, ez = self.er, self.ez
        nc = lib().or_step(ctypes.byref(self.P), n, _ptr(self.r), _ptr(self.z), _ptr(self.vr),
                           _ptr(self.vt), _ptr(self.vz), _ptr(self.uid), _ptr(event),
                           _ptr(margin), _ptr(er), _ptr(ez),
                           self.step_index & 0xFFFFFFFF, self.uid_next, cap,
                           _ptr(ch[0]), _ptr(ch[1]), _ptr(ch[2]), _ptr(ch[3]), _ptr(ch[4]),
                           _ptr(cu), _ptr(b), _ptr(tally))
        if nc < 0:
            raise RuntimeError("oracle child buffer overflow")
        keep = event < EV_WALL
        self.r = np.concatenate([self.r[keep], ch[0][:nc]])
        self.z = np.concatenate([self.z[keep], ch[1][:nc]])
        self.vr = np.concatenate([self.vr[keep], ch[2][:nc]])
        self.vt = np.concatenate([self.vt[keep], ch[3][:nc]])
        self.vz = np.concatenate([self.vz[keep], ch[4][:nc]])
        self.uid = np.concatenate([self.uid[keep], cu[:nc]])
        self.uid_next += int(nc)
        # volumetric seed source (Sec. II.A): source_rate macro-electrons per
        # second, whole ones injected, the fraction carried over (FP64)
        rate = self.cfg.get("source_rate", 0.0)
        if rate > 0:
            self.src_acc += rate * self.cfg["dt"]
            k = int(np.floor(self.src_acc))
            self.src_acc -= k
            if k > 0:
                new = source(self.cfg, k, self.uid_next, self.step_index)
                b = b + deposit(self.cfg, new[0], new[1])
                for name, arr in zip(("r", "z", "vr", "vt", "vz"), new):
                    setattr(self, name, np.concatenate([getattr(self, name), arr]))
                self.uid = np.concatenate([self.uid, np.arange(self.uid_next, self.uid_next + k,
                                                               dtype=np.uint64)])
                self.uid_next += k
                self.n_source += k
                self.ke_source += lib().or_kinetic_energy(ctypes.byref(self.P), k, _ptr(new[2]),
                                                          _ptr(new[3]), _ptr(new[4]))
        self.step_index += 1
        self.tally += tally
        if self.spline is not None:
            # every particle after the step (survivors, children, source)
            # deposits with the spline basis
            self.b = self.spline.deposit(self.r, self.z, self.qw)
            if self.solve_field:
                self.coef = self.spline.solve(self.b)
            return StepResult(int(nc), event, margin, self.b, tally)
        self.b = b
        if self.solve_field:
            self.phi = poisson_solve(self.cfg, b)
            self.er, self.ez = efield(self.cfg, self.phi)
        return StepResult(int(nc), event, margin, b, tally)

    def ledger_residual(self) -> float:
        """KE_now - KE_0 - (W_E - KE_absorbed - ionisation loss - recoil loss
        + KE brought in by the seed source)."""
        t = self.tally
        return (self.kinetic_energy() - self.ke0) - (
            t[T_WORK_E] - t[T_KE_ABSORBED] - t[T_ION_LOSS] - t[T_RECOIL_LOSS] + self.ke_source)
