"""Fluid moments of the particle distribution on the nodes and the terms of
the electron fluid's force balance (arXiv 2206.14662, Sec. IV.A: the forces
on the electron fluid are evaluated from moments of the distribution
function, and their sum is approximately zero) -- plain numpy, FP64.

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's
CPU baseline use this package.

moments(): for node i with hat function Lambda_i (bilinear on the (r, z)
cell) and volume V_i,
    M_c(i) = (w / V_i) sum_p Lambda_i(r_p, z_p) g_c(v_p),
    g = (1, v_r, v_t, v_z, v_r v_r, v_r v_t, v_r v_z, v_t v_t, v_t v_z,
         v_z v_z, nu_d(|v|), nu_io(|v|)),
so M_0 = n, M_1..3 = n u, M_4..9 = n <v v>, M_10 = n <nu_d> (momentum
exchange: elastic + ionisation), M_11 = n <nu_io>.

force_terms(): with u = (n u) / n, P = m (n <v v> - n u u) (u = 0, P = 0
where n = 0), q = -e, m = m_e, components (r, theta, z):
    F_E = q n (E_r, 0, E_z)
    F_B = q n u x B,  B = (B_r, 0, B_z) of the config
    F_i = -m n [u_r d_r u + u_z d_z u + (-u_t^2 / r, u_r u_t / r, 0)]
    F_p = -div P = -[(1/r) d_r(r P_rr) + d_z P_rz - P_tt / r,
                     (1/r^2) d_r(r^2 P_rt) + d_z P_tz,
                     (1/r) d_r(r P_rz) + d_z P_zz]
    F_d = -m n <nu_d> u
    F_a = m n (u - u_prev) / dt_prev
    S   = F_i + F_E + F_B + F_p + F_d - F_a
with derivatives by central differences and one-sided second-order ones on
the boundary lines.

fluid_model(): the fluid-Poisson model of Sec. V.A (force balance without
pressure, continuity, Gauss's law) evaluated per node, with
Omega_c = e B_z / m and omega_p^2 = e^2 n / (eps0 m):
    u_theta = -E_r / B_z                                 (radial balance)
    <nu_d>, <nu_io> = M_10 / n, M_11 / n
    u_r = -(q <nu_d> / m) E_r / (omega_p^2 - Omega_c^2)  (azimuthal balance)
    omega_p,max^2 = Omega_c^2 <nu_io> / (<nu_io> + <nu_d>)  (peak density)
    n_max = eps0 m omega_p,max^2 / e^2
    nu_d, nu_io at the drift speed |E x B| / |B|^2         (Sec. V.B)
    j = -eps0 E_r <nu_io>     (peak current 2 pi L r_+ j, L and r_+ the
                               cloud's length and outer radius)
zero where n = 0 or a denominator vanishes.
"""
from __future__ import annotations

import numpy as np

from . import ME, QE, grid, node_volumes, nu_parts

EPS0 = 8.8541878128e-12
MOMENTS = 12
FLUID_MODEL = ("u_theta", "nu_d", "nu_io", "u_r", "omega_p2_max", "n_max",
               "nu_d_drift", "nu_io_drift", "j")
TERMS = ("F_E", "F_B", "F_i", "F_p", "F_d", "F_a", "sum")


def moments(cfg: dict, r, z, vr, vt, vz, weight: float) -> np.ndarray:
    """(11, nr + 1, nz + 1) moments of the particles (absolute positions)."""
    nr, nz = cfg["nr"], cfg["nz"]
    hr = (cfg["r_out"] - cfg["r_in"]) / nr
    hz = (cfg["z_max"] - cfg["z_min"]) / nz
    sr = (np.asarray(r, float) - cfg["r_in"]) / hr
    sz = (np.asarray(z, float) - cfg["z_min"]) / hz
    ir = np.clip(np.floor(sr).astype(int), 0, nr - 1)
    iz = np.clip(np.floor(sz).astype(int), 0, nz - 1)
    fr, fz = sr - ir, sz - iz
    vr, vt, vz = (np.asarray(a, float) for a in (vr, vt, vz))
    nu_el, nu_io = nu_parts(cfg, np.sqrt(vr * vr + vt * vt + vz * vz))
    g = [np.ones_like(vr), vr, vt, vz, vr * vr, vr * vt, vr * vz, vt * vt, vt * vz, vz * vz,
         nu_el + nu_io, nu_io]
    corners = [(0, 0, (1 - fr) * (1 - fz)), (1, 0, fr * (1 - fz)), (0, 1, (1 - fr) * fz),
               (1, 1, fr * fz)]
    M = np.zeros((MOMENTS, nr + 1, nz + 1))
    for c in range(MOMENTS):
        for di, dj, lam in corners:
            np.add.at(M[c], (ir + di, iz + dj), lam * g[c])
    V = node_volumes(cfg).reshape(nr + 1, nz + 1)
    return M * (weight / V)


def _d(f: np.ndarray, h: float, axis: int) -> np.ndarray:
    """Derivative along `axis`: central inside, one-sided second order at
    the two ends."""
    f = np.moveaxis(f, axis, 0)
    d = np.empty_like(f)
    d[1:-1] = (f[2:] - f[:-2]) / (2 * h)
    d[0] = (-3 * f[0] + 4 * f[1] - f[2]) / (2 * h)
    d[-1] = (3 * f[-1] - 4 * f[-2] + f[-3]) / (2 * h)
    return np.moveaxis(d, 0, axis)


def _fluid(M: np.ndarray):
    n = M[0]
    has = n > 0
    u = np.where(has, M[1:4] / np.where(has, n, 1.0), 0.0)
    pairs = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))
    P = np.array([np.where(has, ME * (M[4 + k] - n * u[a] * u[b]), 0.0)
                  for k, (a, b) in enumerate(pairs)])
    return n, u, P


def magnetic_field(cfg: dict):
    """(B_r, B_z) on the nodes: uniform b0, or the mirror field."""
    r, z = grid(cfg)
    R, Z = np.meshgrid(r, z, indexing="ij")
    b0 = cfg["b0"]
    if cfg["bfield_kind"] == 1:
        L = cfg["z_max"] - cfg["z_min"]
        zeta = Z - 0.5 * (cfg["z_min"] + cfg["z_max"])
        return -2 * b0 * R * zeta / L ** 2, b0 * (1 + 2 * zeta ** 2 / L ** 2)
    return np.zeros_like(R), np.full_like(R, b0)


def force_terms(cfg: dict, M: np.ndarray, Er: np.ndarray, Ez: np.ndarray,
                M_prev: np.ndarray | None = None, dt_prev: float = 0.0) -> np.ndarray:
    """(7, 3, nr + 1, nz + 1): F_E, F_B, F_i, F_p, F_d, F_a, sum."""
    nr, nz = cfg["nr"], cfg["nz"]
    hr = (cfg["r_out"] - cfg["r_in"]) / nr
    hz = (cfg["z_max"] - cfg["z_min"]) / nz
    r, _ = grid(cfg)
    R = np.broadcast_to(r[:, None], (nr + 1, nz + 1))
    n, u, P = _fluid(M)
    q, m = -QE, ME
    Br, Bz = magnetic_field(cfg)
    Er = np.asarray(Er, float).reshape(nr + 1, nz + 1)
    Ez = np.asarray(Ez, float).reshape(nr + 1, nz + 1)
    T = np.zeros((7, 3, nr + 1, nz + 1))
    T[0] = [q * n * Er, np.zeros_like(n), q * n * Ez]
    T[1] = [q * n * u[1] * Bz, q * n * (u[2] * Br - u[0] * Bz), -q * n * u[1] * Br]
    dur = [_d(u[a], hr, 0) for a in range(3)]
    duz = [_d(u[a], hz, 1) for a in range(3)]
    T[2] = [-m * n * (u[0] * dur[0] + u[2] * duz[0] - u[1] ** 2 / R),
            -m * n * (u[0] * dur[1] + u[2] * duz[1] + u[0] * u[1] / R),
            -m * n * (u[0] * dur[2] + u[2] * duz[2])]
    Prr, Prt, Prz, Ptt, Ptz, Pzz = P
    T[3] = [-(_d(R * Prr, hr, 0) / R + _d(Prz, hz, 1) - Ptt / R),
            -(_d(R * R * Prt, hr, 0) / (R * R) + _d(Ptz, hz, 1)),
            -(_d(R * Prz, hr, 0) / R + _d(Pzz, hz, 1))]
    T[4] = -m * M[10] * u
    if M_prev is not None and dt_prev > 0:
        _, u_prev, _ = _fluid(M_prev)
        T[5] = m * n * (u - u_prev) / dt_prev
    T[6] = T[2] + T[0] + T[1] + T[3] + T[4] - T[5]
    return T


def fluid_model(cfg: dict, M: np.ndarray, Er: np.ndarray, Ez: np.ndarray) -> np.ndarray:
    """(9, nr + 1, nz + 1) fluid-model grids in the order of FLUID_MODEL."""
    shp = (cfg["nr"] + 1, cfg["nz"] + 1)
    Er = np.asarray(Er, float).reshape(shp)
    Ez = np.asarray(Ez, float).reshape(shp)
    Br, Bz = magnetic_field(cfg)
    q, m = -QE, ME
    n = M[0]
    has = n > 0
    safe = np.where(has, n, 1.0)
    nu_d = np.where(has, M[10] / safe, 0.0)
    nu_io = np.where(has, M[11] / safe, 0.0)
    Oc2 = (QE * Bz / m) ** 2
    wp2 = QE ** 2 * n / (EPS0 * m)
    den = wp2 - Oc2
    u_r = np.where(den != 0, -(q * nu_d / m) * Er / np.where(den != 0, den, 1.0), 0.0)
    tot = nu_io + nu_d
    w2 = np.where(tot > 0, Oc2 * nu_io / np.where(tot > 0, tot, 1.0), 0.0)
    # drift speed |E x B| / |B|^2 with E = (E_r, 0, E_z), B = (B_r, 0, B_z)
    E3 = np.stack([Er, np.zeros_like(Er), Ez], axis=-1)
    B3 = np.stack([Br, np.zeros_like(Br), Bz], axis=-1)
    B2 = (B3 ** 2).sum(-1)
    vd = np.linalg.norm(np.cross(E3, B3), axis=-1) / B2
    d_el, d_io = nu_parts(cfg, vd.ravel())
    out = np.zeros((len(FLUID_MODEL),) + shp)
    out[0] = np.where(Bz != 0, -Er / np.where(Bz != 0, Bz, 1.0), 0.0)
    out[1], out[2], out[3], out[4] = nu_d, nu_io, u_r, w2
    out[5] = EPS0 * m * w2 / QE ** 2
    out[6] = (d_el + d_io).reshape(shp)
    out[7] = d_io.reshape(shp)
    out[8] = -EPS0 * Er * nu_io
    return out
