"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module holds workload descriptions (plain numbers) and the seeded
initial particle load.  It contains none of the method's arithmetic: the
derived quantities (neutral density, macro weight, collision majorant,
fields) are computed separately by the library and by the oracle.

Workloads follow the paper's problem statement (arXiv 2206.14662, Sec. II.A
and II.B): a coaxial gap with the inner electrode biased, an applied
magnetic field, a uniform neutral gas at rest, and a volumetric seed load of
electrons, uniform in space with a Maxwellian velocity distribution (Sec.
II.A; n0 = 1e15 m^-3 and T0 = 1 eV, Sec. III.A).  The paper's own geometry
(an elliptic bump on the outer electrode) and its LXCat neon cross-sections
are replaced by straight coaxial walls and analytic cross-section fits.
"""
from __future__ import annotations

import numpy as np

# Field names and order of the C struct pic_config (include/pic.h).
_BASE = dict(
    r_in=1.0e-3, r_out=10.0e-3, z_min=-20.0e-3, z_max=20.0e-3,
    nr=32, nz=64,
    v_inner=-10.0e3, v_outer=0.0,
    bfield_kind=0, b0=0.2,
    p_mbar=1.0e-4, t_gas_K=300.0,
    sigma_el=1.0e-19,
    ion_E_th_eV=15.0, ion_sigma_pk=1.0e-20, ion_E_pk_eV=100.0,
    opal_B_eV=10.0, xi_param=0.0,
    elastic_recoil=1, gas_mass_amu=20.1797,
    n_init=10_000, n0=1.0e15, T0_eV=1.0,
    weight=0.0,
    dt=1.0e-12, sort_every=20,
    poisson_rtol=1.0e-8, poisson_maxit=2, warm_start=1,
    capacity=0,
    seed=1,
    precision=32,
    nu_max=0.0,
    source_rate=0.0,
)

#: The synthetic workloads.  ``steps`` is the length of the run the workload
#: describes; the benchmark times a window of it.
WORKLOADS = {
    # plain FP64 method, small: 32x64 cells, uniform Bz = 0.2 T, -10 kV
    "coax_32x64_1e4": dict(_BASE, steps=500, precision=64),
    # single run: 128x512 cells, mirror B0 = 0.3 T, -20 kV, 1e-5 mbar, 1e7
    # macro-electrons, cell sort every 20 steps
    "mirror_128x512_1e7": dict(
        _BASE, nr=128, nz=512, bfield_kind=1, b0=0.3, v_inner=-20.0e3,
        p_mbar=1.0e-5, n_init=10_000_000, steps=20_000, precision=32),
    # large single run: 256x1024 cells, mirror B0 = 0.5 T, -30 kV, 1e-6 mbar,
    # 2e8 macro-electrons with room for 3e8
    "mirror_256x1024_2e8": dict(
        _BASE, nr=256, nz=1024, bfield_kind=1, b0=0.5, v_inner=-30.0e3,
        p_mbar=1.0e-6, n_init=200_000_000, capacity=300_000_000,
        steps=50_000, precision=32),
}


def workload(name: str, **overrides) -> dict:
    """A copy of a named workload with fields overridden."""
    cfg = dict(WORKLOADS[name])
    cfg.update(overrides)
    return cfg


# The parametric scan (the paper's scans over pressure, applied voltage and
# magnetic field, Sec. III-IV): a 4 x 4 x 4 grid of pressure, inner-electrode
# voltage and mirror field B0, 64 x 256 cells each, run as one batch.
SCAN_PRESSURES_MBAR = (1.0e-6, 1.0e-5, 1.0e-4, 1.0e-3)
SCAN_VOLTAGES_V = (-5.0e3, -13.333e3, -21.667e3, -30.0e3)
SCAN_B0_T = (0.1, 0.2333, 0.3667, 0.5)


def scan_configs(n_sims: int = 64, nr: int = 64, nz: int = 256, n_min: int = 100_000,
                 n_max: int = 5_000_000, **overrides) -> list[dict]:
    """Configurations of the scan "scan_64x256_64sims".  Simulation k takes
    pressure SCAN_PRESSURES_MBAR[(k // 16) % 4], voltage
    SCAN_VOLTAGES_V[(k // 4) % 4] and field SCAN_B0_T[k % 4] (mirror field),
    and N_k = round(n_min (n_max / n_min)^(k / (n_sims - 1))) macro-electrons
    (log-spaced: a 50x spread of work between the smallest and the largest
    simulation), with the macro weight n0 V_gap / N_k.  ``overrides`` apply
    to every simulation."""
    cfgs = []
    for k in range(n_sims):
        frac = k / (n_sims - 1) if n_sims > 1 else 0.0
        n_k = int(round(n_min * (n_max / n_min) ** frac))
        cfg = dict(_BASE, nr=nr, nz=nz, bfield_kind=1,
                   p_mbar=SCAN_PRESSURES_MBAR[(k // 16) % 4],
                   v_inner=SCAN_VOLTAGES_V[(k // 4) % 4],
                   b0=SCAN_B0_T[k % 4],
                   n_init=n_k, steps=20_000, precision=32)
        cfg.update(overrides)
        cfgs.append(cfg)
    return cfgs


ELECTRON_MASS = 9.1093837015e-31   # kg, CODATA 2018 (input recipe only)
ELEMENTARY_CHARGE = 1.602176634e-19  # C


def seed_particles(cfg: dict, n: int | None = None, seed: int | None = None,
                   margin_cells: float = 0.0):
    """Initial macro-electrons: r with density uniform in volume between the
    walls (r = sqrt(a^2 + u (b^2 - a^2))), z uniform, each velocity component
    normal with variance k T0 / m_e.  Returns float64 arrays
    (r, z, vr, vtheta, vz) and uint64 uids 0..n-1.

    ``margin_cells`` keeps the load that many cells away from every wall.
    The generator is numpy's PCG64 seeded with ``seed`` (default cfg['seed']).
    """
    n = int(cfg["n_init"] if n is None else n)
    rng = np.random.Generator(np.random.PCG64(cfg["seed"] if seed is None else seed))
    a, b = cfg["r_in"], cfg["r_out"]
    z0, z1 = cfg["z_min"], cfg["z_max"]
    hr = (b - a) / cfg["nr"]
    hz = (z1 - z0) / cfg["nz"]
    a_ = a + margin_cells * hr
    b_ = b - margin_cells * hr
    u = rng.random(n)
    r = np.sqrt(a_ * a_ + u * (b_ * b_ - a_ * a_))
    z = (z0 + margin_cells * hz) + rng.random(n) * ((z1 - z0) - 2 * margin_cells * hz)
    # keep strictly inside the open domain
    r = np.clip(r, np.nextafter(a, b), np.nextafter(b, a))
    z = np.clip(z, np.nextafter(z0, z1), np.nextafter(z1, z0))
    vth = np.sqrt(cfg["T0_eV"] * ELEMENTARY_CHARGE / ELECTRON_MASS)
    v = rng.standard_normal((3, n)) * vth
    uid = np.arange(n, dtype=np.uint64)
    return r, z, v[0].copy(), v[1].copy(), v[2].copy(), uid


def uniform_field_node_arrays(cfg: dict, er_value: float, ez_value: float = 0.0):
    """Constant node fields (E_r, E_z) for tests that inject E."""
    shape = ((cfg["nr"] + 1) * (cfg["nz"] + 1),)
    return np.full(shape, er_value), np.full(shape, ez_value)


def random_field_node_arrays(cfg: dict, scale: float, seed: int = 7):
    """Smooth random node fields for parity tests that inject E: a sum of a
    few low-order sinusoids with random amplitudes of size ``scale``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nr, nz = cfg["nr"], cfg["nz"]
    x = np.linspace(0.0, 1.0, nr + 1)[:, None]
    y = np.linspace(0.0, 1.0, nz + 1)[None, :]
    er = np.zeros((nr + 1, nz + 1))
    ez = np.zeros((nr + 1, nz + 1))
    for _ in range(4):
        kx, ky = rng.integers(1, 4, size=2)
        ph = rng.random(2) * 2 * np.pi
        er += scale * rng.standard_normal() * np.sin(np.pi * kx * x + ph[0]) * np.cos(np.pi * ky * y + ph[1])
        ez += 0.3 * scale * rng.standard_normal() * np.cos(np.pi * kx * x + ph[1]) * np.sin(np.pi * ky * y + ph[0])
    return er.ravel(), ez.ravel()


# Initial weights of the learned field-solve warm start (a U-Net of base
# width c, see the library's pic_unet_* entry points for the layer order).
# Each layer's weights are drawn N(0, 2 / fan_in) (fan_in = kernel taps x
# input channels), biases are zero; the head starts at N(0, head_std^2).
def cross_section_tables(E_th_eV: float = 21.56, n: int = 64, E_max_eV: float = 3.0e4,
                         sigma_el_scale: float = 1.0e-19, sigma_io_scale: float = 2.0e-20,
                         with_xi: bool = True):
    """Synthetic tables for pic_set_cross_sections (the LXCat data the paper
    uses are not available): n energies, 0 then log-spaced from 0.1 eV to
    E_max_eV, with the ionisation threshold among them; an elastic
    momentum-transfer cross-section falling as (1 + E / 10 eV)^-1/2, an
    ionisation cross-section zero up to the threshold, rising to its peak
    at e E_th and falling as log(E) / E; an angle-law anisotropy rising
    from 0 to 0.6 with energy (None when with_xi is false).  Returns
    (E_eV, sigma_el, sigma_io, xi)."""
    E = np.concatenate([[0.0], np.geomspace(0.1, E_max_eV, n - 2)])
    E = np.unique(np.concatenate([E, [E_th_eV]]))
    while len(E) < n:   # keep n points when the threshold was already there
        E = np.unique(np.concatenate([E, [0.5 * (E[-1] + E[-2])]]))
    sigma_el = sigma_el_scale / np.sqrt(1.0 + E / 10.0)
    x = np.maximum(E / E_th_eV, 1.0)
    sigma_io = np.where(E > E_th_eV, sigma_io_scale * 5.0 * np.log(x) / x, 0.0)
    xi = 0.6 * E / (E + 100.0) if with_xi else None
    return E, sigma_el, sigma_io, xi


def unet_layer_shapes(c: int, cin: int = 2) -> list[tuple[str, tuple]]:
    """(name, weight shape) in the flat parameter order: conv layers
    (3, 3, in, out), transposed convolutions (2, 2, in, out), head (c,)."""
    return [("enc1a", (3, 3, cin, c)), ("enc1b", (3, 3, c, c)),
            ("enc2a", (3, 3, c, 2 * c)), ("enc2b", (3, 3, 2 * c, 2 * c)),
            ("enc3a", (3, 3, 2 * c, 4 * c)), ("enc3b", (3, 3, 4 * c, 4 * c)),
            ("enc4a", (3, 3, 4 * c, 8 * c)), ("enc4b", (3, 3, 8 * c, 8 * c)),
            ("up3", (2, 2, 8 * c, 4 * c)), ("dec3a", (3, 3, 8 * c, 4 * c)),
            ("dec3b", (3, 3, 4 * c, 4 * c)),
            ("up2", (2, 2, 4 * c, 2 * c)), ("dec2a", (3, 3, 4 * c, 2 * c)),
            ("dec2b", (3, 3, 2 * c, 2 * c)),
            ("up1", (2, 2, 2 * c, c)), ("dec1a", (3, 3, 2 * c, c)), ("dec1b", (3, 3, c, c)),
            ("head", (c,))]


def unet_init_flat(c: int, seed: int = 0, cin: int = 2, head_std: float = 1e-2,
                   bias_std: float = 0.0) -> np.ndarray:
    """Flat float64 parameter vector: per layer its weights (C order), then
    its bias (out channels; one value for the head)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for name, shp in unet_layer_shapes(c, cin):
        if name == "head":
            parts.append(rng.standard_normal(shp) * head_std)
            parts.append(rng.standard_normal(1) * bias_std)
        else:
            fan_in = shp[0] * shp[1] * shp[2]
            parts.append(rng.standard_normal(shp).ravel() * np.sqrt(2.0 / fan_in))
            parts.append(rng.standard_normal(shp[3]) * bias_std)
    return np.concatenate([np.ravel(p) for p in parts])
