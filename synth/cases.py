"""Case parameters of the synthetic plume and nozzle workloads, and their random draws.

Everything here is plain parameter bookkeeping: geometry, boundary and ambient conditions,
and uniform random numbers from a splitmix64 stream.  The conversion of these parameters
into conserved states is done independently by the oracle and by the CUDA library.

Workloads (sizes and conditions follow the paper's turbofan plume, Sec. 4.1, scaled to the
benchmark grids; the seeded perturbations are the only random inputs):
  * nozzle_case            -- quasi-1D converging-diverging nozzle, 400 cells over 0.2 m
  * plume_case             -- axisymmetric coaxial plume, 1024 x 256, FP64 workload
  * plume_case_mixed_precision -- the same plume on 4096 x 1024 with 1 % inlet
                              velocity perturbations per inflow row
  * batch_cases            -- 64 uneven plume cases (ambient, fuel water and nozzle sweep)
  * mixing_layer_case      -- small, strongly supersaturated plume for parity tests
  * closed_box_case        -- walls everywhere, for conservation tests
  * shock_tube_case        -- constant-area dry tube with walls, for the Riemann pin
"""
from __future__ import annotations

import math

import numpy as np

# Parameter names of one case, in the order of the C structs of both implementations.
CASE_KEYS = (
    ("geom", "i"), ("nx", "i"), ("nr", "i"), ("bc_xlo", "i"), ("bc_xhi", "i"),
    ("bc_rhi", "i"), ("phase_change", "i"), ("freezing", "i"),
    ("lx", "d"), ("lr", "d"), ("area_a", "d"), ("x_throat", "d"),
    ("d_core", "d"), ("d_fan", "d"), ("wall_len", "d"),
    ("T_amb", "d"), ("p_amb", "d"), ("S_ice_amb", "d"), ("mach_coflow", "d"),
    ("T_core", "d"), ("u_core", "d"), ("Yv_core", "d"), ("T_byp", "d"), ("u_byp", "d"),
    ("n_soot", "d"), ("soot_rm", "d"), ("soot_sigma", "d"),
    ("p0", "d"), ("T0", "d"), ("Yv_inlet", "d"),
    ("seed_l_n", "d"), ("seed_l_r", "d"), ("seed_s_n", "d"), ("seed_s_r", "d"),
    ("mix_width", "d"), ("nu_t", "d"), ("viscous", "i"), ("tables", "i"), ("equilibrium", "i"), ("bimodal", "i"),
)

_MASK = (1 << 64) - 1


def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    """n uniform doubles in [0, 1) from splitmix64 (Steele, Lea, Flood 2014), 53-bit."""
    out = np.empty(n, dtype=np.float64)
    x = seed & _MASK
    for k in range(n):
        x = (x + 0x9E3779B97F4A7C15) & _MASK
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        z = z ^ (z >> 31)
        out[k] = (z >> 11) * (1.0 / 9007199254740992.0)
    return out


def _blank() -> dict:
    c = {k: (0 if t == "i" else 0.0) for k, t in CASE_KEYS}
    c["soot_sigma"] = 1.0
    return c


def nozzle_case(seed: int = 1, nx: int = 400, phase_change: bool = True) -> dict:
    """Quasi-1D nozzle: 0.2 m, A/A_t = 1 + 2.5 (x/0.1 - 1)^2, p0 = 40 kPa, T0 = 300 K
    +- 0.5 K from the seed, moist air with Y_v = 0.02, no soot, no freezing."""
    c = _blank()
    c.update(geom=0, nx=nx, nr=1, bc_xlo=0, bc_xhi=0, bc_rhi=0,
             phase_change=int(phase_change), freezing=0,
             lx=0.2, lr=1.0, area_a=2.5, x_throat=0.1,
             p0=40.0e3, T0=300.0 + (splitmix64_uniform(seed, 1)[0] - 0.5),
             Yv_inlet=0.02)
    return c


def _plume_base(nx: int, nr: int) -> dict:
    c = _blank()
    d_core, d_fan = 0.8, 2.0
    c.update(geom=1, nx=nx, nr=nr, bc_xlo=0, bc_xhi=0, bc_rhi=0, phase_change=1, freezing=1,
             lx=40.0 * d_core, lr=4.0 * d_fan, d_core=d_core, d_fan=d_fan, wall_len=0.0,
             T_amb=220.0, p_amb=24.0e3, S_ice_amb=1.1, mach_coflow=0.8,
             T_core=580.0, u_core=450.0, Yv_core=0.03, T_byp=250.0, u_byp=300.0,
             n_soot=1.0e12, soot_rm=15.0e-9, soot_sigma=1.6)
    return c


def plume_case(nx: int = 1024, nr: int = 256) -> tuple[dict, np.ndarray]:
    """Coaxial turbofan plume (FP64 workload): core 580 K / 450 m/s / Y_v 0.03 with
    1e12 m^-3 lognormal soot (median 15 nm, sigma_g 1.6), bypass 250 K / 300 m/s dry,
    ambient 220 K, 24 kPa, ice supersaturation 1.1, coflow Mach 0.8.  Returns the case
    and the per-row inlet velocity factors (all 1: no perturbation)."""
    return _plume_base(nx, nr), np.ones(nr)


def plume_case_mixed_precision(seed: int = 3, nx: int = 4096, nr: int = 1024) -> tuple[dict, np.ndarray]:
    """The same plume with inlet velocities multiplied by 1 + 0.01 U(-1, 1) per row."""
    ufac = 1.0 + 0.01 * (2.0 * splitmix64_uniform(seed, nr) - 1.0)
    return _plume_base(nx, nr), ufac


def batch_cases(seed: int = 5, n: int = 64) -> list[tuple[dict, np.ndarray]]:
    """Sweep of n plume cases with uneven grids n_x in {256, 512, 1024, 2048}, n_r = n_x/4;
    T_amb ~ U(205, 235) K, S_ice ~ U(0.9, 1.3), water per fuel EI ~ U(1.25, 8.9) kg/kg
    mapped to Y_v,core = 0.03 (EI/1.25)(43.2/LHV) with LHV linear from 43.2 to 120 MJ/kg,
    nozzle duct length in {0, 2 D_core}, soot ~ logU(1e10, 1e13) m^-3."""
    u = splitmix64_uniform(seed, 7 * n).reshape(n, 7)
    out = []
    for k in range(n):
        nx = (256, 512, 1024, 2048)[min(3, int(u[k, 0] * 4))]
        c = _plume_base(nx, nx // 4)
        ei = 1.25 + (8.9 - 1.25) * u[k, 3]
        lhv = 43.2 + (ei - 1.25) / (8.9 - 1.25) * (120.0 - 43.2)
        c.update(T_amb=205.0 + 30.0 * u[k, 1], S_ice_amb=0.9 + 0.4 * u[k, 2],
                 Yv_core=0.03 * (ei / 1.25) * (43.2 / lhv),
                 wall_len=0.0 if u[k, 4] < 0.5 else 2.0 * c["d_core"],
                 n_soot=10.0 ** (10.0 + 3.0 * u[k, 5]))
        out.append((c, np.ones(c["nr"])))
    return out


def mixing_layer_case(nx: int = 96, nr: int = 40, seeded: bool = True, freezing: bool = True) -> tuple[dict, np.ndarray]:
    """Small plume whose hydrogen-like core (Y_v = 0.2) meets cold ambient air directly
    (no bypass) through a pre-mixed tanh layer 0.15 m wide, so that the mixing layer is
    strongly supersaturated over liquid from the first step.  With `seeded`, the core starts with droplet and
    crystal populations so that growth, evaporation and freezing run from the first step.
    Domain 6 m x 2.4 m; sized for the oracle to finish in seconds."""
    c = _blank()
    c.update(geom=1, nx=nx, nr=nr, bc_xlo=0, bc_xhi=0, bc_rhi=0, phase_change=1,
             freezing=int(freezing), lx=6.0, lr=2.4, d_core=0.8, d_fan=0.8, wall_len=0.0,
             T_amb=205.0, p_amb=24.0e3, S_ice_amb=1.3, mach_coflow=0.6,
             T_core=330.0, u_core=420.0, Yv_core=0.20, T_byp=250.0, u_byp=300.0,
             n_soot=1.0e12, soot_rm=15.0e-9, soot_sigma=1.6, mix_width=0.15)
    if seeded:
        c.update(seed_l_n=1.0e10, seed_l_r=2.0e-7, seed_s_n=1.0e8, seed_s_r=1.0e-6)
    ufac = 1.0 + 0.01 * (2.0 * splitmix64_uniform(11, nr) - 1.0)
    return c, ufac


def freezing_case(nx: int = 96, nr: int = 40) -> tuple[dict, np.ndarray]:
    """Cold core (232 K, vapour at about 0.97 of liquid saturation, 1.45 of ice saturation)
    carrying seeded droplets (0.2 um, 1e10/kg) and crystals (1 um, 1e8/kg) next to
    ice-supersaturated ambient air: homogeneous and immersion freezing, ice deposition
    growth and droplet evaporation run everywhere in the core, without nucleation bursts."""
    c, ufac = mixing_layer_case(nx=nx, nr=nr, seeded=True)
    c.update(mix_width=0.0, T_core=232.0, Yv_core=4.2468e-4, T_amb=225.0, S_ice_amb=1.3,
             u_core=250.0, mach_coflow=0.6)
    return c, ufac


def closed_box_case(geom: int = 1, nx: int = 48, nr: int = 24) -> tuple[dict, np.ndarray]:
    """Mixing-layer physics at rest with reflective walls on every side (the axis is a
    mirror): a closed box, whose total mass, water and energy stay constant.  For geom 0
    (constant-area-law nozzle with walls) the caller supplies the initial state."""
    c, ufac = mixing_layer_case(nx=nx, nr=nr, seeded=True)
    c.update(bc_xlo=1, bc_xhi=1, bc_rhi=1, u_core=0.0, u_byp=0.0, mach_coflow=0.0)
    if geom == 0:
        c.update(geom=0, nr=1, lx=0.2, area_a=2.5, x_throat=0.1, p0=40.0e3, T0=300.0,
                 Yv_inlet=0.02, freezing=0)
        ufac = np.ones(1)
    return c, ufac


def shock_tube_case(nx: int = 200) -> dict:
    """Constant-area dry tube of length 1 m with walls at both ends (sources off)."""
    c = _blank()
    c.update(geom=0, nx=nx, nr=1, bc_xlo=1, bc_xhi=1, phase_change=0, freezing=0,
             lx=1.0, lr=1.0, area_a=0.0, x_throat=0.5, p0=1.0e5, T0=300.0, Yv_inlet=0.0)
    return c


def perturbation_rows(c: dict) -> np.ndarray:
    return np.ones(c["nr"]) if c["geom"] == 1 else np.ones(1)


def describe(c: dict) -> str:
    if c["geom"] == 0:
        return f"nozzle {c['nx']} cells"
    return f"plume {c['nx']}x{c['nr']} (T_amb {c['T_amb']:.1f} K, Y_v,core {c['Yv_core']:.3f})"


def cells(c: dict) -> int:
    return int(c["nx"]) * (int(c["nr"]) if c["geom"] == 1 else 1)

