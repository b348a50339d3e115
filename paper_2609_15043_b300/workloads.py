"""Seeded synthetic inputs: cell configurations and initial particle
populations.

This module is the only code shared by the CUDA path and the oracle's tests.
It holds parameters and random-number plumbing, none of the method's
arithmetic: a configuration is a record of numbers, and a population is
positions uniform in r^2 and z over the plasma region with Maxwellian
velocities, drawn with numpy's PCG64 from a stated seed.

Workloads (sizes of the phasor-PIC hot path, argon ICP at 13.56 MHz):
  small   32x48 cells over r in [0, 0.10] m, z in [0, 0.15] m, quartz window
          eps_r = 3.8, 3-turn planar coil (radii 0.03/0.05/0.07 m, 2 mm
          wire), dt = T/400, Ar 20 mTorr 300 K, 2e4 macroparticles per
          species, Te = 3 eV, Ti = 0.026 eV, n = 1e16 m^-3, fixed source.
  cell60  128x192 cells, 4e6 macroparticles per species, same geometry and
          gas, power controller targeting 60 W.
  cell100 256x384 cells, 1.6e7 per species, 5-turn coil (radii 0.02-0.08 m),
          Ar 10 mTorr, dt = T/800, target 100 W.
"""
import dataclasses
import math
from dataclasses import dataclass, field
from typing import List

import numpy as np

# physical constants needed to draw Maxwellian velocities
_QE = 1.602176634e-19
_ME = 9.1093837015e-31
_M_AR = 39.948 * 1.66053906660e-27
_TORR = 133.322368
MAX_TURNS = 8


@dataclass
class CellConfig:
    # grid (cell counts) and domain
    nr: int = 32
    nz: int = 48
    r_max: float = 0.10
    z_max: float = 0.15
    # dielectric window slab and coil compartment
    z_win_lo: float = 0.125
    z_win_hi: float = 0.1375
    eps_win: float = 3.8
    z_coil: float = 0.14375
    turn_r: List[float] = field(default_factory=lambda: [0.03, 0.05, 0.07])
    winding: List[int] = field(default_factory=lambda: [1, 1, 1])
    wire_radius: float = 1.0e-3
    # RF
    freq: float = 13.56e6
    dt: float = 1.0 / (400 * 13.56e6)
    full_helmholtz: int = 1
    magnetic_force: int = 1
    # gas
    pressure_pa: float = 20e-3 * _TORR
    t_gas: float = 300.0
    # circuit
    r_g: float = 50.0
    r_m: float = 0.0
    l_m: float = 0.0
    c_m: float = 200e-12
    c_stray: List[float] = field(default_factory=lambda: [0.0] * MAX_TURNS)
    rho20: float = 1.68e-8
    alpha_cu: float = 3.93e-3
    t_coil_c: float = 20.0
    r_rf_override: float = -1.0
    # source and controller
    v_g: float = 300.0
    phase_g: float = 0.0
    power_control: int = 0
    p_target: float = 60.0
    gamma: float = 0.2
    n_trend: float = 5.0
    eps_p: float = 1e-3
    alpha_v: float = 0.5
    f_step: float = 0.05
    v_min: float = 1.0
    v_max: float = 1e4
    alpha: float = 0.5
    # particles
    n_init: int = 20000
    density: float = 1e16
    te_ev: float = 3.0
    ti_ev: float = 0.026
    seed: int = 20260915
    plain_fp64: int = 0            # 1: the plain FP64 particle form (comparison baseline)
    implicit_es: int = 0           # 1: direct-implicit electrostatics (susceptibility chi in the Poisson solve)
    n_harmonics: int = 1           # retained circuit harmonics m = 1..M (Sec. 4 extension); 1: fundamental only
    # particle control (off by default): ion-induced secondary emission, per-particle relative
    # weights and the split-merge pass (every sm_every steps: merge above sm_max particles per
    # cell, split below sm_min, towards sm_target)
    see_gamma: float = 0.0
    see_t_ev: float = 2.0
    particle_weights: int = 0
    sm_every: int = 0
    sm_target: int = 0
    sm_min: int = 0
    sm_max: int = 0
    capacity_factor: float = 1.5
    sort_every_e: int = 8
    sort_every_i: int = 50

    def replace(self, **kw):
        return dataclasses.replace(self, **kw)


def small():
    return CellConfig()


def cell60():
    return CellConfig(nr=128, nz=192, n_init=4_000_000, power_control=1, p_target=60.0)


def coarse60():
    """The plasma of the 128x192 cell (same geometry, gas, density and 60 W
    target) on a 64x96 grid with 5e5 macroparticles per species: a cell that
    reaches a stationary state within a few hundred periods in both the
    fused and the plain FP64 form."""
    return CellConfig(nr=64, nz=96, n_init=500_000, power_control=1, p_target=60.0)


def cell100():
    return CellConfig(nr=256, nz=384, n_init=16_000_000, pressure_pa=10e-3 * _TORR,
                      dt=1.0 / (800 * 13.56e6), turn_r=[0.02, 0.035, 0.05, 0.065, 0.08],
                      winding=[1] * 5, power_control=1, p_target=100.0)


def batch_cells(n_cells=32, seed=20260915):
    """A batch of independent cells of mixed size: nr from {64, 80, ..., 192}
    and nz = 1.5 nr (every nz is a multiple of 24, so the window and coil
    planes lie on grid lines), macroparticles per species log-uniform in
    [5e5, 8e6], controller target uniform in [20, 150] W, pressure uniform in
    [5, 50] mTorr, 3 to 5 turns spread evenly over r in [0.02, 0.08] m.
    Drawn with PCG64 from `seed`; cell i gets PIC seed `seed + i`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_cells):
        nr = int(rng.choice(np.arange(64, 193, 16)))
        n_init = int(round(math.exp(rng.uniform(math.log(5e5), math.log(8e6)))))
        p_target = float(rng.uniform(20.0, 150.0))
        p_mtorr = float(rng.uniform(5.0, 50.0))
        nt = int(rng.integers(3, 6))
        radii = [0.02 + 0.06 * k / (nt - 1) for k in range(nt)]
        out.append(CellConfig(nr=nr, nz=3 * nr // 2, n_init=n_init, pressure_pa=p_mtorr * 1e-3 * _TORR,
                              turn_r=radii, winding=[1] * nt, power_control=1, p_target=p_target,
                              seed=seed + i))
    return out


WORKLOADS = {"small": small, "cell60": cell60, "coarse60": coarse60, "cell100": cell100}


def load_config(src):
    """A CellConfig from a JSON object given as a dict, a JSON string or a file
    path: an optional "workload" key names the starting configuration (one of
    WORKLOADS; the defaults otherwise) and every other key overrides the field
    of that name.  Unknown keys and values of the wrong kind are refused."""
    import json
    import os
    if isinstance(src, dict):
        d = dict(src)
    elif isinstance(src, str) and os.path.exists(src):
        with open(src) as fh:
            d = json.load(fh)
    else:
        d = json.loads(src)
    base = WORKLOADS[d.pop("workload")]() if "workload" in d else CellConfig()
    names = {f.name: f for f in dataclasses.fields(CellConfig)}
    over = {}
    for k, v in d.items():
        if k not in names:
            raise KeyError("unknown configuration key %r" % k)
        cur = getattr(base, k)
        if isinstance(cur, list):
            if not isinstance(v, list):
                raise TypeError("%s must be a list" % k)
            over[k] = [type(cur[0])(x) for x in v] if cur else list(v)
        elif isinstance(cur, bool) or not isinstance(v, (int, float)):
            raise TypeError("%s must be a number" % k)
        else:
            over[k] = type(cur)(v)
    return base.replace(**over)


def dump_config(cfg):
    """The JSON text of a CellConfig (every field), readable by load_config."""
    import json
    return json.dumps(dataclasses.asdict(cfg), indent=1)


def macro_weight(cfg):
    """Physical particles per macroparticle: n V_plasma / N."""
    v_plasma = math.pi * cfg.r_max ** 2 * cfg.z_win_lo
    return cfg.density * v_plasma / cfg.n_init


def population(cfg, species, seed=None, n=None):
    """Initial macroparticles of one species (0 = e-, 1 = Ar+).

    Returns dict(cell uint32, dr, dz, vr, vt, vz float32, uid uint32) with
    cell = iz*nr + ir and (dr, dz) the offsets in [0, 1) inside the cell.
    Positions are uniform in r^2 over [0, r_max) and uniform in z over
    [0, z_win_lo); velocities Maxwellian at te_ev / ti_ev."""
    n = cfg.n_init if n is None else n
    rng = np.random.Generator(np.random.PCG64((cfg.seed if seed is None else seed) * 2 + species))
    dr_m, dz_m = cfg.r_max / cfg.nr, cfg.z_max / cfg.nz
    r = cfg.r_max * np.sqrt(rng.random(n))
    z = cfg.z_win_lo * rng.random(n)
    xr, xz = r / dr_m, z / dz_m
    ir = np.minimum(np.floor(xr).astype(np.int64), cfg.nr - 1)
    iz = np.minimum(np.floor(xz).astype(np.int64), int(round(cfg.z_win_lo / dz_m)) - 1)
    fr = np.clip(xr - ir, 0.0, np.nextafter(1.0, 0.0)).astype(np.float32)
    fz = np.clip(xz - iz, 0.0, np.nextafter(1.0, 0.0)).astype(np.float32)
    fr = np.where(fr >= 1.0, np.float32(0.99999994), fr).astype(np.float32)
    fz = np.where(fz >= 1.0, np.float32(0.99999994), fz).astype(np.float32)
    mass = _ME if species == 0 else _M_AR
    t_ev = cfg.te_ev if species == 0 else cfg.ti_ev
    vth = math.sqrt(t_ev * _QE / mass)
    v = (rng.standard_normal((3, n)) * vth).astype(np.float32)
    order = np.argsort(iz * cfg.nr + ir, kind="stable")
    return dict(cell=(iz * cfg.nr + ir).astype(np.uint32)[order],
                dr=fr[order], dz=fz[order],
                vr=v[0][order], vt=v[1][order], vz=v[2][order],
                uid=np.arange(n, dtype=np.uint32)[order])
