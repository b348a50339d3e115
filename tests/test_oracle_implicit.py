"""Pins of the direct-implicit electrostatics (Sec. 2.3: Eq. poisson with the
susceptibility chi, Eq. epseff, Eq. implicit_charge_relation, Eq. facecharge
with the effective face permittivity) in the oracle:

* with no electrostatic field the implicit step is the explicit step, bit for
  bit (the two forms differ only in when E_r, E_z act);
* one particle in a uniform field: the implicit kick and its position
  response in closed form;
* chi of a uniform lattice population equals sum_s w_ps^2 dt^2 (the plasma
  frequency of the deposited density) on interior nodes;
* a uniform chi scales every face of the operator by 1 + chi, so the potential
  of a charge with grounded boundaries scales by 1 / (1 + chi);
* the discrete Gauss law holds with chi in the faces (turn charges plus metal
  fluxes equal minus the free charge);
* stability: a cold dense plasma at w_pe dt = 4, where the explicit leapfrog
  is unstable (w_pe dt > 2), keeps its energy bounded in the implicit form;
* the defining property (Eq. implicit_charge_relation): the potential solved
  with chi from the predicted positions is, to first order in the
  displacement, the chi-free potential of the corrected positions."""
import math

import numpy as np
import pytest

from oracle import particles, fields
from oracle.constants import QE, ME, M_AR, EPS0
from oracle.grid import CellGeometry, Grid
from oracle.cell import OracleCell
from paper_2609_15043_b300 import workloads
from paper_2609_15043_b300.workloads import CellConfig

from test_oracle_particles import _cfg, _particles, _uniform_F


def _run(cfg, P, F, sp, T, implicit, weight=1.0, step=0):
    geo = CellGeometry(cfg)
    sc = particles.SpeciesConstants(cfg, sp, weight, T)
    Q = np.zeros((cfg.nz + 1, cfg.nr + 1))
    J = np.zeros_like(Q)
    win = np.zeros_like(Q)
    stats = dict(p_ind=0.0, p_es=0.0, absorbed=0, pushed=0, nu_viol=0, coll=np.zeros((2, 3), np.int64))
    ev = particles.push_species(P, F, sc, geo, step, cfg.seed, T, Q, J, win, stats, implicit=implicit)
    return dict(Q=Q, J=J, win=win, stats=stats, events=ev, sc=sc)


@pytest.mark.parametrize("T", [np.float32, np.float64])
def test_implicit_equals_explicit_without_electrostatic_field(T):
    """E_r = E_z = 0 with an inductive E_theta and an RF B: both forms take the
    same Boris step, move, collisions and deposits, bit for bit."""
    cfg = _cfg(pressure_pa=2.0)
    rng = np.random.default_rng(5)
    n = 4000
    geo = CellGeometry(cfg)
    cells = rng.integers(0, geo.i_win * cfg.nr, n)
    args = (cells, rng.random(n), rng.random(n), rng.normal(size=n) * 1e6, rng.normal(size=n) * 1e6,
            rng.normal(size=n) * 1e6)
    F = _uniform_F(cfg, T, Et=300.0, Br=2e-4, Bz=-1e-4)
    for sp in (0, 1):
        Pa = _particles(T, *[np.array(a) for a in args])
        Pb = _particles(T, *[np.array(a) for a in args])
        a = _run(cfg, Pa, F, sp, T, implicit=False)
        b = _run(cfg, Pb, F, sp, T, implicit=True)
        for k in Pa:
            assert np.array_equal(Pa[k], Pb[k]), k
        for k in ("Q", "J", "win"):
            assert np.array_equal(a[k], b[k]), k
        assert a["stats"]["absorbed"] == b["stats"]["absorbed"]
        assert np.array_equal(a["stats"]["coll"], b["stats"]["coll"])
        assert a["stats"]["p_ind"] == b["stats"]["p_ind"]


def test_implicit_kick_in_a_uniform_field():
    """A particle at the predicted state (z~, v~) in a uniform E_z: the pass
    applies v = v~ + (q/m) dt E, z = z~ + (q/m) dt^2 E, then moves by dt v, so
    the next predicted position is z~ + dt v~ + 2 (q/m) dt^2 E and the
    predicted velocity v~ + (q/m) dt E (FP64, closed form)."""
    T = np.float64
    cfg = _cfg()
    E = 250.0
    dz = cfg.z_max / cfg.nz
    geo = CellGeometry(cfg)
    cell = 10 * cfg.nr + 7
    P = _particles(T, [cell], [0.25], [0.4], [0.0], [0.0], [3.0e4])
    F = _uniform_F(cfg, T, Ez=E)
    for sp, q, m in ((0, -QE, ME), (1, QE, M_AR)):
        P = _particles(T, [cell], [0.25], [0.4], [0.0], [0.0], [3.0e4])
        _run(cfg, P, F, sp, T, implicit=True)
        z0 = (10 + 0.4) * dz
        z1 = z0 + cfg.dt * 3.0e4 + 2.0 * q / m * cfg.dt ** 2 * E
        iz, ir = divmod(int(P["cell"][0]), cfg.nr)
        assert ir == 7
        assert (iz + P["dz"][0]) * dz == pytest.approx(z1, rel=1e-13)
        assert P["vz"][0] == pytest.approx(3.0e4 + q / m * cfg.dt * E, rel=1e-13)
        assert P["dr"][0] == pytest.approx(0.25, abs=1e-14)


def test_chi_of_a_lattice_population():
    """Electrons and ions on a regular lattice of 4 x 4 points per cell
    (offsets 1/8, 3/8, 5/8, 7/8): an interior node collects 16 w of each
    species (each of its four cells gives 4 w), its weighting volume is
    2 pi R_j dR dz, and chi there is (e^2 n / eps0)(1/m_e + 1/m_Ar) dt^2 with
    n = 16 w / V -- the plasma-frequency form w_pe^2 dt^2 + w_pi^2 dt^2."""
    cfg = workloads.small().replace(implicit_es=1)
    geo = CellGeometry(cfg)
    nr, iw = cfg.nr, geo.i_win
    offs = (np.arange(4) + 0.5) / 4.0
    cells = np.repeat(np.arange(iw * nr), 16)
    dr = np.tile(np.repeat(offs, 4), iw * nr)
    dz = np.tile(np.tile(offs, 4), iw * nr)
    w = 3.0e6
    oc = OracleCell(cfg, [w, w])
    for sp in (0, 1):
        z = np.zeros(cells.size)
        oc.set_particles(sp, cells, dr, dz, z, z, z, np.arange(cells.size))
    chi = oc.susceptibility(oc.deposit_species(np.float64), np.float64)
    g = geo.grid
    for i in (1, iw // 2, iw - 1):
        for j in (1, 5, nr // 2, nr - 1):
            n = 16 * w / (2 * math.pi * g.R[j] * g.dr * g.dz)
            ref = QE * QE * n / EPS0 * (1.0 / ME + 1.0 / M_AR) * cfg.dt ** 2
            assert chi[i, j] == pytest.approx(ref, rel=1e-12), (i, j)
    assert np.all(chi[iw + 1:, :] == 0.0)              # no particles above the plasma region
    assert np.all(chi >= 0.0)


def test_uniform_chi_scales_the_potential():
    """Eq. epseff with a uniform chi = c multiplies every face coefficient by
    1 + c: with grounded boundaries the potential of a charge is 1/(1 + c)
    of the chi-free one."""
    cfg = workloads.small()
    geo = CellGeometry(cfg)
    g = geo.grid
    ps = fields.PoissonSolver(g, geo.poisson_dirichlet())
    rng = np.random.default_rng(1)
    Q = np.where(geo.poisson_dirichlet(), 0.0, rng.normal(size=(g.NZ, g.NR)) * 1e-13)
    zero = np.zeros((g.NZ, g.NR))
    phi0 = ps.solve(Q, zero)
    for c in (0.5, 3.0, 40.0):
        phic = ps.solve_chi(Q, zero, np.full((g.NZ, g.NR), c))
        assert np.max(np.abs(phic * (1.0 + c) - phi0)) <= 1e-10 * np.max(np.abs(phi0))


def test_gauss_law_global_with_chi():
    """The discrete Gauss law with the susceptibility in the faces: the face
    charges of Eq. facecharge (with Eq. epseff) summed over the turns and the
    grounded metal equal minus the free charge."""
    rng = np.random.default_rng(4)
    g = Grid(10, 8, 1e-3, 1e-3, np.where(np.arange(10)[:, None] >= 6, 3.8, 1.0) * np.ones((10, 8)))
    dirm = np.zeros((g.NZ, g.NR), bool)
    dirm[0, :] = dirm[-1, :] = True
    dirm[:, -1] = True
    turn = [[(8, 3), (8, 4)], [(8, 6)]]
    for nodes in turn:
        for nd in nodes:
            dirm[nd] = True
    ps = fields.PoissonSolver(g, dirm)
    Q = np.where(dirm, 0.0, rng.normal(size=(g.NZ, g.NR)) * 1e-12)
    chi = rng.random((g.NZ, g.NR)) * 5.0            # nonzero at the turns too
    vals = np.zeros((g.NZ, g.NR))
    vals[8, 3] = vals[8, 4] = 5.0
    vals[8, 6] = -3.0
    phi = ps.solve_chi(Q, vals, chi)
    metal = [[(i, j)] for i in range(g.NZ) for j in range(g.NR) if dirm[i, j] and
             not any((i, j) in t for t in turn)]
    qt = fields.turn_charge(g, phi, turn + metal, chi=chi)
    assert np.sum(qt) == pytest.approx(-np.sum(Q), rel=1e-9)
    # without chi in the face charge the balance fails by the polarisation flux
    q0 = fields.turn_charge(g, phi, turn + metal)
    assert abs(np.sum(q0) + np.sum(Q)) > 1e-3 * abs(np.sum(Q))


def _cold_plasma(implicit, w_dt):
    """Small cell, no gas, no coil drive, cold electrons and ions on a lattice
    with a sinusoidal axial displacement of the electrons; the density sets
    w_pe dt."""
    cfg = workloads.small().replace(pressure_pa=0.0, v_g=0.0, implicit_es=int(implicit), magnetic_force=0)
    n0 = (w_dt / cfg.dt) ** 2 * EPS0 * ME / QE ** 2
    geo = CellGeometry(cfg)
    nr, iw = cfg.nr, geo.i_win
    offs = (np.arange(4) + 0.5) / 4.0
    cells = np.repeat(np.arange(iw * nr), 16)
    dr = np.tile(np.repeat(offs, 4), iw * nr)
    dzl = np.tile(np.tile(offs, 4), iw * nr)
    vol = math.pi * cfg.r_max ** 2 * cfg.z_win_lo
    # weight so that the lattice (uniform in R, not in R^2) has mean density n0
    w = n0 * vol / cells.size
    oc = OracleCell(cfg.replace(n_init=cells.size, density=n0), [w, w])
    iz, ir = cells // nr, cells % nr
    zc = (iz + dzl) / iw
    dze = (dzl + 0.1 * np.sin(2 * math.pi * zc)).astype(np.float64)
    izp, dzp = particles._carry(iz, dze, np.float64)
    ok = (izp >= 0) & (izp < iw)
    z = np.zeros(cells.size)
    oc.set_particles(0, (izp * nr + ir)[ok], dr[ok], dzp[ok], z[ok], z[ok], z[ok], np.arange(cells.size)[ok])
    oc.set_particles(1, cells, dr, dzl, z, z, z, np.arange(cells.size))
    oc.prime(np.float64)
    return oc


def _electron_energy(oc):
    P = oc.P[0]
    live = P["cell"] >= 0
    return 0.5 * ME * float(np.sum(P["vr"][live] ** 2 + P["vt"][live] ** 2 + P["vz"][live] ** 2))


def test_cold_plasma_stability_beyond_the_explicit_limit():
    """w_pe dt = 4 (explicit leapfrog needs w_pe dt < 2) on a cold electron
    lattice with an axial sine displacement: the explicit form's electron
    energy grows by orders of magnitude and the electrons leave the domain
    within a few steps; the implicit form (backward kick, amplification
    1/sqrt(1 + w^2 dt^2) per step for a plasma oscillation) damps the
    oscillation and keeps its electrons."""
    runs = {}
    for implicit in (False, True):
        oc = _cold_plasma(implicit, 4.0)
        n0 = int(np.sum(oc.P[0]["cell"] >= 0))
        e = []
        for _ in range(30):
            oc.step(np.float64)
            e.append(_electron_energy(oc))
        runs[implicit] = (np.array(e), n0, int(np.sum(oc.P[0]["cell"] >= 0)))
    (e_exp, n0e, n1e), (e_imp, n0i, n1i) = runs[False], runs[True]
    assert np.max(e_exp) > 1e3 * np.max(e_imp)
    assert n1e < 0.1 * n0e
    assert n1i >= 0.99 * n0i                 # only edge electrons of the initial displacement leave
    assert e_imp[-1] < 1e-2 * e_imp[0]


def test_chi_potential_is_the_potential_of_the_corrected_charge():
    """Eq. implicit_charge_relation: after a step, phi^{s+1} (solved with chi of
    the predicted populations) and the charge of the corrected positions
    x = x~ + (q/m) dt^2 E(x~) satisfy the chi-free Poisson equation to first
    order in the displacement: its residual is far below the residual of the
    predicted charge, which the chi-term accounts for."""
    oc = _cold_plasma(True, 1.5)
    for _ in range(3):
        oc.step(np.float64)
    g = oc.g
    # corrected positions from the current predicted state and phi^{s+1}
    th = oc.theta(oc.s)
    F = oc.node_fields(th, np.float64)
    Qc = np.zeros((g.NZ, g.NR))
    for sp in (0, 1):
        P = {k: v.copy() for k, v in oc.P[sp].items()}
        live = P["cell"] >= 0
        idx = np.nonzero(live)[0]
        cell = P["cell"][idx]
        ir, iz = cell % oc.cfg.nr, cell // oc.cfg.nr
        w = particles.bilinear(P["dr"][idx], P["dz"][idx], np.float64)
        Er = particles._gather(F, cell, w, 0)
        Ez = particles._gather(F, cell, w, 1)
        sc = oc.species(sp, np.float64)
        stats = dict(absorbed=0, p_es=0.0)
        irc, izc, drc, dzc, _, _, ok, _ = particles._implicit_correction(
            P, idx, ir, iz, P["dr"][idx], P["dz"][idx], P["vr"][idx], P["vz"][idx], Er, Ez, sc, oc.geo,
            np.float64, np.zeros((g.NZ, g.NR)), stats)
        wc = particles.bilinear(drc[ok], dzc[ok], np.float64)
        for (di, dj), wk in zip(((0, 0), (0, 1), (1, 0), (1, 1)), wc):
            np.add.at(Qc, (izc[ok] + di, irc[ok] + dj), sc.qw * wk)
    Qp = oc.Q_last
    dv = oc.dirichlet_values(th)
    r_corr = oc.poisson.residual(oc.phi, Qc + oc.window_q, dv)
    r_pred = oc.poisson.residual(oc.phi, Qp + oc.window_q, dv)
    inner = ~oc.pdir
    inner[:, :3] = False                     # away from the axis rows of the lattice
    inner[oc.geo.i_win - 2:, :] = False
    inner[:3, :] = False
    inner[:, -4:] = False
    a, b = np.abs(r_corr[inner]), np.abs(r_pred[inner])
    ratio = np.sqrt(np.mean(a ** 2)) / np.sqrt(np.mean(b ** 2))
    print("residual ratio", ratio)
    assert ratio < 0.1
