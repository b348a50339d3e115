"""Oracle pins for the particle step: closed-form orbits, exact energy and
charge bookkeeping, null-collision statistics, Philox known answers."""
import math

import numpy as np
import pytest

from oracle import philox, particles
from oracle.constants import QE, ME, M_AR, KB, E_EXC, E_ION
from oracle.grid import CellGeometry
from paper_2609_15043_b300.workloads import CellConfig


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Philox4x32-10 known-answer vectors (Salmon et al. 2011 / Random123)."""
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
        ((0xffffffff,) * 4, (0xffffffff, 0xffffffff), (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
        ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
         (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
    ]
    for ctr, key, out in cases:
        got = philox.philox4x32(*[[c] for c in ctr], *key)
        assert tuple(int(g[0]) for g in got) == out


def test_philox2x32_known_answers():
    """Philox2x32-10 known-answer vectors (Salmon et al. 2011 / Random123);
    this generator draws the per-particle null-collision uniform."""
    cases = [((0, 0), 0, (0xff1dae59, 0x6cd10df2)),
             ((0xffffffff, 0xffffffff), 0xffffffff, (0x2c3f628b, 0xab4fd7ad)),
             ((0x243f6a88, 0x85a308d3), 0x13198a2e, (0xdd7ce038, 0xf62a4c12))]
    for ctr, key, out in cases:
        a, b = philox.philox2x32([ctr[0]], [ctr[1]], key)
        assert (int(a[0]), int(b[0])) == out


def test_uniform_conversion_exact():
    x = np.array([0, 1, 511, 512, 0xFFFFFFFF, 0x80000000], np.uint32)
    u = philox.to_uniform(x, np.float32)
    assert np.all(u > 0) and np.all(u < 1)
    ref = ((x >> 9).astype(np.float64) + 0.5) * 2.0 ** -23
    assert np.array_equal(u.astype(np.float64), ref)          # exact in float32
    d = philox.draws(np.arange(200000), 7, 0, 0, 12345, np.float32)
    for ui in d:
        assert abs(ui.mean() - 0.5) < 5 * math.sqrt(1 / 12 / ui.size)


# ---------------------------------------------------------------- helpers
def _cfg(**kw):
    base = dict(nr=16, nz=24, r_max=0.16, z_max=0.24, z_win_lo=0.20, z_win_hi=0.21,
                z_coil=0.225, turn_r=[0.05], winding=[1], pressure_pa=0.0)
    base.update(kw)
    return CellConfig(**base)


def _particles(T, cell, dr, dz, vr, vt, vz, uid=None):
    n = len(cell)
    return dict(cell=np.asarray(cell, np.int64), dr=np.asarray(dr, T), dz=np.asarray(dz, T),
                vr=np.asarray(vr, T), vt=np.asarray(vt, T), vz=np.asarray(vz, T),
                uid=np.arange(n, dtype=np.int64) if uid is None else np.asarray(uid, np.int64))


def _run(cfg, P, F, sp, T, steps=1, weight=1.0, step0=0):
    geo = CellGeometry(cfg)
    sc = particles.SpeciesConstants(cfg, sp, weight, T)
    Q = np.zeros((cfg.nz + 1, cfg.nr + 1))
    J = np.zeros_like(Q)
    win = np.zeros_like(Q)
    stats = dict(p_ind=0.0, p_es=0.0, absorbed=0, pushed=0, nu_viol=0, coll=np.zeros((2, 3), np.int64))
    events = []
    for s in range(steps):
        events += particles.push_species(P, F, sc, geo, step0 + s, cfg.seed, T, Q, J, win, stats)
    return dict(Q=Q, J=J, win=win, stats=stats, events=events, sc=sc, geo=geo)


def _uniform_F(cfg, T, Er=0.0, Ez=0.0, Et=0.0, Br=0.0, Bz=0.0):
    geo = CellGeometry(cfg)
    n = geo.i_win * cfg.nr
    F = np.zeros((n, 5, 4), T)
    for c, v in enumerate((Er, Ez, Et, Br, Bz)):
        F[:, c, :] = v
    return F


# ---------------------------------------------------------------- orbits
def test_boris_gyration_closed_form():
    """Uniform B_z, no E: the Boris step rotates v by alpha = -2 atan(qBdt/2m)
    per step (Boris 1970) and the leapfrog positions lie on the discrete
    circle x^N = x^0 + dt sum_{k=1..N} e^{i k alpha} v^{-1/2}; r = |x^N|."""
    cfg = _cfg(r_max=1.6, z_max=2.4, z_win_lo=2.0, z_win_hi=2.1, z_coil=2.25, turn_r=[0.5])
    T = np.float64
    B = 3e-4
    F = _uniform_F(cfg, T, Bz=B)
    dr_cell = cfg.r_max / cfg.nr
    r0 = 0.73
    ir0 = int(r0 // dr_cell)
    v = 2.0e6
    P = _particles(T, [8 * cfg.nr + ir0], [r0 / dr_cell - ir0], [0.5], [0.3 * v], [v], [1e4])
    steps = 300
    out = _run(cfg, P, F, 0, T, steps=steps)
    qm = -QE / ME
    alpha = -2.0 * math.atan(qm * B * cfg.dt / 2.0)
    v0 = complex(0.3 * v, v)
    k = np.arange(1, steps + 1)
    xN = r0 + cfg.dt * np.sum(np.exp(1j * k * alpha)) * v0
    r_num = (P['cell'][0] % cfg.nr + P['dr'][0]) * dr_cell
    assert r_num == pytest.approx(abs(xN), rel=1e-10)
    assert math.hypot(P['vr'][0], P['vt'][0]) == pytest.approx(abs(v0), rel=1e-13)
    z_num = (P['cell'][0] // cfg.nr + P['dz'][0]) * (cfg.z_max / cfg.nz)
    assert z_num == pytest.approx(8.5 * cfg.z_max / cfg.nz + 1e4 * cfg.dt * steps, rel=1e-12)


def test_free_streaming_through_axis():
    """No fields: straight lines in Cartesian space, including the passage
    through the axis: r(n) = |(r0 + n vx dt, n vy dt)|."""
    cfg = _cfg()
    T = np.float64
    F = _uniform_F(cfg, T)
    dr_cell = cfg.r_max / cfg.nr
    r0 = 0.0234
    vx, vy = -1.0e6, 1.3e5
    P = _particles(T, [3 * cfg.nr + 2], [r0 / dr_cell - 2], [0.25], [vx], [vy], [0.0])
    for n in range(1, 301):
        _run(cfg, P, F, 0, T, steps=1, step0=n)
        r = (P['cell'][0] % cfg.nr + P['dr'][0]) * dr_cell
        assert r == pytest.approx(math.hypot(r0 + n * vx * cfg.dt, n * vy * cfg.dt), rel=1e-9, abs=1e-15)
    assert math.hypot(P['vr'][0], P['vt'][0]) == pytest.approx(math.hypot(vx, vy), rel=1e-13)


def test_uniform_ez_acceleration():
    """Uniform E_z: v_z grows by (q/m) E dt per step exactly and z follows the
    leapfrog sum."""
    cfg = _cfg()
    T = np.float64
    E = 50.0
    F = _uniform_F(cfg, T, Ez=E)
    dz_cell = cfg.z_max / cfg.nz
    P = _particles(T, [10 * cfg.nr + 5], [0.5], [0.5], [0.0], [0.0], [0.0])
    _run(cfg, P, F, 1, T, steps=100)
    a = QE / M_AR * E
    assert P['vz'][0] == pytest.approx(100 * a * cfg.dt, rel=1e-12)
    z = (P['cell'][0] // cfg.nr + P['dz'][0]) * dz_cell
    assert z == pytest.approx(10.5 * dz_cell + a * cfg.dt ** 2 * 100 * 101 / 2, rel=1e-12)


# ---------------------------------------------------------------- bookkeeping
def _random_population(cfg, T, n, rng, vscale=1e6):
    geo = CellGeometry(cfg)
    cell = rng.integers(0, geo.i_win * cfg.nr, n)
    return _particles(T, cell, rng.random(n), rng.random(n), rng.normal(size=n) * vscale,
                      rng.normal(size=n) * vscale, rng.normal(size=n) * vscale)


def test_energy_bookkeeping_exact():
    """With random node fields (E and B) and no collisions, the kinetic energy
    gained in a step equals dt times the time-centred work sum
    q w vbar.E = dt (P_ind + P_es): the Boris rotation conserves |v| and the
    current is deposited with vbar = (v^{n-1/2} + v^{n+1/2}) / 2."""
    cfg = _cfg()
    T = np.float64
    rng = np.random.default_rng(5)
    geo = CellGeometry(cfg)
    F = rng.normal(size=(geo.i_win * cfg.nr, 5, 4)) * np.array([3e3, 3e3, 3e3, 1e-3, 1e-3])[None, :, None]
    P = _random_population(cfg, T, 5000, rng)
    w = 3.0e7
    e0 = 0.5 * ME * w * np.sum(P['vr'] ** 2 + P['vt'] ** 2 + P['vz'] ** 2)
    out = _run(cfg, P, F, 0, T, weight=w)
    e1 = 0.5 * ME * w * np.sum(P['vr'] ** 2 + P['vt'] ** 2 + P['vz'] ** 2)
    work = cfg.dt * (out['stats']['p_ind'] + out['stats']['p_es'])
    assert e1 - e0 == pytest.approx(work, rel=1e-9)


def test_deposit_conserves_charge():
    """Sum of node charges = q w N (area weights sum to one); sum of the
    current moments = sum q w vbar_theta."""
    cfg = _cfg()
    rng = np.random.default_rng(6)
    for T in (np.float64, np.float32):
        P = _random_population(cfg, T, 4000, rng, vscale=1e5)
        vt0 = P['vt'].astype(np.float64).copy()
        out = _run(cfg, P, _uniform_F(cfg, T), 0, T, weight=2e7)
        n_alive = np.count_nonzero(P['cell'] >= 0)
        qw = float(out['sc'].qw)
        assert out['Q'].sum() == pytest.approx(qw * n_alive, rel=1e-6 if T == np.float32 else 1e-12)
        vbar = 0.5 * (vt0 + P['vt'].astype(np.float64))   # no field: v_theta unchanged in
        # the old frame, rotated in the new one, so only check the FP64 case exactly
        if T == np.float64:
            assert out['J'].sum() == pytest.approx(qw * vt0.sum(), rel=1e-12)


def test_uniform_density_flat_charge_density():
    """Particles uniform in r^2 and z give a flat node charge density
    Q / V_node away from the boundaries (annular node volumes)."""
    cfg = _cfg()
    rng = np.random.default_rng(7)
    geo = CellGeometry(cfg)
    n = 400000
    dr_c, dz_c = cfg.r_max / cfg.nr, cfg.z_max / cfg.nz
    r = cfg.r_max * np.sqrt(rng.random(n))
    z = cfg.z_win_lo * rng.random(n)
    ir, iz = np.floor(r / dr_c).astype(int), np.floor(z / dz_c).astype(int)
    P = _particles(np.float64, iz * cfg.nr + ir, r / dr_c - ir, z / dz_c - iz,
                   np.zeros(n), np.zeros(n), np.zeros(n))
    Q = np.zeros((cfg.nz + 1, cfg.nr + 1))
    w = particles.bilinear(P['dr'], P['dz'], np.float64)
    for (di, dj), wk in zip(((0, 0), (0, 1), (1, 0), (1, 1)), w):
        np.add.at(Q, (iz + di, ir + dj), wk)
    rho = Q[3:geo.i_win - 2, 2:cfg.nr - 1] / geo.vol[3:geo.i_win - 2, 2:cfg.nr - 1]
    mean = n / (math.pi * cfg.r_max ** 2 * cfg.z_win_lo)
    assert abs(rho.mean() / mean - 1) < 0.01
    # axis and wall nodes with the weighting volumes: same density within noise
    assert abs(np.mean(Q[3:geo.i_win - 2, 0] / geo.vol[3:geo.i_win - 2, 0]) / mean - 1) < 0.05
    assert abs(np.mean(Q[3:geo.i_win - 2, -1] / geo.vol[3:geo.i_win - 2, -1]) / mean - 1) < 0.02


def test_absorption_and_window_charge():
    """A particle crossing z = 0 is absorbed; one crossing the window plane
    leaves exactly q w on the window node row; one crossing r = R is
    absorbed without window charge."""
    cfg = _cfg()
    T = np.float64
    geo = CellGeometry(cfg)
    iw = geo.i_win
    P = _particles(T, [0 * cfg.nr + 4, (iw - 1) * cfg.nr + 4, 5 * cfg.nr + cfg.nr - 1],
                   [0.5, 0.3, 0.99], [0.01, 0.99, 0.5], [0.0, 0.0, 1e7], [0.0, 0.0, 0.0],
                   [-1e7, 1e7, 0.0])
    out = _run(cfg, P, _uniform_F(cfg, T), 1, T, weight=5.0)
    assert list(P['cell']) == [particles.DEAD] * 3
    assert out['win'].sum() == pytest.approx(QE * 5.0, rel=1e-14)
    assert np.count_nonzero(out['win'][iw]) == 2 and out['win'][:iw].sum() == 0
    assert out['stats']['absorbed'] == 3


# ---------------------------------------------------------------- MCC
def test_cross_section_thresholds_and_bound():
    x = np.linspace(0, 1000, 200001)
    se, sx, si = particles.sigma_e(x, np.float64)
    assert np.all(sx[x <= E_EXC] == 0) and np.all(sx[x > E_EXC + 1e-3] > 0)
    assert np.all(si[x <= E_ION] == 0) and np.all(si[x > E_ION + 1e-3] > 0)
    assert np.all(se > 0)
    n_gas = 2.666 / (KB * 300)
    nue, nui = particles.nu_max(n_gas)
    g = np.sqrt(2 * QE * x / ME)
    assert np.max(n_gas * 1e-20 * (se + sx + si) * g) < nue
    gi = np.sqrt(2 * QE * x / M_AR)
    scx, siso = particles.sigma_i(x, np.float64)
    assert np.max(n_gas * 1e-19 * (scx + siso) * gi) < nui


def _mono_electrons(cfg, T, n, e_ev, rng):
    geo = CellGeometry(cfg)
    v = math.sqrt(2 * QE * e_ev / ME)
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    cell = rng.integers(cfg.nr * 4, cfg.nr * 5, n) + 2
    return _particles(T, cell, np.full(n, 0.5), np.full(n, 0.5), v * d[0], v * d[1], v * d[2])


@pytest.mark.parametrize("e_ev", [5.0, 30.0])
def test_null_collision_statistics(e_ev):
    """Monoenergetic electrons, no fields, one step: each process fires with
    probability P_null nu_j / nu_max (Vahedi & Surendra), within 5 sigma;
    excitation and ionisation never fire below threshold; post-collision
    energies: excitation E - 11.55, ionisation (E - 15.76)/2 for both
    electrons, elastic mean loss 2m/M E (isotropic)."""
    cfg = _cfg(pressure_pa=20e-3 * 133.322368)
    T = np.float64
    rng = np.random.default_rng(8)
    n = 200000
    P = _mono_electrons(cfg, T, n, e_ev, rng)
    out = _run(cfg, P, _uniform_F(cfg, T), 0, T)
    sc = out['sc']
    se, sx, si = particles.sigma_e(np.array([e_ev]), T)
    g = math.sqrt(2 * QE * e_ev / ME)
    nus = [float(sc.ng * s[0] * g) for s in (se, sx, si)]
    for j in range(3):
        p = float(sc.pnull) * nus[j] / float(sc.numax)
        mu, sd = n * p, math.sqrt(n * p * (1 - p)) + 1e-9
        assert abs(out['stats']['coll'][0, j] - mu) <= 5 * sd + 1e-9
    if e_ev < E_EXC:
        assert out['stats']['coll'][0, 1] == 0 and out['stats']['coll'][0, 2] == 0
    e_new = 0.5 * ME * (P['vr'] ** 2 + P['vt'] ** 2 + P['vz'] ** 2) / QE
    changed = np.abs(e_new - e_ev) > 1e-9 * e_ev
    exc = np.isclose(e_new, e_ev - E_EXC, rtol=1e-12)
    ion = np.isclose(e_new, (e_ev - E_ION) / 2, rtol=1e-12)
    el = changed & ~exc & ~ion
    assert np.count_nonzero(exc) == out['stats']['coll'][0, 1]
    assert np.count_nonzero(ion) == out['stats']['coll'][0, 2]
    assert np.count_nonzero(el) <= out['stats']['coll'][0, 0]
    loss = (e_ev - e_new[el]) / e_ev
    assert np.all(loss >= -1e-12) and np.all(loss <= 2 * 2 * ME / M_AR * (1 + 1e-9))
    assert loss.mean() == pytest.approx(2 * ME / M_AR, rel=0.05)
    for ev in out['events']:
        ve = np.array(ev['ve'])
        assert 0.5 * ME * ve @ ve / QE == pytest.approx((e_ev - E_ION) / 2, rel=1e-12)
    assert len(out['events']) == out['stats']['coll'][0, 2]


def test_ion_collisions_statistics():
    """Ions at rest in a 300 K neutral background: every real collision leaves
    the ion with a velocity built from one sampled Maxwellian neutral (charge
    exchange: the neutral's velocity; isotropic: (v_n + |v_n| d) / 2); the
    collision rate grows with g, so the collided velocities have the
    flux-weighted spread sqrt(E[v^3] / (3 E[v])) = sqrt(4/3) vth for a
    constant sigma (lower for the decreasing sigma); candidates follow
    Binomial(N, P_null)."""
    cfg = _cfg(pressure_pa=20e-3 * 133.322368)
    T = np.float64
    rng = np.random.default_rng(9)
    n = 3000000
    cell = rng.integers(cfg.nr * 4, cfg.nr * 5, n) + 2
    P = _particles(T, cell, np.full(n, 0.5), np.full(n, 0.5), np.zeros(n), np.zeros(n), np.zeros(n))
    out = _run(cfg, P, _uniform_F(cfg, T), 1, T)
    ncx, niso = out['stats']['coll'][1, 0], out['stats']['coll'][1, 1]
    assert ncx > 20 and niso > 10
    moved = (P['vr'] != 0)
    assert np.count_nonzero(moved) == ncx + niso
    vth = math.sqrt(KB * 300 / M_AR)
    s = np.std(np.concatenate([P['vr'][moved], P['vt'][moved], P['vz'][moved]]))
    assert 0.5 * vth < s < math.sqrt(4.0 / 3.0) * vth * 1.25


def test_fp32_matches_fp64_step():
    """The float32 instantiation tracks the float64 one within float32
    rounding for one step (cells identical away from boundaries)."""
    cfg = _cfg(pressure_pa=20e-3 * 133.322368)
    rng = np.random.default_rng(10)
    geo = CellGeometry(cfg)
    F64 = rng.normal(size=(geo.i_win * cfg.nr, 5, 4)) * np.array([3e3, 3e3, 3e3, 1e-4, 1e-4])[None, :, None]
    P64 = _random_population(cfg, np.float64, 20000, rng)
    P32 = {k: (v.astype(np.float32) if v.dtype == np.float64 else v.copy()) for k, v in P64.items()}
    P64 = {k: (v.astype(np.float32).astype(np.float64) if v.dtype == np.float64 else v) for k, v in P64.items()}
    _run(cfg, P64, F64.astype(np.float32).astype(np.float64), 0, np.float64)
    _run(cfg, P32, F64.astype(np.float32), 0, np.float32)
    same = P64['cell'] == P32['cell']
    assert np.count_nonzero(~same) <= 3
    for k in ('vr', 'vt', 'vz'):
        a, b = P64[k][same], P32[k][same].astype(np.float64)
        assert np.max(np.abs(a - b) / (np.abs(a) + 1e3)) < 2e-5
