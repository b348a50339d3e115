"""Pins of the oracle's particle control (the GEC application of Sec. 3.4 runs
with secondary-electron emission and weighted split-merge; the readings are
stated in oracle.particles and oracle.control): emission yield and the
half-space Maxwellian of the emitted electrons (closed-form moments), the
window's surface charge, weights as exact charge multipliers, the counts the
split-merge pass leaves, charge conservation, exact conservation by splits,
conservation in expectation by merges, and independence from storage order."""
import math

import numpy as np
import pytest

from oracle import control, particles
from oracle.constants import QE, ME
from oracle.grid import CellGeometry
from paper_2609_15043_b300.workloads import CellConfig

T = np.float32


def _cfg(**kw):
    base = dict(nr=16, nz=24, r_max=0.16, z_max=0.24, z_win_lo=0.20, z_win_hi=0.21,
                z_coil=0.225, turn_r=[0.05], winding=[1], pressure_pa=0.0)
    base.update(kw)
    return CellConfig(**base)


def _zero_F(cfg):
    geo = CellGeometry(cfg)
    return np.zeros((geo.i_win * cfg.nr, 5, 4), T)


def _push(cfg, P, sp, see=None, weight=1.0, step=0):
    geo = CellGeometry(cfg)
    sc = particles.SpeciesConstants(cfg, sp, weight, T)
    Q = np.zeros((cfg.nz + 1, cfg.nr + 1))
    J = np.zeros_like(Q)
    win = np.zeros_like(Q)
    stats = dict(p_ind=0.0, p_es=0.0, absorbed=0, pushed=0, nu_viol=0, coll=np.zeros((2, 3), np.int64))
    ev = particles.push_species(P, _zero_F(cfg), sc, geo, step, cfg.seed, T, Q, J, win, stats, see=see)
    return dict(Q=Q, J=J, win=win, stats=stats, events=ev, sc=sc, geo=geo)


def _ions_at(cfg, surface, n, rng):
    """n ions one step from the given surface, moving into it at 1e6 m/s."""
    geo = CellGeometry(cfg)
    nr = cfg.nr
    dr = rng.uniform(0.05, 0.95, n).astype(T)
    dz = rng.uniform(0.05, 0.95, n).astype(T)
    vr = np.zeros(n, T)
    vz = np.zeros(n, T)
    if surface == 0:               # electrode: bottom row, moving down
        ir = rng.integers(0, nr, n)
        iz = np.zeros(n, np.int64)
        dz[:] = T(0.005)
        vz[:] = T(-1e6)
    elif surface == 1:             # side wall: last column, moving out
        ir = np.full(n, nr - 1)
        iz = rng.integers(0, geo.i_win, n)
        dr[:] = T(0.995)
        vr[:] = T(1e6)
    else:                          # window: top plasma row, moving up
        ir = rng.integers(0, nr, n)
        iz = np.full(n, geo.i_win - 1)
        dz[:] = T(0.995)
        vz[:] = T(1e6)
    return dict(cell=(iz * nr + ir).astype(np.int64), dr=dr, dz=dz, vr=vr, vt=np.zeros(n, T), vz=vz,
                uid=rng.permutation(n).astype(np.int64) + 1000)


def _see(gamma, t_ev=2.0):
    return (T(gamma), T(math.sqrt(QE * t_ev / ME)))


@pytest.mark.parametrize("surface", [0, 1, 2])
def test_secondary_emission_yield_and_half_maxwellian(surface):
    """gamma = 0.3: the number of emitted electrons is binomial(N, gamma)
    (within 5 sigma); each starts at its ion's position before the move; the
    normal component points into the plasma with the Rayleigh mean
    v_s sqrt(pi/2) and second moment 2 v_s^2, the tangential components have
    mean 0 and variance v_s^2 (half-space Maxwellian flux at T_see = 2 eV)."""
    cfg = _cfg()
    rng = np.random.default_rng(11 + surface)
    n = 20000
    P = _ions_at(cfg, surface, n, rng)
    P0 = {k: v.copy() for k, v in P.items()}
    out = _push(cfg, P, 1, see=_see(0.3))
    assert out["stats"]["absorbed"] == n
    ev = out["events"]
    assert all(e["kind"] == 1 for e in ev)
    m = len(ev)
    assert abs(m - 0.3 * n) < 5 * math.sqrt(n * 0.3 * 0.7)
    pos = {int(u): (int(c), float(a), float(b)) for u, c, a, b in zip(P0["uid"], P0["cell"], P0["dr"], P0["dz"])}
    for e in ev:
        assert (e["cell"], float(e["dr"]), float(e["dz"])) == pos[e["parent"]]
    v = np.array([e["ve"] for e in ev], np.float64)
    vs = math.sqrt(QE * 2.0 / ME)
    normal = {0: v[:, 2], 1: -v[:, 0], 2: -v[:, 2]}[surface]
    tang = {0: (v[:, 0], v[:, 1]), 1: (v[:, 1], v[:, 2]), 2: (v[:, 0], v[:, 1])}[surface]
    assert np.all(normal > 0)
    se_mean = vs * math.sqrt((4 - math.pi) / 2) / math.sqrt(m)
    assert abs(normal.mean() - vs * math.sqrt(math.pi / 2)) < 5 * se_mean
    assert abs(np.mean(normal ** 2) / (2 * vs ** 2) - 1) < 5 * 1.0 / math.sqrt(m)
    for t in tang:
        assert abs(t.mean()) < 5 * vs / math.sqrt(m)
        assert abs(np.mean(t ** 2) / vs ** 2 - 1) < 5 * math.sqrt(2.0 / m)


def test_window_keeps_the_charge_of_emitted_electrons():
    """On the window each absorbed ion leaves q W w and each emitted electron
    another q W w: the surface charge totals q W w (N_abs + N_emit)."""
    cfg = _cfg()
    rng = np.random.default_rng(5)
    n = 4000
    P = _ions_at(cfg, 2, n, rng)
    out = _push(cfg, P, 1, see=_see(0.4), weight=1e6)
    m = len(out["events"])
    qw = float(out["sc"].qw)
    assert out["win"].sum() == pytest.approx(qw * (n + m), rel=1e-6)
    P2 = _ions_at(cfg, 2, n, np.random.default_rng(5))
    out2 = _push(cfg, P2, 1, see=None, weight=1e6)
    assert out2["win"].sum() == pytest.approx(qw * n, rel=1e-6)


def test_zero_and_unit_yield():
    """gamma = 0 is the step without emission, bit for bit; gamma = 1 emits one
    electron per absorbed ion (the uniform is < 1)."""
    cfg = _cfg()
    for surface in (0, 1, 2):
        P = _ions_at(cfg, surface, 500, np.random.default_rng(surface))
        Pa = {k: v.copy() for k, v in P.items()}
        Pb = {k: v.copy() for k, v in P.items()}
        a = _push(cfg, Pa, 1, see=None)
        b = _push(cfg, Pb, 1, see=_see(0.0))
        assert b["events"] == [] and np.array_equal(a["win"], b["win"])
        for k in Pa:
            assert np.array_equal(Pa[k], Pb[k])
        c = _push(cfg, {k: v.copy() for k, v in P.items()}, 1, see=_see(1.0))
        assert len(c["events"]) == 500


def _plasma(cfg, n, rng, sp):
    geo = CellGeometry(cfg)
    cells = rng.integers(0, geo.i_win * cfg.nr, n)
    vth = 1e6 if sp == 0 else 1e3
    return dict(cell=cells.astype(np.int64), dr=rng.random(n).astype(T), dz=rng.random(n).astype(T),
                vr=(rng.standard_normal(n) * vth).astype(T), vt=(rng.standard_normal(n) * vth).astype(T),
                vz=(rng.standard_normal(n) * vth).astype(T), uid=np.arange(n, dtype=np.int64))


def test_unit_weights_and_uniform_weights():
    """w = 1 reproduces the unweighted step bit for bit; w = 2 doubles Q, J,
    the window charge and P_ind exactly (a power-of-two charge multiplier)."""
    cfg = _cfg()
    base = _plasma(cfg, 6000, np.random.default_rng(2), 0)
    F = _zero_F(cfg)
    F[:, 2, :] = T(300.0)          # an E_theta so that J and P_ind are nonzero
    F[:, 0, :] = T(1e3)

    def run(w):
        P = {k: v.copy() for k, v in base.items()}
        if w is not None:
            P["w"] = np.full(P["dr"].shape, w, T)
        geo = CellGeometry(cfg)
        sc = particles.SpeciesConstants(cfg, 0, 1e5, T)
        Q = np.zeros((cfg.nz + 1, cfg.nr + 1))
        J, win = np.zeros_like(Q), np.zeros_like(Q)
        st = dict(p_ind=0.0, p_es=0.0, absorbed=0, pushed=0, nu_viol=0, coll=np.zeros((2, 3), np.int64))
        particles.push_species(P, F, sc, geo, 3, cfg.seed, T, Q, J, win, st)
        return P, Q, J, win, st

    P0, Q0, J0, W0, s0 = run(None)
    P1, Q1, J1, W1, s1 = run(1.0)
    P2, Q2, J2, W2, s2 = run(2.0)
    for k in ("cell", "dr", "dz", "vr", "vt", "vz"):
        assert np.array_equal(P0[k], P1[k]) and np.array_equal(P0[k], P2[k])
    assert np.array_equal(Q0, Q1) and np.array_equal(J0, J1) and s0["p_ind"] == s1["p_ind"]
    assert np.array_equal(Q2, 2 * Q0) and np.array_equal(J2, 2 * J0) and np.array_equal(W2, 2 * W0)
    assert s2["p_ind"] == 2 * s0["p_ind"] and s2["p_es"] == 2 * s0["p_es"]
    assert np.any(J0 != 0) and s0["p_ind"] != 0


def test_ionisation_products_inherit_the_parent_weight():
    cfg = _cfg(pressure_pa=20e-3 * 133.322368)
    rng = np.random.default_rng(4)
    P = _plasma(cfg, 20000, rng, 0)
    P["vr"] = (rng.standard_normal(P["vr"].size) * 3e6).astype(T)
    P["w"] = rng.uniform(0.5, 2.0, P["vr"].size).astype(T)
    wmap = dict(zip(P["uid"].tolist(), P["w"].tolist()))
    geo = CellGeometry(cfg)
    sc = particles.SpeciesConstants(cfg, 0, 1e5, T)
    Q = np.zeros((cfg.nz + 1, cfg.nr + 1))
    st = dict(p_ind=0.0, p_es=0.0, absorbed=0, pushed=0, nu_viol=0, coll=np.zeros((2, 3), np.int64))
    ev = []
    for s in range(20):
        ev += particles.push_species(P, _zero_F(cfg), sc, geo, s, cfg.seed, T, Q, np.zeros_like(Q),
                                     np.zeros_like(Q), st)
    assert len(ev) > 10
    for e in ev:
        assert e["kind"] == 0 and float(e["w"]) == wmap[e["parent"]]


# ---------------------------------------------------------------- split-merge
def _store(counts, rng, ncell):
    cells = np.concatenate([np.full(n, c, np.int64) for c, n in counts.items()])
    n = cells.size
    P = dict(cell=cells, dr=rng.random(n).astype(T), dz=rng.random(n).astype(T),
             vr=rng.standard_normal(n).astype(T), vt=rng.standard_normal(n).astype(T),
             vz=rng.standard_normal(n).astype(T), w=rng.uniform(0.5, 2.0, n).astype(T),
             uid=rng.permutation(n).astype(np.int64) * 3 + 7)
    perm = rng.permutation(n)
    return {k: v[perm] for k, v in P.items()}


def _cell_sums(P, ncell):
    live = P["cell"] >= 0
    c = P["cell"][live]
    w = P["w"][live].astype(np.float64)
    out = dict(n=np.bincount(c, minlength=ncell), w=np.bincount(c, w, ncell))
    for k in ("vr", "vt", "vz"):
        v = P[k][live].astype(np.float64)
        out["p" + k] = np.bincount(c, w * v, ncell)
        out["e" + k] = np.bincount(c, w * v * v, ncell)
    return out


def test_split_merge_counts_and_conservation():
    """target 40, split below 20, merge above 60: n = 100 -> 50 (n // 2
    merges), n = 70 -> 40, n = 10 -> 20 (every particle splits), n = 13 -> 26,
    n = 30 and 60 untouched, n = 5000 > CELL_CAP skipped.  Charge (sum of w)
    is conserved per cell to the rounding of the pair sums; in split cells the
    weighted momentum and energy sums are exact; the copies carry the new uids
    in cell order, then in the originals' uid order."""
    ncell = 8
    counts = {0: 100, 1: 70, 2: 10, 3: 30, 4: 5000, 5: 13, 6: 60}
    P = _store(counts, np.random.default_rng(9), ncell)
    before = _cell_sums(P, ncell)
    src_state = {int(u): (int(c), float(a), float(b), float(x), float(y), float(z))
                 for u, c, a, b, x, y, z in zip(P["uid"], P["cell"], P["dr"], P["dz"], P["vr"], P["vt"], P["vz"])}
    n_old = P["uid"].size
    st, nu = control.split_merge(P, 0, 17, 99, ncell, 40, 20, 60, 10 ** 6, T)
    after = _cell_sums(P, ncell)
    expect = {0: 50, 1: 40, 2: 20, 3: 30, 4: 5000, 5: 26, 6: 60, 7: 0}
    assert [int(after["n"][c]) for c in range(ncell)] == [expect[c] for c in range(ncell)]
    assert st == dict(split=10 + 13, merged=50 + 30, skipped=1)
    assert nu == 10 ** 6 + 23
    assert np.allclose(after["w"], before["w"], rtol=1e-6, atol=0)
    for c in (2, 5):
        for k in ("pvr", "pvt", "pvz", "evr", "evt", "evz"):
            assert after[k][c] == pytest.approx(before[k][c], rel=1e-12, abs=1e-12)
    # copies: uids 10^6.. in cell order (2 then 5), originals' uid order within a cell
    new_uid = P["uid"][n_old:]
    assert np.array_equal(new_uid, np.arange(10 ** 6, 10 ** 6 + 23))
    orig = {}
    for c in (2, 5):
        live = np.nonzero((P["cell"][:n_old] == c))[0]
        orig[c] = np.sort(P["uid"][live])[:counts[c]]
    want = np.concatenate([orig[2], orig[5]])
    for j, u in enumerate(want):
        q = n_old + j
        s = src_state[int(u)]
        assert (int(P["cell"][q]), float(P["dr"][q]), float(P["dz"][q]), float(P["vr"][q]), float(P["vt"][q]),
                float(P["vz"][q])) == s
        po = np.nonzero(P["uid"] == u)[0][0]
        assert P["w"][q] == P["w"][po]
    # untouched cells keep their particles as they were
    for c in (3, 4, 6):
        assert after["w"][c] == before["w"][c]


def test_merge_keeps_a_state_with_probability_proportional_to_its_weight():
    """2000 pairs (w_a = 1, v_z = +1; w_b = 3, v_z = -1; a the lower uid):
    the survivor has v_z = +1 with probability 1/4, so the weighted momentum
    1 - 3 = -2 is conserved in expectation (a rule with the probabilities
    swapped would give +2)."""
    k = 2000
    n = 2 * k
    uid = np.arange(n, dtype=np.int64)
    a = uid % 2 == 0
    P = dict(cell=np.zeros(n, np.int64), dr=np.full(n, 0.5, T), dz=np.full(n, 0.5, T),
             vr=np.zeros(n, T), vt=np.zeros(n, T), vz=np.where(a, 1.0, -1.0).astype(T),
             w=np.where(a, 1.0, 3.0).astype(T), uid=uid)
    st, _ = control.split_merge(P, 1, 5, 2026, 1, 1, 1, 2, n, T)
    assert st["merged"] == k
    live = P["cell"] >= 0
    assert np.count_nonzero(live) == k and np.all(P["w"][live] == 4.0)
    frac = np.mean(P["vz"][live] > 0)
    assert abs(frac - 0.25) < 5 * math.sqrt(0.25 * 0.75 / k)
    mom = float(np.sum(P["w"][live] * P["vz"][live]))
    assert abs(mom / k - (-2.0)) < 5 * 4 * 2 * math.sqrt(0.25 * 0.75 / k)


def test_split_merge_does_not_depend_on_storage_order():
    ncell = 4
    counts = {0: 90, 1: 8, 2: 45, 3: 200}
    P = _store(counts, np.random.default_rng(3), ncell)
    perm = np.random.default_rng(8).permutation(P["uid"].size)
    Q = {k: v[perm].copy() for k, v in P.items()}
    control.split_merge(P, 0, 4, 1, ncell, 30, 10, 50, 5000, T)
    control.split_merge(Q, 0, 4, 1, ncell, 30, 10, 50, 5000, T)

    def table(R):
        live = R["cell"] >= 0
        o = np.argsort(R["uid"][live])
        return {k: R[k][live][o] for k in R}
    a, b = table(P), table(Q)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
