"""Particle control on the GPU against the oracle (the GEC-type runs of Sec.
3.4: secondary-electron emission and weighted split-merge; readings stated
with pp_config): steps with ions absorbed on every surface and emitting,
steps with per-particle weights, split-merge passes (bit-exact: a merge
selects a state, a split copies one), the plain FP64 form against the
oracle's float64 instantiation, and checkpoints of weighted cells."""
import numpy as np
import pytest

from gpu_common import require_gpu, oracle_cell, gpu_cell, by_uid, oracle_live

pytestmark = pytest.mark.gpu


def _boundary_ions(cfg, n, seed):
    """n ions one step from the electrode, the side wall or the window (a
    third each), moving into the surface at 1e6 m/s."""
    rng = np.random.default_rng(seed)
    nr = cfg.nr
    i_win = int(round(cfg.z_win_lo / (cfg.z_max / cfg.nz)))
    surf = np.arange(n) % 3
    ir = rng.integers(0, nr, n)
    iz = rng.integers(0, i_win, n)
    dr = rng.uniform(0.05, 0.95, n)
    dz = rng.uniform(0.05, 0.95, n)
    vr = rng.normal(0, 1e3, n)
    vz = rng.normal(0, 1e3, n)
    e, w, d = surf == 0, surf == 1, surf == 2
    iz[e], dz[e], vz[e] = 0, 0.005, -1e6
    ir[w], dr[w], vr[w] = nr - 1, 0.995, 1e6
    iz[d], dz[d], vz[d] = i_win - 1, 0.995, 1e6
    return dict(cell=(iz * nr + ir).astype(np.uint32), dr=dr.astype(np.float32), dz=dz.astype(np.float32),
                vr=vr.astype(np.float32), vt=rng.normal(0, 1e3, n).astype(np.float32), vz=vz.astype(np.float32),
                uid=(rng.permutation(n) + 5).astype(np.uint32))


def _empty():
    e = np.zeros(0, np.float32)
    return dict(cell=np.zeros(0, np.uint32), dr=e, dz=e, vr=e, vt=e, vz=e, uid=np.zeros(0, np.uint32))


def _pair(cfg, pops, weights=None, T=np.float32):
    """Oracle and GPU cells on the same populations (and weights), the GPU
    started from the oracle's primed potential."""
    oc = oracle_cell(cfg, pops, T)
    if weights is not None:
        for sp in (0, 1):
            oc.P[sp]["w"] = np.asarray(weights[sp], T).copy()
    oc.prime(T)
    gp = []
    for sp in (0, 1):
        p = dict(pops[sp])
        if weights is not None:
            p["w"] = np.asarray(weights[sp], np.float64)
        gp.append(p)
    g = gpu_cell(cfg, gp)
    g.set_potential(oc.phi)
    return oc, g


def _compare_particles(oc, g, exact_v=False, T=np.float32):
    for sp in (0, 1):
        pg = by_uid(g.get_particles(sp, dtype=T))
        po = oracle_live(oc.P[sp])
        assert np.array_equal(pg["uid"], po["uid"].astype(np.uint32)), sp
        assert np.array_equal(pg["cell"], po["cell"].astype(np.uint32)), sp
        if "w" in pg:
            assert np.array_equal(pg["w"], po["w"].astype(np.float64)), sp
        for k in ("dr", "dz", "vr", "vt", "vz"):
            if exact_v:
                assert np.array_equal(pg[k], po[k].astype(T)), (sp, k)
            else:
                scale = np.maximum(np.abs(po[k]), 1e-3 * max(np.max(np.abs(po[k]), initial=0.0), 1e-30))
                assert np.max(np.abs(pg[k] - po[k]) / scale, initial=0.0) <= 2e-5, (sp, k)


@pytest.mark.parametrize("implicit", [0, 1])
def test_secondary_emission_step(implicit):
    """6000 ions leave through the electrode, the wall and the window in one
    step with gamma = 0.4: the same ions emit on both sides (count, uids,
    cells and offsets of the new electrons exact, velocities to the float32
    rounding of their transcendentals), and the window's surface charge,
    doubled where an ion emitted, agrees."""
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp, workloads
    cfg = workloads.small().replace(pressure_pa=0.0, see_gamma=0.4, implicit_es=implicit)
    pops = [_empty(), _boundary_ions(cfg, 6000, 3)]
    oc, g = _pair(cfg, pops)
    info = oc.step(np.float32)
    g.advance_steps(1)
    assert info["see"] > 1500
    assert g.control_counters()["see"] == oc.see_emitted == info["see"]
    assert g.counters()["absorbed"] == info["stats"]["absorbed"]
    _compare_particles(oc, g)
    win = oc.window_q
    assert np.max(np.abs(g.grid(pp.GRID_WINDOW) - win)) <= 1e-6 * np.sum(np.abs(win))
    assert g.status() == 0
    g.close()


@pytest.mark.parametrize("implicit", [0, 1])
def test_weighted_steps(implicit):
    """Both species with weights uniform in [0.5, 2] over five steps from the
    small workload's populations (gas on): cells, absorptions and collisions
    exact, ionisation products carrying their parents' weights, charge and
    current deposits within 1e-6 of their totals."""
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp, workloads
    cfg = workloads.small().replace(particle_weights=1, implicit_es=implicit)
    pops = [workloads.population(cfg, sp) for sp in (0, 1)]
    rng = np.random.default_rng(7)
    ws = [rng.uniform(0.5, 2.0, len(p["uid"])).astype(np.float32) for p in pops]
    oc, g = _pair(cfg, pops, ws)
    created = 0
    for _ in range(5):
        info = oc.step(np.float32)
        created += info["events"]
        g.advance_steps(1)
        g.set_potential(oc.phi)
    assert created > 0
    assert g.counters()["created"] == oc.created
    _compare_particles(oc, g)
    q_g = g.grid(pp.GRID_CHARGE)
    assert np.max(np.abs(q_g - info["Q"])) <= 1e-6 * np.sum(np.abs(info["Q"]))
    j_g = g.grid(pp.GRID_JMOM)
    assert np.max(np.abs(j_g - info["J"])) <= 1e-6 * np.sum(np.abs(info["J"]))
    g.close()


def _sm_cfg(**kw):
    from paper_2609_15043_b300 import workloads
    base = dict(sm_every=1, sm_target=12, sm_min=8, sm_max=20)
    base.update(kw)
    return workloads.small().replace(**base)


@pytest.mark.parametrize("implicit", [0, 1])
def test_split_merge_passes(implicit):
    """A pass after each of three steps on the small workload (about 15
    particles per cell, target 12, split below 8, merge above 20): the
    populations, weights and new uids are bit-identical to the oracle's, the
    split and merge counts equal, and the live counters match the store."""
    require_gpu()
    from paper_2609_15043_b300 import workloads
    cfg = _sm_cfg(implicit_es=implicit)
    pops = [workloads.population(cfg, sp) for sp in (0, 1)]
    oc, g = _pair(cfg, pops)
    for _ in range(3):
        oc.step(np.float32)
        g.advance_steps(1)
        g.set_potential(oc.phi)
    cc = g.control_counters()
    assert cc["split"] == oc.sm_stats["split"] > 0
    assert cc["merged"] == oc.sm_stats["merged"] > 0
    assert cc["skipped"] == oc.sm_stats["skipped"] == 0
    _compare_particles(oc, g)
    cnt = g.counters()
    assert cnt["live_e"] == len(g.get_particles(0)["uid"]) and cnt["live_i"] == len(g.get_particles(1)["uid"])
    assert g.status() == 0
    g.close()


def test_plain_fp64_control_against_float64_oracle():
    """The plain FP64 form with secondary emission and split-merge against
    the oracle's float64 instantiation over three steps: integer state and
    weights exact, offsets and velocities within 1e-9."""
    require_gpu()
    from paper_2609_15043_b300 import workloads
    cfg = _sm_cfg(plain_fp64=1, see_gamma=0.5, implicit_es=1)
    pops = [workloads.population(cfg, 0), _boundary_ions(cfg, 3000, 9)]
    pops[1]["uid"] = pops[1]["uid"] + np.uint32(10 ** 6)
    oc, g = _pair(cfg, pops, T=np.float64)
    for _ in range(3):
        oc.step(np.float64)
        g.advance_steps(1)
        g.set_potential(oc.phi)
    assert g.control_counters()["see"] == oc.see_emitted > 0
    assert g.control_counters()["merged"] == oc.sm_stats["merged"]
    assert g.control_counters()["split"] == oc.sm_stats["split"]
    for sp in (0, 1):
        pg = by_uid(g.get_particles(sp, dtype=np.float64))
        po = oracle_live(oc.P[sp])
        assert np.array_equal(pg["uid"], po["uid"].astype(np.uint32))
        assert np.array_equal(pg["cell"], po["cell"].astype(np.uint32))
        assert np.array_equal(pg["w"], po["w"])
        for k in ("dr", "dz", "vr", "vt", "vz"):
            scale = max(np.max(np.abs(po[k])), 1e-30)
            assert np.max(np.abs(pg[k] - po[k])) <= 1e-9 * scale, (sp, k)
    g.close()


def test_checkpoint_of_a_weighted_cell():
    """A weighted cell with split-merge and emission restores bit for bit and
    continues identically in its integer state."""
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp, workloads
    cfg = _sm_cfg(sm_every=4, see_gamma=0.3)
    pops = [workloads.population(cfg, sp) for sp in (0, 1)]
    a = gpu_cell(cfg, pops)
    a.prime()
    a.advance_steps(6)
    img = a.checkpoint()
    b = pp.Cell(cfg)
    b.restore(img)
    assert b.checkpoint() == img
    a.advance_steps(3)
    b.advance_steps(3)
    for sp in (0, 1):
        pa, pb = by_uid(a.get_particles(sp)), by_uid(b.get_particles(sp))
        for k in ("uid", "cell", "w"):
            assert np.array_equal(pa[k], pb[k]), (sp, k)
    assert a.control_counters() == b.control_counters()
    a.close()
    b.close()


def test_weights_need_a_weighted_cell():
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp, workloads
    cfg = workloads.small()
    g = pp.Cell(cfg)
    p = workloads.population(cfg, 0)
    p["w"] = np.ones(len(p["uid"]))
    with pytest.raises(pp.PhasorPICError):
        g.set_particles(0, p)
    g.close()


def test_control_inside_the_period_graph():
    """With sm_every dividing N_RF the captured period graph carries the
    split-merge passes (and the emission branches): two whole periods run
    through pp_advance_period, the passes act, the live counters equal the
    stored populations, the applied weights stay positive and the cell's
    status stays clear."""
    require_gpu()
    from paper_2609_15043_b300 import workloads
    cfg = _sm_cfg(sm_every=100, see_gamma=0.3, implicit_es=1)
    g = gpu_cell(cfg, [workloads.population(cfg, sp) for sp in (0, 1)])
    g.prime()
    g.advance_period(2)
    cc = g.control_counters()
    assert cc["split"] > 0 and cc["merged"] > 0 and cc["see"] > 0
    cnt = g.counters()
    for sp, key in ((0, "live_e"), (1, "live_i")):
        p = g.get_particles(sp)
        assert cnt[key] == len(p["uid"])
        assert np.all(p["w"] > 0) and len(np.unique(p["uid"])) == len(p["uid"])
    rec = g.turn_phasors()
    assert rec["period"] == 1 and rec["accepted"]
    assert g.status() == 0
    g.close()
