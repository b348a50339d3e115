"""The plain FP64 particle form (pp_config.plain_fp64 = 1) against the
oracle's float64 instantiation on identical seeded inputs: integer cells,
absorptions, uids and collision counts bit-exact, FP64 positions and
velocities within 1e-9 relative (both sides are FP64 with the operation order
of the float32 path; the node fields and the transcendental functions of the
collision kinematics may differ in the last bits), deposited charge and
current within 1e-12 of the total (atomic summation order)."""
import numpy as np
import pytest

from gpu_common import require_gpu, oracle_cell, gpu_cell, by_uid, oracle_live, check_step_potential

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small_fp64():
    from paper_2609_15043_b300 import workloads
    cfg = workloads.small().replace(plain_fp64=1)
    pops = [workloads.population(cfg, sp) for sp in (0, 1)]
    return cfg, pops


def _run(cfg, pops, steps):
    oc = oracle_cell(cfg, pops, T=np.float64)
    oc.prime(np.float64)
    g = gpu_cell(cfg, pops)
    g.set_potential(oc.phi)
    tot = dict(coll=np.zeros((2, 3), np.int64), absorbed=0, created=0, pushed=0)
    info = None
    for _ in range(steps):
        info = oc.step(np.float64)
        tot['coll'] += info['stats']['coll']
        tot['absorbed'] += info['stats']['absorbed']
        tot['created'] += info['events']
        tot['pushed'] += info['stats']['pushed']
        g.advance_steps(1)
        if steps > 1:
            g.set_potential(oc.phi)
    return oc, g, info, tot


@pytest.mark.parametrize("implicit", [0, 1])
def test_fp64_one_step_parity(small_fp64, implicit):
    """One step in each electrostatic form; in the direct-implicit form also
    the potential of the step's chi solve (from the FP64 species charges)."""
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp
    cfg, pops = small_fp64
    cfg = cfg.replace(implicit_es=implicit)
    oc, g, info, tot = _run(cfg, pops, 1)
    cnt = g.counters()
    assert cnt["particle_steps"] == tot["pushed"]
    assert cnt["absorbed"] == tot["absorbed"]
    assert cnt["created"] == tot["created"]
    assert [cnt["e_elastic"], cnt["e_excitation"], cnt["e_ionisation"]] == list(tot["coll"][0])
    assert [cnt["i_cx"], cnt["i_isotropic"]] == list(tot["coll"][1][:2])
    for sp in (0, 1):
        pg = by_uid(g.get_particles(sp, dtype=np.float64))
        po = oracle_live(oc.P[sp])
        assert np.array_equal(pg["uid"], po["uid"].astype(np.uint32))
        assert np.array_equal(pg["cell"], po["cell"].astype(np.uint32))
        for k in ("dr", "dz"):
            assert np.max(np.abs(pg[k] - po[k])) <= 1e-12
        for k in ("vr", "vt", "vz"):
            scale = np.maximum(np.abs(po[k]), 1e-3 * np.max(np.abs(po[k])))
            assert np.max(np.abs(pg[k] - po[k]) / scale) <= 1e-9
    q = g.grid(pp.GRID_CHARGE)
    assert np.max(np.abs(q - info["Q"])) <= 1e-12 * np.sum(np.abs(info["Q"]))
    j = g.grid(pp.GRID_JMOM)
    assert np.max(np.abs(j - info["J"])) <= 1e-12 * np.sum(np.abs(info["J"]))
    if implicit:
        for sp, grid in ((0, pp.GRID_CHARGE_E), (1, pp.GRID_CHARGE_I)):
            qs = g.grid(grid)
            assert np.max(np.abs(qs - info["Qs"][sp])) <= 1e-12 * np.sum(np.abs(info["Qs"][sp]))
        check_step_potential(oc, g, T=np.float64, tol_oracle=1e-8)
    g.close()


@pytest.mark.parametrize("implicit", [0, 1])
def test_fp64_ten_steps(small_fp64, implicit):
    require_gpu()
    cfg, pops = small_fp64
    cfg = cfg.replace(implicit_es=implicit)
    oc, g, info, tot = _run(cfg, pops, 10)
    cnt = g.counters()
    assert cnt["absorbed"] == tot["absorbed"]
    assert cnt["created"] == tot["created"]
    for sp in (0, 1):
        pg = by_uid(g.get_particles(sp, dtype=np.float64))
        po = oracle_live(oc.P[sp])
        assert np.array_equal(pg["uid"], po["uid"].astype(np.uint32))
        assert np.array_equal(pg["cell"], po["cell"].astype(np.uint32))
    g.close()


def test_fp64_period_and_checkpoint(small_fp64):
    """A whole period of the FP64 form runs through the period graph, and its
    checkpoint restores into a fresh FP64 cell."""
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp
    cfg, pops = small_fp64
    g = gpu_cell(cfg, pops)
    g.advance_period(1)
    r = g.turn_phasors()
    assert r["n_samples"] == g.n_rf and r["accepted"]
    # the violent 2e4-particle cell may fill its particle or event storage
    # within a period (reported, not an error of the step)
    assert g.status() & ~(2 | 4) == 0
    img = g.checkpoint()
    h = pp.Cell(cfg)
    h.restore(img)
    assert h.checkpoint() == img
    a, b = by_uid(g.get_particles(0, dtype=np.float64)), by_uid(h.get_particles(0, dtype=np.float64))
    for k in a:
        assert np.array_equal(a[k], b[k])
    g.close()
    h.close()
