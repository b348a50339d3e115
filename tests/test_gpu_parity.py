"""GPU (CUDA, sm_103a) vs oracle parity through the C ABI on identical seeded
inputs.  Contract: integer cell indices, particle counts and collision counts
bit-exact; float32 positions and velocities within 2e-5 relative; deposited
grid charge within 1e-6 of the total; FP64 field solves within 1e-9."""
import math

import numpy as np
import pytest

from gpu_common import require_gpu, oracle_cell, gpu_cell, by_uid, oracle_live, check_step_potential

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small_inputs():
    from paper_2609_15043_b300 import workloads
    cfg = workloads.small()
    pops = [workloads.population(cfg, sp) for sp in (0, 1)]
    return cfg, pops


def test_vacuum_impedance_and_unit_fields(small_inputs):
    """Eq. unitfield / Eq. zvac: FP64 separable Helmholtz on the GPU vs the
    oracle's sparse direct solve; R_rf of Eq. skin."""
    require_gpu()
    cfg, pops = small_inputs
    from oracle.cell import OracleCell
    from paper_2609_15043_b300 import phasorpic as pp
    oc = OracleCell(cfg, [1.0, 1.0])
    g = pp.Cell(cfg)
    Z, eps_rec, rrf = g.vacuum_impedance()
    assert np.max(np.abs(Z - oc.zvac)) <= 1e-10 * np.max(np.abs(oc.zvac))
    assert eps_rec < 1e-9
    assert np.allclose(rrf, oc.r_rf, rtol=1e-14)
    for k in range(len(cfg.turn_r)):
        U = g.grid(pp.GRID_U0 + k)
        assert np.max(np.abs(U - oc.U[k])) <= 1e-10 * np.max(np.abs(oc.U[k]))
    # the composed first-cycle field (Eq. compose with the zero-load state)
    assert np.max(np.abs(g.grid(pp.GRID_EC) - oc.Ec)) <= 1e-9 * np.max(np.abs(oc.Ec))
    assert np.max(np.abs(g.grid(pp.GRID_ESS) - oc.Ess)) <= 1e-9 * np.max(np.abs(oc.Ess))
    x, vg = g.circuit_state()
    assert np.max(np.abs(x - oc.x)) <= 1e-10 * np.max(np.abs(oc.x))
    g.close()


@pytest.mark.parametrize("workload", ["small", "cell60", "cell100"])
def test_poisson_solve(workload):
    """Eq. poisson (chi = 0) with the dielectric window and equipotential
    turns: FP32 separable solves inside FP64 residual refinement vs the
    oracle's sparse LU; Gauss-law turn charges (Eq. facecharge)."""
    require_gpu()
    from paper_2609_15043_b300 import workloads, phasorpic as pp
    from oracle.grid import CellGeometry
    from oracle import fields
    cfg = getattr(workloads, workload)().replace(n_init=1000)
    geo = CellGeometry(cfg)
    ps = fields.PoissonSolver(geo.grid, geo.poisson_dirichlet())
    rng = np.random.default_rng(11)
    NZ, NR = cfg.nz + 1, cfg.nr + 1
    q = np.zeros((NZ, NR))
    q[:geo.i_win + 1] = rng.normal(size=(geo.i_win + 1, NR)) * 1e-12
    turn_phi = rng.normal(size=len(cfg.turn_r)) * 200.0
    vals = np.zeros((NZ, NR))
    for k, nodes in enumerate(geo.turn_nodes):
        for n in nodes:
            vals[n] = turn_phi[k]
    phi_o = ps.solve(np.where(geo.poisson_dirichlet(), 0.0, q), vals)
    qk_o = fields.turn_charge(geo.grid, phi_o, geo.turn_nodes)
    g = pp.Cell(cfg)
    phi_g, qk_g, iters, rel = g.poisson_solve(np.where(geo.poisson_dirichlet(), 0.0, q), turn_phi)
    assert rel <= 1e-10
    scale = np.max(np.abs(phi_o))
    assert np.max(np.abs(phi_g - phi_o)) <= 1e-9 * scale
    assert np.max(np.abs(qk_g - qk_o)) <= 1e-8 * np.max(np.abs(qk_o))
    g.close()


def test_helmholtz_solve(small_inputs):
    """Eq. helmholtz_op (full operator with the window's eps_r w^2/c^2)."""
    require_gpu()
    cfg, _ = small_inputs
    from oracle.cell import OracleCell
    from paper_2609_15043_b300 import phasorpic as pp
    oc = OracleCell(cfg, [1.0, 1.0])
    g = pp.Cell(cfg)
    rng = np.random.default_rng(12)
    rhs = rng.normal(size=(cfg.nz + 1, cfg.nr + 1))
    e_o = oc.helm.solve(rhs)
    e_g = g.helmholtz_solve(rhs)
    # both solvers are backward stable; the operator conditioning (~N^2) bounds
    # their agreement near 1e-10 relative for a white-noise right-hand side
    assert np.max(np.abs(e_g - e_o)) <= 1e-8 * np.max(np.abs(e_o))
    g.close()


def _step_compare(cfg, pops, steps=1):
    from paper_2609_15043_b300 import phasorpic as pp
    oc = oracle_cell(cfg, pops)
    oc.prime(np.float32)
    g = gpu_cell(cfg, pops)
    g.set_potential(oc.phi)
    tot = dict(coll=np.zeros((2, 3), np.int64), absorbed=0, created=0, pushed=0)
    for _ in range(steps):
        info = oc.step(np.float32)
        tot['coll'] += info['stats']['coll']
        tot['absorbed'] += info['stats']['absorbed']
        tot['created'] += info['events']
        tot['pushed'] += info['stats']['pushed']
        g.advance_steps(1)
        if steps > 1:
            g.set_potential(oc.phi)      # restart each step from the oracle's field
    return oc, g, info, tot


@pytest.mark.parametrize("implicit", [0, 1])
def test_one_step_parity(small_inputs, implicit):
    """One full PIC step from identical state and field: cells, absorptions,
    collision counts and ionisation products bit-exact, float32 state within
    2e-5, deposited charge within 1e-6 of the total.  In the direct-implicit
    form (Sec. 2.3) the step also solves Eq. poisson with the susceptibility of
    the predicted populations: the new potential against the oracle's direct
    solve of the same operator."""
    require_gpu()
    cfg, pops = small_inputs
    cfg = cfg.replace(implicit_es=implicit)
    from paper_2609_15043_b300 import phasorpic as pp
    oc, g, info, tot = _step_compare(cfg, pops)
    check_step_potential(oc, g)
    assert g.poisson_stats()[g.poisson_stats() > 0][-1] <= 1e-10
    cnt = g.counters()
    assert cnt["particle_steps"] == tot['pushed']
    assert cnt["absorbed"] == tot['absorbed']
    assert cnt["created"] == tot['created']
    assert [cnt["e_elastic"], cnt["e_excitation"], cnt["e_ionisation"]] == list(tot['coll'][0])
    assert [cnt["i_cx"], cnt["i_isotropic"]] == list(tot['coll'][1][:2])
    for sp in (0, 1):
        pg = by_uid(g.get_particles(sp))
        po = oracle_live(oc.P[sp])
        assert len(pg["uid"]) == len(po["uid"])
        assert np.array_equal(pg["uid"], po["uid"].astype(np.uint32))
        assert np.array_equal(pg["cell"], po["cell"].astype(np.uint32))
        for k in ("dr", "dz"):
            assert np.max(np.abs(pg[k] - po[k])) <= 2e-5
        for k in ("vr", "vt", "vz"):
            scale = np.maximum(np.abs(po[k]), 1e-3 * np.max(np.abs(po[k])))
            assert np.max(np.abs(pg[k] - po[k]) / scale) <= 2e-5
    q_g = g.grid(pp.GRID_CHARGE)
    tot_q = np.sum(np.abs(info['Q']))
    assert np.max(np.abs(q_g - info['Q'])) <= 1e-6 * tot_q
    j_g = g.grid(pp.GRID_JMOM)
    assert np.max(np.abs(j_g - info['J'])) <= 1e-6 * np.sum(np.abs(info['J']))
    assert np.max(np.abs(g.grid(pp.GRID_WINDOW) - oc.window_q)) <= 1e-6 * max(np.sum(np.abs(oc.window_q)), 1e-30)
    g.close()


@pytest.mark.parametrize("implicit", [0, 1])
def test_ten_steps_from_shared_fields(small_inputs, implicit):
    """Ten consecutive steps, each started from the oracle's potential: the
    particle populations (including ionisation products and their uids) stay
    bit-identical in their integer state."""
    require_gpu()
    cfg, pops = small_inputs
    cfg = cfg.replace(implicit_es=implicit)
    oc, g, info, tot = _step_compare(cfg, pops, steps=10)
    cnt = g.counters()
    assert cnt["absorbed"] == tot['absorbed']
    assert cnt["created"] == tot['created']
    for sp in (0, 1):
        pg = by_uid(g.get_particles(sp))
        po = oracle_live(oc.P[sp])
        assert np.array_equal(pg["uid"], po["uid"].astype(np.uint32))
        assert np.array_equal(pg["cell"], po["cell"].astype(np.uint32))
    g.close()
