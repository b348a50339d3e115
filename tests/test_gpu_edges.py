"""Edge cases of the particle step against the oracle, in both
electrostatic forms: particles exactly on cell edges (offsets 0), on the axis
moving inward (through r = 0), a float32 step below the next cell edge, next
to every boundary, at rest, and fast enough to cross a cell in one step; and
the largest radial grid the kernels take (512 cells) with a ragged last
chunk.  Cells, uids, absorptions and collision counts bit-exact, float32
state within 2e-5, deposits within 1e-6 of their totals."""
import numpy as np
import pytest

from gpu_common import require_gpu, oracle_cell, gpu_cell, by_uid, oracle_live

pytestmark = pytest.mark.gpu


def _edge_population(cfg, sp, n, seed):
    rng = np.random.default_rng(seed)
    nr = cfg.nr
    i_win = int(round(cfg.z_win_lo / (cfg.z_max / cfg.nz)))
    kind = np.arange(n) % 6
    ir = rng.integers(0, nr, n)
    iz = rng.integers(0, i_win, n)
    dr = rng.random(n).astype(np.float32)
    dz = rng.random(n).astype(np.float32)
    vth = 2e6 if sp == 0 else 3e3
    v = (rng.standard_normal((3, n)) * vth).astype(np.float32)
    below_one = np.float32(np.nextafter(np.float32(1.0), np.float32(0.0)))
    m = kind == 0                                  # on the cell edges
    dr[m], dz[m] = 0.0, 0.0
    m = kind == 1                                  # on the axis, moving inward
    ir[m], dr[m] = 0, 0.0
    v[0][m] = -np.abs(v[0][m]) * 4
    m = kind == 2                                  # one float32 step below the next edge
    dr[m], dz[m] = below_one, below_one
    m = kind == 3                                  # next to the wall / the window / the electrode
    ir[m[:]] = np.where(rng.random(n) < 0.5, nr - 1, ir)[m]
    iz[m] = np.where(rng.random(m.sum()) < 0.5, i_win - 1, 0)
    m = kind == 4                                  # at rest
    v[:, m] = 0.0
    m = kind == 5                                  # fast: about a cell per step
    v[:, m] *= 8 if sp == 0 else 400
    return dict(cell=(iz * nr + ir).astype(np.uint32), dr=dr, dz=dz, vr=v[0], vt=v[1], vz=v[2],
                uid=(rng.permutation(n) + 7).astype(np.uint32))


def _compare(oc, g, info):
    from paper_2609_15043_b300 import phasorpic as pp
    cnt = g.counters()
    assert cnt["absorbed"] == info["stats"]["absorbed"]
    assert cnt["created"] == info["events"]
    assert [cnt["e_elastic"], cnt["e_excitation"], cnt["e_ionisation"]] == list(info["stats"]["coll"][0])
    for sp in (0, 1):
        pg = by_uid(g.get_particles(sp))
        po = oracle_live(oc.P[sp])
        assert np.array_equal(pg["uid"], po["uid"].astype(np.uint32))
        assert np.array_equal(pg["cell"], po["cell"].astype(np.uint32))
        for k in ("dr", "dz"):
            assert np.max(np.abs(pg[k] - po[k]), initial=0.0) <= 2e-5
        for k in ("vr", "vt", "vz"):
            scale = np.maximum(np.abs(po[k]), 1e-3 * max(np.max(np.abs(po[k]), initial=0.0), 1e-30))
            assert np.max(np.abs(pg[k] - po[k]) / scale, initial=0.0) <= 2e-5
    q = g.grid(pp.GRID_CHARGE)
    assert np.max(np.abs(q - info["Q"])) <= 1e-6 * np.sum(np.abs(info["Q"]))
    j = g.grid(pp.GRID_JMOM)
    assert np.max(np.abs(j - info["J"])) <= 1e-6 * max(np.sum(np.abs(info["J"])), 1e-30)


@pytest.mark.parametrize("implicit", [0, 1])
def test_edge_population_step(implicit):
    require_gpu()
    from paper_2609_15043_b300 import workloads
    cfg = workloads.small().replace(implicit_es=implicit)
    pops = [_edge_population(cfg, sp, 24000, 40 + sp) for sp in (0, 1)]
    oc = oracle_cell(cfg, pops)
    oc.prime(np.float32)
    g = gpu_cell(cfg, pops)
    g.set_potential(oc.phi)
    info = oc.step(np.float32)
    g.advance_steps(1)
    assert info["stats"]["absorbed"] > 0
    _compare(oc, g, info)
    assert g.status() == 0
    g.close()


def test_largest_radial_grid_step():
    """512 x 768 cells (513 radial nodes, the deposit tile's limit) in the
    explicit form, 1.5e5 particles per species (a ragged last chunk): one
    step from the oracle's potential, the refinement reaching its 1e-10
    target within four sweeps, and the step's separable solve against the
    oracle's direct solve."""
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp, workloads
    cfg = workloads.small().replace(nr=512, nz=768, n_init=150001, implicit_es=0, wire_radius=0.3e-3)
    pops = [workloads.population(cfg, sp) for sp in (0, 1)]
    oc = oracle_cell(cfg, pops)
    oc.prime(np.float32)
    # two refinement sweeps (the default, enough on the bench grids) leave this
    # grid above the 1e-10 target and the cell reports PP_ST_NOCONV; four reach it
    g = gpu_cell(cfg, pops, poisson_max_iter=4)
    g.set_potential(oc.phi)
    info = oc.step(np.float32)
    g.advance_steps(1)
    _compare(oc, g, info)
    rel = g.poisson_stats()
    assert rel[rel > 0][-1] <= 1e-10
    q = g.grid(pp.GRID_CHARGE_E) + g.grid(pp.GRID_CHARGE_I) + g.grid(pp.GRID_WINDOW)
    ref = oc.solve_potential(q, oc.theta(1), None)
    phi = g.grid(pp.GRID_PHI)
    assert np.max(np.abs(phi - ref)) <= 1e-8 * np.max(np.abs(ref))
    assert g.status() == 0
    g.close()
