"""The batched ensemble at its full size: 32 independent cells of mixed grids
(64x96 to 192x288), 5e5 to 8e6 macroparticles per species (8.0e7 per species
in all), pressures 5-50 mTorr, 3-5 turn coils and 20-150 W targets, in the
direct-implicit form, set up as the benchmark sets it up (one pp_batch, every
cell's populations resident).  Sampled cells of the batch step against the
oracle on sampled particles; a whole batched period (per-cell streams and
period graphs, the benchmark's launch) is checked on every cell through
properties that hold at any size."""
import numpy as np
import pytest

from gpu_common import require_gpu, oracle_cell, by_uid, oracle_live

pytestmark = pytest.mark.gpu


def _full_batch():
    from paper_2609_15043_b300 import phasorpic as pp, workloads
    cfgs = [c.replace(implicit_es=1) for c in workloads.batch_cells()]
    pops = [[workloads.population(c, sp) for sp in (0, 1)] for c in cfgs]
    batch = pp.Batch(cfgs)
    for c, p in zip(batch.cells, pops):
        for sp in (0, 1):
            c.set_particles(sp, p[sp])
    return cfgs, pops, batch


def _sampled_cells(cfgs):
    """The smallest and the largest grid, the highest and the lowest
    pressure, the most macroparticles (distinct cells, in batch order)."""
    nr = [c.nr for c in cfgs]
    pr = [c.pressure_pa for c in cfgs]
    ni = [c.n_init for c in cfgs]
    return sorted({int(np.argmin(nr)), int(np.argmax(nr)), int(np.argmax(pr)), int(np.argmin(pr)),
                   int(np.argmax(ni))})


def test_batch32_cells_step_on_sampled_particles():
    """Five cells of the full batch, each advanced one step inside the batch
    (its own stream, tile shape and blocks per SM) from the oracle's
    potential of its full population; the oracle advances 2e4 sampled
    particles per species of the same cell in the same fields: cells and
    collisions bit-exact, float32 state within 2e-5; and each step's cluster
    solve against the oracle's direct solve of the same operator on the GPU's
    charges."""
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp
    cfgs, pops, batch = _full_batch()
    picks = _sampled_cells(cfgs)
    assert len(picks) >= 3
    rng = np.random.default_rng(32)
    for i in picks:
        oc = oracle_cell(cfgs[i], pops[i])
        oc.prime(np.float32)
        g = batch.cells[i]
        g.set_potential(oc.phi)
        g.advance_steps(1)
        sampled = []
        for sp in (0, 1):
            P = oc.P[sp]
            pick = np.sort(rng.choice(len(P["uid"]), min(20000, len(P["uid"])), replace=False))
            oc.P[sp] = {k: v[pick].copy() for k, v in P.items()}
            sampled.append(oc.P[sp]["uid"].astype(np.uint32))
        oc.step(np.float32)
        for sp in (0, 1):
            pg = by_uid(g.get_particles(sp))
            po = oracle_live(oc.P[sp])
            # the sample's own particles (pairs it creates are numbered
            # within the sample, the GPU's within the whole population)
            po = {k: v[np.isin(po["uid"].astype(np.uint32), sampled[sp])] for k, v in po.items()}
            gone = np.setdiff1d(sampled[sp], po["uid"].astype(np.uint32))
            assert not np.any(np.isin(gone, pg["uid"])), (i, sp)      # absorbed on both sides
            idx = np.searchsorted(pg["uid"], po["uid"].astype(np.uint32))
            assert np.all(idx < len(pg["uid"])), (i, sp)
            assert np.array_equal(pg["uid"][idx], po["uid"].astype(np.uint32)), (i, sp)
            assert np.array_equal(pg["cell"][idx], po["cell"].astype(np.uint32)), (i, sp)
            for k in ("dr", "dz"):
                assert np.max(np.abs(pg[k][idx] - po[k])) <= 2e-5, (i, sp, k)
            for k in ("vr", "vt", "vz"):
                ref = po[k]
                scale = np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)))
                assert np.max(np.abs(pg[k][idx] - ref) / scale) <= 2e-5, (i, sp, k)
        qe, qi = g.grid(pp.GRID_CHARGE_E), g.grid(pp.GRID_CHARGE_I)
        chi = oc.susceptibility([qe, qi], np.float32)
        ref = oc.solve_potential(qe + qi + g.grid(pp.GRID_WINDOW), oc.theta(1), chi)
        phi = g.grid(pp.GRID_PHI)
        assert np.max(np.abs(phi - ref)) <= 1e-8 * np.max(np.abs(ref)), i
        assert g.status() == 0, i
    batch.close()


def test_batch32_period_in_the_benchmark_launch():
    """One batched period of all 32 cells (pp_batch_advance_period): every
    cell's record is its first, accepted, with N_RF samples and finite
    powers; the live counters equal the stored populations and balance the
    initial ones against creations and absorptions; every particle lies in
    the plasma region with offsets in [0, 1) and a unique uid; no status bit
    is set."""
    require_gpu()
    cfgs, pops, batch = _full_batch()
    batch.advance_period(1)
    for i, (cfg, c) in enumerate(zip(cfgs, batch.cells)):
        rec = c.turn_phasors()
        assert rec["period"] == 0 and rec["accepted"] and rec["n_samples"] == c.n_rf, i
        for k in ("p_port", "p_ind", "p_cu"):
            assert np.isfinite(rec[k]), (i, k)
        assert rec["p_port"] > 0, i
        cnt = c.counters()
        assert cnt["steps"] == c.n_rf, i
        live = 0
        for sp, key in ((0, "live_e"), (1, "live_i")):
            p = c.get_particles(sp)
            n = len(p["uid"])
            assert cnt[key] == n, (i, sp)
            live += n
            assert len(np.unique(p["uid"])) == n, (i, sp)
            i_win = int(round(cfg.z_win_lo / (cfg.z_max / cfg.nz)))
            assert np.all(p["cell"] < i_win * cfg.nr), (i, sp)
            for k in ("dr", "dz"):
                assert np.all((p[k] >= 0) & (p[k] < 1)), (i, sp, k)
            for k in ("vr", "vt", "vz"):
                assert np.all(np.isfinite(p[k])), (i, sp, k)
        n0 = sum(len(pops[i][sp]["uid"]) for sp in (0, 1))
        assert live == n0 + 2 * cnt["created"] - cnt["absorbed"], i
        assert c.status() == 0, i
    batch.close()
