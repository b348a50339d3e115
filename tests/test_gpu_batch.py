"""Batches of independent cells (pp_init_batch / pp_batch_advance_period):
every cell of a batch evolves exactly as the same cell run alone.  The
comparison uses cells whose periods are deterministic up to float-atomic
rounding (particle-free, and ions-only without gas), on different grids, so
that a mix-up of per-cell state between the concurrent streams would show."""
import numpy as np
import pytest

from gpu_common import require_gpu, gpu_cell

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _cases():
    from paper_2609_15043_b300 import workloads
    base = workloads.small()
    empty = lambda c, sp: {k: v[:0] for k, v in workloads.population(c, sp).items()}
    cfgs = [base,
            base.replace(nr=48, nz=72, seed=base.seed + 1, pressure_pa=0.0),
            base.replace(pressure_pa=0.0, seed=base.seed + 2, turn_r=[0.03, 0.06], winding=[1, 1], v_g=200.0)]
    pops = [[empty(cfgs[0], 0), empty(cfgs[0], 1)],
            [empty(cfgs[1], 0), workloads.population(cfgs[1], 1)],
            [empty(cfgs[2], 0), workloads.population(cfgs[2], 1)]]
    return cfgs, pops


def _mixed_cases():
    """Cells whose forms differ within one batch: direct-implicit ions-only,
    explicit particle-free with a retained second harmonic, and
    direct-implicit ions-only with per-particle weights."""
    from paper_2609_15043_b300 import workloads
    base = workloads.small()
    empty = lambda c, sp: {k: v[:0] for k, v in workloads.population(c, sp).items()}
    cfgs = [base.replace(nr=48, nz=72, seed=base.seed + 1, pressure_pa=0.0, implicit_es=1),
            base.replace(n_harmonics=2),
            base.replace(pressure_pa=0.0, seed=base.seed + 3, implicit_es=1, particle_weights=1)]
    pops = [[empty(cfgs[0], 0), workloads.population(cfgs[0], 1)],
            [empty(cfgs[1], 0), empty(cfgs[1], 1)],
            [empty(cfgs[2], 0), workloads.population(cfgs[2], 1)]]
    w = np.random.default_rng(4).uniform(0.5, 2.0, len(pops[2][1]["uid"]))
    pops[2][1] = dict(pops[2][1], w=w)
    return cfgs, pops


@pytest.mark.parametrize("cases", ["plain", "mixed"])
def test_batch_matches_cells_run_alone(cases):
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp
    cfgs, pops = _cases() if cases == "plain" else _mixed_cases()
    batch = pp.Batch(cfgs)
    assert pp.lib.pp_batch_size(batch.h) == len(cfgs)
    for c, p in zip(batch.cells, pops):
        for sp in (0, 1):
            c.set_particles(sp, p[sp])
    batch.advance_period(2)
    alone = []
    for cfg, p in zip(cfgs, pops):
        g = gpu_cell(cfg, p)
        g.advance_period(2)
        alone.append(g)
    for i, (b, a) in enumerate(zip(batch.cells, alone)):
        rb, ra = b.turn_phasors(), a.turn_phasors()
        assert rb["period"] == ra["period"] == 1, i
        assert rb["n_samples"] == b.n_rf and rb["accepted"], i
        assert b.counters()["live_i"] == a.counters()["live_i"], i
        particle_free = all(len(x["uid"]) == 0 for x in pops[i])
        tol = 1e-9 if particle_free else 1e-5
        for k in ("icap", "qhat", "x_next"):
            assert _rel(rb[k], ra[k]) < tol, (i, k)
        if not particle_free:
            assert _rel(rb["vp"], ra["vp"]) < 1e-5, i
        assert len(rb["harmonics"]) == len(ra["harmonics"]), i
        for hb, ha in zip(rb["harmonics"], ra["harmonics"]):
            assert _rel(hb["x_next"], ha["x_next"]) < tol, i
        assert b.status() == 0
        a.close()
    # a batch cell is destroyed with its batch only
    assert pp.lib.pp_destroy(batch.cells[0].h) == -7
    assert not pp.lib.pp_batch_cell(batch.h, len(cfgs))
    batch.close()


def test_batch_rejects_cells_off_the_period_boundary():
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp
    cfgs, pops = _cases()
    batch = pp.Batch(cfgs[:2])
    for c, p in zip(batch.cells, pops):
        for sp in (0, 1):
            c.set_particles(sp, p[sp])
    batch.cells[1].advance_steps(3)
    with pytest.raises(pp.PhasorPICError):
        batch.advance_period(1)
    batch.close()


def test_batch_cells_against_oracle():
    """Each cell of a batch against the oracle over one period (the oracle
    runs each cell alone): the particle-free cell to rounding, the ions-only
    cells to the period tolerances of the single-cell parity tests."""
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp
    from gpu_common import oracle_cell
    cfgs, pops = _cases()
    batch = pp.Batch(cfgs)
    for c, p in zip(batch.cells, pops):
        for sp in (0, 1):
            c.set_particles(sp, p[sp])
    batch.advance_period(1)
    for i, (cfg, p, b) in enumerate(zip(cfgs, pops, batch.cells)):
        oc = oracle_cell(cfg, p)
        oc.prime(np.float32)
        for _ in range(oc.n_rf):
            oc.step(np.float32)
        ro, rb = oc.records[-1], b.turn_phasors()
        assert rb["n_samples"] == ro["n_samples"] == oc.n_rf, i
        assert rb["n_live"] == ro["n_live"], i
        tol = 1e-8 if i == 0 else 1e-3
        for k in ("icap", "qhat"):
            assert _rel(rb[k], ro[k]) < tol, (i, k, _rel(rb[k], ro[k]))
        assert _rel(rb["x_next"], ro["x_next"]) < (1e-9 if i == 0 else 1e-4), i
        if i > 0:
            assert _rel(rb["vp"], ro["vp"]) < 1e-3, i
        assert b.status() == 0
    batch.close()
