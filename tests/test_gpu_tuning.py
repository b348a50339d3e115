"""Run-time tuning (pp_get_tuning / pp_set_tuning / pp_autotune /
pp_batch_autotune): the knobs (sort cadences, blocks per SM and the particle
kernel's tile shape, particles per thread) round-trip and are validated, a
different tuning leaves the physics unchanged (cells whose periods are deterministic up
to float-atomic order give the same records), and the tuner returns a valid
tuning, leaves the cell on it and the cell keeps running."""
import numpy as np
import pytest

from gpu_common import require_gpu, gpu_cell

pytestmark = pytest.mark.gpu


def _valid_cadences(n_rf, lo, hi):
    return [d for d in range(lo, hi + 1) if n_rf % d == 0 and (n_rf // d) % 2 == 0]


def test_tuning_roundtrip_and_validation():
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp, workloads
    cfg = workloads.small()
    g = gpu_cell(cfg, [workloads.population(cfg, sp) for sp in (0, 1)])
    t = g.tuning()
    assert t == {"sort_every": [cfg.sort_every_e, cfg.sort_every_i], "push_blocks_per_sm": 0,
                 "push_particles_per_thread": 8}
    g.set_tuning(sort_every=(4, 25), push_blocks_per_sm=1, push_particles_per_thread=16)
    want = {"sort_every": [4, 25], "push_blocks_per_sm": 1, "push_particles_per_thread": 16}
    assert g.tuning() == want
    with pytest.raises(pp.PhasorPICError):
        g.set_tuning(sort_every=(0, 25))
    with pytest.raises(pp.PhasorPICError):
        g.set_tuning(push_blocks_per_sm=-1)
    with pytest.raises(pp.PhasorPICError):
        g.set_tuning(push_particles_per_thread=5)
    assert g.tuning() == want
    g.advance_steps(3)
    with pytest.raises(pp.PhasorPICError):       # not on a period boundary
        g.autotune(1)
    g.close()


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_tuning_leaves_the_physics_unchanged():
    """An ions-only cell without gas (no random draws depend on order) run two
    periods under the default tuning and under another: same live counts, and
    phasors equal to float-atomic rounding."""
    require_gpu()
    from paper_2609_15043_b300 import workloads
    base = workloads.small()
    cfg = base.replace(nr=48, nz=72, seed=base.seed + 1, pressure_pa=0.0)
    pops = [{k: v[:0] for k, v in workloads.population(cfg, 0).items()}, workloads.population(cfg, 1)]
    recs = []
    for tuning in (None, dict(sort_every=(4, 10), push_blocks_per_sm=1), dict(push_particles_per_thread=4),
                   dict(push_particles_per_thread=16, push_blocks_per_sm=1)):
        g = gpu_cell(cfg, pops)
        if tuning:
            g.set_tuning(**tuning)
        g.advance_period(2)
        recs.append((g.turn_phasors(), g.counters()["live_i"]))
        assert g.status() == 0
        g.close()
    ra, la = recs[0]
    for rb, lb in recs[1:]:
        assert la == lb
        for k in ("icap", "qhat", "x_next", "vp"):
            assert _rel(rb[k], ra[k]) < 1e-5, k


def test_autotune_cell_and_batch():
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp, workloads
    cfg = workloads.small()
    g = gpu_cell(cfg, [workloads.population(cfg, sp) for sp in (0, 1)])
    t = g.autotune(trial_periods=1)
    n_rf = g.n_rf
    assert t["sort_every"][0] in _valid_cadences(n_rf, 2, 40) + [cfg.sort_every_e]
    assert t["sort_every"][1] in _valid_cadences(n_rf, 10, 200) + [cfg.sort_every_i]
    assert 0 <= t["push_blocks_per_sm"] <= 8 and t["ms_per_period"] > 0
    assert t["push_particles_per_thread"] in (4, 8, 16)
    keys = ("sort_every", "push_blocks_per_sm", "push_particles_per_thread")
    assert {k: t[k] for k in keys} == g.tuning()
    periods = g.step_index // n_rf
    assert g.step_index % n_rf == 0 and periods >= 2
    g.advance_period(1)
    r = g.turn_phasors()
    assert r["accepted"] and r["period"] == periods
    g.close()
    cfgs = [cfg, cfg.replace(nr=48, nz=72, seed=cfg.seed + 5)]
    batch = pp.Batch(cfgs)
    for c, cf in zip(batch.cells, cfgs):
        for sp in (0, 1):
            c.set_particles(sp, workloads.population(cf, sp))
    tb = batch.autotune(trial_periods=1)
    for c in batch.cells:
        assert c.tuning() == {k: tb[k] for k in keys}
    batch.advance_period(1)
    for c in batch.cells:
        assert c.turn_phasors()["accepted"]
    batch.close()
