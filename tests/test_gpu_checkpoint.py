"""pp_checkpoint / pp_restore: a restored cell carries the same step-to-step
state as the original, and the next steps agree.  Deposits use float
atomics, whose order varies between runs, so the comparison after a step is
bit-exact for everything a step computes per particle from the restored field
(cells, offsets, velocities, uids, collision counts) and close for the
period-end quantities that integrate the deposits."""
import numpy as np
import pytest

from gpu_common import require_gpu, gpu_cell, by_uid

pytestmark = pytest.mark.gpu


def _small():
    from paper_2609_15043_b300 import workloads
    cfg = workloads.small()
    return cfg, [workloads.population(cfg, sp) for sp in (0, 1)]


def _state(g):
    return [by_uid(g.get_particles(sp)) for sp in (0, 1)]


def test_checkpoint_round_trip_and_continuation():
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp
    cfg, pops = _small()
    a = gpu_cell(cfg, pops)
    n0 = a.n_rf - 1
    a.advance_steps(n0)
    img = a.checkpoint()
    b = pp.Cell(cfg)
    b.restore(img)
    assert b.step_index == n0
    assert b.checkpoint() == img, "the restored cell's image differs from the one loaded"
    for k in (pp.GRID_PHI, pp.GRID_EC):
        assert np.array_equal(a.grid(k), b.grid(k))
    ca0, cb0 = a.counters(), b.counters()
    assert ca0 == cb0
    # one more step crosses the RF-period end
    a.advance_steps(1)
    b.advance_steps(1)
    sa, sb = _state(a), _state(b)
    for sp in (0, 1):
        for k in ("cell", "uid", "dr", "dz", "vr", "vt", "vz"):
            assert np.array_equal(sa[sp][k], sb[sp][k]), (sp, k)
    assert a.counters() == b.counters()
    ra, rb = a.turn_phasors(), b.turn_phasors()
    assert ra["period"] == rb["period"] == 0 and ra["n_samples"] == rb["n_samples"] == a.n_rf
    for k in ("vp", "icap", "qhat", "x_next"):
        scale = max(np.max(np.abs(ra[k])), 1e-300)
        assert np.max(np.abs(np.asarray(ra[k]) - np.asarray(rb[k]))) <= 1e-5 * scale, k
    a.close()
    b.close()


def test_restore_rejects_foreign_and_truncated_images():
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp
    cfg, pops = _small()
    a = gpu_cell(cfg, pops)
    a.advance_steps(3)
    img = a.checkpoint()
    other = pp.Cell(cfg.replace(seed=cfg.seed + 1))
    with pytest.raises(pp.PhasorPICError):
        other.restore(img)
    same = pp.Cell(cfg)
    with pytest.raises(pp.PhasorPICError):
        same.restore(img[: len(img) // 2])
    with pytest.raises(pp.PhasorPICError):
        same.restore(b"\0" * 64)
    same.restore(img)
    assert same.checkpoint() == img
    for c in (a, other, same):
        c.close()
