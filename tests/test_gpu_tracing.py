"""Tracing: per-phase CUDA-event times (pp_set_profiling) and host-side NVTX
ranges (pp_set_nvtx) leave the physics untouched: a period traced both ways
gives the same record as the same cell's period untraced (ions only, no gas,
so the period is deterministic up to float-atomic rounding), and the phase
times cover every phase of every step."""
import numpy as np
import pytest

from gpu_common import require_gpu, gpu_cell

pytestmark = pytest.mark.gpu


def test_traced_period_matches_untraced():
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp, workloads
    cfg = workloads.small().replace(pressure_pa=0.0, implicit_es=1)
    pops = [{k: v[:0] for k, v in workloads.population(cfg, 0).items()}, workloads.population(cfg, 1)]
    recs = []
    for traced in (False, True):
        g = gpu_cell(cfg, pops)
        if traced:
            pp.set_nvtx(True)
            g.set_profiling(True, 2)
        g.advance_period(1)
        recs.append(g.turn_phasors())
        if traced:
            t = g.phase_times()
            assert t["push"][1] == g.n_rf and t["poisson"][1] >= g.n_rf and t["period_end"][1] == 1
            assert all(v[0] > 0 for k, v in t.items() if k != "sort")
            pp.set_nvtx(False)
        assert g.status() == 0
        g.close()
    a, b = recs
    for k in ("vp", "icap", "x_next"):
        assert np.max(np.abs(np.asarray(a[k]) - b[k])) <= 1e-5 * np.max(np.abs(np.asarray(a[k])))
