"""Edge cases of the step on the GPU: more ionisations in one step than the
event buffer holds (they are dropped and reported, the bookkeeping stays
consistent), and global charge conservation of the deposit at the benchmark
size."""
import numpy as np
import pytest

from gpu_common import require_gpu, gpu_cell

pytestmark = pytest.mark.gpu

EVENT_CAP = 8192        # ionisation events a step can record


def test_event_overflow_is_reported_not_fatal():
    """1e5 electrons at 60 eV in 3 Torr of argon: nearly every electron is a
    collision candidate and a sizeable share ionises, well over the event
    buffer.  The step appends exactly the buffered pairs, sets PP_ST_EVENTS,
    and the live counts, uids and counters agree with each other."""
    require_gpu()
    from paper_2609_15043_b300 import workloads
    cfg = workloads.small().replace(n_init=100000, te_ev=60.0, pressure_pa=3.0 * 133.322368)
    pops = [workloads.population(cfg, sp) for sp in (0, 1)]
    g = gpu_cell(cfg, pops)
    g.advance_steps(1)
    c = g.counters()
    assert c["e_ionisation"] > EVENT_CAP
    assert c["created"] == EVENT_CAP
    assert g.status() & 2
    e, i = g.get_particles(0), g.get_particles(1)
    assert len(e["uid"]) == c["live_e"] and len(i["uid"]) == c["live_i"]
    assert len(np.unique(e["uid"])) == len(e["uid"]) and len(np.unique(i["uid"])) == len(i["uid"])
    assert np.sum(e["uid"] >= cfg.n_init) == EVENT_CAP and np.sum(i["uid"] >= cfg.n_init) == EVENT_CAP
    assert c["live_e"] + c["live_i"] == 2 * cfg.n_init - c["absorbed"] + 2 * EVENT_CAP
    g.close()


def test_deposit_conserves_charge_at_bench_size():
    """Sum of the deposited node charge after a step equals q w (N_i - N_e)
    of the live particles (float32 atomics: within 1e-5 of the ion charge)."""
    require_gpu()
    from paper_2609_15043_b300 import workloads, phasorpic as pp
    cfg = workloads.cell60()
    g = gpu_cell(cfg, [workloads.population(cfg, sp) for sp in (0, 1)])
    g.advance_steps(3)
    c = g.counters()
    w = workloads.macro_weight(cfg)
    qe = 1.602176634e-19
    total = qe * w * (c["live_i"] - c["live_e"])
    q = g.grid(pp.GRID_CHARGE)
    assert abs(q.sum() - total) <= 1e-5 * qe * w * c["live_i"]
    g.close()


def test_event_buffer_scales_with_the_population():
    """The step's event buffer holds 1/64 of the electron capacity (at least
    8192): with room for 4e6 electrons, a burst of well over 8192 ionisations
    in one step is appended in full, in parent-uid order, exactly as the
    oracle appends it (new pairs, uids, cells and offsets bit-exact)."""
    require_gpu()
    from paper_2609_15043_b300 import workloads
    from gpu_common import oracle_cell, oracle_live, by_uid
    cfg = workloads.small().replace(n_init=100000, te_ev=60.0, pressure_pa=3.0 * 133.322368,
                                    capacity_factor=40.0)
    pops = [workloads.population(cfg, sp) for sp in (0, 1)]
    oc = oracle_cell(cfg, pops)
    oc.prime(np.float32)
    g = gpu_cell(cfg, pops)
    g.set_potential(oc.phi)
    g.advance_steps(1)
    info = oc.step(np.float32)
    c = g.counters()
    assert c["e_ionisation"] > EVENT_CAP
    assert c["created"] == c["e_ionisation"] == info["events"]
    assert g.status() == 0
    for sp in (0, 1):
        pg = by_uid(g.get_particles(sp))
        po = oracle_live(oc.P[sp])
        assert np.array_equal(pg["uid"], po["uid"].astype(np.uint32))
        assert np.array_equal(pg["cell"], po["cell"].astype(np.uint32))
        new = pg["uid"] >= cfg.n_init
        assert np.sum(new) == info["events"]
        for k in ("dr", "dz"):
            assert np.array_equal(pg[k][new], po[k][new])
    g.close()
