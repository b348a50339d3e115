"""Whole RF periods on the GPU (Sec. 2.5 workflow: per-step sampling, two
plasma-only Helmholtz solves, V_p, I_cap, powers, controller, network,
relaxation, composed field).  Periods of the violent 2e4-particle cell are
chaotic and noise-dominated (two runs of the same code differ by tens of
percent in I_cap), so period-level parity uses deterministic periods: a
particle-free cell (pure field-circuit closure, like the paper's Test 3) and
an ions-only cell without collisions (smooth dynamics for 400 steps)."""
import numpy as np
import pytest

from gpu_common import require_gpu, oracle_cell, gpu_cell

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _pops(cfg, electrons=True, ions=True):
    from paper_2609_15043_b300 import workloads
    out = []
    for sp, keep in ((0, electrons), (1, ions)):
        p = workloads.population(cfg, sp)
        out.append(p if keep else {k: v[:0] for k, v in p.items()})
    return out


def _period_pair(cfg, pops):
    oc = oracle_cell(cfg, pops)
    oc.prime(np.float32)
    g = gpu_cell(cfg, pops)
    g.set_potential(oc.phi)
    for _ in range(oc.n_rf):
        oc.step(np.float32)
    g.advance_steps(g.n_rf)
    return oc, g, oc.records[-1], g.turn_phasors()


def test_particle_free_period_against_oracle():
    """No particles: the period samples the Laplace charges of the applied
    turn potentials, so I_cap = i w C_h V and P_cap follow deterministically;
    V_p = 0; the network update and relaxation must agree to rounding."""
    require_gpu()
    from paper_2609_15043_b300 import workloads
    cfg = workloads.small()
    oc, g, ro, rg = _period_pair(cfg, _pops(cfg, False, False))
    assert rg["n_samples"] == ro["n_samples"] == oc.n_rf and rg["accepted"]
    assert np.max(np.abs(rg["vp"])) == 0.0
    assert _rel(rg["icap"], ro["icap"]) < 1e-8
    assert _rel(rg["qhat"], ro["qhat"]) < 1e-8
    # a lossless capacitor: both powers vanish; compare on the reactive scale
    n = len(cfg.turn_r)
    q_scale = 0.5 * np.max(np.abs(ro["x_applied"][1 + n:])) * np.max(np.abs(ro["icap"]))
    assert abs(rg["p_cap"] - ro["p_cap"]) <= 1e-9 * q_scale
    assert abs(rg["p_cap_ph"] - ro["p_cap_ph"]) <= 1e-9 * q_scale
    assert abs(ro["p_cap"]) <= 1e-9 * q_scale
    assert _rel(rg["x_next"], ro["x_next"]) < 1e-9
    assert rg["r_kcl"] == pytest.approx(ro["r_kcl"], rel=1e-6, abs=1e-12)
    # the composed field of the next period (Eq. compose)
    from paper_2609_15043_b300 import phasorpic as pp
    assert _rel(g.grid(pp.GRID_EC), oc.Ec) < 1e-8
    g.close()


def test_ions_only_period_against_oracle():
    """Ions only, no gas: the period's current harmonics, back-emf, charge
    harmonics and powers against the oracle (deterministic dynamics; FP32
    particle arithmetic against the float32 oracle instantiation)."""
    require_gpu()
    from paper_2609_15043_b300 import workloads
    cfg = workloads.small().replace(pressure_pa=0.0)
    oc, g, ro, rg = _period_pair(cfg, _pops(cfg, False, True))
    report = {k: _rel(rg[k], ro[k]) for k in ("vp", "icap", "x_next")}
    for k in ("p_ind", "p_cap", "p_es"):
        report[k] = abs(rg[k] - ro[k]) / max(abs(ro[k]), 1e-300)
    print(report)
    assert rg["n_samples"] == oc.n_rf
    assert rg["n_live"][1] == ro["n_live"][1]
    for k, tol in (("vp", 1e-3), ("icap", 1e-3), ("x_next", 1e-4), ("p_ind", 1e-2), ("p_cap", 1e-3)):
        assert report[k] < tol, (k, report[k])
    g.close()


def test_graph_period_equals_step_loop():
    """The captured period graph replays the step loop: on the deterministic
    ions-only cell the two paths agree to float-atomic rounding, and the
    graph keeps running over a second period."""
    require_gpu()
    from paper_2609_15043_b300 import workloads
    cfg = workloads.small().replace(pressure_pa=0.0)
    pops = _pops(cfg, False, True)
    a = gpu_cell(cfg, pops)
    b = gpu_cell(cfg, pops)
    a.advance_period(1)
    b.advance_steps(b.n_rf)
    ra, rb = a.turn_phasors(), b.turn_phasors()
    for k in ("vp", "icap", "x_next"):
        assert _rel(ra[k], rb[k]) < 1e-5, k
    assert a.counters()["live_i"] == b.counters()["live_i"]
    a.set_profiling(True)
    a.advance_period(1)
    t = a.phase_times()
    assert t["push"][1] == a.n_rf and t["push"][0] > 0
    assert a.turn_phasors()["period"] == 1 and a.counters()["steps"] == 2 * a.n_rf
    a.close()
    b.close()


def _periods_pair(cfg, pops, n_periods):
    oc = oracle_cell(cfg, pops)
    oc.prime(np.float32)
    g = gpu_cell(cfg, pops)
    g.set_potential(oc.phi)
    recs = []
    for _ in range(n_periods):
        for _ in range(oc.n_rf):
            oc.step(np.float32)
        g.advance_steps(g.n_rf)
        recs.append((oc.records[-1], g.turn_phasors()))
    return oc, g, recs


def test_controller_particle_free_periods_against_oracle():
    """The port-power controller (Eqs. pfilter, ptrend, pcontrol with the
    symmetric limiter) on the device against the oracle's PowerController over
    four particle-free periods: the filtered power carries state from period
    to period, so every period's V_g and relaxed state must agree."""
    require_gpu()
    from paper_2609_15043_b300 import workloads
    cfg = workloads.small().replace(power_control=1, p_target=3.0)
    oc, g, recs = _periods_pair(cfg, _pops(cfg, False, False), 4)
    moved = 0
    for ro, rg in recs:
        assert rg["accepted"] and rg["n_samples"] == oc.n_rf
        assert rg["vg"] == pytest.approx(ro["vg"], rel=1e-12)
        assert rg["p_port"] == pytest.approx(ro["p_port"], rel=1e-9)
        assert rg["vg_next"] == pytest.approx(ro["vg_next"], rel=1e-12)
        assert _rel(rg["x_next"], ro["x_next"]) < 1e-9
        moved += rg["vg_next"] != rg["vg"]
    assert moved == len(recs)                  # the controller acted every period
    assert g.status() == 0
    g.close()


def test_controller_ions_only_periods_against_oracle():
    """The controller with a kinetic load (ions only, no gas) over two
    periods: the first period's V_g update sees the same applied state on
    both sides, the second one the relaxed states of the first."""
    require_gpu()
    from paper_2609_15043_b300 import workloads
    cfg = workloads.small().replace(pressure_pa=0.0, power_control=1, p_target=3.0)
    oc, g, recs = _periods_pair(cfg, _pops(cfg, False, True), 2)
    (ro1, rg1), (ro2, rg2) = recs
    assert rg1["vg_next"] == pytest.approx(ro1["vg_next"], rel=1e-9)
    assert rg2["vg"] == pytest.approx(ro2["vg"], rel=1e-9)
    assert rg2["vg_next"] == pytest.approx(ro2["vg_next"], rel=1e-4)
    for ro, rg in recs:
        assert _rel(rg["x_next"], ro["x_next"]) < 1e-4
        assert rg["p_port"] == pytest.approx(ro["p_port"], rel=1e-4)
    assert g.status() == 0
    g.close()
