"""The multiharmonic circuit (Sec. 4 extension, pp_config.n_harmonics) on the
GPU against the oracle: per retained frequency m w the charge harmonics of
the waveform-reconstructed turn potentials, I_cap^(m) = i m w Q^(m), the
sourceless network at m w and its relaxation, the powers summed over the
harmonics, and the harmonic fields composed for the next period; then the
same with ions carrying current (V_p at every harmonic)."""
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


def _set_harmonics(oc, g, rng):
    """The same nonzero applied state at every retained harmonic on both sides
    (the fundamental's state scaled by 0.3 / m and rotated)."""
    for h in oc.harm:
        x = oc.x * (0.3 / h["m"]) * np.exp(1j * (0.7 + rng.uniform(-1, 1)))
        h["x"] = x.copy()
        oc._compose_h(h)
        g.set_harmonic_state(h["m"], x)
        assert np.array_equal(g.harmonic_state(h["m"]), x)


def _run(cfg, pops, periods, seed=3):
    rng = np.random.default_rng(seed)
    oc = oracle_cell(cfg, pops)
    g = gpu_cell(cfg, pops)
    _set_harmonics(oc, g, rng)
    oc.prime(np.float32)
    g.set_potential(oc.phi)
    recs = []
    for _ in range(periods):
        for _ in range(oc.n_rf):
            oc.step(np.float32)
        g.advance_steps(g.n_rf)
        recs.append((oc.records[-1], g.turn_phasors()))
    return oc, g, recs


def test_particle_free_harmonic_periods_against_oracle():
    """No particles, three retained harmonics with nonzero applied states:
    the Laplace charges of the summed turn-potential waveform give every
    harmonic's I_cap deterministically, the harmonic networks relax, and the
    records (per harmonic and summed powers) and next-period fields agree
    with the oracle to rounding over two periods."""
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp, workloads
    cfg = workloads.small().replace(n_harmonics=3)
    oc, g, recs = _run(cfg, _pops(cfg, False, False), 2)
    n = len(cfg.turn_r)
    for ro, rg in recs:
        assert rg["accepted"] and rg["n_samples"] == oc.n_rf
        assert _rel(rg["icap"], ro["icap"]) < 1e-8
        assert _rel(rg["x_next"], ro["x_next"]) < 1e-9
        assert len(rg["harmonics"]) == 2
        for hg, ho in zip(rg["harmonics"], ro["harmonics"]):
            assert hg["m"] == ho["m"]
            assert np.max(np.abs(ho["icap"])) > 0
            assert _rel(hg["icap"], ho["icap"]) < 1e-8
            assert _rel(hg["qhat"], ho["qhat"]) < 1e-8
            assert _rel(hg["x_applied"], ho["x_applied"]) < 1e-12
            assert _rel(hg["x_next"], ho["x_next"]) < 1e-9
            assert np.max(np.abs(hg["vp"])) == 0.0
            # the residuals of the relaxed state with the period's loads
            assert hg["r_kcl"] == pytest.approx(ho["r_kcl"], rel=1e-6, abs=1e-12)
            assert hg["r_kvl"] == pytest.approx(ho["r_kvl"], rel=1e-6, abs=1e-12)
        scale = 0.5 * np.max(np.abs(ro["x_applied"][1 + n:])) * np.max(np.abs(ro["icap"]))
        for k in ("p_cap", "p_cap_ph"):
            assert abs(rg[k] - ro[k]) <= 1e-9 * scale, k
        assert rg["p_port"] == pytest.approx(ro["p_port"], rel=1e-9)
        assert rg["p_cu"] == pytest.approx(ro["p_cu"], rel=1e-9)
    # the composed fields of the next period
    assert _rel(g.grid(pp.GRID_EC), oc.Ec) < 1e-8
    for h in oc.harm:
        assert _rel(g.harmonic_state(h["m"]), h["x"]) < 1e-9
    assert g.status() == 0
    g.close()


@pytest.mark.parametrize("implicit", [0, 1])
def test_ions_only_harmonic_period_against_oracle(implicit):
    """Ions only, no gas, two retained harmonics, in both electrostatic
    forms: the ions respond to the summed E_theta waveform, so every
    harmonic's current has a V_p; the period's loads, powers and relaxed
    states agree with the oracle at the tolerances of the one-harmonic
    ions-only period."""
    require_gpu()
    from paper_2609_15043_b300 import workloads
    cfg = workloads.small().replace(pressure_pa=0.0, n_harmonics=2, implicit_es=implicit)
    oc, g, recs = _run(cfg, _pops(cfg, False, True), 1)
    ro, rg = recs[0]
    assert rg["n_live"][1] == ro["n_live"][1]
    for k, tol in (("vp", 1e-3), ("icap", 1e-3), ("x_next", 1e-4)):
        assert _rel(rg[k], ro[k]) < tol, k
    hg, ho = rg["harmonics"][0], ro["harmonics"][0]
    assert np.max(np.abs(ho["vp"])) > 0
    for k, tol in (("vp", 1e-3), ("icap", 1e-3), ("x_next", 1e-4)):
        assert _rel(hg[k], ho[k]) < tol, ("m=2", k)
    for k, tol in (("p_ind", 1e-2), ("p_port", 1e-6)):
        assert abs(rg[k] - ro[k]) <= tol * abs(ro[k]), k
    assert g.status() == 0
    g.close()


def test_one_harmonic_record_has_no_harmonics():
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp, workloads
    cfg = workloads.small()
    g = gpu_cell(cfg, _pops(cfg, False, False))
    g.advance_period(1)
    assert g.turn_phasors()["harmonics"] == []
    with pytest.raises(pp.PhasorPICError):
        g.set_harmonic_state(2, np.zeros(2 * len(cfg.turn_r) + 1, complex))
    g.close()
