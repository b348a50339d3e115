"""Pins of the oracle's multiharmonic extension (Sec. 4: the network solved at
each retained frequency m w with the field responses and impedances of that
frequency, Q and J harmonics as the feedback, I_cap^(m) = i m w Q^(m), and the
waveforms reconstructed from all harmonics).  Each test names the closed form
or invariant it checks."""
import math

import numpy as np
import pytest

from oracle import circuit
from oracle.cell import OracleCell
from paper_2609_15043_b300 import workloads


def _empty_cell(cfg):
    oc = OracleCell(cfg, [1.0, 1.0])
    e = np.zeros(0)
    for sp in (0, 1):
        oc.set_particles(sp, e.astype(np.int64), e, e, e, e, e, e.astype(np.int64))
    return oc


def test_one_harmonic_is_the_fundamental_code():
    """n_harmonics = 1 keeps no harmonic state and the record has none."""
    oc = _empty_cell(workloads.small())
    assert oc.harm == [] and oc.M == 1


def test_particle_free_cell_keeps_its_harmonics_at_zero():
    """Without particles the turn charges are linear in the turn potentials,
    which start purely fundamental: the discrete Fourier sums of Eq. fourier
    are orthogonal across harmonics (m != 1), so every harmonic load, and
    with it every harmonic state, stays zero to rounding, and the fundamental
    records equal those of the one-harmonic run."""
    cfg = workloads.small().replace(full_helmholtz=1)
    a = _empty_cell(cfg)
    b = _empty_cell(cfg.replace(n_harmonics=3))
    for oc in (a, b):
        oc.prime(np.float64)
        for _ in range(2 * oc.n_rf):
            oc.step(np.float64)
    for ra, rb in zip(a.records, b.records):
        sx = np.max(np.abs(ra["x_next"]))
        assert np.max(np.abs(rb["x_next"] - ra["x_next"])) <= 1e-12 * sx
        assert rb["p_port"] == pytest.approx(ra["p_port"], rel=1e-12)
        for hr in rb["harmonics"]:
            assert np.max(np.abs(hr["x_next"])) <= 1e-12 * sx
            assert np.max(np.abs(hr["qhat"])) <= 1e-12 * np.max(np.abs(ra["qhat"]))


def test_zvac_scales_with_the_harmonic_in_mqs():
    """Without the w^2/c^2 term K U = mu0 w g gives U^(m) = m U and so
    Z_vac(m w) = m Z_vac(w) (Eq. zvac)."""
    oc = _empty_cell(workloads.small().replace(full_helmholtz=0, n_harmonics=3))
    for h in oc.harm:
        assert np.max(np.abs(h["zvac"] - h["m"] * oc.zvac)) <= 1e-12 * np.max(np.abs(h["m"] * oc.zvac))
        # skin resistance grows as sqrt(m) while the skin depth is below the wire radius
        rr = circuit.skin_resistance(oc.cfg.turn_r, oc.cfg.wire_radius, h["omega"], oc.cfg.rho20,
                                     oc.cfg.alpha_cu, oc.cfg.t_coil_c)
        assert np.allclose(h["r_rf"], rr)


def _coil_current_drive(oc, Ihat, m):
    """A prescribed current shaped like the coil's own pattern, sum_l I_l g_l,
    oscillating at m w (peak phasors I_l, exp(+i m w t))."""
    pattern = np.tensordot(Ihat, oc.geo.gk, axes=1)
    vol = np.where(oc.geo.vol > 0, oc.geo.vol, 0.0)
    oc.geo.vol = np.where(vol > 0, vol, 1.0)       # unit volume on the coil rows (test-only)

    def drive(th, Et):
        return (pattern * complex(math.cos(m * th), math.sin(m * th))).real * oc.geo.vol
    return drive


def test_harmonic_vp_and_network_of_a_coil_shaped_current():
    """A 2 w current J = sum_l I_l g_l: Eq. fourier at m = 2 recovers I_l
    exactly, the Helmholtz solves at 2 w and Eq. vpind give V_p^(2) =
    Z_vac(2 w) I (no fundamental or third-harmonic load); the network at 2 w
    has no source, so its Thevenin row gives V_1 = -Z_s(2 w) I_f and the port
    power -1/2 Re Z_s(2 w) |I_f|^2; its KCL/KVL residuals vanish."""
    cfg = workloads.small().replace(full_helmholtz=1, n_harmonics=3, alpha=1.0)
    oc = _empty_cell(cfg)
    oc.prime(np.float64)
    Ihat = np.array([1.0 - 0.5j, -0.3 + 2.0j, 0.7 + 0.1j])
    drive = _coil_current_drive(oc, Ihat, 2)
    for _ in range(oc.n_rf):
        oc.step(np.float64, drive=drive)
    rec = oc.records[-1]
    h2, h3 = oc.harm
    vp2 = rec["harmonics"][0]["vp"]
    ref = h2["zvac"] @ Ihat
    assert np.max(np.abs(vp2 - ref)) <= 1e-9 * np.max(np.abs(ref))
    assert np.max(np.abs(rec["vp"])) <= 1e-9 * np.max(np.abs(ref))
    assert np.max(np.abs(rec["harmonics"][1]["vp"])) <= 1e-9 * np.max(np.abs(ref))
    x2 = h2["x"]
    N = oc.N
    assert np.max(np.abs(x2)) > 0
    assert x2[1 + N] == pytest.approx(-h2["zs"] * x2[0], rel=1e-10)
    assert circuit.port_power(x2, N) == pytest.approx(-0.5 * h2["zs"].real * abs(x2[0]) ** 2, rel=1e-10)
    hr = rec["harmonics"][0]
    assert hr["r_kcl"] < 1e-12 and hr["r_kvl"] < 1e-12


@pytest.mark.slow
def test_power_balance_of_a_coupled_run_with_a_cubic_load():
    """Eq. pbalance with a nonlinear load J = sigma E (E / E0)^2 (odd in E, so
    it generates the third harmonic and no even one): at the fixed point of the
    coupled loop with three retained harmonics the port power, summed over the
    harmonics (the source's power at w less what the third-harmonic currents
    return to the source resistance), equals the time-domain inductive power
    sum(J E) plus the copper power of every harmonic.  The third harmonic
    carries current, the second stays zero."""
    cfg = workloads.small().replace(alpha=1.0, full_helmholtz=1, n_harmonics=3)
    oc = _empty_cell(cfg)
    oc.prime(np.float64)
    g, iw = oc.g, oc.geo.i_win
    mask = np.zeros((g.NZ, g.NR), bool)
    mask[iw // 3: iw - 2, 2: int(0.8 * cfg.nr)] = True
    vol = 2 * math.pi * g.R[None, :] * g.dr * g.dz * np.ones((g.NZ, 1))
    E0 = 30.0

    def drive(th, Et):
        return np.where(mask, 2.0 * Et * (Et / E0) ** 2 * vol, 0.0)

    for _ in range(16 * oc.n_rf):
        oc.step(np.float64, drive=drive)
    rec = oc.records[-1]
    s = np.max(np.abs(rec["x_applied"]))
    drift = np.max(np.abs(rec["x_next"] - rec["x_applied"])) / s
    assert drift < 1e-6
    h2, h3 = rec["harmonics"]
    assert np.max(np.abs(h3["x_applied"][1:1 + oc.N])) > 1e-4 * np.max(np.abs(rec["x_applied"][1:1 + oc.N]))
    assert np.max(np.abs(h2["x_applied"])) <= 1e-9 * s
    assert rec["p_ind"] > 0.05 * rec["p_port"]
    bal = abs(rec["p_port"] - (rec["p_ind"] + rec["p_cap"] + rec["p_cu"])) / rec["p_port"]
    assert bal < 1e-5, bal
