"""Oracle pins for the field and circuit parts of the method: the paper's
particle-free Tests 1-3 (Sec. 3.1-3.3, appendix) and closed forms."""
import math

import numpy as np
import pytest

from conftest import load_golden
from oracle import verification as v
from oracle import circuit, fields
from oracle.grid import Grid


def _golden(name):
    out = {}
    for row in load_golden(name):
        out.setdefault(row[0], []).append([float(x) for x in row[1:]])
    return out


G12 = _golden("test12_solenoids.txt")


@pytest.fixture(scope="module")
def two_sheets():
    Z, eps_rec, g, U = v.solenoid_impedance([0.01, 0.02])
    return Z, eps_rec


def test_test2_inductance_matrix(two_sheets):
    """Table S2results: L1, L2, M to the printed digits (single node-row
    sheets, Eq. zvac projection)."""
    Z, eps_rec = two_sheets
    L = Z.imag / v.OMEGA * 1e9
    assert L[0, 0] == pytest.approx(G12["t2_L1"][0][0], rel=2e-6)
    assert L[1, 1] == pytest.approx(G12["t2_L2"][0][0], rel=2e-6)
    assert L[0, 1] == pytest.approx(G12["t2_M"][0][0], rel=2e-6)
    k = L[0, 1] / math.sqrt(L[0, 0] * L[1, 1])
    assert k == pytest.approx(G12["t2_k"][0][0], abs=2e-6)
    assert eps_rec < 1e-10                       # Eq. reciprocity
    assert np.all(np.abs(Z.real) < 1e-14)        # purely reactive in vacuum


def test_test2_loops(two_sheets):
    """Eq. S2solution with the field-derived matrix reproduces the model
    column of Table S2results."""
    Z, _ = two_sheets
    I1, I2, U1, U2 = v.two_loop(1.0, 0.1, 0.1, 10e-9, Z)
    for key, val in (("t2_I1", I1), ("t2_I2", I2), ("t2_U1", U1), ("t2_U2", U2)):
        mag, ang = G12[key][0]
        assert abs(val) == pytest.approx(mag, rel=2e-5)
        assert math.degrees(np.angle(val)) == pytest.approx(ang, abs=2e-3)


def test_test1_base_case():
    """Table S1results: Im Z_vac, the series-circuit current and coil voltage,
    and the analytic references of Eq. sol_L."""
    Z, _, g, U = v.solenoid_impedance([0.01])
    z = Z[0, 0]
    assert z.imag == pytest.approx(G12["t1_imz_model"][0][0], rel=1e-4)
    I, UL = v.series_current(1.0, 0.1, z)
    mag, ang = G12["t1_I_model"][0]
    assert abs(I) == pytest.approx(mag, abs=2e-4)
    assert math.degrees(np.angle(I)) == pytest.approx(ang, abs=6e-3)
    mag, ang = G12["t1_UL_model"][0]
    assert abs(UL) == pytest.approx(mag, abs=1e-4)
    assert math.degrees(np.angle(UL)) == pytest.approx(ang, abs=6e-3)
    # the analytic references of Tests 1-2 (Eqs. sol_L, S2ind) use the exact
    # mu0 = 4 pi 1e-7: 0.394784 nH; the field code uses 1.2566e-6
    L_ana = 4e-7 * math.pi * math.pi * 0.01 ** 2 / 1.0
    assert L_ana * 1e9 == pytest.approx(G12["t1_L_ana"][0][0], rel=2e-6)
    I_ana, _ = v.series_current(1.0, 0.1, 1j * v.OMEGA * L_ana)
    assert abs(I_ana) == pytest.approx(G12["t1_I_ana"][0][0], abs=1e-4)
    # Eq. sol_field: the interior field of a long sheet approaches -w A_theta
    # = -w mu0 R / (2 L) per ampere-turn at mid-length, well inside the sheet
    i_mid = int(round(0.62 / 1e-3))
    R = g.R[3]
    assert U[0][i_mid, 3] / (1.2566e-6 * v.OMEGA) * (1.2566e-6 * v.OMEGA) == pytest.approx(
        -v.OMEGA * 1.2566e-6 * R / 2.0, rel=0.03)


@pytest.mark.parametrize("case", range(1, 7))
def test_test1_sensitivity_cases(case):
    """Table S1cases: every non-base row of the boundary/grid/length scans."""
    h, L, b, Lnum, eps = G12["t1_case"][case]
    if h == 0.5:
        pytest.skip("the h = 0.5 mm case is covered by the slow marker")
    Z, _, _, _ = v.solenoid_impedance([0.01], h=h * 1e-3, L=L, b=b)
    Lh = Z[0, 0].imag / v.OMEGA * 1e9
    assert Lh == pytest.approx(Lnum, rel=1e-4)
    L_ana = 4e-7 * math.pi * math.pi * 0.01 ** 2 / L * 1e9
    assert 100 * (Lh - L_ana) / L_ana == pytest.approx(eps, abs=0.011)


@pytest.mark.slow
def test_test1_fine_grid():
    h, L, b, Lnum, eps = G12["t1_case"][4]
    Z, _, _, _ = v.solenoid_impedance([0.01], h=h * 1e-3, L=L, b=b)
    assert Z[0, 0].imag / v.OMEGA * 1e9 == pytest.approx(Lnum, rel=1e-4)


# ---------------------------------------------------------------- Test 3
G3 = load_golden("test3_five_node.txt")
X_CALC = np.array([float(r[2]) + 1j * float(r[3]) for r in G3 if r[0] == "x"])
X_CONT = np.array([float(r[4]) + 1j * float(r[5]) for r in G3 if r[0] == "x"])
S3 = {r[1]: float(r[2]) for r in G3 if r[0] == "s"}


def test_test3_continuous_reference():
    """Eq. t7network with Eqs. t7C/t7M reproduces the continuous column of
    Table t7phasors; Eq. t7recurrence has rho = 0.359062."""
    x, _ = v.t3_network(v.t3_continuous_C(), v.t3_continuous_M())
    assert np.max(np.abs(x - X_CONT)) < 6e-9
    c, G = v.t3_recurrence(v.t3_continuous_C(), v.t3_continuous_M())
    assert max(abs(np.linalg.eigvals(G))) == pytest.approx(S3["rho_cont"], abs=1e-6)
    # closed-form fixed point of the recurrence equals the network solution
    xf = np.linalg.solve(np.eye(11) - G, c)
    assert np.max(np.abs(xf - x)) < 1e-10


@pytest.fixture(scope="module")
def five_node():
    return v.FiveNode(1e-3)


def test_test3_extracted_matrices(five_node):
    """C_h from five Laplace basis runs through the Gauss-law charge, M_h from
    the unit-field projection: relative Frobenius errors 1.21e-4 / 7.44e-5,
    reciprocity defect eta_M 6.27e-6 (Sec. 3.3)."""
    C, M = v.t3_continuous_C(), v.t3_continuous_M()
    ec = np.linalg.norm(five_node.Ch - C) / np.linalg.norm(C)
    em = np.linalg.norm(five_node.Mh - M) / np.linalg.norm(M)
    assert ec == pytest.approx(S3["Ch_err_h1"], rel=0.01)
    assert em == pytest.approx(S3["Mh_err_h1"], rel=0.01)
    eta_m = np.linalg.norm(five_node.Mh - five_node.Mh.T) / np.linalg.norm(five_node.Mh)
    assert eta_m == pytest.approx(S3["eta_M_h1"], rel=0.02)
    # zero conductor potentials give zero charge (appendix)
    assert np.max(np.abs(five_node.charges(np.zeros(5)))) == 0.0


def test_test3_semidiscrete_state(five_node):
    """x_{h,*} from C_h, M_h equals the field-circuit column of Table
    t7phasors; its distance to x_* is 1.90e-5 (Eq. t7error); rho(G_h) =
    0.359069."""
    xh, _ = v.t3_network(five_node.Ch, five_node.Mh)
    assert np.max(np.abs(xh - X_CALC)) < 6e-8
    assert v.t3_error(xh, X_CONT) == pytest.approx(S3["state_err_cont_h1"], rel=0.01)
    c, G = v.t3_recurrence(five_node.Ch, five_node.Mh)
    assert max(abs(np.linalg.eigvals(G))) == pytest.approx(S3["rho_h"], abs=1e-6)


def test_test3_coupled_run(five_node):
    """The sampled, period-delayed field-circuit loop (400 Laplace solves per
    period, I_cap = i w Q_hat, alpha = 1) reproduces the recurrence and its
    fixed point; KCL/KVL residuals vanish; power identities of Eq. t7power."""
    hist, last = five_node.coupled_run(periods=30)
    xh, _ = v.t3_network(five_node.Ch, five_node.Mh)
    c, G = v.t3_recurrence(five_node.Ch, five_node.Mh)
    xr = c.copy()
    for n in range(1, len(hist)):
        assert v.t3_error(hist[n - 1], xr) < 1e-10       # history = recurrence
        xr = c + G @ xr
    assert v.t3_error(hist[-1], xh) < 1e-10
    assert v.t3_error(hist[-1], X_CONT) == pytest.approx(S3["state_err_cont_h1"], rel=0.01)
    assert np.max(np.abs(hist[-1] - X_CALC)) < 6e-8
    rI, rV = last["residuals"]
    assert rI < 1e-13 and rV < 1e-13
    # reactive powers Q_L, Q_C of Eq. t7power at the fixed point
    x = hist[-1]
    I, V = x[1:6], x[6:]
    WM = np.conj(I) @ five_node.Mh @ I
    WC = np.conj(V) @ five_node.Ch @ V
    assert v.OMEGA / 2 * WM.real == pytest.approx(S3["QL_var"], rel=1e-5)
    assert -v.OMEGA / 2 * WC.real == pytest.approx(S3["QC_var"], rel=1e-5)
    Sg = 0.5 * v.T3_VG * np.conj(x[0])
    rhs = v.T3_RG * abs(x[0]) ** 2 / 2 + 20.0 * np.sum(np.abs(I) ** 2) / 2 \
        + 1j * v.OMEGA / 2 * (WM - np.conj(WC))
    assert abs(Sg - rhs) / abs(Sg) < 1e-10
    # normalised active-power defects on the final completed period
    ql, qc = v.OMEGA / 2 * WM.real, -v.OMEGA / 2 * WC.real
    assert abs(last["p_cap"]) / (abs(ql) + abs(qc)) < 1e-5
    assert abs(last["p_port"] - last["p_cu"]) / abs(last["p_port"]) < 1e-5


@pytest.mark.slow
def test_test3_second_order_convergence():
    """State error against x_*: 7.63e-5 at h = 2 mm, order about 2."""
    x = v.t3_network(v.t3_continuous_C(), v.t3_continuous_M())[0]
    errs = []
    for h in (2e-3, 1e-3, 0.5e-3):
        fn = v.FiveNode(h)
        errs.append(v.t3_error(v.t3_network(fn.Ch, fn.Mh)[0], x))
    assert errs[0] == pytest.approx(S3["state_err_cont_h2"], rel=0.01)
    for a, b in zip(errs, errs[1:]):
        assert 1.9 < math.log2(a / b) < 2.1


def test_rotation_covariance():
    """A 37-degree rotation of the source rotates the network solution by the
    same phasor factor (appendix consistency check)."""
    C, M = v.t3_continuous_C(), v.t3_continuous_M()
    x0, _ = v.t3_network(C, M)
    rot = np.exp(1j * math.radians(37.0))
    x1, _ = v.t3_network(C, M, vg=v.T3_VG * rot)
    assert np.max(np.abs(x1 - rot * x0)) / np.max(np.abs(x0)) < 1e-14


# ---------------------------------------------------------------- powers
def test_pcap_quadrature_identity():
    """Eq. pcap_quadrature: for a pure fundamental V and the same charge
    samples, P_cap = sinc(2 pi / N) P_cap^ph; a lossless capacitor gives 0
    active power; <V dQ/dt> = w V0 Q_s / 2 (Sec. 2.4)."""
    rng = np.random.default_rng(1)
    for n_rf in (7, 40, 400):
        th = 2 * np.pi * (np.arange(1, n_rf + 1) % n_rf) / n_rf
        Vh = rng.normal(size=3) + 1j * rng.normal(size=3)
        Qh = rng.normal(size=3) + 1j * rng.normal(size=3)
        V = Vh.real[None] * np.cos(th)[:, None] - Vh.imag[None] * np.sin(th)[:, None]
        Q = Qh.real[None] * np.cos(th)[:, None] - Qh.imag[None] * np.sin(th)[:, None]
        f = 13.56e6
        w = 2 * np.pi * f
        p_trap, _ = circuit.cap_power_trapezoid(V, Q, f)
        Qc = 2 / n_rf * np.sum(Q * np.cos(th)[:, None], axis=0)
        Qs = 2 / n_rf * np.sum(Q * np.sin(th)[:, None], axis=0)
        icap = 1j * w * (Qc - 1j * Qs)
        x = np.concatenate([[0], np.zeros(3), Vh])
        p_ph = circuit.cap_power_phasor(x, 3, icap)
        a = 2 * np.pi / n_rf
        assert p_trap == pytest.approx(math.sin(a) / a * p_ph, rel=1e-12, abs=1e-14)
        # lossless linear capacitor Q = C V: zero active power
        Cm = rng.normal(size=(3, 3))
        Cm = Cm + Cm.T
        p0, _ = circuit.cap_power_trapezoid(V, V @ Cm.T, f)
        assert abs(p0) < 1e-12 * np.max(np.abs(V)) ** 2 * f * np.max(np.abs(Cm))
    # <V dQ/dt> with V = V0 cos, Q = Qc cos + Qs sin  ->  w V0 Qs / 2
    V0, Qc_, Qs_ = 2.0, 0.3, -0.7
    assert 0.5 * (V0 * (w * Qs_)) == pytest.approx(w * V0 * Qs_ / 2)


def test_skin_resistance_limits():
    """Eq. skin: thick wire -> rho 2 pi R / (pi (R_w^2 - (R_w - d)^2)); thin wire
    (R_w < delta) -> the DC resistance rho 2 pi R / (pi R_w^2)."""
    w = 2 * np.pi * 13.56e6
    rho = 1.68e-8
    delta = math.sqrt(2 * rho / (w * 1.2566e-6))
    r = circuit.skin_resistance([0.05], 1e-3, w, rho, 3.93e-3, 20.0)[0]
    assert r == pytest.approx(rho * 2 * math.pi * 0.05 / (math.pi * (1e-6 - (1e-3 - delta) ** 2)))
    r_thin = circuit.skin_resistance([0.05], 0.5 * delta, w, rho, 3.93e-3, 20.0)[0]
    assert r_thin == pytest.approx(rho * 2 * 0.05 / (0.5 * delta) ** 2)
    r_hot = circuit.skin_resistance([0.05], 1e-3, w, rho, 3.93e-3, 120.0)[0]
    assert r_hot > r


def test_controller_steps():
    """Eqs. pfilter-pcontrol: at target power the amplitude holds; far below it
    the limiter allows at most +f_step per cycle; bounds apply."""
    c = circuit.PowerController(60.0, 0.2, 5.0, 1e-3, 0.5, 0.05, 1.0, 1e4)
    assert c.update(100.0, 60.0) == pytest.approx(100.0)
    c = circuit.PowerController(60.0, 0.2, 5.0, 1e-3, 0.5, 0.05, 1.0, 1e4)
    assert c.update(100.0, 1.0) == pytest.approx(105.0)
    c = circuit.PowerController(60.0, 0.2, 5.0, 1e-3, 0.5, 0.05, 1.0, 102.0)
    assert c.update(100.0, 1.0) == pytest.approx(102.0)
    c = circuit.PowerController(60.0, 1.0, 0.0, 1e-3, 1.0, 10.0, 1.0, 1e4)
    assert c.update(100.0, 15.0) == pytest.approx(200.0)       # sqrt(60/15) = 2


def test_gauss_law_global():
    """Discrete Gauss law: with a random interior charge and random turn
    potentials, the charge on the Dirichlet nodes (turns and grounded metal)
    computed face by face equals minus the free charge plus the induced
    charge balance: sum over all Dirichlet nodes of the face flux equals
    -(total interior charge)."""
    rng = np.random.default_rng(3)
    g = Grid(10, 8, 1e-3, 1e-3, np.where(np.arange(10)[:, None] >= 6, 3.8, 1.0) * np.ones((10, 8)))
    dirm = np.zeros((g.NZ, g.NR), bool)
    dirm[0, :] = dirm[-1, :] = True
    dirm[:, -1] = True
    turn = [[(8, 3), (8, 4)], [(8, 6)]]
    for nodes in turn:
        for n in nodes:
            dirm[n] = True
    ps = fields.PoissonSolver(g, dirm)
    Q = np.where(dirm, 0.0, rng.normal(size=(g.NZ, g.NR)) * 1e-12)
    vals = np.zeros((g.NZ, g.NR))
    vals[8, 3] = vals[8, 4] = 5.0
    vals[8, 6] = -3.0
    phi = ps.solve(Q, vals)
    metal = [[(i, j)] for i in range(g.NZ) for j in range(g.NR) if dirm[i, j] and
             not any((i, j) in t for t in turn)]
    qt = fields.turn_charge(g, phi, turn + metal)
    assert np.sum(qt) == pytest.approx(-np.sum(Q), rel=1e-9)
