"""The paper's particle-free verification problems on the GPU
(pp_vacuum_impedance: the unit problems of Eq. unitfield solved by the
device's FP64 separable Helmholtz solver, then the projection of Eq. zvac):
Tests 1 and 2 (Sec. 3.1-3.2, Tables S1results, S1cases, S2results) on the
paper's 1241 x 121 node grid and its sensitivity grids, and Test 3 (Sec. 3.3):
M_h with the manufactured axial boundaries, C_h from the Laplace solves with
the sheets as conductors (pp_vacuum_capacitance), and the semidiscrete
network state they give.
Each result is checked against the printed numbers and against the oracle's
sparse direct solve of the same problem."""
import math

import numpy as np
import pytest

from conftest import load_golden
from gpu_common import require_gpu

pytestmark = pytest.mark.gpu

F_RF = 13.56e6
OMEGA = 2 * math.pi * F_RF


def _golden(name):
    out = {}
    for row in load_golden(name):
        out.setdefault(row[0], []).append([float(x) for x in row[1:]])
    return out


G12 = _golden("test12_solenoids.txt")
G3 = load_golden("test3_five_node.txt")
S3 = {r[1]: float(r[2]) for r in G3 if r[0] == "s"}


def _solenoids(radii, h=1e-3, L=1.0, b=0.12):
    """Sheets of length L at the given radii on 0 <= z <= L + 2b, 0 <= R <= b
    (node rows b/h + 1 .. b/h + L/h)."""
    from paper_2609_15043_b300 import phasorpic as pp
    nz, nr = int(round((L + 2 * b) / h)), int(round(b / h))
    i0, i1 = int(round(b / h)) + 1, int(round(b / h)) + int(round(L / h))
    sheets = [(int(round(a / h)), i0, i1) for a in radii]
    return pp.vacuum_impedance(nr, nz, b, L + 2 * b, F_RF, sheets)


def test_test2_inductance_matrix_on_the_gpu():
    require_gpu()
    from oracle import verification as v
    Z, eps_rec = _solenoids([0.01, 0.02])
    L = Z.imag / OMEGA * 1e9
    assert L[0, 0] == pytest.approx(G12["t2_L1"][0][0], rel=2e-6)
    assert L[1, 1] == pytest.approx(G12["t2_L2"][0][0], rel=2e-6)
    assert L[0, 1] == pytest.approx(G12["t2_M"][0][0], rel=2e-6)
    assert eps_rec < 1e-10
    assert np.all(Z.real == 0.0)
    Zo, _, _, _ = v.solenoid_impedance([0.01, 0.02])
    assert np.max(np.abs(Z - Zo)) <= 1e-9 * np.max(np.abs(Zo))


@pytest.mark.parametrize("case", range(0, 7))
def test_test1_cases_on_the_gpu(case):
    """Table S1results (case 0) and every row of Table S1cases, the
    h = 0.5 mm grid (2481 x 241 nodes) included."""
    require_gpu()
    h, L, b, Lnum, eps = G12["t1_case"][case]
    Z, _ = _solenoids([0.01], h=h * 1e-3, L=L, b=b)
    Lh = Z[0, 0].imag / OMEGA * 1e9
    assert Lh == pytest.approx(Lnum, rel=1e-4)
    L_ana = 4e-7 * math.pi * math.pi * 0.01 ** 2 / L * 1e9
    assert 100 * (Lh - L_ana) / L_ana == pytest.approx(eps, abs=0.011)
    if case == 0:
        assert Z[0, 0].imag == pytest.approx(G12["t1_imz_model"][0][0], rel=1e-4)


def test_test3_inductance_on_the_gpu():
    """Test 3's M_h (sheets at a = 8, 20, 32, 48, 64 mm, b = 80 mm, l = 0.1 m,
    grid length l + h) with the analytic unit fields of Eq. t7unitfield on
    both axial boundary rows: the relative Frobenius error against the
    continuous M of Eq. t7M (Sec. 3.3: 7.44e-5) and the reciprocity defect
    eta_M (6.27e-6), and the oracle's M_h to solver precision."""
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp
    from oracle import verification as v
    h = 1e-3
    nsrc = int(round(v.T3_ELL / h))
    nz, nr = nsrc + 1, int(round(v.T3_B / h))
    R = np.arange(nr + 1) * h
    sheets, bnd = [], np.zeros((5, nz + 1, nr + 1))
    for k, a in enumerate(v.T3_A):
        sheets.append((int(round(a / h)), 1, nz - 1))
        prof = v.t3_unit_analytic(R, a)
        bnd[k, 0, :] = prof
        bnd[k, -1, :] = prof
    Z, _ = pp.vacuum_impedance(nr, nz, v.T3_B, nz * h, F_RF, sheets, boundary=bnd)
    Mh = Z.imag / OMEGA
    M = v.t3_continuous_M()
    em = np.linalg.norm(Mh - M) / np.linalg.norm(M)
    assert em == pytest.approx(S3["Mh_err_h1"], rel=0.01)
    eta_m = np.linalg.norm(Mh - Mh.T) / np.linalg.norm(Mh)
    assert eta_m == pytest.approx(S3["eta_M_h1"], rel=0.02)
    ref = v.FiveNode(h).Mh
    assert np.max(np.abs(Mh - ref)) <= 1e-9 * np.max(np.abs(ref))


def _t3_capacitance(h=1e-3):
    from paper_2609_15043_b300 import phasorpic as pp
    from oracle import verification as v
    nsrc = int(round(v.T3_ELL / h))
    nz, nr = nsrc + 1, int(round(v.T3_B / h))
    R = np.arange(nr + 1) * h
    cols = [int(round(a / h)) for a in v.T3_A]
    bnd = np.zeros((5, nz + 1, nr + 1))
    for l in range(5):
        V = np.zeros(5)
        V[l] = 1.0
        prof = v.t3_potential_analytic(R, V)
        bnd[l, 0, :] = prof
        bnd[l, -1, :] = prof
        bnd[l, :, -1] = 0.0                      # the grounded outer radius
    return pp.vacuum_capacitance(nr, nz, v.T3_B, nz * h, cols, v.T3_EPS, np.eye(5), bnd)


def test_test3_capacitance_and_state_on_the_gpu():
    """C_h of Test 3 from five Laplace solves on the GPU: its relative
    Frobenius error against the continuous C of Eq. t7C (Sec. 3.3: 1.21e-4),
    the oracle's C_h to solver precision, zero charge for zero potentials
    (appendix), and with the GPU's M_h the field-circuit column of Table
    t7phasors (Eq. t7network) and its distance 1.90e-5 to the continuous state
    (Eq. t7error)."""
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp
    from oracle import verification as v
    Ch = _t3_capacitance()
    C = v.t3_continuous_C()
    ec = np.linalg.norm(Ch - C) / np.linalg.norm(C)
    assert ec == pytest.approx(S3["Ch_err_h1"], rel=0.01)
    five = v.FiveNode(1e-3)
    assert np.max(np.abs(Ch - five.Ch)) <= 1e-9 * np.max(np.abs(five.Ch))
    # zero potentials everywhere give zero charge
    h = 1e-3
    nz, nr = int(round(v.T3_ELL / h)) + 1, int(round(v.T3_B / h))
    cols = [int(round(a / h)) for a in v.T3_A]
    Z0 = pp.vacuum_capacitance(nr, nz, v.T3_B, nz * h, cols, v.T3_EPS, np.zeros((5, 5)),
                               np.zeros((5, nz + 1, nr + 1)))
    assert np.max(np.abs(Z0)) == 0.0
    # the semidiscrete state from the GPU's C_h and M_h
    R = np.arange(nr + 1) * h
    sheets, bnd = [], np.zeros((5, nz + 1, nr + 1))
    for k, a in enumerate(v.T3_A):
        sheets.append((int(round(a / h)), 1, nz - 1))
        prof = v.t3_unit_analytic(R, a)
        bnd[k, 0, :] = prof
        bnd[k, -1, :] = prof
    Z, _ = pp.vacuum_impedance(nr, nz, v.T3_B, nz * h, F_RF, sheets, boundary=bnd)
    xh, _ = v.t3_network(Ch, Z.imag / OMEGA)
    x_calc = np.array([float(r[2]) + 1j * float(r[3]) for r in G3 if r[0] == "x"])
    x_cont = np.array([float(r[4]) + 1j * float(r[5]) for r in G3 if r[0] == "x"])
    assert np.max(np.abs(xh - x_calc)) < 6e-8
    assert v.t3_error(xh, x_cont) == pytest.approx(S3["state_err_cont_h1"], rel=0.01)
