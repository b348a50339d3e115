"""The paper's particle-free verification problems (Sec. 3.1-3.3 and the
appendix on the joint benchmark), set up on the oracle's field and circuit
routines.  They are the oracle's external pins: the paper prints the numbers
these functions must reproduce.

Test 1/2 (solenoids): MQS vacuum Helmholtz on 0 <= z <= L + 2b,
0 <= R <= b, homogeneous Dirichlet on the three outer edges and the axis
(Eq. S1bc); each sheet is one node row at R = a over the z nodes
b/h + 1 .. b/h + L/h with g = 1/(N_k h^2).

Test 3 (five-node MQS-EQS benchmark): sheets at a = 8, 20, 32, 48, 64 mm,
outer radius b = 80 mm, eps_r = 9, source length l = N_src h, grid length
l + h; both axial boundaries carry the analytic radial solutions of Eqs.
t7unitfield and t7potential.
"""
import math
import numpy as np

from .constants import EPS0, MU0
from .grid import Grid
from . import fields, circuit

F_RF = 13.56e6
OMEGA = 2 * math.pi * F_RF


# ----------------------------------------------------------------------------
# Tests 1 and 2
# ----------------------------------------------------------------------------
def solenoid_impedance(radii, h=1e-3, L=1.0, b=0.12):
    """Z_vac of coaxial current sheets of length L at the given radii."""
    nz_c = int(round((L + 2 * b) / h))
    nr_c = int(round(b / h))
    g = Grid(nz_c, nr_c, h, h)
    hs = fields.HelmholtzSolver(g)
    i0 = int(round(b / h)) + 1
    i1 = int(round(b / h)) + int(round(L / h))
    gk = np.zeros((len(radii), g.NZ, g.NR))
    for k, a in enumerate(radii):
        j = int(round(a / h))
        n = i1 - i0 + 1
        gk[k, i0:i1 + 1, j] = 1.0 / (n * h * h)
    U = fields.unit_fields(hs, gk, OMEGA)
    Z, eps_rec = fields.vacuum_impedance(g, gk, U)
    return Z, eps_rec, g, U


def series_current(u_rf, R, Z):
    """Eq. S1circuit: I = U / (R + Z), U_L = Z I."""
    I = u_rf / (R + Z)
    return I, Z * I


def two_loop(u_rf, R1, R2, C, Z):
    """Eqs. S2loops-S2solution with the field-derived Z (2x2)."""
    ZA = R1 + Z[0, 0]
    ZB = Z[1, 1] + R2 - 1j / (OMEGA * C)
    Zm = Z[0, 1]
    det = ZA * ZB - Zm * Zm
    I1 = u_rf * ZB / det
    I2 = -Zm * u_rf / det
    U1 = Z[0, 0] * I1 + Z[0, 1] * I2
    U2 = Z[1, 0] * I1 + Z[1, 1] * I2
    return I1, I2, U1, U2


# ----------------------------------------------------------------------------
# Test 3
# ----------------------------------------------------------------------------
T3_A = np.array([8e-3, 20e-3, 32e-3, 48e-3, 64e-3])
T3_B = 80e-3
T3_ELL = 0.1
T3_EPS = 9.0
T3_VG = 100.0
T3_RG = 50.0
T3_RRF = 20.0


def t3_continuous_C(a=T3_A, b=T3_B, ell=T3_ELL, eps=T3_EPS):
    """Eq. t7C."""
    ak = np.concatenate([a, [b]])
    c = np.array([2 * math.pi * EPS0 * eps * ell / math.log(ak[k + 1] / ak[k]) for k in range(len(a))])
    n = len(a)
    C = np.zeros((n, n))
    for k in range(n):
        C[k, k] = (c[k - 1] if k > 0 else 0.0) + c[k]
        if k + 1 < n:
            C[k, k + 1] = C[k + 1, k] = -c[k]
    return C


def t3_continuous_M(a=T3_A, b=T3_B, ell=T3_ELL):
    """Eq. t7M."""
    n = len(a)
    M = np.zeros((n, n))
    for k in range(n):
        for l in range(n):
            lo, hi = min(a[k], a[l]), max(a[k], a[l])
            M[k, l] = MU0 * math.pi / ell * lo * lo * (1 - hi * hi / (b * b))
    return M


def t3_network(C, M, vg=T3_VG, rg=T3_RG, rrf=T3_RRF):
    """Eq. t7network as the general block system with Z_source = R_g,
    Z_turn = R_rf + i w M and the linear capacitive load I_cap = i w C V moved
    to the left-hand side."""
    n = C.shape[0]
    A = circuit.network_matrix(rg, 1j * OMEGA * M + rrf * np.eye(n), np.zeros(n), OMEGA)
    A[1:1 + n, 1 + n:] -= 1j * OMEGA * C
    b = np.zeros(2 * n + 1, complex)
    b[0] = vg
    return np.linalg.solve(A, b), A


def t3_recurrence(C, M, vg=T3_VG, rg=T3_RG, rrf=T3_RRF):
    """Eq. t7recurrence: x^{n+1} = c + G x^n with G = A0^-1 T (i w C) S_V."""
    n = C.shape[0]
    A0 = circuit.network_matrix(rg, 1j * OMEGA * M + rrf * np.eye(n), np.zeros(n), OMEGA)
    b0 = np.zeros(2 * n + 1, complex)
    b0[0] = vg
    T = np.zeros((2 * n + 1, n))
    T[1:1 + n, :] = np.eye(n)
    SV = np.zeros((n, 2 * n + 1))
    SV[:, 1 + n:] = np.eye(n)
    G = np.linalg.solve(A0, T @ (1j * OMEGA * C) @ SV)
    c = np.linalg.solve(A0, b0)
    return c, G


def t3_error(x, xref, vg=T3_VG):
    """Eq. t7error."""
    n = (len(x) - 1) // 2
    s = np.concatenate([np.full(n + 1, abs(xref[0])), np.full(n, abs(vg))])
    return np.linalg.norm((x - xref) / s) / np.linalg.norm(xref / s)


def t3_unit_analytic(R, a, b=T3_B, ell=T3_ELL):
    """Eq. t7unitfield."""
    R = np.asarray(R, float)
    pre = -OMEGA * MU0 / (2 * ell)
    with np.errstate(divide='ignore'):
        out = np.where(R <= a, (1 - a * a / (b * b)) * R, a * a * (1 / np.where(R > 0, R, 1) - R / (b * b)))
    return pre * out


def t3_potential_analytic(R, V, a=T3_A, b=T3_B):
    """Eq. t7potential (real potentials V, one value per sheet)."""
    ak = np.concatenate([a, [b]])
    Vk = np.concatenate([V, [0.0]])
    R = np.asarray(R, float)
    out = np.empty_like(R)
    for idx, r in enumerate(R):
        if r <= ak[0]:
            out[idx] = Vk[0]
            continue
        for k in range(len(a)):
            if ak[k] < r <= ak[k + 1]:
                out[idx] = (Vk[k] * math.log(ak[k + 1] / r) + Vk[k + 1] * math.log(r / ak[k])) \
                    / math.log(ak[k + 1] / ak[k])
                break
        else:
            out[idx] = 0.0
    return out


class FiveNode:
    """The Test 3 grid with its unit fields, Laplace basis and Gauss charge."""

    def __init__(self, h=1e-3):
        self.h = h
        self.nsrc = int(round(T3_ELL / h))
        nz_c = self.nsrc + 1                      # grid length l + h
        nr_c = int(round(T3_B / h))
        self.g = Grid(nz_c, nr_c, h, h, np.full((nz_c, nr_c), T3_EPS))
        g = self.g
        self.jk = [int(round(a / h)) for a in T3_A]
        self.turn_nodes = [[(i, j) for i in range(1, g.NZ - 1)] for j in self.jk]
        # inductive unit fields with manufactured axial boundaries
        hs = fields.HelmholtzSolver(g)
        gk = np.zeros((5, g.NZ, g.NR))
        for k, j in enumerate(self.jk):
            gk[k, 1:g.NZ - 1, j] = 1.0 / (self.nsrc * h * h)
        self.gk = gk
        bnds = []
        for a in T3_A:
            bnd = np.zeros((g.NZ, g.NR))
            prof = t3_unit_analytic(g.R, a)
            bnd[0, :] = prof
            bnd[-1, :] = prof
            bnds.append(bnd)
        self.U = fields.unit_fields(hs, gk, OMEGA, bnds)
        Z, self.eps_rec = fields.vacuum_impedance(g, gk, self.U)
        self.Mh = Z.imag / OMEGA
        # electrostatics: sheets and axial boundary rows Dirichlet, R = b grounded
        self.dir = np.zeros((g.NZ, g.NR), bool)
        self.dir[0, :] = self.dir[-1, :] = True
        self.dir[:, -1] = True
        for nodes in self.turn_nodes:
            for (i, j) in nodes:
                self.dir[i, j] = True
        self.ps = fields.PoissonSolver(g, self.dir)
        self.Ch = np.zeros((5, 5))
        for l in range(5):
            V = np.zeros(5)
            V[l] = 1.0
            self.Ch[:, l] = self.charges(V)

    def dirichlet_values(self, V):
        g = self.g
        vals = np.zeros((g.NZ, g.NR))
        prof = t3_potential_analytic(g.R, V)
        vals[0, :] = prof
        vals[-1, :] = prof
        for k, nodes in enumerate(self.turn_nodes):
            for (i, j) in nodes:
                vals[i, j] = V[k]
        return vals

    def charges(self, V):
        phi = self.ps.solve(np.zeros((self.g.NZ, self.g.NR)), self.dirichlet_values(V))
        return fields.turn_charge(self.g, phi, self.turn_nodes)

    def coupled_run(self, periods=30, n_rf=400, alpha=1.0, vg=T3_VG, rrf=T3_RRF):
        """Period-delayed field-circuit iteration of Sec. 2.5 without particles:
        each period samples Q_k(t_n) from n_rf Laplace solves with the applied
        turn potentials, projects I_cap = i w Q_hat, and solves the network
        with Z_vac = i w M_h.  Returns the applied states x^1..x^{periods+1}
        and the last period's diagnostics."""
        n = 5
        A = circuit.network_matrix(T3_RG, 1j * OMEGA * self.Mh + rrf * np.eye(n), np.zeros(n), OMEGA)
        zero = np.zeros(n, complex)
        x = circuit.solve_target(A, vg, zero, zero)
        hist = [x.copy()]
        last = None
        for _ in range(periods):
            V = x[1 + n:]
            Qc = np.zeros(n)
            Qs = np.zeros(n)
            Vs, Qsm = [], []
            for m in range(1, n_rf + 1):
                th = 2 * math.pi * (m % n_rf) / n_rf
                phik = V.real * math.cos(th) + (-V.imag) * math.sin(th)
                Q = self.charges(phik)
                Qc += 2.0 / n_rf * Q * math.cos(th)
                Qs += 2.0 / n_rf * Q * math.sin(th)
                Vs.append(phik)
                Qsm.append(Q)
            qhat = Qc - 1j * Qs
            icap = 1j * OMEGA * qhat
            p_cap, _ = circuit.cap_power_trapezoid(np.array(Vs), np.array(Qsm), F_RF)
            p_port = circuit.port_power(x, n)
            p_cu = circuit.copper_power(x, n, np.full(n, rrf))
            last = dict(x_applied=x.copy(), icap=icap, p_cap=p_cap, p_port=p_port, p_cu=p_cu,
                        p_cap_ph=circuit.cap_power_phasor(x, n, icap))
            xt = circuit.solve_target(A, vg, icap, zero)
            x = (1 - alpha) * x + alpha * xt
            hist.append(x.copy())
            last['residuals'] = circuit.residuals(x, T3_RG, 1j * OMEGA * self.Mh + rrf * np.eye(n),
                                                  np.zeros(n), OMEGA, vg, icap, zero)
        return np.array(hist), last
