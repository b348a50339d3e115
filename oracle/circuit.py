"""Turn-resolved coil circuit of Sec. 2.4, FP64 complex.

Unknowns x = (I_f, I_1..I_N, V_1..V_N) (Eq. unknowns), peak phasors under
exp(+i w t).  The block system of Eq. blockmatrix is assembled from its three
row blocks: the Thevenin source row (Eq. thevenin), the N KCL rows (Eq. kcl)
and the N KVL rows (Eq. kvl), and solved with numpy.linalg.solve.
"""
import math
import numpy as np

from .constants import MU0


def skin_resistance(turn_r, wire_radius, omega, rho20, alpha_cu, t_c):
    """R_rf,k of Eq. skin with rho(T) = rho20 [1 + alpha (T - 20 C)]."""
    rho = rho20 * (1.0 + alpha_cu * (t_c - 20.0))
    delta = math.sqrt(2.0 * rho / (omega * MU0))
    inner = max(wire_radius - delta, 0.0)
    return np.array([rho * 2 * math.pi * rk / (math.pi * (wire_radius ** 2 - inner ** 2))
                     for rk in turn_r])


def z_source(r_g, r_m, l_m, c_m, omega):
    """Eq. zsource; the capacitor term is dropped when C_m <= 0."""
    x = omega * l_m
    if c_m > 0:
        x -= 1.0 / (omega * c_m)
    return r_g + r_m + 1j * x


def network_matrix(zs, zturn, c_stray, omega):
    """(2N+1)x(2N+1) matrix of Eq. blockmatrix."""
    N = zturn.shape[0]
    A = np.zeros((2 * N + 1, 2 * N + 1), complex)
    # Thevenin row: Z_source I_f + V_1 = V_g
    A[0, 0] = zs
    A[0, 1 + N] = 1.0
    for k in range(N):
        r = 1 + k
        # KCL at node k: I_in,k - I_k - i w C_stray,k V_k = I_cap,k
        if k == 0:
            A[r, 0] = 1.0
        else:
            A[r, 1 + (k - 1)] = 1.0
        A[r, 1 + k] = -1.0
        A[r, 1 + N + k] = -1j * omega * c_stray[k]
        # KVL along segment k: V_k - V_{k+1} - sum_l Z_turn,kl I_l = V_p,k
        r2 = 1 + N + k
        for l in range(N):
            A[r2, 1 + l] = -zturn[k, l]
        A[r2, 1 + N + k] = 1.0
        if k + 1 < N:
            A[r2, 1 + N + k + 1] = -1.0
    return A


def solve_target(A, vg, icap, vp):
    """x_target = C(V_p, I_cap, V_g) (Eq. target)."""
    b = np.concatenate([[vg], icap, vp]).astype(complex)
    return np.linalg.solve(A, b)


def residuals(x, zs, zturn, c_stray, omega, vg, icap, vp, v_scale=None):
    """Eqs. kclres, kvlres, normalised by |I_f| and |V_g| (the scales the
    paper uses for Test 3; v_scale replaces |V_g| where the source is zero,
    as at a harmonic); returns (max KCL, max KVL)."""
    N = zturn.shape[0]
    If, I, V = x[0], x[1:1 + N], x[1 + N:]
    Iin = np.concatenate([[If], I[:-1]])
    rI = Iin - I - icap - 1j * omega * np.asarray(c_stray) * V
    Vnext = np.concatenate([V[1:], [0.0]])
    rV = V - Vnext - zturn @ I - vp
    rV0 = vg - zs * If - V[0]
    si = max(abs(If), 1e-300)
    sv = max(abs(vg) if v_scale is None else v_scale, 1e-300)
    return np.max(np.abs(rI)) / si, max(np.max(np.abs(rV)), abs(rV0)) / sv


def port_power(x, N):
    """P_port = 1/2 Re(V_1 I_f*) (Eq. pport)."""
    return 0.5 * (x[1 + N] * np.conj(x[0])).real


def copper_power(x, N, r_rf):
    """P_Cu = 1/2 sum R_rf,k |I_k|^2."""
    return 0.5 * float(np.sum(r_rf * np.abs(x[1:1 + N]) ** 2))


def cap_power_phasor(x, N, icap):
    """P_cap^ph = 1/2 Re sum V_k I_cap,k* (Eq. pcap_phasor)."""
    return 0.5 * float(np.sum(x[1 + N:] * np.conj(icap)).real)


def cap_power_trapezoid(V, Q, f):
    """P_cap = f sum_k W_k with the closed-cycle trapezoid of Eq. pcap.
    V, Q: arrays (N_RF, N_turns) of the samples n = 1..N_RF; the interval
    before sample 1 is closed with sample N_RF."""
    Vp = np.roll(V, 1, axis=0)
    Qp = np.roll(Q, 1, axis=0)
    W = np.sum(0.5 * (V + Vp) * (Q - Qp), axis=0)
    return f * float(np.sum(W)), W


class PowerController:
    """Eqs. pfilter, ptrend, pcontrol with the symmetric limiter and the
    absolute bounds.  The filter starts from the first measurement."""

    def __init__(self, p_target, gamma, n_trend, eps_p, alpha_v, f_step, v_min, v_max):
        self.p_target, self.gamma, self.n_trend = p_target, gamma, n_trend
        self.eps_p, self.alpha_v, self.f_step = eps_p, alpha_v, f_step
        self.v_min, self.v_max = v_min, v_max
        self.pf_prev = None

    def update(self, v_old, p_port):
        prev = p_port if self.pf_prev is None else self.pf_prev
        pf = self.gamma * p_port + (1.0 - self.gamma) * prev
        pc = max(pf + self.n_trend * (pf - prev), self.eps_p)
        v_des = v_old * math.sqrt(self.p_target / pc)
        v_new = v_old + self.alpha_v * (v_des - v_old)
        v_new = min(max(v_new, (1.0 - self.f_step) * v_old), (1.0 + self.f_step) * v_old)
        v_new = min(max(v_new, self.v_min), self.v_max)
        self.pf_prev = pf
        return v_new
