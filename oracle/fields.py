"""Field equations of the method, written as sparse linear systems and solved
directly (scipy.sparse.linalg).  All FP64.

Poisson (Sec. 2.3, Eq. poisson with chi = 0, Eq. epseff, Eq. areas): the
finite-volume balance of node (i, j)
    sum_f eps_f A_f (phi_nb - phi_ij) / d_f = -Q_ij / eps0
with Q_ij the charge (C) in the node's control volume; Neumann on the axis
(Eq. axis_electrostatic_bc), Dirichlet on metal and on the turn nodes
(Eq. dirichlet).

Helmholtz (Sec. 2.2, Eqs. helmholtz_op, helmholtz_phasor): the plain
five-point central-difference operator
    L E = E_zz + E_RR + E_R / R - E / R^2 + k^2 E,  k^2 = mu0 eps0 eps_r w^2,
with E = 0 on the axis (Eq. axis_inductive_bc) and on the outer boundaries.

Gauss-law turn charge (Eq. facecharge): Q_k = sum over the faces between a
node of turn k and a node outside turn k of eps0 eps_f (phi_k - phi_nb) A_f / d_f.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .constants import EPS0, MU0


# ----------------------------------------------------------------------------
# Poisson
# ----------------------------------------------------------------------------
def poisson_matrix(g, dirichlet):
    """Sparse FV operator over all nodes; Dirichlet rows are identity rows."""
    N = g.NZ * g.NR
    rows, cols, vals = [], [], []
    for i in range(g.NZ):
        for j in range(g.NR):
            p = g.idx(i, j)
            if dirichlet[i, j]:
                rows.append(p); cols.append(p); vals.append(1.0)
                continue
            diag = 0.0
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                if j == 0 and dj == -1:
                    continue                     # no R- face on the axis
                ii, jj = i + di, j + dj
                if di != 0:
                    A, d = g.area_z(j), g.dz
                else:
                    A, d = g.area_r(j, dj), g.dr
                c = g.eps_face(i, j, di, dj) * A / d
                rows.append(p); cols.append(g.idx(ii, jj)); vals.append(c)
                diag -= c
            rows.append(p); cols.append(p); vals.append(diag)
    return sp.csc_matrix((vals, (rows, cols)), shape=(N, N))


class PoissonSolver:
    """Factorises the Poisson matrix once; solve() takes node charges (C) and
    the Dirichlet values."""

    def __init__(self, g, dirichlet):
        self.g = g
        self.dirichlet = dirichlet
        self.A = poisson_matrix(g, dirichlet)
        self.lu = spla.splu(self.A)

    def rhs(self, Q, phi_dirichlet):
        b = -np.asarray(Q, dtype=np.float64) / EPS0
        b = np.where(self.dirichlet, phi_dirichlet, b)
        return b.ravel()

    def solve(self, Q, phi_dirichlet):
        b = self.rhs(Q, phi_dirichlet)
        return self.lu.solve(b).reshape(self.g.NZ, self.g.NR)

    def solve_chi(self, Q, phi_dirichlet, chi):
        """Eq. poisson with the susceptibility chi (a fresh factorisation:
        chi changes every step)."""
        A = poisson_matrix_chi(self.A, self.dirichlet, chi)
        b = self.rhs(Q, phi_dirichlet)
        return spla.spsolve(A, b).reshape(self.g.NZ, self.g.NR)

    def residual(self, phi, Q, phi_dirichlet):
        b = self.rhs(Q, phi_dirichlet)
        return (self.A @ phi.ravel() - b).reshape(self.g.NZ, self.g.NR)


def poisson_matrix_chi(A0, dirichlet, chi):
    """The operator of Eq. poisson with the susceptibility chi on the nodes:
    every face coefficient eps_f A_f / d_f of the chi = 0 operator A0 (rows of
    non-Dirichlet nodes) is multiplied by 1 + (chi_p + chi_nb)/2, the face
    factor of Eq. epseff, and the diagonal is minus the row's face sum."""
    A = A0.tocoo()
    r, c, v = A.row, A.col, A.data.copy()
    d = dirichlet.ravel()
    x = np.asarray(chi, dtype=np.float64).ravel()
    off = (r != c) & ~d[r]
    v[off] = v[off] * (1.0 + 0.5 * (x[r[off]] + x[c[off]]))
    on = (r == c) & ~d[r]
    face_sum = np.bincount(r[off], weights=v[off], minlength=A.shape[0])
    v[on] = -face_sum[r[on]]
    return sp.csc_matrix((v, (r, c)), shape=A.shape)


def turn_charge(g, phi, turn_nodes, chi=None):
    """Q_k of Eq. facecharge summed over the external faces of each turn.
    Faces to a node of another turn count for both turns; faces to metal or
    boundary nodes count with the node's Dirichlet value.  With a
    susceptibility chi the face coefficient is that of Eq. epseff."""
    member = {}
    for k, nodes in enumerate(turn_nodes):
        for n in nodes:
            member[n] = k
    Q = np.zeros(len(turn_nodes))
    for k, nodes in enumerate(turn_nodes):
        for (i, j) in nodes:
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                if j == 0 and dj == -1:
                    continue
                ii, jj = i + di, j + dj
                if not (0 <= ii < g.NZ and 0 <= jj < g.NR):
                    continue
                if member.get((ii, jj)) == k:
                    continue                     # internal face of turn k
                if di != 0:
                    A, d = g.area_z(j), g.dz
                else:
                    A, d = g.area_r(j, dj), g.dr
                eps = g.eps_face(i, j, di, dj)
                if chi is not None:
                    eps = eps * (1.0 + 0.5 * (chi[i, j] + chi[ii, jj]))
                Q[k] += EPS0 * eps * (phi[i, j] - phi[ii, jj]) / d * A
    return Q


# ----------------------------------------------------------------------------
# Helmholtz
# ----------------------------------------------------------------------------
def helmholtz_matrix(g, dirichlet, k2=None):
    """Five-point FD operator L of Eq. helmholtz_op over all nodes; Dirichlet
    rows are identity rows.  k2 is mu0 eps0 eps_r w^2 per node (None: MQS).
    Row (i, j), R = R_j:
        E[i+-1, j] / dz^2 + E[i, j+-1] (1/dr^2 +- 1/(2 R dr))
        + E[i, j] (-2/dz^2 - 2/dr^2 - 1/R^2 + k2)."""
    NZ, NR = g.NZ, g.NR
    hz2, hr2 = g.dz * g.dz, g.dr * g.dr
    I, Jn = np.meshgrid(np.arange(NZ), np.arange(NR), indexing="ij")
    p = (I * NR + Jn).ravel()
    inner = ~dirichlet.ravel()
    Rn = np.broadcast_to(g.R[None, :], (NZ, NR)).ravel()
    rows, cols, vals = [p[~inner]], [p[~inner]], [np.ones(np.count_nonzero(~inner))]
    pi, Ri = p[inner], Rn[inner]
    diag = -2.0 / hz2 - 2.0 / hr2 - 1.0 / (Ri * Ri)
    if k2 is not None:
        diag = diag + k2.ravel()[inner]
    for off, c in ((NR, np.full(pi.shape, 1.0 / hz2)), (-NR, np.full(pi.shape, 1.0 / hz2)),
                   (1, 1.0 / hr2 + 1.0 / (2.0 * Ri * g.dr)), (-1, 1.0 / hr2 - 1.0 / (2.0 * Ri * g.dr))):
        rows.append(pi); cols.append(pi + off); vals.append(c)
    rows.append(pi); cols.append(pi); vals.append(diag)
    N = NZ * NR
    return sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N))


def helmholtz_dirichlet(g):
    m = np.zeros((g.NZ, g.NR), bool)
    m[0, :] = m[-1, :] = True
    m[:, 0] = m[:, -1] = True
    return m


class HelmholtzSolver:
    """Factorises L once; solve(rhs, boundary) returns E on all nodes."""

    def __init__(self, g, k2=None, dirichlet=None):
        self.g = g
        self.dirichlet = helmholtz_dirichlet(g) if dirichlet is None else dirichlet
        self.A = helmholtz_matrix(g, self.dirichlet, k2)
        self.lu = spla.splu(self.A)

    def solve(self, rhs, boundary=None):
        b = np.where(self.dirichlet, 0.0 if boundary is None else boundary, rhs)
        return self.lu.solve(b.ravel()).reshape(self.g.NZ, self.g.NR)


def unit_fields(hs, gk, omega, boundaries=None):
    """U_k from K U_k = g_k with K = L/(mu0 w) (Eq. unitfield)."""
    out = []
    for k in range(gk.shape[0]):
        bnd = None if boundaries is None else boundaries[k]
        out.append(hs.solve(MU0 * omega * gk[k], bnd))
    return np.array(out)


def vacuum_impedance(g, gk, U):
    """Z_vac,kl = -i sum g_k U_l 2 pi R dz dR (Eq. zvac) and eps_rec
    (Eq. reciprocity)."""
    w = 2 * np.pi * g.R[None, :] * g.dz * g.dr
    n = gk.shape[0]
    Z = np.zeros((n, n), complex)
    for k in range(n):
        for l in range(n):
            Z[k, l] = -1j * np.sum(gk[k] * U[l] * w)
    eps_rec = np.max(np.abs(Z - Z.T)) / np.max(np.abs(Z))
    return Z, eps_rec


def project(g, gk, field):
    """int g_k field dV for every turn (used by Eq. vpind)."""
    w = 2 * np.pi * g.R[None, :] * g.dz * g.dr
    return np.array([np.sum(gk[k] * field * w) for k in range(gk.shape[0])])


# ----------------------------------------------------------------------------
# node fields for the particle gather
# ----------------------------------------------------------------------------
def efield_from_phi(g, phi):
    """E_r, E_z at nodes: centred differences, one-sided at the first and last
    node, E_r = 0 on the axis (Eq. axis_electrostatic_bc)."""
    Ez = np.empty_like(phi)
    Er = np.empty_like(phi)
    Ez[1:-1, :] = -(phi[2:, :] - phi[:-2, :]) / (2.0 * g.dz)
    Ez[0, :] = -(phi[1, :] - phi[0, :]) / g.dz
    Ez[-1, :] = -(phi[-1, :] - phi[-2, :]) / g.dz
    Er[:, 1:-1] = -(phi[:, 2:] - phi[:, :-2]) / (2.0 * g.dr)
    Er[:, 0] = 0.0
    Er[:, -1] = -(phi[:, -1] - phi[:, -2]) / g.dr
    return Er, Ez


def b_phasors(g, Ec, Es_sto, omega):
    """RF magnetic field from Faraday's law under exp(+i w t):
    B_r = -(i/w) dE/dz, B_z = (i/w)(1/R) d(R E)/dR with E = Ec + i Es_sto.
    Returns (Brc, Brs, Bzc, Bzs) with B(t) = Bc cos(theta) + Bs sin(theta)."""
    def ddz(f):
        d = np.empty_like(f)
        d[1:-1] = (f[2:] - f[:-2]) / (2.0 * g.dz)
        d[0] = (f[1] - f[0]) / g.dz
        d[-1] = (f[-1] - f[-2]) / g.dz
        return d

    def curl_r(f):
        R = g.R
        d = np.empty_like(f)
        d[:, 1:-1] = (R[2:] * f[:, 2:] - R[:-2] * f[:, :-2]) / (2.0 * g.dr * R[1:-1])
        d[:, 0] = 2.0 * (f[:, 1] - f[:, 0]) / g.dr
        d[:, -1] = (R[-1] * f[:, -1] - R[-2] * f[:, -2]) / (g.dr * R[-1])
        return d

    Brc = ddz(Es_sto) / omega
    Brs = ddz(Ec) / omega
    Bzc = -curl_r(Es_sto) / omega
    Bzs = -curl_r(Ec) / omega
    return Brc, Brs, Bzc, Bzs
