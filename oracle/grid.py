"""RZ grid geometry for the oracle.

Nodes (i, j) sit at z_i = i*dz, R_j = j*dr, i = 0..nz, j = 0..nr; cell (i, j)
spans [z_i, z_{i+1}] x [R_j, R_{j+1}].  Readings of the paper's silent
points: the configured sizes are cell counts; a quartz slab over the full
radius separates the plasma region from a particle-free coil compartment
under a grounded lid; a turn is the set of nodes inside its wire disc (the
nearest node when the disc holds none); the axis node's control volume uses
A_z = pi*(dr/2)**2 and has no R- face.

Node control volumes and faces follow Sec. 2.3 (Eq. areas):
    A_z = 2*pi*R_j*dr (j >= 1),   A_z = pi*(dr/2)**2 on the axis (j = 0),
    A_R+- = 2*pi*(R_j +- dr/2)*dz,  no R- face on the axis.
"""
import math
import numpy as np


class Grid:
    """Uniform (z, R) node grid with a cell permittivity array."""

    def __init__(self, nz, nr, dz, dr, eps_cell=None):
        self.nz, self.nr = int(nz), int(nr)          # cells
        self.dz, self.dr = float(dz), float(dr)
        self.NZ, self.NR = self.nz + 1, self.nr + 1  # nodes
        self.z = np.arange(self.NZ) * self.dz
        self.R = np.arange(self.NR) * self.dr
        if eps_cell is None:
            eps_cell = np.ones((self.nz, self.nr))
        self.eps_cell = np.asarray(eps_cell, dtype=np.float64)

    def idx(self, i, j):
        return i * self.NR + j

    # --- face areas (Eq. areas) and the axis reading --------------------------
    def area_z(self, j):
        if j == 0:
            return math.pi * (self.dr / 2) ** 2
        return 2 * math.pi * self.R[j] * self.dr

    def area_r(self, j, sign):
        return 2 * math.pi * (self.R[j] + sign * self.dr / 2) * self.dz

    # --- face permittivities (Eq. epseff with chi = 0) ------------------------
    def _cell_eps(self, ic, jc):
        if 0 <= ic < self.nz and 0 <= jc < self.nr:
            return self.eps_cell[ic, jc]
        return None

    def eps_face(self, i, j, di, dj):
        """Mean permittivity of the existing cells that touch the face between
        node (i, j) and its neighbour (i+di, j+dj)."""
        if di != 0:
            ic = i if di > 0 else i - 1
            cells = [self._cell_eps(ic, j - 1), self._cell_eps(ic, j)]
        else:
            jc = j if dj > 0 else j - 1
            cells = [self._cell_eps(i - 1, jc), self._cell_eps(i, jc)]
        cells = [c for c in cells if c is not None]
        return sum(cells) / len(cells)

    def node_volume(self, i, j, z_lo=0.0, z_hi=None):
        """Annular control volume of node (i, j) clipped to [z_lo, z_hi] and to
        [0, R_max]."""
        if z_hi is None:
            z_hi = self.z[-1]
        za = max(self.z[i] - self.dz / 2, z_lo)
        zb = min(self.z[i] + self.dz / 2, z_hi)
        ra = max(self.R[j] - self.dr / 2, 0.0)
        rb = min(self.R[j] + self.dr / 2, self.R[-1])
        if zb <= za:
            return 0.0
        return math.pi * (rb * rb - ra * ra) * (zb - za)


class CellGeometry:
    """The PIC cell of the workloads: grounded electrode z=0, grounded wall
    r=r_max, grounded lid z=z_max, dielectric slab [z_win_lo, z_win_hi] over
    the full radius, and N turns centred at (turn_r[k], z_coil)."""

    def __init__(self, cfg):
        self.cfg = cfg
        nr, nz = cfg.nr, cfg.nz
        dr, dz = cfg.r_max / nr, cfg.z_max / nz
        self.i_win = _exact_index(cfg.z_win_lo, dz, "z_win_lo")
        self.i_win_hi = _exact_index(cfg.z_win_hi, dz, "z_win_hi")
        eps = np.ones((nz, nr))
        eps[self.i_win:self.i_win_hi, :] = cfg.eps_win
        self.grid = Grid(nz, nr, dz, dr, eps)
        g = self.grid
        # turn node sets Omega_k (Eq. shape): nodes inside the wire disc, else
        # the nearest node; every conductor node belongs to exactly one turn.
        self.turn_nodes = []
        owner = {}
        for k, rk in enumerate(cfg.turn_r):
            nodes = []
            for i in range(1, g.NZ - 1):
                for j in range(0, g.NR - 1):
                    d2 = (g.R[j] - rk) ** 2 + (g.z[i] - cfg.z_coil) ** 2
                    if d2 <= cfg.wire_radius ** 2:
                        nodes.append((i, j))
            if not nodes:
                best = None
                for i in range(1, g.NZ - 1):
                    for j in range(0, g.NR - 1):
                        d2 = (g.R[j] - rk) ** 2 + (g.z[i] - cfg.z_coil) ** 2
                        if best is None or d2 < best[0]:
                            best = (d2, i, j)
                nodes = [(best[1], best[2])]
            for n in nodes:
                if n in owner:
                    raise ValueError("conductor node %s belongs to turns %d and %d" % (n, owner[n], k))
                owner[n] = k
            self.turn_nodes.append(nodes)
        self.owner = owner
        self.n_turns = len(cfg.turn_r)
        # shape functions g_k = s_k / A_k on Omega_k, checked as in Eq. shape
        self.gk = np.zeros((self.n_turns, g.NZ, g.NR))
        for k, nodes in enumerate(self.turn_nodes):
            A = len(nodes) * dz * dr
            for (i, j) in nodes:
                self.gk[k, i, j] = cfg.winding[k] / A
            s = self.gk[k].sum() * dz * dr
            if abs(s - cfg.winding[k]) > 1e-12:
                raise ValueError("shape normalisation failed for turn %d" % k)
        # node volumes of the plasma region (rows 0..i_win) for densities:
        # the volume each node's bilinear weight covers, V = int S dV, so a
        # uniform population gives a flat density up to the axis
        # (Verboncoeur, J. Comput. Phys. 174 (2001)): 2 pi R_j dr in r, pi dr^2/3
        # on the axis, pi (R dr - dr^2/3) at the wall; dz in z, dz/2 on the
        # electrode and window rows.
        vr = np.array([2 * np.pi * g.R[j] * dr for j in range(g.NR)])
        vr[0] = np.pi * dr * dr / 3.0
        vr[-1] = np.pi * (g.R[-1] * dr - dr * dr / 3.0)
        vz = np.zeros(g.NZ)
        vz[:self.i_win + 1] = dz
        vz[0] = vz[self.i_win] = dz / 2.0
        self.vol = vz[:, None] * vr[None, :]
        # relative permittivity at nodes for the omega^2/c^2 Helmholtz term:
        # mean of the adjacent cells
        self.eps_node = np.zeros((g.NZ, g.NR))
        for i in range(g.NZ):
            for j in range(g.NR):
                cs = [eps[ic, jc] for ic in (i - 1, i) for jc in (j - 1, j)
                      if 0 <= ic < nz and 0 <= jc < nr]
                self.eps_node[i, j] = sum(cs) / len(cs)

    def poisson_dirichlet(self):
        """Mask of Dirichlet nodes: the grounded electrode, lid and wall, and
        the turn nodes; axis nodes are Neumann (Eq. axis_electrostatic_bc)."""
        g = self.grid
        m = np.zeros((g.NZ, g.NR), bool)
        m[0, :] = m[-1, :] = True
        m[:, -1] = True
        for nodes in self.turn_nodes:
            for (i, j) in nodes:
                m[i, j] = True
        return m


def _exact_index(x, h, name):
    k = x / h
    if abs(k - round(k)) > 1e-9:
        raise ValueError("%s=%g is not on a grid line" % (name, x))
    return int(round(k))
