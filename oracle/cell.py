"""One RF cell advanced by the phasor-PIC algorithm (Sec. 2.5, Fig.
algorithm_workflow), plainly and in FP64 except for the particle step
(float32 or float64, see oracle.particles).

Time levels.  Global step s (0-based) takes positions x^s and potential phi^s
(solved at t_s) to x^{s+1} and phi^{s+1}.  theta_s = 2 pi (s mod N_RF)/N_RF
(Eq. et_reconstruct).  Cycle c runs steps s = c N_RF .. c N_RF + N_RF - 1:
  * the current harmonics sample J_theta(t_s) (time-centred current at the
    old positions) for s in the cycle;
  * the turn charges sample Q_k(t_{s+1}) after each step's Poisson solve, so
    the last sample of the cycle has theta = 0;
  * both are projected with Eq. fourier (factor 2/N_RF).
At the end of the cycle: two plasma-only Helmholtz solves (Eq.
helmholtz_two_real), V_p (Eq. vpind), I_cap (Eq. icap), the sample-count check,
powers (Eqs. pind, pcap, pcap_phasor, pport), the controller, the target
network solve, relaxation (Eq. relaxation), residuals, and the composed field
for the next cycle (Eq. compose).  phi at the cycle boundary is then re-solved
with the new turn potentials so the first step of the next cycle sees them.

Multiharmonic extension (Sec. 4, with n_harmonics = M > 1): every retained
frequency m w, m = 2..M, has its own Helmholtz operator (the eps_r (m w)^2/c^2
term), unit fields, Z_vac, skin resistance, source impedance and network.  The
per-step accumulation projects J and Q on cos m theta, sin m theta as on the
fundamental (Eq. fourier), the period end turns them into V_p^(m) and
I_cap^(m) = i m w Q^(m), and the network at m w is solved and relaxed with no
source (the generator is sinusoidal: V_g drives the fundamental only).  The
turn potentials and E_theta, B used by the next period's steps are the sums of
all retained harmonics (waveform reconstruction, exp(+i m w t) peak phasors);
the powers of the record are the sums over the harmonics (the time-domain
P_ind and P_cap carry them by construction).

Particle control (oracle.particles, oracle.control): with see_gamma > 0 the
ions absorbed on the electrode, wall or window emit secondary electrons; with
particle_weights (or sm_every > 0) every particle carries a relative weight,
and with sm_every > 0 a split-merge pass follows the append of every
sm_every-th step.  Creation events are appended ionisations first (electron
and ion, ordered by the parent electron's uid), then secondary electrons
(ordered by the parent ion's uid); both species number their new particles
in that order.
"""
import math
import numpy as np

from .constants import EPS0, MU0, QE, ME, M_AR, KB
from .grid import CellGeometry
from . import fields, circuit, particles, control


class OracleCell:
    def __init__(self, cfg, weights):
        self.cfg = cfg
        self.geo = CellGeometry(cfg)
        g = self.geo.grid
        self.g = g
        self.omega = 2 * math.pi * cfg.freq
        self.n_rf = int(round(1.0 / (cfg.freq * cfg.dt)))
        if abs(cfg.freq * cfg.dt * self.n_rf - 1.0) >= 1e-10:      # Eq. phaseclosure
            raise ValueError("phase closure violated")
        self.N = self.geo.n_turns
        # --- Poisson ----------------------------------------------------------
        self.pdir = self.geo.poisson_dirichlet()
        self.poisson = fields.PoissonSolver(g, self.pdir)
        # --- Helmholtz, unit fields, Z_vac -------------------------------------
        k2 = None
        if cfg.full_helmholtz:
            k2 = MU0 * EPS0 * self.omega ** 2 * self.geo.eps_node
        self.helm = fields.HelmholtzSolver(g, k2)
        self.U = fields.unit_fields(self.helm, self.geo.gk, self.omega)
        self.zvac, self.eps_rec = fields.vacuum_impedance(g, self.geo.gk, self.U)
        # --- circuit ------------------------------------------------------------
        if cfg.r_rf_override >= 0:
            self.r_rf = np.full(self.N, cfg.r_rf_override)
        else:
            self.r_rf = circuit.skin_resistance(cfg.turn_r, cfg.wire_radius, self.omega,
                                                cfg.rho20, cfg.alpha_cu, cfg.t_coil_c)
        self.zs = circuit.z_source(cfg.r_g, cfg.r_m, cfg.l_m, cfg.c_m, self.omega)
        self.zturn = self.zvac + np.diag(self.r_rf)
        self.c_stray = np.asarray(cfg.c_stray[:self.N], dtype=float)
        self.A = circuit.network_matrix(self.zs, self.zturn, self.c_stray, self.omega)
        self.vg_amp = cfg.v_g
        self.vg = cfg.v_g * complex(math.cos(cfg.phase_g), math.sin(cfg.phase_g))
        self.ctrl = None
        if cfg.power_control:
            self.ctrl = circuit.PowerController(cfg.p_target, cfg.gamma, cfg.n_trend, cfg.eps_p,
                                                cfg.alpha_v, cfg.f_step, cfg.v_min, cfg.v_max)
        # x^1: zero-load network solution
        zeros = np.zeros(self.N, complex)
        self.x = circuit.solve_target(self.A, self.vg, zeros, zeros)
        self.Ecp = np.zeros((g.NZ, g.NR))
        self.Essp = np.zeros((g.NZ, g.NR))
        self._compose()
        # --- retained harmonics m = 2..M (zero state: no source at m w) ------
        self.M = max(1, int(getattr(cfg, "n_harmonics", 1)))
        self.harm = []
        for m in range(2, self.M + 1):
            wm = m * self.omega
            k2m = None if k2 is None else MU0 * EPS0 * wm ** 2 * self.geo.eps_node
            hm = fields.HelmholtzSolver(g, k2m)
            Um = fields.unit_fields(hm, self.geo.gk, wm)
            zvm, _ = fields.vacuum_impedance(g, self.geo.gk, Um)
            if cfg.r_rf_override >= 0:
                rrf = np.full(self.N, cfg.r_rf_override)
            else:
                rrf = circuit.skin_resistance(cfg.turn_r, cfg.wire_radius, wm, cfg.rho20, cfg.alpha_cu,
                                              cfg.t_coil_c)
            zsm = circuit.z_source(cfg.r_g, cfg.r_m, cfg.l_m, cfg.c_m, wm)
            ztm = zvm + np.diag(rrf)
            h = dict(m=m, omega=wm, helm=hm, U=Um, zvac=zvm, r_rf=rrf, zs=zsm, zturn=ztm,
                     A=circuit.network_matrix(zsm, ztm, self.c_stray, wm),
                     x=np.zeros(2 * self.N + 1, complex),
                     Ecp=np.zeros((g.NZ, g.NR)), Essp=np.zeros((g.NZ, g.NR)))
            self._compose_h(h)
            self.harm.append(h)
        # --- particles ----------------------------------------------------------
        self.weights = weights
        self._species = {}
        self.implicit = bool(getattr(cfg, "implicit_es", 0))
        self.chi_last = None
        self.P = [None, None]
        self.next_uid = [0, 0]
        self.window_q = np.zeros((g.NZ, g.NR))
        self.see_gamma = float(getattr(cfg, "see_gamma", 0.0))
        self.see_t_ev = float(getattr(cfg, "see_t_ev", 2.0))
        self.sm_every = int(getattr(cfg, "sm_every", 0))
        self.sm = (int(getattr(cfg, "sm_target", 0)), int(getattr(cfg, "sm_min", 0)),
                   int(getattr(cfg, "sm_max", 0)))
        self.see_emitted = 0
        self.sm_stats = dict(split=0, merged=0, skipped=0)
        self.s = 0
        self.phi = np.zeros((g.NZ, g.NR))
        self._reset_accumulators()
        self.records = []

    # ------------------------------------------------------------------------
    def set_particles(self, sp, cell, dr, dz, vr, vt, vz, uid, w=None):
        """w: relative weights (default 1, in the state's dtype)."""
        dr = np.array(dr)
        self.P[sp] = dict(cell=np.asarray(cell, np.int64).copy(), dr=dr, dz=np.array(dz),
                          vr=np.array(vr), vt=np.array(vt), vz=np.array(vz),
                          w=(np.ones(dr.shape, dr.dtype) if w is None else np.array(w, dr.dtype)),
                          uid=np.asarray(uid, np.int64).copy())
        self.next_uid[sp] = int(np.max(uid)) + 1 if len(uid) else 0

    def species(self, sp, T):
        """Species constants in T (computed once per species and type; they
        depend only on the configuration and the macro weight)."""
        key = (sp, np.dtype(T).name)
        if key not in self._species:
            self._species[key] = particles.SpeciesConstants(self.cfg, sp, self.weights[sp], T)
        return self._species[key]

    def theta(self, s):
        return 2.0 * math.pi * (s % self.n_rf) / self.n_rf

    def turn_potentials(self, th):
        V = self.x[1 + self.N:]
        out = V.real * math.cos(th) + (-V.imag) * math.sin(th)       # Eq. dirichlet
        for h in self.harm:
            Vm, mt = h["x"][1 + self.N:], h["m"] * th
            out = out + (Vm.real * math.cos(mt) + (-Vm.imag) * math.sin(mt))
        return out

    def etheta(self, th):
        """E_theta at phase th (Eq. et_reconstruct, summed over the retained
        harmonics)."""
        Et = self.Ec * math.cos(th) - self.Ess * math.sin(th)
        for h in self.harm:
            mt = h["m"] * th
            Et = Et + (h["Ec"] * math.cos(mt) - h["Ess"] * math.sin(mt))
        return Et

    def dirichlet_values(self, th):
        vals = np.zeros((self.g.NZ, self.g.NR))
        phik = self.turn_potentials(th)
        for k, nodes in enumerate(self.geo.turn_nodes):
            for (i, j) in nodes:
                vals[i, j] = phik[k]
        return vals

    def deposit_species(self, T):
        """Charge of each species at the current positions (C per node)."""
        Qs = [np.zeros((self.g.NZ, self.g.NR)), np.zeros((self.g.NZ, self.g.NR))]
        for sp in (0, 1):
            P = self.P[sp]
            sc = self.species(sp, T)
            live = P['cell'] >= 0
            cell = P['cell'][live]
            ir, iz = cell % self.cfg.nr, cell // self.cfg.nr
            w = particles.bilinear(P['dr'][live].astype(T), P['dz'][live].astype(T), T)
            qwp = (sc.qw * P['w'][live].astype(T)).astype(T)
            for (di, dj), wk in zip(((0, 0), (0, 1), (1, 0), (1, 1)), w):
                np.add.at(Qs[sp], (iz + di, ir + dj), (qwp * wk).astype(np.float64))
        return Qs

    def deposit_charge(self, T):
        """Q at the current positions (used once before the first step)."""
        Qs = self.deposit_species(T)
        return Qs[0] + Qs[1]

    def susceptibility(self, Qs, T):
        """chi on the nodes from the species charges of the predicted
        populations (Sec. 2.3): chi = sum_s (q_s/m_s) dt^2 (Q_s / V) /
        (eps0 eps_r), with V the node weighting volume and eps_r the node mean
        of the adjacent cells; zero where no particle deposits."""
        vol = self.geo.vol
        chi = np.zeros((self.g.NZ, self.g.NR))
        m = vol > 0
        for sp in (0, 1):
            chi[m] += self.species(sp, T).chi_per_charge * Qs[sp][m] / vol[m]
        chi[m] /= self.geo.eps_node[m]
        return chi

    def solve_potential(self, Q, th, chi):
        dv = self.dirichlet_values(th)
        if chi is None:
            return self.poisson.solve(Q, dv)
        return self.poisson.solve_chi(Q, dv, chi)

    def prime(self, T=np.float32):
        """phi^0 from the initial positions and theta_0 (with the initial
        populations' susceptibility in the direct-implicit form)."""
        Qs = self.deposit_species(T)
        self.chi_last = self.susceptibility(Qs, T) if self.implicit else None
        self.phi = self.solve_potential(Qs[0] + Qs[1] + self.window_q, self.theta(0), self.chi_last)

    # ------------------------------------------------------------------------
    def node_fields(self, th, T):
        """Per-cell corner fields for the gather at phase th: E_r, E_z from phi;
        E_theta = E_c cos - E_s^sto sin (Eq. et_reconstruct); B from Faraday."""
        g = self.g
        Er, Ez = fields.efield_from_phi(g, self.phi)
        c, s = math.cos(th), math.sin(th)
        Et = self.Ec * c - self.Ess * s
        Br = self.Brc * c + self.Brs * s
        Bz = self.Bzc * c + self.Bzs * s
        for h in self.harm:
            cm, sm = math.cos(h["m"] * th), math.sin(h["m"] * th)
            Et = Et + (h["Ec"] * cm - h["Ess"] * sm)
            Br = Br + (h["Brc"] * cm + h["Brs"] * sm)
            Bz = Bz + (h["Bzc"] * cm + h["Bzs"] * sm)
        if not self.cfg.magnetic_force:
            Br = np.zeros_like(Br)
            Bz = np.zeros_like(Bz)
        nr, iw = self.cfg.nr, self.geo.i_win
        F = np.zeros((iw * nr, 5, 4), T)
        for comp, f in enumerate((Er, Ez, Et, Br, Bz)):
            f32 = f.astype(T)
            F[:, comp, 0] = f32[:iw, :nr].ravel()
            F[:, comp, 1] = f32[:iw, 1:nr + 1].ravel()
            F[:, comp, 2] = f32[1:iw + 1, :nr].ravel()
            F[:, comp, 3] = f32[1:iw + 1, 1:nr + 1].ravel()
        return F

    def step(self, T=np.float32, drive=None):
        """One PIC step; returns per-step information.

        drive: optional callable (theta_s, E_theta nodes at theta_s) -> node
        current moment (A m) of a prescribed, non-particle current carrier
        (a test load such as an ohmic conductor).  Its moment is added to the
        particles' J_theta deposit and its work sum(J E) to the field-side
        inductive power, exactly as a particle's q w v_theta is."""
        cfg, g = self.cfg, self.g
        s = self.s
        th_old = self.theta(s)
        F = self.node_fields(th_old, T)
        Qs = [np.zeros((g.NZ, g.NR)), np.zeros((g.NZ, g.NR))]
        J = np.zeros((g.NZ, g.NR))
        stats = dict(p_ind=0.0, p_es=0.0, absorbed=0, pushed=0, nu_viol=0,
                     coll=np.zeros((2, 3), np.int64))
        events = []
        see = None
        if self.see_gamma > 0:
            see = (T(self.see_gamma), T(math.sqrt(QE * self.see_t_ev / ME)))
        for sp in (0, 1):
            if self.P[sp] is None:
                continue
            sc = self.species(sp, T)
            ev = particles.push_species(self.P[sp], F, sc, self.geo, s, cfg.seed, T,
                                        Qs[sp], J, self.window_q, stats, implicit=self.implicit, see=see)
            events.extend(ev)
        Q = Qs[0] + Qs[1]
        if drive is not None:
            Et = self.etheta(th_old)                                        # Eq. et_reconstruct
            Jd = np.asarray(drive(th_old, Et), dtype=np.float64)
            J += Jd
            stats['p_ind'] += float(np.sum(Jd * Et))
        self._append(events, T)
        if self.sm_every > 0 and (s + 1) % self.sm_every == 0:
            ncell = self.geo.i_win * cfg.nr
            for sp in (0, 1):
                if self.P[sp] is None:
                    continue
                st_sm, self.next_uid[sp] = control.split_merge(self.P[sp], sp, s, cfg.seed, ncell, *self.sm,
                                                               self.next_uid[sp], T)
                for key in st_sm:
                    self.sm_stats[key] += st_sm[key]
        # Poisson at t_{s+1}
        th_new = self.theta(s + 1)
        chi = self.susceptibility(Qs, T) if self.implicit else None
        self.phi = self.solve_potential(Q + self.window_q, th_new, chi)
        Qk = fields.turn_charge(g, self.phi, self.geo.turn_nodes, chi=chi)
        self.chi_last = chi
        Vk = self.turn_potentials(th_new)
        # accumulations (Eq. fourier, Eq. pind, Eq. pcap samples)
        N = self.n_rf
        with np.errstate(divide='ignore', invalid='ignore'):
            Jd = np.where(self.geo.vol > 0, J / np.where(self.geo.vol > 0, self.geo.vol, 1.0), 0.0)
        self.Jc += (2.0 / N) * Jd * math.cos(th_old)
        self.Js += (2.0 / N) * Jd * math.sin(th_old)
        self.Qc += (2.0 / N) * Qk * math.cos(th_new)
        self.Qs += (2.0 / N) * Qk * math.sin(th_new)
        for h in self.harm:
            m = h["m"]
            h["Jc"] += (2.0 / N) * Jd * math.cos(m * th_old)
            h["Js"] += (2.0 / N) * Jd * math.sin(m * th_old)
            h["Qc"] += (2.0 / N) * Qk * math.cos(m * th_new)
            h["Qs"] += (2.0 / N) * Qk * math.sin(m * th_new)
        self.p_ind += stats['p_ind'] / N
        self.p_es += stats['p_es'] / N
        self.samples_V.append(Vk)
        self.samples_Q.append(Qk)
        self.n_samples += 1
        self.pushed += stats['pushed']
        self.coll += stats['coll']
        self.absorbed += stats['absorbed']
        n_see = sum(1 for e in events if e['kind'] == 1)
        self.created += len(events) - n_see
        self.see_emitted += n_see
        self.s += 1
        self.Q_last = Q
        info = dict(stats=stats, events=len(events), see=n_see, Q=Q, J=J, Qk=Qk, Qs=Qs)
        if self.s % N == 0:
            info['record'] = self.period_end()
        return info

    def _append(self, events, T):
        """Creation events: ionisations (kind 0) give an electron and an ion,
        secondary emissions (kind 1) an electron; ordered by (kind, parent
        uid), numbered in that order per species."""
        events = sorted(events, key=lambda e: (e['kind'], e['parent']))
        if not events:
            return
        for sp in (0, 1):
            evs = events if sp == 0 else [e for e in events if e['kind'] == 0]
            n = len(evs)
            if n == 0:
                continue
            P = self.P[sp]
            uid0 = self.next_uid[sp]
            new = dict(cell=np.array([e['cell'] for e in evs], np.int64),
                       dr=np.array([e['dr'] for e in evs], T),
                       dz=np.array([e['dz'] for e in evs], T),
                       vr=np.array([(e['ve'] if sp == 0 else e['vi'])[0] for e in evs], T),
                       vt=np.array([(e['ve'] if sp == 0 else e['vi'])[1] for e in evs], T),
                       vz=np.array([(e['ve'] if sp == 0 else e['vi'])[2] for e in evs], T),
                       w=np.array([e['w'] for e in evs], T),
                       uid=np.arange(uid0, uid0 + n, dtype=np.int64))
            for key in P:
                P[key] = np.concatenate([P[key], new[key].astype(P[key].dtype)])
            self.next_uid[sp] = uid0 + n

    # ------------------------------------------------------------------------
    def _reset_accumulators(self):
        g = self.g
        self.Jc = np.zeros((g.NZ, g.NR))
        self.Js = np.zeros((g.NZ, g.NR))
        self.Qc = np.zeros(self.N)
        self.Qs = np.zeros(self.N)
        self.p_ind = 0.0
        self.p_es = 0.0
        self.samples_V = []
        self.samples_Q = []
        self.n_samples = 0
        self.pushed = 0
        self.coll = np.zeros((2, 3), np.int64)
        self.absorbed = 0
        self.created = 0
        for h in getattr(self, "harm", []):
            h["Jc"] = np.zeros((g.NZ, g.NR))
            h["Js"] = np.zeros((g.NZ, g.NR))
            h["Qc"] = np.zeros(self.N)
            h["Qs"] = np.zeros(self.N)

    def _compose_h(self, h):
        """Eq. compose and the B phasors at harmonic m (Faraday's law at m w)."""
        I = h["x"][1:1 + self.N]
        h["Ec"] = h["Ecp"] + np.tensordot(-I.imag, h["U"], axes=1)
        h["Ess"] = h["Essp"] + np.tensordot(I.real, h["U"], axes=1)
        h["Brc"], h["Brs"], h["Bzc"], h["Bzs"] = fields.b_phasors(self.g, h["Ec"], h["Ess"], h["omega"])

    def _compose(self):
        """Eq. compose with I_k = I_c - i I_s, and the B phasors."""
        I = self.x[1:1 + self.N]
        self.Ec = self.Ecp + np.tensordot(-I.imag, self.U, axes=1)
        self.Ess = self.Essp + np.tensordot(I.real, self.U, axes=1)
        self.Brc, self.Brs, self.Bzc, self.Bzs = fields.b_phasors(self.g, self.Ec, self.Ess,
                                                                  self.omega)

    def period_end(self):
        cfg, N = self.cfg, self.N
        # plasma-only Helmholtz solves (Eq. helmholtz_two_real)
        rhs_c = MU0 * self.omega * self.Js
        rhs_s = MU0 * self.omega * self.Jc
        Ecp = self.helm.solve(rhs_c)
        Essp = self.helm.solve(rhs_s)
        vp = -(fields.project(self.g, self.geo.gk, Ecp) +
               1j * fields.project(self.g, self.geo.gk, Essp))          # Eq. vpind
        qhat = self.Qc - 1j * self.Qs
        icap = 1j * self.omega * qhat                                     # Eq. icap
        accepted = self.n_samples == self.n_rf
        x_app = self.x.copy()
        p_port = circuit.port_power(x_app, N)
        p_cu = circuit.copper_power(x_app, N, self.r_rf)
        p_cap, W = circuit.cap_power_trapezoid(np.array(self.samples_V), np.array(self.samples_Q),
                                               cfg.freq)
        p_cap_ph = circuit.cap_power_phasor(x_app, N, icap)
        # the retained harmonics: V_p^(m), I_cap^(m) = i m w Q^(m), and their
        # port, copper and capacitive powers
        hrec = []
        for h in self.harm:
            wm = h["omega"]
            Ecp_m = h["helm"].solve(MU0 * wm * h["Js"])
            Essp_m = h["helm"].solve(MU0 * wm * h["Jc"])
            vp_m = -(fields.project(self.g, self.geo.gk, Ecp_m) +
                     1j * fields.project(self.g, self.geo.gk, Essp_m))
            qhat_m = h["Qc"] - 1j * h["Qs"]
            icap_m = 1j * wm * qhat_m
            xa = h["x"].copy()
            p_port += circuit.port_power(xa, N)
            p_cu += circuit.copper_power(xa, N, h["r_rf"])
            p_cap_ph += circuit.cap_power_phasor(xa, N, icap_m)
            hrec.append(dict(m=h["m"], vp=vp_m, icap=icap_m, qhat=qhat_m, x_applied=xa,
                             Ecp=Ecp_m, Essp=Essp_m))
        vg_applied = self.vg_amp
        rec = dict(period=self.s // self.n_rf - 1, n_samples=self.n_samples, accepted=accepted,
                   vp=vp, icap=icap, qhat=qhat, x_applied=x_app, vg=vg_applied,
                   p_port=p_port, p_cu=p_cu, p_cap=p_cap, p_cap_ph=p_cap_ph,
                   p_ind=self.p_ind, p_es=self.p_es, pushed=self.pushed,
                   coll=self.coll.copy(), absorbed=self.absorbed, created=self.created,
                   n_live=[int(np.count_nonzero(self.P[sp]['cell'] >= 0)) for sp in (0, 1)])
        rec['eps_bal'] = abs(p_port - (self.p_ind + p_cap + p_cu)) / max(abs(p_port), 1e-300)
        if accepted:
            if self.ctrl is not None:
                self.vg_amp = self.ctrl.update(self.vg_amp, p_port)
                self.vg = self.vg_amp * complex(math.cos(cfg.phase_g), math.sin(cfg.phase_g))
            xt = circuit.solve_target(self.A, self.vg, icap, vp)
            self.x = (1.0 - cfg.alpha) * self.x + cfg.alpha * xt
            rec['x_target'] = xt
            self.Ecp, self.Essp = Ecp, Essp
            self._compose()
            for h, hr in zip(self.harm, hrec):
                xt_m = circuit.solve_target(h["A"], 0.0, hr["icap"], hr["vp"])   # no source at m w
                h["x"] = (1.0 - cfg.alpha) * h["x"] + cfg.alpha * xt_m
                h["Ecp"], h["Essp"] = hr["Ecp"], hr["Essp"]
                self._compose_h(h)
        rec['x_next'] = self.x.copy()
        rec['vg_next'] = self.vg_amp
        rec['r_kcl'], rec['r_kvl'] = circuit.residuals(self.x, self.zs, self.zturn, self.c_stray,
                                                       self.omega, self.vg, icap, vp)
        for h, hr in zip(self.harm, hrec):
            hr['x_next'] = h["x"].copy()
            hr['r_kcl'], hr['r_kvl'] = circuit.residuals(h["x"], h["zs"], h["zturn"], self.c_stray, h["omega"],
                                                         0.0, hr["icap"], hr["vp"],
                                                         v_scale=float(np.max(np.abs(h["x"][1 + N:]))))
            del hr['Ecp'], hr['Essp']
        rec['harmonics'] = hrec
        self._reset_accumulators()
        # phi at the cycle boundary with the new turn potentials
        self.phi = self.solve_potential(self.Q_last + self.window_q, self.theta(self.s), self.chi_last)
        self.records.append(rec)
        return rec
