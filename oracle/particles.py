"""Particle step of the PIC/MCC cycle: gather, cylindrical Boris push,
boundaries, null-collision MCC and area-weighted deposition.

The paper inherits its particle engine and does not specify it (Sec. 2.1,
Sec. 3.4); the step below is the explicit scheme the workload names, written
from the textbook methods:
  * gather/deposit: bilinear (area) weights in the cell-relative offsets
    (dr, dz) on the four nodes of the cell;
  * Boris rotation (Boris 1970) in the local Cartesian frame (x = r, y = theta,
    z), then the move in that frame, r' = |(r + dx, dy)|, and the velocity
    rotated by the angle between the old and new radial directions;
  * null-collision MCC (Vahedi & Surendra 1995, cited in Sec. 3.4): a particle
    is a candidate with probability P_null = 1 - exp(-nu_max dt) (uniform from
    Philox2x32-10); a candidate's process is chosen by comparing u * nu_max
    with the cumulative real frequencies (uniforms from Philox4x32-10).

Direct-implicit form (Sec. 2.3, Eq. poisson with chi; Langdon, Cohen &
Friedman 1983): the stored state is the predicted one, (x~^s, v~^{s-1/2}).
The electrostatic force of a step is applied implicitly at the new time level,
v^{s-1/2} = v~^{s-1/2} + (q/m) dt E^s(x~^s), x^s = x~^s + (q/m) dt^2 E^s(x~^s),
by the next step's particle pass, once E^s has been solved with the
susceptibility of the predicted populations (chi = sum_s q_s n_s (q_s/m_s)
dt^2 / (eps0 eps_r)).  The inductive E_theta and the RF B stay explicit
(the Boris step with E_r = E_z = 0); every field is gathered at the predicted
position.  The current moment is taken at the corrected position x^s; the
charge is deposited at the next predicted position, per species.

The step is written once over a dtype T.  With T = float32 every operation is
a single IEEE float32 operation in the order the kernels use, so integer
outcomes (cells, absorptions, collisions) are decided exactly as on the GPU;
with T = float64 it is the accuracy reference.  Transcendental functions
(cos/sin of scattering angles, log in Box-Muller) only shape continuous
values, never a decision of the same step.

Cross sections are this project's analytic rational functions of energy (a
reading: the paper gives none): thresholds 11.55 and 15.76 eV, magnitudes of
the right order for argon; they are not database fits.

Particle control (the GEC application of Sec. 3.4 runs with secondary-electron
emission and weighted split-merge, which the paper inherits and does not
define; readings):
  * per-particle relative weights w (P['w'], 1 when absent): a particle
    carries the charge q W_s w, with W_s the species' macro weight; every
    deposit, current moment and power sum uses (q W_s) w, rounded once in T,
    which equals q W_s exactly when w = 1;
  * ion-induced secondary emission: an Ar+ absorbed on the electrode, the side
    wall or the window emits one electron with probability gamma, decided by
    the first uniform of draw call 3 (keyed by the ion's uid and the step).
    The electron starts at the ion's last position inside the plasma (before
    the move or correction that took it out, at most one ion step from the
    surface), carries the ion's relative weight, and leaves with a half-space
    Maxwellian flux at temperature T_see: the normal speed is Rayleigh,
    v_s sqrt(-2 ln u_b), directed into the plasma, and the two tangential
    components are Gaussian, v_s sqrt(-2 ln u_c) (cos, sin)(2 pi u_d), with
    v_s = sqrt(e T_see / m_e).  On the window the departing electron leaves
    its positive charge on the surface as well (twice the ion's charge).
"""
import math
import numpy as np

from .constants import QE, ME, M_AR, KB, E_EXC, E_ION, EPS0
from . import philox

DEAD = -1


# ----------------------------------------------------------------------------
# cross sections (units: 1e-20 m^2 for electrons, 1e-19 m^2 for ions)
# ----------------------------------------------------------------------------
def sigma_e(x, T):
    """Electron-Ar elastic, excitation, ionisation at energy x (eV)."""
    x = np.asarray(x, T)
    one = T(1.0)
    y = x - T(0.23)
    y2 = y * y
    s_el = (T(0.1) + T(14.0) * y2 / (y2 + T(4.0))) / (one + x / T(50.0))
    ye = x - T(E_EXC)
    s_ex = np.where(x > T(E_EXC), T(1.2) * ye / (ye * ye / T(30.0) + ye + T(8.0)), T(0.0))
    yi = x - T(E_ION)
    s_iz = np.where(x > T(E_ION), T(3.0) * yi / (yi * yi / T(60.0) + yi + T(30.0)), T(0.0))
    return s_el.astype(T), s_ex.astype(T), s_iz.astype(T)


def sigma_i(x, T):
    """Ar+-Ar charge exchange and isotropic elastic at lab energy x (eV)."""
    x = np.asarray(x, T)
    sq = np.sqrt(x)
    one = T(1.0)
    s_cx = T(2.0) + T(3.0) / (one + sq)
    s_iso = T(1.0) + T(2.0) / (one + sq)
    return s_cx.astype(T), s_iso.astype(T)


def nu_max(n_gas):
    """Upper bounds of the total collision frequency, FP64, with a 5 % margin:
    electrons: max over x = 1000 k / 100000 eV, k = 0..100000;
    ions: at the relative speed of a 1 keV ion (sigma*g increases with g)."""
    k = np.arange(100001, dtype=np.float64)
    x = 1000.0 * k / 100000.0
    se, sx, si = sigma_e(x, np.float64)
    g = np.sqrt(2.0 * QE * x / ME)
    nu_e = np.max(n_gas * 1e-20 * (se + sx + si) * g) * 1.05
    gcap = math.sqrt(2.0 * QE * 1000.0 / M_AR)
    scx, siso = sigma_i(np.array([1000.0]), np.float64)
    nu_i = float(n_gas * 1e-19 * (scx[0] + siso[0]) * gcap) * 1.05
    return float(nu_e), nu_i


class SpeciesConstants:
    """Per-species constants, computed in FP64 and rounded once to T."""

    def __init__(self, cfg, sp, weight, T):
        q = -QE if sp == 0 else QE
        m = ME if sp == 0 else M_AR
        dr, dz = cfg.r_max / cfg.nr, cfg.z_max / cfg.nz
        n_gas = cfg.pressure_pa / (KB * cfg.t_gas)
        nue, nui = nu_max(n_gas)
        nu = nue if sp == 0 else nui
        self.T = T
        self.sp = sp
        self.q, self.m, self.w = q, m, weight
        self.qmh = T(q / m * cfg.dt / 2.0)
        # direct-implicit electrostatic kick (Sec. 2.3): velocity and
        # position response to E^{s} at the predicted position, per unit field
        self.qmd = T(q / m * cfg.dt)
        self.kres = T(q / m * cfg.dt * cfg.dt / dr)     # cells per (V/m), radial
        self.kzes = T(q / m * cfg.dt * cfg.dt / dz)     # cells per (V/m), axial
        self.chi_per_charge = q / m * cfg.dt * cfg.dt / EPS0   # FP64: chi = this * (charge / volume)
        self.dtr = T(cfg.dt / dr)
        self.dtz = T(cfg.dt / dz)
        self.qw = T(q * weight)
        self.numax = T(nu)
        self.pnull = T(-math.expm1(-nu * cfg.dt))
        self.ng = T(n_gas * (1e-20 if sp == 0 else 1e-19))
        self.ce = T(0.5 * m / QE)                      # v^2 -> eV
        self.inv_ce = T(QE / (0.5 * m))                # eV -> v^2
        self.loss = T(2.0 * ME / M_AR)
        self.vth_gas = T(math.sqrt(KB * cfg.t_gas / M_AR))


def bilinear(dr, dz, T):
    one = T(1.0)
    a = one - dr
    b = one - dz
    return a * b, dr * b, a * dz, dr * dz


def _gather(F, cell, w, comp):
    w00, w01, w10, w11 = w
    f = F[cell, comp]
    return w00 * f[:, 0] + w01 * f[:, 1] + w10 * f[:, 2] + w11 * f[:, 3]


def _iso_dir(u2, u3, T):
    """Uniform direction on the sphere: cos(chi) = 1 - 2 u2, phi = 2 pi u3."""
    c = T(1.0) - T(2.0) * u2
    s = np.sqrt(np.maximum(T(1.0) - c * c, T(0.0)))
    ang = 2.0 * np.pi * u3.astype(np.float64)
    cp = np.cos(ang).astype(T)
    spn = np.sin(ang).astype(T)
    return s * cp, s * spn, c


def _gauss3(ua, ub, uc, ud, T):
    """Three standard normals by Box-Muller from four uniforms."""
    ra = np.sqrt(-2.0 * np.log(ua.astype(np.float64)))
    rc = np.sqrt(-2.0 * np.log(uc.astype(np.float64)))
    angb = 2.0 * np.pi * ub.astype(np.float64)
    angd = 2.0 * np.pi * ud.astype(np.float64)
    return ((ra * np.cos(angb)).astype(T), (ra * np.sin(angb)).astype(T),
            (rc * np.cos(angd)).astype(T))


def _carry(i, f, T):
    """Integer cell carry of an offset f (cells) added to cell index i: the
    offset is brought back into [0, 1) (a rounding to exactly 1 moves on)."""
    one = T(1.0)
    k = np.clip(np.floor(f), T(-1048576.0), T(1048576.0))       # beyond this: outside anyway
    f = (f - k).astype(T)
    i = i + k.astype(np.int64)
    fix = f >= one
    f = np.where(fix, f - one, f).astype(T)
    return i + fix, f


def _window_charge(window_q, ir2, drn, qd, i_win, nr, T):
    """Permanent window charge of particles absorbed on the window surface:
    linear weights in R on the surface nodes; qd is the charge each one
    leaves (T)."""
    one = T(1.0)
    rpos = ir2.astype(T) + drn
    j0 = np.floor(rpos).astype(np.int64)
    f = (rpos - j0.astype(T)).astype(T)
    qd = np.asarray(qd, T)
    np.add.at(window_q, (np.full(j0.shape, i_win), j0), (qd * (one - f)).astype(np.float64))
    np.add.at(window_q, (np.full(j0.shape, i_win), np.minimum(j0 + 1, nr)), (qd * f).astype(np.float64))


def secondary_electrons(uid, surface, ir, iz, dr, dz, w, step, seed, see, T, nr):
    """Ion-induced secondary emission (module docstring) for absorbed ions:
    uid, surface (0 electrode, 1 side wall, 2 window), the ions' last
    positions inside the plasma (ir, iz, dr, dz), their relative weights w;
    see = (gamma, v_s) in T.  Returns the mask of ions that emit and the
    emission events (kind 1: an electron only)."""
    gamma, vs = see
    a, b, c, d = philox.draws(uid, step, 3, 1, seed, T)
    emit = a < gamma
    events = []
    if np.any(emit):
        rn = np.sqrt(-2.0 * np.log(b.astype(np.float64))).astype(T)
        rt = np.sqrt(-2.0 * np.log(c.astype(np.float64)))
        ang = 2.0 * np.pi * d.astype(np.float64)
        vn = (vs * rn).astype(T)
        t1 = (vs * (rt * np.cos(ang)).astype(T)).astype(T)
        t2 = (vs * (rt * np.sin(ang)).astype(T)).astype(T)
        for q in np.nonzero(emit)[0]:
            if surface[q] == 0:          # electrode z = 0: into +z
                ve = (t1[q], t2[q], vn[q])
            elif surface[q] == 1:        # side wall r = R: into -r
                ve = (-vn[q], t1[q], t2[q])
            else:                        # window z = z_win: into -z
                ve = (t1[q], t2[q], -vn[q])
            events.append(dict(kind=1, parent=int(uid[q]), cell=int(iz[q] * nr + ir[q]), dr=dr[q], dz=dz[q],
                               ve=ve, vi=None, w=w[q]))
    return emit, events


def _absorb(window_q, hit_e, hit_w, hit_d, ir_in, iz_in, dr_in, dz_in, ir_out, dr_out, uid, wrel, qwp, sc,
            geo, step, seed, see, T):
    """Boundary bookkeeping of the particles that left the plasma region:
    secondary emission for ions (positions _in: the last ones inside), and the
    window charge at the surface crossing (positions _out), doubled where the
    ion emitted.  Returns the emission events."""
    nr, i_win = geo.cfg.nr, geo.i_win
    hit = hit_e | hit_w | hit_d
    emit = np.zeros(hit.shape, bool)
    events = []
    if see is not None and sc.sp == 1 and np.any(hit):
        hi = np.nonzero(hit)[0]
        surf = np.where(hit_e[hi], 0, np.where(hit_w[hi], 1, 2))
        em, events = secondary_electrons(uid[hi], surf, ir_in[hi], iz_in[hi], dr_in[hi], dz_in[hi], wrel[hi],
                                         step, seed, see, T, nr)
        emit[hi] = em
    if np.any(hit_d):
        qd = np.where(emit, qwp * T(2.0), qwp).astype(T)[hit_d]
        _window_charge(window_q, ir_out[hit_d], dr_out[hit_d], qd, i_win, nr, T)
    return events


def _implicit_correction(P, idx, ir, iz, dr, dz, vr, vz, Er, Ez, sc, geo, T, window_q, stats, wrel=None,
                         qwp=None, step=0, seed=0, see=None):
    """The implicit electrostatic kick of the previous step at the predicted
    position (v += (q/m) dt E, x += (q/m) dt^2 E).  A correction through the
    axis reflects (r -> -r, v_r -> -v_r); a correction out of the plasma region
    absorbs the particle there (window charge on the window surface, secondary
    emission from the position before the correction).
    Returns the corrected arrays, the mask of particles still alive and the
    emission events."""
    nr, i_win = geo.cfg.nr, geo.i_win
    if wrel is None:
        wrel = np.ones(idx.size, T)
        qwp = np.full(idx.size, sc.qw, T)
    vr_c = (vr + sc.qmd * Er).astype(T)
    vz_c = (vz + sc.qmd * Ez).astype(T)
    # electrostatic work of the kick with the mean of the pre- and post-kick velocities
    half = T(0.5)
    vbr = ((vr + vr_c) * half).astype(np.float64)
    vbz = ((vz + vz_c) * half).astype(np.float64)
    irc, drc = _carry(ir, (dr + sc.kres * Er).astype(T), T)
    izc, dzc = _carry(iz, (dz + sc.kzes * Ez).astype(T), T)
    neg = irc < 0
    if np.any(neg):
        rpos = (-(irc[neg].astype(T) + drc[neg])).astype(T)
        j = np.floor(rpos)
        irc[neg] = j.astype(np.int64)
        drc[neg] = (rpos - j).astype(T)
        vr_c[neg] = -vr_c[neg]
    hit_e = izc < 0
    hit_w = (~hit_e) & (irc >= nr)
    hit_d = (~hit_e) & (~hit_w) & (izc >= i_win)
    stats['absorbed'] += int(np.count_nonzero(hit_e | hit_w | hit_d))
    events = _absorb(window_q, hit_e, hit_w, hit_d, ir, iz, dr, dz, irc, drc, P['uid'][idx], wrel, qwp, sc,
                     geo, step, seed, see, T)
    alive = ~(hit_e | hit_w | hit_d)
    stats['p_es'] += float(np.sum(qwp[alive].astype(np.float64) * (vbr[alive] * Er[alive].astype(np.float64) +
                                                                   vbz[alive] * Ez[alive].astype(np.float64))))
    P['cell'][idx[~alive]] = DEAD
    P['dr'][idx[~alive]] = T(0.0)
    P['dz'][idx[~alive]] = T(0.0)
    return irc, izc, drc, dzc, vr_c, vz_c, alive, events


def push_species(P, F, sc, geo, step, seed, T, Q, J, window_q, stats, implicit=False, see=None):
    """Advance one species one step in place.

    P: dict with int64 'cell' (DEAD when absorbed), T arrays 'dr','dz','vr',
       'vt','vz', int64 'uid'.
    F: (n_plasma_cells, 5, 4) T array of node fields per cell (Er, Ez, Et, Br,
       Bz at corners 00, 01, 10, 11).
    Q, J: FP64 node grids receiving the charge (C) at the new positions and the
       current moment q w vbar_theta (A m) at the old positions.
    window_q: FP64 node grid of the permanent window surface charge.
    implicit: the direct-implicit form (module docstring): the stored state is
       the predicted one; the gathered E_r, E_z are applied as the previous
       step's implicit kick, the Boris step carries E_theta and B only, J is
       taken at the corrected position and Q at the next predicted one.
    see: (gamma, v_s) in T to let absorbed ions emit secondary electrons, or
       None.
    P may carry relative weights 'w' (module docstring; 1 when absent).
    Returns the list of creation events: ionisations (kind 0, from electrons)
    and secondary emissions (kind 1, from ions).
    """
    nr = geo.cfg.nr
    i_win = geo.i_win
    live = P['cell'] >= 0
    idx = np.nonzero(live)[0]
    cell = P['cell'][idx]
    ir = cell % nr
    iz = cell // nr
    dr, dz = P['dr'][idx], P['dz'][idx]
    vr, vt, vz = P['vr'][idx], P['vt'][idx], P['vz'][idx]
    one, half, zero = T(1.0), T(0.5), T(0.0)
    wrel = P['w'][idx].astype(T) if 'w' in P else np.ones(idx.size, T)
    qwp = (sc.qw * wrel).astype(T)          # = sc.qw exactly when w = 1
    events = []

    # --- gather at the old position ------------------------------------------
    w = bilinear(dr, dz, T)
    Er = _gather(F, cell, w, 0)
    Ez = _gather(F, cell, w, 1)
    Et = _gather(F, cell, w, 2)
    Br = _gather(F, cell, w, 3)
    Bz = _gather(F, cell, w, 4)
    n_entry = int(idx.size)

    if implicit:
        ir, iz, dr, dz, vr, vz, ok, ev = _implicit_correction(P, idx, ir, iz, dr, dz, vr, vz, Er, Ez, sc, geo,
                                                             T, window_q, stats, wrel, qwp, step, seed, see)
        events.extend(ev)
        idx, ir, iz, dr, dz, vr, vt, vz = (a[ok] for a in (idx, ir, iz, dr, dz, vr, vt, vz))
        wrel, qwp = wrel[ok], qwp[ok]
        Et, Br, Bz = Et[ok], Br[ok], Bz[ok]
        cell = iz * nr + ir
        w = bilinear(dr, dz, T)             # current moment at the corrected position
        Er = np.zeros_like(Et)
        Ez = np.zeros_like(Et)

    # --- Boris in the local frame (x = r, y = theta, z); B_theta = 0 ----------
    hx, hy, hz = sc.qmh * Er, sc.qmh * Et, sc.qmh * Ez
    vmx, vmy, vmz = vr + hx, vt + hy, vz + hz
    tx, tz = sc.qmh * Br, sc.qmh * Bz
    t2 = tx * tx + tz * tz
    sf = T(2.0) / (one + t2)
    sx, sz = tx * sf, tz * sf
    v1x = vmx + vmy * tz
    v1y = vmy + (vmz * tx - vmx * tz)
    v1z = vmz - vmy * tx
    vpx = vmx + v1y * sz
    vpy = vmy + (v1z * sx - v1x * sz)
    vpz = vmz - v1y * sx
    vnx, vny, vnz = vpx + hx, vpy + hy, vpz + hz

    # --- current moment at the old position with the time-centred velocity ----
    vbt = (vt + vny) * half
    vbr = (vr + vnx) * half
    vbz = (vz + vnz) * half
    jm = qwp * vbt
    for (di, dj), wk in zip(((0, 0), (0, 1), (1, 0), (1, 1)), w):
        np.add.at(J, (iz + di, ir + dj), (jm * wk).astype(np.float64))
    stats['p_ind'] += float(np.sum(jm.astype(np.float64) * Et.astype(np.float64)))
    if not implicit:
        stats['p_es'] += float(np.sum(qwp.astype(np.float64) *
                                      (vbr.astype(np.float64) * Er.astype(np.float64) +
                                       vbz.astype(np.float64) * Ez.astype(np.float64))))

    # --- move ------------------------------------------------------------------
    a = vnx * sc.dtr
    b = vny * sc.dtr
    c = vnz * sc.dtz
    rho = ir.astype(T) + dr
    x1 = rho + a
    rp = np.sqrt(x1 * x1 + b * b)
    den = rho + rp
    with np.errstate(divide='ignore', invalid='ignore'):
        delta = np.where(den > zero, (a * (rho + x1) + b * b) / den, zero).astype(T)
        inv = np.where(rp > zero, one / rp, zero).astype(T)
        ca = np.where(rp > zero, x1 * inv, one).astype(T)
        sa = np.where(rp > zero, b * inv, zero).astype(T)
    vr2 = np.where(rp > zero, ca * vnx + sa * vny, vnx).astype(T)
    vt2 = np.where(rp > zero, ca * vny - sa * vnx, vny).astype(T)
    drn = dr + delta
    dzn = dz + c
    kr = np.clip(np.floor(drn), T(-1048576.0), T(1048576.0))     # beyond this: outside anyway
    drn = (drn - kr).astype(T)
    ir2 = ir + kr.astype(np.int64)
    fix = drn >= one
    drn = np.where(fix, drn - one, drn).astype(T)
    ir2 = ir2 + fix
    kz = np.clip(np.floor(dzn), T(-1048576.0), T(1048576.0))
    dzn = (dzn - kz).astype(T)
    iz2 = iz + kz.astype(np.int64)
    fix = dzn >= one
    dzn = np.where(fix, dzn - one, dzn).astype(T)
    iz2 = iz2 + fix
    neg = ir2 < 0
    ir2 = np.where(neg, 0, ir2)
    drn = np.where(neg, zero, drn).astype(T)

    # --- boundaries: electrode z<0, wall r>=R, window z>=z_win ---------------
    hit_e = iz2 < 0
    hit_w = (~hit_e) & (ir2 >= nr)
    hit_d = (~hit_e) & (~hit_w) & (iz2 >= i_win)
    stats['absorbed'] += int(np.count_nonzero(hit_e | hit_w | hit_d))
    events.extend(_absorb(window_q, hit_e, hit_w, hit_d, ir, iz, dr, dz, ir2, drn, P['uid'][idx], wrel, qwp,
                          sc, geo, step, seed, see, T))
    alive = ~(hit_e | hit_w | hit_d)

    # --- null-collision MCC at the new position -------------------------------
    uid = P['uid'][idx]
    u0 = philox.null_draw(uid, step, sc.sp, seed, T)
    _, u1, u2, u3 = philox.draws(uid, step, 0, sc.sp, seed, T)
    cand = alive & (u0 < sc.pnull)
    ci = np.nonzero(cand)[0]
    if ci.size:
        if sc.sp == 0:
            events.extend(_collide_electrons(ci, vr2, vt2, vnz, u1, u2, u3, uid, step, seed,
                                             sc, T, stats, ir2, iz2, drn, dzn, nr, wrel))
        else:
            _collide_ions(ci, vr2, vt2, vnz, u1, u2, u3, uid, step, seed, sc, T, stats)

    # --- charge at the new position -------------------------------------------
    ai = np.nonzero(alive)[0]
    wn = bilinear(drn[ai], dzn[ai], T)
    for (di, dj), wk in zip(((0, 0), (0, 1), (1, 0), (1, 1)), wn):
        np.add.at(Q, (iz2[ai] + di, ir2[ai] + dj), (qwp[ai] * wk).astype(np.float64))

    # --- write back ------------------------------------------------------------
    newcell = np.where(alive, iz2 * nr + ir2, DEAD)
    P['cell'][idx] = newcell
    P['dr'][idx] = np.where(alive, drn, zero)
    P['dz'][idx] = np.where(alive, dzn, zero)
    P['vr'][idx] = vr2
    P['vt'][idx] = vt2
    P['vz'][idx] = vnz
    stats['pushed'] += n_entry
    return events


def _collide_electrons(ci, vr, vt, vz, u1, u2, u3, uid, step, seed, sc, T, stats,
                       ir2, iz2, drn, dzn, nr, wrel):
    x, y, z = vr[ci], vt[ci], vz[ci]
    v2 = x * x + y * y + z * z
    g = np.sqrt(v2)
    en = v2 * sc.ce
    s_el, s_ex, s_iz = sigma_e(en, T)
    nu_el = sc.ng * s_el * g
    nu_ex = sc.ng * s_ex * g
    nu_iz = sc.ng * s_iz * g
    r = u1[ci] * sc.numax
    c1 = nu_el
    c2 = c1 + nu_ex
    c3 = c2 + nu_iz
    el = r < c1
    ex = (~el) & (r < c2)
    iz_ = (~el) & (~ex) & (r < c3)
    stats['coll'][0, 0] += int(np.count_nonzero(el))
    stats['coll'][0, 1] += int(np.count_nonzero(ex))
    stats['coll'][0, 2] += int(np.count_nonzero(iz_))
    stats['nu_viol'] += int(np.count_nonzero(c3 > sc.numax))
    dx, dy, dz = _iso_dir(u2[ci], u3[ci], T)
    one = T(1.0)
    # elastic: isotropic, energy loss 2m/M (1 - cos chi)
    with np.errstate(divide='ignore', invalid='ignore'):
        cosx = np.where(g > 0, (x * dx + y * dy + z * dz) / g, T(0.0)).astype(T)
    g_el = g * np.sqrt(one - sc.loss * (one - cosx))
    g_ex = np.sqrt(np.maximum(en - T(E_EXC), T(0.0)) * sc.inv_ce)
    e_half = np.maximum(en - T(E_ION), T(0.0)) * T(0.5)
    g_iz = np.sqrt(e_half * sc.inv_ce)
    gnew = np.where(el, g_el, np.where(ex, g_ex, g_iz)).astype(T)
    hit = el | ex | iz_
    sel = ci[hit]
    vr[sel] = (gnew * dx)[hit]
    vt[sel] = (gnew * dy)[hit]
    vz[sel] = (gnew * dz)[hit]
    events = []
    ii = np.nonzero(iz_)[0]
    if ii.size:
        p = ci[ii]
        a0, a1, a2, a3 = philox.draws(uid[p], step, 1, 0, seed, T)
        b0, b1, _, _ = philox.draws(uid[p], step, 2, 0, seed, T)
        ex_, ey_, ez_ = _iso_dir(a0, a1, T)
        ge = g_iz[ii]
        n0, n1, n2 = _gauss3(a2, a3, b0, b1, T)
        for q in range(ii.size):
            k = p[q]
            events.append(dict(kind=0, parent=int(uid[k]), cell=int(iz2[k] * nr + ir2[k]),
                               dr=drn[k], dz=dzn[k],
                               ve=(ge[q] * ex_[q], ge[q] * ey_[q], ge[q] * ez_[q]),
                               vi=(sc.vth_gas * n0[q], sc.vth_gas * n1[q], sc.vth_gas * n2[q]),
                               w=wrel[k]))
    return events


def _collide_ions(ci, vr, vt, vz, u1, u2, u3, uid, step, seed, sc, T, stats):
    a0, a1, a2, a3 = philox.draws(uid[ci], step, 1, 1, seed, T)
    n0, n1, n2 = _gauss3(a0, a1, a2, a3, T)
    vnx, vny, vnz = sc.vth_gas * n0, sc.vth_gas * n1, sc.vth_gas * n2
    x, y, z = vr[ci], vt[ci], vz[ci]
    gx, gy, gz = x - vnx, y - vny, z - vnz
    g2 = gx * gx + gy * gy + gz * gz
    g = np.sqrt(g2)
    en = g2 * sc.ce
    s_cx, s_iso = sigma_i(en, T)
    nu_cx = sc.ng * s_cx * g
    nu_iso = sc.ng * s_iso * g
    r = u1[ci] * sc.numax
    c1 = nu_cx
    c2 = c1 + nu_iso
    cx = r < c1
    iso = (~cx) & (r < c2)
    stats['coll'][1, 0] += int(np.count_nonzero(cx))
    stats['coll'][1, 1] += int(np.count_nonzero(iso))
    stats['nu_viol'] += int(np.count_nonzero(c2 > sc.numax))
    half = T(0.5)
    dx, dy, dz = _iso_dir(u2[ci], u3[ci], T)
    hg = g * half
    ix = (x + vnx) * half + hg * dx
    iy = (y + vny) * half + hg * dy
    iz_ = (z + vnz) * half + hg * dz
    nxv = np.where(cx, vnx, np.where(iso, ix, x)).astype(T)
    nyv = np.where(cx, vny, np.where(iso, iy, y)).astype(T)
    nzv = np.where(cx, vnz, np.where(iso, iz_, z)).astype(T)
    vr[ci], vt[ci], vz[ci] = nxv, nyv, nzv
