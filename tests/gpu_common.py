"""Shared helpers of the GPU parity tests (inputs from workloads, oracle and
CUDA path each run on them independently)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def oracle_cell(cfg, populations, T=np.float32):
    from oracle.cell import OracleCell
    from paper_2609_15043_b300 import workloads
    w = workloads.macro_weight(cfg)
    c = OracleCell(cfg, [w, w])
    for sp in (0, 1):
        p = populations[sp]
        c.set_particles(sp, p["cell"].astype(np.int64), p["dr"].astype(T), p["dz"].astype(T),
                        p["vr"].astype(T), p["vt"].astype(T), p["vz"].astype(T), p["uid"])
    return c


def gpu_cell(cfg, populations, **kw):
    from paper_2609_15043_b300 import phasorpic as pp
    g = pp.Cell(cfg, **kw)
    for sp in (0, 1):
        g.set_particles(sp, populations[sp])
    return g


def by_uid(p):
    o = np.argsort(p["uid"])
    return {k: np.asarray(v)[o] for k, v in p.items()}


def oracle_live(P):
    live = P["cell"] >= 0
    return by_uid({k: v[live] for k, v in P.items()})


def check_step_potential(oc, g, tol_solve=1e-8, tol_oracle=1e-4, T=np.float32):
    """The step's Poisson solve on the GPU: its potential against the
    oracle's solve of the same operator (Eq. poisson, with the susceptibility
    of the GPU's own species charges in the direct-implicit form) applied to the
    GPU's deposited charges, to solver precision; and against the oracle's own
    step, to the bound that the float32 charge deposit allows (the net charge
    of a quasi-neutral plasma is a small difference of the species' charges)."""
    from paper_2609_15043_b300 import phasorpic as pp
    qe, qi = g.grid(pp.GRID_CHARGE_E), g.grid(pp.GRID_CHARGE_I)
    chi = oc.susceptibility([qe, qi], T) if oc.implicit else None
    ref = oc.solve_potential(qe + qi + g.grid(pp.GRID_WINDOW), oc.theta(oc.s), chi)
    phi = g.grid(pp.GRID_PHI)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(phi - ref)) <= tol_solve * scale, np.max(np.abs(phi - ref)) / scale
    assert np.max(np.abs(phi - oc.phi)) <= tol_oracle * np.max(np.abs(oc.phi))
