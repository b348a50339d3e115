"""Detection of a statistically stationary state from completed-period
records (host logic over pp_period_record values).

The paper judges convergence by the period-to-period behaviour of the turn
phasors and the power balance (Sec. 2.5, Sec. 4); this module fixes the test
as numbers.  The state is stationary at period n when, over the trailing
window of W periods ending at n:

  * with the power controller on, |mean(P_port) - P_target| / P_target <= tol_p;
  * the power balance of the window means,
        |P_port - (P_ind + P_cap + P_Cu)| / |P_port|  (Eq. power_imbalance),
    is <= tol_bal;
  * the means over the two halves of the window of P_port, P_ind, P_cap,
    P_Cu and of every |V_k|, |I_k| of the applied circuit state differ by at
    most tol_drift relative to the whole-window mean.

Quantities whose window mean is below `floor` times the largest power (or
phasor magnitude) are exempt from the relative drift test: a relative test
on a mean that is zero up to noise never passes.

With plasma_drift = False the drift test covers the circuit state only, not
the four powers: the state then counts as stationary when the power balance
holds within tol_bal (the coupled field-circuit state is converged), the
controller holds P_port and the circuit phasors have settled, while the
plasma's particle inventory may still relax on ion time scales (a density
set by the initial load that the target power cannot sustain decays over
thousands of periods).
"""
from dataclasses import dataclass
from typing import Optional

import numpy as np


@dataclass
class StationarityCriteria:
    window: int = 100
    tol_p: float = 0.01
    tol_bal: float = 0.005
    tol_drift: float = 0.005
    floor: float = 1e-3
    plasma_drift: bool = True


def _drift(series, floor_abs):
    """max over columns of |mean(first half) - mean(second half)| / |mean|,
    skipping columns whose mean magnitude is below floor_abs."""
    s = np.asarray(series, float)
    if s.ndim == 1:
        s = s[:, None]
    h = s.shape[0] // 2
    m = s.mean(axis=0)
    d = np.abs(s[:h].mean(axis=0) - s[h:].mean(axis=0))
    keep = np.abs(m) >= floor_abs
    if not np.any(keep):
        return 0.0
    return float(np.max(d[keep] / np.abs(m[keep])))


class StationarityMonitor:
    """Feed completed-period records (dicts from Cell.turn_phasors()) in
    order; `update` returns True from the first period at which the trailing
    window satisfies every criterion."""

    def __init__(self, n_turns, p_target=None, criteria: Optional[StationarityCriteria] = None):
        self.n = n_turns
        self.p_target = p_target
        self.c = criteria or StationarityCriteria()
        self.rows = []          # per period: p_port, p_ind, p_cap, p_cu
        self.mags = []          # per period: |x_applied| (2N+1 phasors)
        self.stationary_at = None
        self.last = {}

    def update(self, rec):
        self.rows.append([rec["p_port"], rec["p_ind"], rec["p_cap"], rec["p_cu"]])
        self.mags.append(np.abs(np.asarray(rec["x_applied"])))
        ok = self.check()
        if ok and self.stationary_at is None:
            self.stationary_at = len(self.rows) - 1
        return ok

    def window_means(self):
        """Means over the trailing window: the four powers (P_port, P_ind,
        P_cap, P_Cu) and the magnitudes of the applied circuit state."""
        W = min(self.c.window, len(self.rows))
        if W == 0:
            return None
        return {"p": np.asarray(self.rows[-W:]).mean(axis=0).tolist(),
                "x_abs": np.asarray(self.mags[-W:]).mean(axis=0).tolist(), "periods": W}

    def check(self):
        W = self.c.window
        if len(self.rows) < W:
            self.last = dict(periods=len(self.rows))
            return False
        P = np.asarray(self.rows[-W:])
        X = np.asarray(self.mags[-W:])
        m = P.mean(axis=0)
        p_port = m[0]
        bal = abs(p_port - (m[1] + m[2] + m[3])) / max(abs(p_port), 1e-300)
        pscale = max(np.max(np.abs(m)), 1e-300)
        drift_p = _drift(P, self.c.floor * pscale)
        drift_x = _drift(X, self.c.floor * max(np.max(X.mean(axis=0)), 1e-300))
        err_p = abs(p_port - self.p_target) / self.p_target if self.p_target else 0.0
        self.last = dict(periods=len(self.rows), err_p=err_p, bal=bal, drift_p=drift_p, drift_x=drift_x)
        return err_p <= self.c.tol_p and bal <= self.c.tol_bal and \
            (drift_p <= self.c.tol_drift or not self.c.plasma_drift) and drift_x <= self.c.tol_drift
