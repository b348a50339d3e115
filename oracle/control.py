"""Stochastic weighted split-merge particle control (oracle; test
infrastructure only).

The GEC application of Sec. 3.4 keeps the macroparticle count of every cell
near a target with a weighted split-merge module that the paper inherits and
does not define.  The reading written here (the same one the CUDA path
implements) is the plain stochastic form:

  * a pass runs after the step's creation events are appended, every
    `sm_every` steps (after step s with (s + 1) % sm_every == 0), for each
    species separately;
  * the live particles of a cell are taken in increasing uid order;
  * a cell with n > n_max particles merges k = min(n - target, n // 2)
    disjoint pairs, the (2j, 2j + 1)-th particles of that order (j < k): the
    pair (a, b) becomes one particle of weight w_a + w_b (rounded once in T)
    whose state (position, velocity, uid) is a's when u (w_a + w_b) < w_a and
    b's otherwise, u the first uniform of draw call 5 keyed by a's uid, the
    step and the species.  The other member is removed.  Charge is conserved
    to the rounding of the sum, momentum and energy in expectation;
  * a cell with 0 < n < n_min particles splits its first k = min(target - n,
    n) particles: each keeps its state with half its weight, and a copy with
    the same state and weight is created.  Charge, momentum and energy are
    conserved exactly;
  * cells with more than CELL_CAP particles are left alone (counted);
  * created copies are numbered next_uid, next_uid + 1, ... in the order of
    their cells and, within a cell, of their originals.
"""
import numpy as np

from . import philox

DEAD = -1
CELL_CAP = 4096


def split_merge(P, sp, step, seed, ncell, target, n_min, n_max, next_uid, T):
    """One pass over species sp of the particle dict P (arrays cell, dr, dz,
    vr, vt, vz, w, uid; cell = DEAD for removed slots).  Returns (stats,
    next_uid) with stats = dict(split, merged, skipped)."""
    live = np.nonzero(P['cell'] >= 0)[0]
    order = live[np.lexsort((P['uid'][live], P['cell'][live]))]
    counts = np.bincount(P['cell'][order], minlength=ncell) if order.size else np.zeros(ncell, np.int64)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    stats = dict(split=0, merged=0, skipped=0)
    copies = []
    act = np.nonzero((counts > n_max) | ((counts > 0) & (counts < n_min)))[0]
    for c in act:
        n = int(counts[c])
        seg = order[starts[c]:starts[c] + n]
        if n > CELL_CAP:
            stats['skipped'] += 1
            continue
        if n > n_max:
            k = min(n - target, n // 2)
            a, b = seg[0:2 * k:2], seg[1:2 * k:2]
            wa, wb = P['w'][a].astype(T), P['w'][b].astype(T)
            ws = (wa + wb).astype(T)
            u = philox.draws(P['uid'][a], step, 5, sp, seed, T)[0]
            keep_a = (u * ws).astype(T) < wa
            surv = np.where(keep_a, a, b)
            gone = np.where(keep_a, b, a)
            P['w'][surv] = ws
            P['cell'][gone] = DEAD
            P['dr'][gone] = 0.0
            P['dz'][gone] = 0.0
            stats['merged'] += k
        else:
            k = min(target - n, n)
            src = seg[:k]
            P['w'][src] = (P['w'][src].astype(T) * T(0.5)).astype(T)
            copies.extend(int(x) for x in src)
            stats['split'] += k
    if copies:
        src = np.asarray(copies, np.int64)
        m = src.size
        for key in ('cell', 'dr', 'dz', 'vr', 'vt', 'vz', 'w'):
            P[key] = np.concatenate([P[key], P[key][src]])
        P['uid'] = np.concatenate([P['uid'], np.arange(next_uid, next_uid + m, dtype=P['uid'].dtype)])
        next_uid += m
    return stats, next_uid
