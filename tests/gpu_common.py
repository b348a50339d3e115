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
