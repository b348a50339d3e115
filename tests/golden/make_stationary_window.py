"""Writes tests/golden/stationary_window_small.txt: the oracle's per-period
records of a small cell (the small workload's geometry, gas, 2e4
macroparticles per species and fixed 300 V source, on 64 x 96 cells at an
initial density of 3e15 m^-3, where its population levels off) in the
direct-implicit form, for the GPU's stationary-window parity test
(period-averaged circuit phasors and absorbed powers).

Calls only the oracle (and the shared seeded input generators).  The run is
the oracle's float32 instantiation, the one whose arithmetic the fused GPU
kernel follows, from the seeded populations; each completed period's
record (Sec. 2.5: P_port, P_ind, P_cap, P_Cu of Eqs. pport, pind, pcap and
the applied circuit state) becomes one row.

    python tests/golden/make_stationary_window.py [periods]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.cell import OracleCell                     # noqa: E402
from paper_2609_15043_b300 import workloads            # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "stationary_window_small.txt")


def window_cell():
    return workloads.small().replace(nr=64, nz=96, density=3e15, implicit_es=1)


def main():
    periods = int(sys.argv[1]) if len(sys.argv) > 1 else 80
    cfg = window_cell()
    w = workloads.macro_weight(cfg)
    oc = OracleCell(cfg, [w, w])
    for sp in (0, 1):
        p = workloads.population(cfg, sp)
        oc.set_particles(sp, p["cell"].astype(np.int64), p["dr"].astype(np.float32), p["dz"].astype(np.float32),
                         p["vr"].astype(np.float32), p["vt"].astype(np.float32), p["vz"].astype(np.float32),
                         p["uid"])
    oc.prime(np.float32)
    n = len(cfg.turn_r)
    # the file grows by one row per completed period, so a long run can be
    # stopped and its rows used
    with open(OUT, "w") as f:
        f.write("# Oracle records of a small cell (64x96 cells, 2e4 macroparticles per species, n0 = 3e15 m^-3,\n")
        f.write("# fixed 300 V source, direct-implicit electrostatics, float32 instantiation, seeded populations), one row\n")
        f.write("# per completed RF period (Sec. 2.5): period p_port p_ind p_cap p_cu |x_1| .. |x_%d| (W, A, V)\n"
                % (2 * n + 1))
        f.write("# written by tests/golden/make_stationary_window.py %d\n" % periods)
    done = 0
    t0 = time.time()
    while done < periods:
        info = oc.step(np.float32)
        rec = info.get("record")
        if rec is None:
            continue
        done += 1
        x = np.abs(np.asarray(rec["x_applied"]))
        row = [rec["p_port"], rec["p_ind"], rec["p_cap"], rec["p_cu"]] + list(x)
        with open(OUT, "a") as f:
            f.write("p %d " % done + " ".join("%.10e" % v for v in row) + "\n")
        print("period %d  %.0f s  p_ind %.4f  live %s" % (done, time.time() - t0, rec["p_ind"], rec["n_live"]),
              flush=True)


if __name__ == "__main__":
    main()
