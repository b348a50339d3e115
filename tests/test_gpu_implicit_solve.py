"""The direct-implicit Poisson solve (Sec. 2.3, Eq. poisson with the
susceptibility, Eq. epseff) on grids that take each of the cluster solve's
shared-memory plans: the radial eigenbasis and the CG vectors in shared
memory (32 and 80 radial nodes), both in global memory (192), and the largest
grid the solve takes (256 radial nodes, 383 interior rows).  After two PIC
steps (the second starts from the extrapolated potential) the GPU's
potential is compared with the oracle's sparse direct solve of the same
operator on the GPU's own deposited charges."""
import numpy as np
import pytest

from gpu_common import require_gpu, gpu_cell

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nr,nz", [(32, 48), (80, 120), (192, 288), (256, 384)])
def test_implicit_solve_on_each_plan(nr, nz):
    require_gpu()
    from oracle.cell import OracleCell
    from paper_2609_15043_b300 import phasorpic as pp, workloads
    # about 40 macroparticles per plasma cell and species: the susceptibility's
    # particle noise stays near the bench workload's
    cfg = workloads.cell60().replace(nr=nr, nz=nz, n_init=35 * nr * nz, implicit_es=1, power_control=0)
    pops = [workloads.population(cfg, sp) for sp in (0, 1)]
    g = gpu_cell(cfg, pops)
    g.prime()
    g.advance_steps(2)
    assert g.status() == 0
    w = workloads.macro_weight(cfg)
    oc = OracleCell(cfg, [w, w])
    qe, qi = g.grid(pp.GRID_CHARGE_E), g.grid(pp.GRID_CHARGE_I)
    chi = oc.susceptibility([qe, qi], np.float32)
    assert np.max(chi) > 0.1          # the susceptibility matters on this grid
    ref = oc.solve_potential(qe + qi + g.grid(pp.GRID_WINDOW), oc.theta(2), chi)
    phi = g.grid(pp.GRID_PHI)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(phi - ref)) <= 1e-8 * scale, np.max(np.abs(phi - ref)) / scale
    rel = g.poisson_stats()
    assert rel[rel > 0][-1] <= 1e-10
    assert g.poisson_evaluations() <= 60
    g.close()
