"""The allocation-free Poisson entry point (pp_poisson_solve_noalloc) gives
the same potential as the allocating pp_poisson_solve.

This entry point serves callers that may not allocate device memory, such as
code recorded into a CUDA graph or a host program whose memory manager owns
the device; its scratch is a fixed array inside the library.  The check runs
two calls in a row with different inputs, so the second one also shows that
left-over contents of the shared scratch do not leak into a new solve.
Collected last (file name) so that a run stopping at the first failure has run
every other test first."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_poisson_matches_allocating_solve():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_15043_b300 import phasorpic as pp, workloads
    cfg = workloads.small().replace(n_init=1000)
    cell = pp.Cell(cfg)
    NZ, NR = cfg.nz + 1, cfg.nr + 1
    i_win = int(round(cfg.z_win_lo / (cfg.z_max / cfg.nz)))
    rng = np.random.default_rng(31)
    stream = torch.cuda.current_stream()
    for call in range(2):
        q = np.zeros((NZ, NR))
        q[1:i_win + 1, :NR - 1] = rng.normal(size=(i_win, NR - 1)) * 1e-12
        turn_phi = rng.normal(size=len(cfg.turn_r)) * 300.0
        phi_ref, _, _, rel = cell.poisson_solve(q, turn_phi)
        assert rel <= 1e-10
        d_q = torch.tensor(q.ravel(), dtype=torch.float64, device="cuda")
        d_t = torch.tensor(turn_phi, dtype=torch.float64, device="cuda")
        d_phi = torch.full((NZ * NR,), float("nan"), dtype=torch.float64, device="cuda")
        d_info = torch.zeros(2, dtype=torch.int32, device="cuda")
        cell.poisson_solve_noalloc(d_q.data_ptr(), d_t.data_ptr(), d_phi.data_ptr(), d_info.data_ptr(),
                                   stream.cuda_stream)
        torch.cuda.synchronize()
        info = d_info.cpu().numpy()
        assert info[1] == 1 and info[0] >= 1
        phi = d_phi.cpu().numpy().reshape(NZ, NR)
        # same refinement on the same inputs: equal to rounding
        assert np.max(np.abs(phi - phi_ref)) <= 1e-12 * np.max(np.abs(phi_ref))
    cell.close()
