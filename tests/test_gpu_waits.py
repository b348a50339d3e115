"""Failure detection without a GPU fault: the library's bounded device waits
(an mbarrier phase that no copy completes, a global flag that no one sets)
expire on a condition that never comes true, report PP_ST_TIMEOUT to the
host, and leave the context usable for the next cell."""
import numpy as np
import pytest

from gpu_common import require_gpu, gpu_cell

pytestmark = pytest.mark.gpu


def test_bounded_waits_expire_and_the_context_survives():
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp, workloads
    st = pp.wait_selftest(1 << 14)
    assert st[0] & pp.ST_TIMEOUT and st[1] & pp.ST_TIMEOUT
    cfg = workloads.small()
    g = gpu_cell(cfg, [workloads.population(cfg, sp) for sp in (0, 1)])
    g.prime()
    g.advance_steps(5)
    assert g.status() == 0 and g.counters()["steps"] == 5
    g.close()
