"""Failure detection of the persistent kernels' grid barriers, exercised without a
fault: a barrier that one block never reaches gives up after its bounded wait,
the host reads AFC_E_TIMEOUT from the barrier state, and the context stays usable
(a CN step with the persistent BiCGStab afterwards matches one before)."""
import numpy as np
import pytest

from paper_2110_15676_gb300 import workloads as W
from pairs import gpu_problem

pytestmark = pytest.mark.gpu


def _cn_steps(afc, wl, steps=2):
    g = gpu_problem(wl.elem, wl.n, wl.b, wl.eps, wl.c, wl.f, wl.dir_mask, wl.u_dir)
    g.set_solution(wl.u0)
    dt = g.cfl_timestep(1.0)
    for _ in range(steps):
        g.step(afc.default_opts(scheme=afc.AFC_CN_NONLINEAR, dt=dt))
    u = g.get_solution()
    g.close()
    return u


@pytest.mark.parametrize("limit_ms", [20.0, 200.0])
def test_expired_grid_wait_reports_timeout_and_context_survives(limit_ms):
    from paper_2110_15676_gb300 import afc
    wl = W.random_transient(np.random.default_rng(70), "q1", (12, 12))
    before = _cn_steps(afc, wl)
    status, waited = afc.selftest_grid_wait(limit_ms)
    assert status == afc.AFC_E_TIMEOUT
    assert waited >= 0.9 * limit_ms and waited < limit_ms + 2000.0
    after = _cn_steps(afc, wl)
    assert np.array_equal(before, after)
