"""Failure detection of the persistent kernels' grid barriers, exercised without a
fault: a barrier that one block never reaches gives up after its bounded wait,
the host reads AFC_E_TIMEOUT from the barrier state, and the context stays usable
(a CN step with the persistent BiCGStab afterwards matches one before); and a CN
step whose solver barriers have a zero wait limit reports AFC_E_TIMEOUT and leaves
a clean barrier state behind."""
import numpy as np
import pytest

from paper_2110_15676_gb300 import workloads as W
from pairs import gpu_problem

pytestmark = pytest.mark.gpu


def _cn_steps(afc, wl, steps=2, graph=1):
    g = gpu_problem(wl.elem, wl.n, wl.b, wl.eps, wl.c, wl.f, wl.dir_mask, wl.u_dir)
    g.set_solution(wl.u0)
    dt = g.cfl_timestep(1.0)
    for _ in range(steps):
        g.step(afc.default_opts(scheme=afc.AFC_CN_NONLINEAR, dt=dt, graph=graph))
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


@pytest.mark.parametrize("graph", [1, 0])
def test_solver_barrier_timeout_is_reported_and_cleared(graph):
    """A CN step whose persistent BiCGStab barriers are given a zero wait limit: the
    first block that finds a barrier still closed gives up at once, the launch ends,
    and afc_step reports AFC_E_TIMEOUT, in the graph (device-side loop) and in the
    host-driven loop alike.  The barrier state is cleared, so the same problem with
    the default limit then steps exactly as a fresh one does."""
    from paper_2110_15676_gb300 import afc
    wl = W.rotating_transient("q1", 33)
    ref = _cn_steps(afc, wl, graph=graph)
    g = gpu_problem(wl.elem, wl.n, wl.b, wl.eps, wl.c, wl.f, wl.dir_mask, wl.u_dir)
    dt = g.cfl_timestep(1.0)
    opts = afc.default_opts(scheme=afc.AFC_CN_NONLINEAR, dt=dt, graph=graph)
    g.set_solution(wl.u0)
    g.set_grid_wait_limit(0.0)
    with pytest.raises(afc.AfcError) as e:
        g.step(opts)
    assert e.value.status == afc.AFC_E_TIMEOUT
    with pytest.raises(afc.AfcError):
        g.set_grid_wait_limit(4001.0)
    g.set_grid_wait_limit(4000.0)
    g.set_solution(wl.u0)
    for _ in range(2):
        g.step(opts)
    assert np.array_equal(g.get_solution(), ref)
    g.close()
