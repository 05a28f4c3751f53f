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


def _split_inputs():
    """Doubles over the whole range the float pairs cover and its edges: random magnitudes
    from 1e-330 (subnormal doubles) to 2^127, values on and next to float roundings and
    rounding ties (hi and lo), the normal/subnormal float boundary, and signed zeros."""
    rng = np.random.default_rng(11)
    parts = [rng.uniform(-1, 1, 200000),
             rng.choice([-1.0, 1.0], 600000) * rng.uniform(1, 2, 600000) * 2.0 ** rng.uniform(-1100, 126.9, 600000)]
    f = np.float64(np.float32(rng.uniform(1, 2, 100000)))
    e = rng.integers(-160, 120, 100000).astype(np.float64)
    half = 2.0 ** -24                                       # half a float ulp of [1, 2)
    for k in (-1.0, 1.0):                                   # ties of hi, and next to them
        parts.append(np.ldexp(f + k * half, e.astype(int)))
        parts.append(np.ldexp(f + k * half * (1 + 2.0 ** -28), e.astype(int)))
    parts.append(np.ldexp(f + half * 2.0 ** -24 * rng.integers(-7, 8, 100000), e.astype(int)))   # lo ties
    b = np.array([2.0 ** -126, 2.0 ** -126 * (1 - 2.0 ** -30), 2.0 ** -126 * (1 + 2.0 ** -29), 2.0 ** -149,
                  2.0 ** -150, 3 * 2.0 ** -151, 2.0 ** -151, 2.0 ** -97, 2.0 ** -74, 2.0 ** -74 * (1 - 2.0 ** -40),
                  2.0 ** 127 * (1 - 2.0 ** -30), 5e-324, 0.0])
    parts.append(np.concatenate([b, -b]))
    x = np.concatenate(parts)
    return x[np.abs(x) < 2.0 ** 127]


def test_float_pair_split_and_widening_match_ieee():
    """The device's float-pair split (integer pipe) against IEEE round-to-nearest-even on the
    host: hi = float32(x) bit for bit, lo = float32(x - hi) in value (the sign of a zero low
    part is not specified), and the exact widening of hi back to double."""
    from paper_2110_15676_gb300 import afc
    x = _split_inputs()
    hi, lo, back = afc.selftest_split(x)
    with np.errstate(over="ignore"):
        hr = x.astype(np.float32)
        lr = (x - hr.astype(np.float64)).astype(np.float32)
    bad = np.flatnonzero(hi.view(np.uint32) != hr.view(np.uint32))
    assert bad.size == 0, (x[bad[:5]], hi[bad[:5]], hr[bad[:5]])
    bad = np.flatnonzero(lo != lr)
    assert bad.size == 0, (x[bad[:5]], lo[bad[:5]], lr[bad[:5]])
    assert np.array_equal(back, hi.astype(np.float64))
    assert np.array_equal(np.signbit(back), np.signbit(hi))
