"""Batched explicit SSP steps (many independent instances per launch) against the
same instances run alone, and against the oracle.

An instance's arithmetic in a batch is the one of the single-problem kernels, so
a batched run must equal the solo run bit for bit, whatever the launch shape,
the tile size or the other instances.  FP64 runs follow the oracle within the
per-step tolerance; mixed runs (single-precision raw fluxes, Sec. 2.1.2 fluxes
with FP64 limiter sums and update) within 1e-6 of the FP64 oracle, with the
maximum principle of the Zalesak stage intact."""
import numpy as np
import pytest

from oracle import afc_oracle as O
from paper_2110_15676_gb300 import workloads as W
from pairs import gpu_problem, oracle_problem, relerr

pytestmark = pytest.mark.gpu

STEPS = 4


@pytest.fixture(scope="module")
def afc():
    from paper_2110_15676_gb300 import afc as A
    return A


def make_instances(seed, count, elems=("q1", "p1"), n_range=(6, 12)):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        wl = W.random_transient(rng, elems[q % len(elems)], n_range)
        out.append(wl)
    return out


def gpu_of(wl):
    g = gpu_problem(wl.elem, wl.n, wl.b, wl.eps, wl.c, wl.f, wl.dir_mask, wl.u_dir)
    g.set_solution(wl.u0)
    return g


def solo_runs(afc, wls, dts, scheme, precision, steps):
    out = []
    for wl, dt in zip(wls, dts):
        g = gpu_of(wl)
        opts = afc.default_opts(scheme=scheme, dt=dt, precision=precision)
        for _ in range(steps):
            g.step(opts)
        out.append(g.get_solution())
        g.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_solo_every_shape(afc, precision):
    wls = make_instances(3, 7)
    gs = [gpu_of(wl) for wl in wls]
    dts = [g.cfl_timestep(0.5) for g in gs]
    prec = afc.AFC_FP64 if precision == "fp64" else afc.AFC_MIXED
    ref = solo_runs(afc, wls, dts, afc.AFC_SSP3, prec, STEPS)
    opts = afc.default_opts(scheme=afc.AFC_SSP3, precision=prec)
    with afc.Batch(gs) as b:
        shapes = [(m, blk) for m in (afc.AFC_BATCH_PER_PASS, afc.AFC_BATCH_PER_STAGE, afc.AFC_BATCH_PER_STEP)
                  for blk in (128, 256, 512)]
        for mode, blk in shapes:
            for g, wl in zip(gs, wls):
                g.set_solution(wl.u0)
            b.set_tuning(mode, blk)
            stats = b.step(opts, dt=dts, nsteps=STEPS)
            for q, g in enumerate(gs):
                u = g.get_solution()
                assert np.array_equal(u, ref[q]), (mode, blk, q, np.abs(u - ref[q]).max())
                assert stats[q]["stages"] == 3 * STEPS
                assert stats[q]["umin"] == u.min() and stats[q]["umax"] == u.max()
        _, launches = b.info()
        assert launches > 0


@pytest.mark.parametrize("scheme", ["ssp2", "ssp3"])
def test_batch_fp64_vs_oracle(afc, scheme):
    wls = make_instances(11, 5)
    gs = [gpu_of(wl) for wl in wls]
    order = 2 if scheme == "ssp2" else 3
    os_ = [oracle_problem(wl.elem, wl.n, wl.b, wl.eps, wl.c, wl.f, wl.dir_mask, wl.u_dir) for wl in wls]
    dts = [O.cfl_timestep(o, 0.5) for o in os_]
    opts = afc.default_opts(scheme=afc.AFC_SSP2 if order == 2 else afc.AFC_SSP3)
    us = [wl.u0.copy() for wl in wls]
    with afc.Batch(gs) as b:
        for step in range(3):
            b.step(opts, dt=dts, nsteps=1)
            for q in range(len(wls)):
                us[q] = O.ssp_step(os_[q], us[q], dts[q], order=order)
                ug = gs[q].get_solution()
                assert relerr(ug, us[q]) < 1e-10, (step, q)
                assert ug.min() >= -1e-14 and ug.max() <= 1 + 1e-14


def test_mixed_ssp_vs_fp64_oracle_and_bounds(afc):
    """Mixed precision: 20 SSP3 steps of the rotating P1 9^3 problem and a random Q1
    instance stay within 1e-6 of the FP64 oracle and inside [0, 1]."""
    cases = [W.rotating_transient("p1", 9)] + make_instances(5, 1, elems=("q1",), n_range=(11, 11))
    for wl in cases:
        o = oracle_problem(wl.elem, wl.n, wl.b, wl.eps, wl.c, wl.f, wl.dir_mask, wl.u_dir)
        dt = O.cfl_timestep(o, 0.5)
        g = gpu_of(wl)
        opts = afc.default_opts(scheme=afc.AFC_SSP3, dt=dt, precision=afc.AFC_MIXED)
        u = wl.u0.copy()
        worst = 0.0
        for _ in range(20):
            u = O.ssp_step(o, u, dt, order=3)
            g.step(opts)
            ug = g.get_solution()
            worst = max(worst, float(np.abs(ug - u).max()))
            assert ug.min() >= -1e-14 and ug.max() <= 1 + 1e-14
        assert worst <= 1e-6 * max(1.0, np.abs(u).max()), worst


def test_batch_mixed_sizes_and_elements_bitwise_independent_of_company(afc):
    """An instance gives the same bits in a batch of 1 and in a batch of 6."""
    wls = make_instances(21, 6, n_range=(5, 14))
    gs = [gpu_of(wl) for wl in wls]
    dts = [g.cfl_timestep(0.4) for g in gs]
    opts = afc.default_opts(scheme=afc.AFC_SSP3, precision=afc.AFC_MIXED)
    with afc.Batch(gs) as b:
        b.step(opts, dt=dts, nsteps=3)
    together = [g.get_solution() for g in gs]
    for q, wl in enumerate(wls):
        gs[q].set_solution(wl.u0)
        with afc.Batch([gs[q]]) as b1:
            b1.step(opts, dt=[dts[q]], nsteps=3)
        assert np.array_equal(gs[q].get_solution(), together[q]), q


def test_batch_tune_restores_state_and_picks_a_shape(afc):
    wls = make_instances(31, 4, n_range=(8, 12))
    gs = [gpu_of(wl) for wl in wls]
    dts = [g.cfl_timestep(0.5) for g in gs]
    opts = afc.default_opts(scheme=afc.AFC_SSP3)
    with afc.Batch(gs) as b:
        before = [g.get_solution() for g in gs]
        best = b.tune(opts, dt=dts)
        assert best["mode"] in (afc.AFC_BATCH_PER_PASS, afc.AFC_BATCH_PER_STAGE, afc.AFC_BATCH_PER_STEP)
        assert best["block"] in (128, 256, 512) and best["ms_per_step"] > 0
        for g, u in zip(gs, before):
            assert np.array_equal(g.get_solution(), u)
        t = b.get_tuning()
        assert t["mode"] == best["mode"] and t["block"] == best["block"]
        # a new batch of the same size class picks the tuned shape up
        b.set_tuning(afc.AFC_BATCH_AUTO)
        auto = b.get_tuning()
        assert auto["block"] == best["block"]


def test_batch_rejects_bad_input(afc):
    wls = make_instances(41, 2, n_range=(5, 6))
    gs = [gpu_of(wl) for wl in wls]
    with pytest.raises(afc.AfcError) as e:
        afc.Batch([gs[0], gs[0]])
    assert e.value.status == afc.AFC_E_INVALID
    raw = afc.Problem.structured("q1", 5)
    with pytest.raises(afc.AfcError) as e:
        afc.Batch([gs[0], raw])
    assert e.value.status == afc.AFC_E_STATE
    with afc.Batch(gs) as b:
        with pytest.raises(afc.AfcError) as e:
            b.step(afc.default_opts(scheme=afc.AFC_CN_NONLINEAR, dt=1e-3))
        assert e.value.status == afc.AFC_E_INVALID
        with pytest.raises(afc.AfcError) as e:
            b.step(afc.default_opts(scheme=afc.AFC_SSP3), dt=[1e-3, -1.0])
        assert e.value.status == afc.AFC_E_INVALID
        with pytest.raises(afc.AfcError):
            b.set_tuning(afc.AFC_BATCH_PER_STAGE, block=100)
