"""The request server: every result is the same as the request run alone (bit
for bit: the batched step and the stationary solve are the calls a lone run
makes), mixed-precision results stay within 1e-6 of FP64, admission keeps the
estimated device memory inside the budget, and cancellation and timeouts
behave as documented."""
import time

import numpy as np
import pytest

from paper_2110_15676_gb300 import workloads as W
from pairs import gpu_problem

pytestmark = pytest.mark.gpu

STEPS = 8


@pytest.fixture(scope="module")
def afc():
    from paper_2110_15676_gb300 import afc as A
    return A


def opts_for(afc, kind, prec):
    if kind == "transient":
        return afc.default_opts(scheme=afc.AFC_SSP3, precision=prec)
    return afc.default_opts(limiter=afc.AFC_LIM_MC, omega=0.5, ksp=afc.AFC_KSP_GMRES, ksp_atol=0.0,
                            ksp_rtol=1e-6, fp_tol=1e-10, fp_maxit=400, precision=prec)


def request_of(afc, kind, wl, prec):
    k = afc.AFC_REQ_TRANSIENT if kind == "transient" else afc.AFC_REQ_STATIONARY
    return afc.Request(k, wl.elem, wl.n, wl.eps, wl.c, wl.b, wl.u0, wl.dir_mask, wl.u_dir, f=wl.f,
                       opts=opts_for(afc, kind, prec), steps=STEPS, cfl=0.5)


def alone(afc, kind, wl, prec):
    g = gpu_problem(wl.elem, wl.n, wl.b, wl.eps, wl.c, wl.f, wl.dir_mask, wl.u_dir,
                    family="fct" if kind == "transient" else "mc",
                    precision="mixed" if prec == afc.AFC_MIXED else "fp64")
    g.set_solution(wl.u0)
    o = opts_for(afc, kind, prec)
    if kind == "transient":
        o.dt = g.cfl_timestep(0.5)
        for _ in range(STEPS):
            g.step(o)
    else:
        g.solve_stationary(o)
    u = g.get_solution()
    g.close()
    return u


def run_mix(afc, srv, mix, prec, gap=0.002):
    ids = []
    for kind, wl in mix:
        ids.append(srv.submit(request_of(afc, kind, wl, prec)))
        time.sleep(gap)
    out = []
    for rid in ids:
        res, u = srv.wait(rid, timeout=300.0)
        assert res["state"] == afc.AFC_REQ_DONE, res
        out.append((res, u))
        srv.release(rid)
    return out


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_results_same_alone_and_in_the_mix(afc, prec):
    p = afc.AFC_MIXED if prec == "mixed" else afc.AFC_FP64
    mix = W.serving_mix(np.random.default_rng(50), 10, n_range=(6, 11))
    with afc.Server(stationary_workers=3, max_chunk=3) as srv:
        got = run_mix(afc, srv, mix, p)
        info = srv.info()
    assert info["completed"] == len(mix) and info["failed"] == 0
    for (kind, wl), (res, u) in zip(mix, got):
        ref = alone(afc, kind, wl, p)
        assert np.array_equal(u, ref), (kind, wl.name, np.abs(u - ref).max())
        if kind == "transient":
            assert res["stats"]["stages"] == 3 * STEPS
            assert u.min() >= -1e-14 and u.max() <= 1 + 1e-14


def test_mixed_within_1e6_of_fp64(afc):
    mix = W.serving_mix(np.random.default_rng(51), 6, n_range=(6, 10))
    with afc.Server(stationary_workers=2) as srv:
        m = run_mix(afc, srv, mix, afc.AFC_MIXED)
        f = run_mix(afc, srv, mix, afc.AFC_FP64)
    for (kind, wl), (_, um), (_, uf) in zip(mix, m, f):
        assert np.abs(um - uf).max() <= 1e-6 * max(1.0, np.abs(uf).max()), (kind, wl.name)


def test_serial_mode_equals_batched(afc):
    mix = W.serving_mix(np.random.default_rng(52), 6, n_range=(6, 10))
    with afc.Server(mode=afc.AFC_SERVE_SERIAL) as s1:
        a = run_mix(afc, s1, mix, afc.AFC_FP64, gap=0.0)
    with afc.Server(mode=afc.AFC_SERVE_BATCHED) as s2:
        b = run_mix(afc, s2, mix, afc.AFC_FP64, gap=0.0)
    for (_, ua), (_, ub) in zip(a, b):
        assert np.array_equal(ua, ub)


def test_admission_respects_the_budget(afc):
    mix = W.serving_mix(np.random.default_rng(53), 8, n_range=(9, 13))
    reqs = [request_of(afc, k, wl, afc.AFC_MIXED) for k, wl in mix]
    est = [r.estimate_bytes() for r in reqs]
    budget = int(2.2 * max(est))
    with afc.Server(hbm_budget=budget, max_active=3) as srv:
        ids = [srv.submit(r) for r in reqs]
        peak = 0
        while True:
            inf = srv.info()
            assert inf["bytes_in_use"] <= budget and inf["active"] <= 3
            peak = max(peak, inf["bytes_in_use"])
            if inf["completed"] + inf["failed"] == len(ids):
                break
            time.sleep(0.001)
        for rid in ids:
            res, _ = srv.wait(rid, timeout=60.0, want_u=False)
            assert res["state"] == afc.AFC_REQ_DONE
            assert res["t_admit"] >= res["t_submit"] and res["t_done"] >= res["t_admit"]
    assert peak > 0


def test_cancel_timeout_and_errors(afc):
    mix = W.serving_mix(np.random.default_rng(54), 4, n_range=(8, 10))
    reqs = [request_of(afc, k, wl, afc.AFC_FP64) for k, wl in mix]
    with afc.Server(mode=afc.AFC_SERVE_SERIAL) as srv:
        ids = [srv.submit(r) for r in reqs]
        srv.cancel(ids[-1])
        for rid in ids[:-1]:
            res, _ = srv.wait(rid, timeout=120.0, want_u=False)
            assert res["state"] == afc.AFC_REQ_DONE
        res, _ = srv.wait(ids[-1], timeout=120.0, want_u=False)
        assert res["state"] == afc.AFC_REQ_CANCELLED
        with pytest.raises(afc.AfcError) as e:
            srv.poll(12345)
        assert e.value.status == afc.AFC_E_INVALID
        with pytest.raises(afc.AfcError) as e:
            srv.release(ids[0]) or srv.release(ids[0])
        assert e.value.status == afc.AFC_E_INVALID
    with afc.Server(hbm_budget=1 << 20) as small:
        with pytest.raises(afc.AfcError) as e:
            small.submit(reqs[0])
        assert e.value.status == afc.AFC_E_INVALID


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_served_results_match_the_oracle(afc, prec):
    """Every request of a served mix against the CPU oracle: transient requests
    against the oracle's SSP3 Zalesak steps, stationary ones against its damped MC
    fixed point (Sec. 3.1, Sec. 4) converged with exact inner solves.  FP64 requests
    (stationary fixed point to 1e-12, inner GMRES to 1e-14) within 1e-10 relative
    max-norm; mixed requests (FP32 fluxes or inner solves, float-pair MC residual,
    fixed point to 1e-10) within 1e-6."""
    from oracle import afc_oracle as O
    p = afc.AFC_MIXED if prec == "mixed" else afc.AFC_FP64
    tol = 1e-6 if prec == "mixed" else 1e-10
    mix = W.serving_mix(np.random.default_rng(55), 8, n_range=(6, 10))

    def sopts():
        if prec == "mixed":
            return afc.default_opts(limiter=afc.AFC_LIM_MC, omega=0.5, ksp=afc.AFC_KSP_GMRES, ksp_atol=0.0,
                                    ksp_rtol=1e-6, fp_tol=1e-10, fp_maxit=1000, precision=p)
        return afc.default_opts(limiter=afc.AFC_LIM_MC, omega=0.5, ksp=afc.AFC_KSP_GMRES, ksp_atol=1e-14,
                                fp_tol=1e-12, fp_maxit=2000, precision=p)

    with afc.Server(stationary_workers=3, max_chunk=3, builders=3) as srv:
        ids = []
        for kind, wl in mix:
            k = afc.AFC_REQ_TRANSIENT if kind == "transient" else afc.AFC_REQ_STATIONARY
            o = opts_for(afc, kind, p) if kind == "transient" else sopts()
            ids.append(srv.submit(afc.Request(k, wl.elem, wl.n, wl.eps, wl.c, wl.b, wl.u0, wl.dir_mask, wl.u_dir,
                                              f=wl.f, opts=o, steps=STEPS, cfl=0.5)))
        got = []
        for rid in ids:
            res, u = srv.wait(rid, timeout=300.0)
            assert res["state"] == afc.AFC_REQ_DONE and res["status"] == afc.AFC_OK, res
            got.append(u)
            srv.release(rid)
    for (kind, wl), u in zip(mix, got):
        mesh = O.structured_mesh(wl.elem, wl.n)
        fam = "fct" if kind == "transient" else "mc"
        o = O.assemble(mesh, wl.eps, wl.b, wl.c, wl.f, wl.dir_mask.astype(bool), wl.u_dir, fam)
        if kind == "transient":
            dt = O.cfl_timestep(o, 0.5)
            ref = wl.u0.copy()
            for _ in range(STEPS):
                ref = O.ssp_step(o, ref, dt, order=3)
        else:
            ref, st = O.mc_stationary(o, u0=wl.u0, tol=1e-12, omega=0.5, ksp="direct", max_outer=4000)
            assert st["converged"]
        err = np.abs(u - ref).max() / max(np.abs(ref).max(), 1e-300)
        assert err <= tol, (kind, wl.name, err)
