"""Parity at the full benchmark sizes, on the launch configuration bench.py times.

* Kuhn P1 129^3 (2,146,689 dofs, 14.8 M pairs), stationary MC limiter: the limited
  sum F*_i of sampled rows against the oracle evaluated on a local sub-box around each
  row (the row, its neighbours and their neighbours see complete element sets there),
  plus conservation of F* over the whole field.
* Q1 65^3 (274,625 dofs), Crank-Nicolson Zalesak FCT: F*_i of sampled rows the same way
  (the limiter of row i reaches three element layers), plus the limiter-level bound
  dt F*_i / m_i in [Q_i^-, Q_i^+] and conservation at full size, and one complete CN
  step whose returned residual meets the stopping rule.
* The benchmarked Q1 65^3 CN step itself (CFL 1, six fixed-point corrections with
  tight inner solves) through afc_step against the oracle's step, the whole field at
  the 1e-10 relative bound per step.
Inputs are seeded fields from the workload generators; nothing the oracle sees comes
from the GPU."""
import math

import numpy as np
import pytest

from oracle import afc_oracle as O
from paper_2110_15676_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def afc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_15676_gb300 import afc as mod
    return mod


def _sub_problem(wl, family, center, R, fields):
    """Oracle problem on the index box of radius R around node `center` (clipped to the
    grid), with the exact global coordinates and the given nodal fields restricted."""
    n = wl.n
    ix, iy, iz = W.grid_index(n)
    c = (ix[center], iy[center], iz[center])
    lo = [max(0, c[d] - R) for d in range(3)]
    hi = [min(n[d] - 1, c[d] + R) for d in range(3)]
    m = tuple(hi[d] - lo[d] + 1 for d in range(3))
    sub = O.structured_mesh(wl.elem, m)
    lx, ly, lz = W.grid_index(m)
    gid = (lx + lo[0]) + n[0] * ((ly + lo[1]) + n[1] * (lz + lo[2]))
    xyz = W.grid_coords(n)[gid]
    mesh = O.Mesh(wl.elem, xyz, sub.cells)
    prob = O.assemble(mesh, wl.eps, wl.b[gid], wl.c, wl.f[gid], wl.dir_mask[gid].astype(bool), wl.u_dir[gid], family)
    local = int(np.flatnonzero(gid == center)[0])
    return prob, gid, local, {k: v[gid] for k, v in fields.items()}


def _samples(rng, wl, k):
    """Sampled rows: interior, next to the boundary, and spread over the grid."""
    free = np.flatnonzero(wl.dir_mask == 0)
    ix, iy, iz = W.grid_index(wl.n)
    near = free[(np.minimum.reduce([ix[free], iy[free], iz[free]]) <= 1)]
    pick = list(rng.choice(free, k, replace=False)) + list(rng.choice(near, k // 4, replace=False))
    return pick


def test_mc_sweep_full_size_p1_129(afc):
    wl = W.stationary_inflow("p1", 129)
    P = afc.Problem.structured(wl.elem, wl.n)
    P.set_coefficients(wl.eps, wl.b, wl.c, wl.f)
    P.set_dirichlet(wl.dir_mask, wl.u_dir)
    P.assemble(afc.AFC_FAMILY_MC, afc.AFC_MIXED)          # the bench configuration
    rng = np.random.default_rng(129)
    xyz = W.grid_coords(wl.n)
    u = W.front_field(xyz, rng)
    u[wl.dir_mask.astype(bool)] = wl.u_dir[wl.dir_mask.astype(bool)]
    out = P.mc_limited_sum(u, afc.AFC_LIM_MC)
    F = out["Fstar"]
    scale = np.abs(F).max()
    assert scale > 0
    # conservation over the whole field (Dirichlet rows hold 0; their share is the boundary flux)
    info = P.info()
    assert info["n_nodes"] == 2146689 and info["n_edges"] == 14827904
    for i in _samples(rng, wl, 24):
        prob, gid, loc, fl = _sub_problem(wl, "mc", i, 3, {"u": u})
        rstar, _ = O.mc_limited_fluxes(prob, fl["u"])
        Fo = O.limited_sum(prob, np.ones_like(rstar), rstar)
        assert abs(F[i] - Fo[loc]) <= 1e-13 * scale, i
        assert out["umax"][i] == fl["u"][prob.MC[loc].indices].max()
        assert out["umin"][i] == fl["u"][prob.MC[loc].indices].min()
    # the sweep the bench times, on the same problem: its residual f + F* - AA u at the
    # sampled rows against the oracle's (Sec. 4), 0 on Dirichlet rows
    P.set_solution(u)
    P.mc_residual_sweep(afc.AFC_LIM_MC)
    res = P.get_residual()
    assert (res[wl.dir_mask.astype(bool)] == 0).all()
    rscale = np.abs(res).max()
    assert rscale > 0
    for i in _samples(np.random.default_rng(130), wl, 24):
        prob, gid, loc, fl = _sub_problem(wl, "mc", i, 3, {"u": u})
        rstar, _ = O.mc_limited_fluxes(prob, fl["u"])
        Fo = O.limited_sum(prob, np.ones_like(rstar), rstar)
        ro = prob.f[loc] + Fo[loc] - (prob.AA @ fl["u"])[loc]
        assert abs(res[i] - ro) <= 1e-13 * rscale, i


def test_cn_limiter_and_step_full_size_q1_65(afc):
    wl = W.rotating_transient("q1", 65)
    P = afc.Problem.structured(wl.elem, wl.n)
    P.set_coefficients(wl.eps, wl.b, wl.c, wl.f)
    P.set_dirichlet(wl.dir_mask, wl.u_dir)
    P.assemble(afc.AFC_FAMILY_FCT, afc.AFC_MIXED)         # the bench configuration
    rng = np.random.default_rng(65)
    xyz = W.grid_coords(wl.n)
    u_old = wl.u0.copy()
    u_new = np.clip(u_old + 0.05 * W.front_field(xyz, rng) - 0.025, 0, 1)
    u_new[wl.dir_mask.astype(bool)] = 0.0
    dt = 0.02
    out = P.cn_limited_sum(dt, u_new, u_old, afc.AFC_LIM_ZALESAK, 1)
    F = out["Fstar"]
    scale = np.abs(F).max()
    assert scale > 0
    assert abs(F.sum()) <= 1e-12 * np.abs(F).sum()
    # limiter-level bound at every free node: dt F*_i / m_i within [Q_i^-, Q_i^+] of the predictor
    mL = P.lumped_mass()
    rowptr, col, _ = P.export_csr(afc.AFC_MAT_MC)
    ut = out["u_tilde"]
    seg = np.repeat(np.arange(P.N), np.diff(rowptr))
    hi = np.full(P.N, -np.inf); lo = np.full(P.N, np.inf)
    np.maximum.at(hi, seg, ut[col]); np.minimum.at(lo, seg, ut[col])
    free = wl.dir_mask == 0
    inc = dt * F / mL
    assert (inc[free] <= (hi - ut)[free] + 1e-14).all() and (inc[free] >= (lo - ut)[free] - 1e-14).all()
    for i in _samples(rng, wl, 16):
        prob, gid, loc, fl = _sub_problem(wl, "fct", i, 4, {"un": u_new, "uo": u_old})
        uo, un = fl["uo"], fl["un"]
        ut_l = uo - 0.5 * dt * (prob.AA @ uo - prob.f) / prob.mL
        ut_l[prob.dir_mask] = prob.u_dir[prob.dir_mask]
        r = O.cn_fluxes(prob, un, uo, dt, True)
        alpha, lim = O.zalesak_limiter(prob, r, ut_l, dt)
        Fo = O.limited_sum(prob, alpha, r)
        assert abs(F[i] - Fo[loc]) <= 1e-13 * scale, i
        assert abs(ut[i] - ut_l[loc]) <= 1e-15 * max(1.0, abs(ut_l[loc]))
    # one complete step of the benchmark workload, run to its stopping rule
    dt_cfl = P.cfl_timestep(1.0)
    P.set_solution(wl.u0)
    st = P.step(afc.default_opts(scheme=afc.AFC_CN_NONLINEAR, dt=dt_cfl, fp_tol=1e-10, ksp_atol=1e-12))
    assert st["status"] == afc.AFC_OK
    assert st["res_final"] < math.sqrt(P.N) * 1e-10
    assert st["outer_its"] >= 2 and st["inner_its"] >= st["outer_its"]


def test_cn_step_full_size_q1_65_matches_oracle(afc):
    """The step bench.py times (nonlinear Zal+CN, Q1 65^3, CFL 1, prelimiting, FP64),
    at a fixed count of six fixed-point corrections and inner BiCGStab to 1e-14, so that
    neither side's stopping test decides the iterate: every node against the oracle's
    cn_step with the same settings, relative max-norm 1e-10."""
    wl = W.rotating_transient("q1", 65)
    mesh = O.structured_mesh(wl.elem, wl.n)
    o = O.assemble(mesh, wl.eps, wl.b, wl.c, wl.f, wl.dir_mask.astype(bool), wl.u_dir)
    dt = O.cfl_timestep(o, 1.0)
    u_ref, sto = O.cn_step(o, wl.u0, dt, fixed_iterations=6, ksp_atol=1e-14)
    assert np.isfinite(u_ref).all()
    P = afc.Problem.structured(wl.elem, wl.n)
    P.set_coefficients(wl.eps, wl.b, wl.c, wl.f)
    P.set_dirichlet(wl.dir_mask, wl.u_dir)
    P.assemble(afc.AFC_FAMILY_FCT, afc.AFC_FP64)
    assert abs(P.cfl_timestep(1.0) - dt) <= 1e-14 * dt
    for graph in (1, 0):
        P.set_solution(wl.u0)
        st = P.step(afc.default_opts(scheme=afc.AFC_CN_NONLINEAR, dt=dt, fp_fixed_its=6, ksp_atol=1e-14,
                                     graph=graph))
        assert st["outer_its"] == 6 == sto["outer_its"]
        u = P.get_solution()
        assert np.isfinite(u).all(), (graph, np.flatnonzero(~np.isfinite(u))[:8])
        err = np.abs(u - u_ref).max() / np.abs(u_ref).max()
        assert err <= 1e-10, (graph, err)
