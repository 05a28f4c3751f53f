"""Pins of the oracle's method variants: the monolithic upwind (MU) limiter
(Sec. 3, MU limiter), checked against what the method fixes: conservation,
0 <= alpha <= 1 with alpha_ij = alpha_ji, the local bound P_i R_i <= Q_i that step
3 enforces, constants give no flux, and alpha = 1 where nothing is limited."""
import numpy as np
import pytest

from oracle import afc_oracle as O
from pairs import oracle_problem, random_workload


@pytest.mark.parametrize("elem,n", [("p1", 7), ("q1", 6)])
def test_mu_conservation_symmetry_and_bounds(elem, n):
    wl = random_workload(elem, n, seed=33)
    o = oracle_problem(wl.elem, wl.n, wl.b, 0.0, 0.0, wl.f, wl.dir_mask, wl.u_dir, family="mc")
    rng = np.random.default_rng(34)
    u = rng.uniform(0.0, 1.0, o.mesh.n_nodes)
    rstar, info = O.mu_limited_fluxes(o, u)
    F = O.limited_sum(o, np.ones_like(rstar), rstar)
    r, alpha = info["r"], info["alpha"]
    assert abs(F.sum()) <= 1e-14 * np.abs(rstar).sum()
    assert alpha.min() >= 0.0 and alpha.max() <= 1.0
    # alpha_ij = alpha_ji and r*_ji = -r*_ij
    I, J = o.pairs
    key = dict(zip(zip(I.tolist(), J.tolist()), range(len(I))))
    rev = np.array([key[(j, i)] for i, j in zip(I.tolist(), J.tolist())])
    assert np.array_equal(alpha, alpha[rev])
    assert np.abs(rstar + rstar[rev]).max() <= 1e-15 * max(np.abs(rstar).max(), 1e-300)
    # step 3: the limited fluxes a node owns stay within its Q bounds
    aij, aji = O.entries(o.K, I, J), O.entries(o.K, J, I)
    tie = np.abs(aij - aji) <= 1e-12 * (np.abs(aij) + np.abs(aji))
    owns = np.where(tie, I < J, aji < aij)
    N = o.mesh.n_nodes
    pos = np.bincount(I[owns], weights=np.maximum(rstar[owns], 0.0), minlength=N)
    neg = np.bincount(I[owns], weights=np.minimum(rstar[owns], 0.0), minlength=N)
    free = ~o.dir_mask
    tol = 1e-14 * np.abs(r).max()
    assert np.all(pos[free] <= info["Qp"][free] + tol)
    assert np.all(neg[free] >= info["Qm"][free] - tol)
    # an unlimited node (R = 1 on both sides) passes its owned fluxes whole
    full = owns & (info["Rp"][I] == 1.0) & (info["Rm"][I] == 1.0)
    assert np.all(alpha[full] == 1.0)


def test_mu_constant_state_has_no_flux():
    wl = random_workload("p1", 6, seed=35)
    o = oracle_problem(wl.elem, wl.n, wl.b, 0.0, 0.0, wl.f, wl.dir_mask, wl.u_dir, family="mc")
    rstar, _ = O.mu_limited_fluxes(o, np.full(o.mesh.n_nodes, 0.42))
    assert np.abs(rstar).max() == 0.0


# ---- linear Zal+CN (Sec. 2.1.1) --------------------------------------------------
def _cn_pair(elem, n):
    from paper_2110_15676_gb300 import workloads as Wk
    wl = Wk.rotating_transient(elem, n)
    o = oracle_problem(wl.elem, wl.n, wl.b, wl.eps, wl.c, wl.f, wl.dir_mask, wl.u_dir)
    return wl, o


def test_linear_cn_with_no_flux_is_the_low_order_cn_step():
    wl, o = _cn_pair("p1", 8)
    dt = O.cfl_timestep(o, 1.0)
    ul, _ = O.cn_linear_step(o, wl.u0, dt, mode="none")
    un, st = O.cn_step(o, wl.u0, dt, mode="none", tol=1e-13, ksp_atol=1e-15, max_outer=50)
    assert st["converged"]
    assert np.abs(ul - un).max() < 1e-12


def test_linear_cn_limiter_bounds_and_conservation():
    wl, o = _cn_pair("q1", 7)
    dt = O.cfl_timestep(o, 1.0)
    u_old = wl.u0
    u_new, st = O.cn_linear_step(o, u_old, dt)
    F, ut = st["Fstar"], st["u_tilde"]
    free = ~o.dir_mask
    # Zalesak bounds at the limiter level, Q from the predictor: dt/m_i F*_i in [Q-, Q+]
    I, J = o.pairs
    N = o.mesh.n_nodes
    Qp = np.zeros(N); Qm = np.zeros(N)
    np.maximum.at(Qp, I, ut[J] - ut[I])
    np.minimum.at(Qm, I, ut[J] - ut[I])
    g = dt * F / o.mL
    assert np.all(g[free] <= Qp[free] + 1e-14) and np.all(g[free] >= Qm[free] - 1e-14)
    assert abs(F.sum()) <= 1e-13 * np.abs(F).sum()
    # the step solves (M_L/dt + AA/2) u = b0 + F*
    b0 = o.mL / dt * u_old - 0.5 * (o.AA @ u_old) + o.f
    resid = (o.mL / dt * u_new + 0.5 * (o.AA @ u_new)) - (b0 + F)
    assert np.abs(resid[free]).max() < 1e-10 * np.abs(b0).max()


def test_linear_and_nonlinear_cn_agree_for_small_steps():
    """Both schemes approximate the same CN step; with dt small the extrapolation
    2 u~ - u_old is close to u^n and the two solutions nearly coincide."""
    wl, o = _cn_pair("p1", 9)
    dt = O.cfl_timestep(o, 0.1)
    ul, _ = O.cn_linear_step(o, wl.u0, dt)
    un, st = O.cn_step(o, wl.u0, dt, tol=1e-13, ksp_atol=1e-15, max_outer=200)
    change = np.abs(un - wl.u0).max()
    assert np.abs(ul - un).max() < 0.05 * change


# ---- transient MC (Sec. 2.2) -----------------------------------------------------
@pytest.mark.parametrize("elem,n", [("p1", 9), ("q1", 8)])
def test_transient_mc_stage_local_bounds_and_conservation(elem, n):
    """At CFL 0.5 (dt sum_j 2|d_ij| <= m_i) every forward-Euler MC stage is a convex
    combination of limited bar states: u_new,i lies in [u_i^min, u_i^max] of the stage
    input (Eq. u_max_min), and the limited fluxes are conservative."""
    from paper_2110_15676_gb300 import workloads as Wk
    wl = Wk.rotating_transient(elem, n)
    o = oracle_problem(wl.elem, wl.n, wl.b, wl.eps, wl.c, wl.f, wl.dir_mask, wl.u_dir, family="mc")
    dt = O.cfl_timestep(o, 0.5)
    u = wl.u0.copy()
    free = ~o.dir_mask
    for _ in range(6):
        un, info = O.fe_mc_stage(o, u, dt, want=True)
        assert np.all(un[free] >= info["umin"][free] - 1e-14)
        assert np.all(un[free] <= info["umax"][free] + 1e-14)
        assert abs(info["Fstar"].sum()) <= 1e-14 * max(np.abs(info["rstar"]).sum(), 1e-300)
        u = O.ssp_step(o, u, dt, order=3, mode="mc")
    assert u.min() >= -1e-14 and u.max() <= 1.0 + 1e-14


def test_transient_mc_preserves_constants():
    from paper_2110_15676_gb300 import workloads as Wk
    n = 7
    xyz = Wk.grid_coords(n)
    N = len(xyz)
    o = oracle_problem("p1", n, Wk.rotating_b(xyz), 1e-4, 0.0, np.zeros(N), Wk.boundary_mask(n), np.full(N, 0.3),
                       family="mc")
    u = O.ssp_step(o, np.full(N, 0.3), O.cfl_timestep(o, 0.5), order=3, mode="mc")
    assert np.abs(u - 0.3).max() < 1e-15


# ---- CN with the MC limiter (Sec. 2.2) -------------------------------------------
def test_cn_mc_agrees_with_ssp_mc_for_small_steps_and_keeps_constants():
    """CN and SSP3 both integrate the same semi-discrete MC scheme: for a small step
    their updates agree to a small fraction of the step's change (second order in
    dt), and a constant state stays constant."""
    from paper_2110_15676_gb300 import workloads as Wk
    wl = Wk.rotating_transient("p1", 9)
    o = oracle_problem(wl.elem, wl.n, wl.b, wl.eps, wl.c, wl.f, wl.dir_mask, wl.u_dir, family="mc")
    dt = O.cfl_timestep(o, 0.05)
    uc, st = O.cn_mc_step(o, wl.u0, dt, tol=1e-13, max_outer=300)
    assert st["converged"]
    us = O.ssp_step(o, wl.u0, dt, order=3, mode="mc")
    assert np.abs(uc - us).max() < 1e-3 * np.abs(us - wl.u0).max()
    N = o.mesh.n_nodes
    oc = oracle_problem("p1", 9, wl.b, wl.eps, 0.0, np.zeros(N), wl.dir_mask, np.full(N, 0.6), family="mc")
    u1, _ = O.cn_mc_step(oc, np.full(N, 0.6), O.cfl_timestep(oc, 1.0), tol=1e-13, max_outer=50)
    assert np.abs(u1 - 0.6).max() < 1e-13
    # both flux halves are conservative
    assert abs(O.mc_transient_flux_sum(o, uc).sum()) < 1e-14 * np.abs(uc).sum()
