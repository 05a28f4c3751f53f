"""Pins for the oracle's implicit parts: nonlinear Crank-Nicolson FCT (Sec. 2.1.1),
the stationary monolithic convex limiter (Sec. 2.2, Sec. 3.1), the damped fixed
point (Sec. 4) and the Krylov solvers.

  * Krylov: BiCGStab and GMRES(m) agree with a dense direct solve and meet atol
    on the true residual.
  * CN with alpha = 1 and no prelimiting satisfies the CN-Galerkin equation
    [M_C/dt + A/2] u^n = [M_C/dt - A/2] u^{n-1} + f; with alpha = 0 it is the
    low-order CN step (direct solve).
  * CN Zalesak: the converged step solves Eq. CNZal, the limited term is
    conservative and within the limiter bounds dt/m_i F*_i in [Q_i^-, Q_i^+].
  * Prelimiting only shrinks fluxes and never flips their sign.
  * MC: r*_ji = -r*_ij; limited bar states stay in the local bounds; alpha = 1
    gives the Galerkin system for the unlimited operator, alpha = 0 the upwind
    system; the converged solution of the inflow problem stays in [0, 1].
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import afc_oracle as O
from paper_2110_15676_gb300 import workloads as W


def _mate(prob):
    I, J = prob.pairs
    key = {(i, j): k for k, (i, j) in enumerate(zip(I, J))}
    return np.array([key[(j, i)] for i, j in zip(I, J)])


# ---------------------------------------------------------------- Krylov
@pytest.mark.parametrize("ksp", ["bicgstab", "gmres"])
def test_krylov_matches_direct_solve(ksp):
    rng = np.random.default_rng(7)
    n = 60
    A = sp.random(n, n, density=0.1, random_state=3, format="csr")
    A = A - sp.diags(np.asarray(abs(A).sum(axis=1)).ravel() + rng.uniform(0.5, 2.0, n))   # diagonally dominant
    A = A.tocsr()
    b = rng.normal(size=n)
    x_ref = np.linalg.solve(A.toarray(), b)
    dinv = 1.0 / A.diagonal()
    x, st = O.krylov_solve(A, b, dinv, ksp, 1e-12, 0.0, 500, 20)
    assert np.linalg.norm(b - A @ x) < 1e-12
    assert np.abs(x - x_ref).max() < 1e-10 * np.abs(x_ref).max()
    assert st["its"] > 0


def test_gmres_full_space_converges_within_n_steps():
    rng = np.random.default_rng(8)
    n = 12
    A = sp.csr_matrix(rng.normal(size=(n, n)) + 4 * np.eye(n))
    b = rng.normal(size=n)
    x, st = O.gmres(A, b, np.ones(n), m=n, atol=1e-11, rtol=0.0, maxit=n)
    assert st["its"] <= n
    assert np.linalg.norm(b - A @ x) < 1e-11


def test_relative_tolerance():
    rng = np.random.default_rng(9)
    n = 80
    A = sp.diags([-1.0, 2.5, -1.2], [-1, 0, 1], shape=(n, n), format="csr")
    b = rng.normal(size=n)
    for ksp in ("bicgstab", "gmres"):
        x, st = O.krylov_solve(A, b, 1.0 / A.diagonal(), ksp, 0.0, 1e-6, 500, 20)
        assert np.linalg.norm(b - A @ x) <= 1e-6 * np.linalg.norm(b) * 1.0001


# ---------------------------------------------------------------- CN
def _cn_problem(elem="q1", n=7, seed=3):
    rng = np.random.default_rng(seed)
    mesh = O.structured_mesh(elem, n)
    N = mesh.n_nodes
    b = W.rotating_b(mesh.xyz)
    dm = W.boundary_mask(n).astype(bool)
    f = rng.uniform(0, 0.5, N)
    prob = O.assemble(mesh, 1e-3, b, 0.2, f, dm, np.zeros(N))
    u_old = W.cosine_hump(mesh.xyz, radius=0.3)
    u_old[dm] = 0.0
    dt = O.cfl_timestep(prob, 1.0)
    return prob, u_old, dt


def test_cn_alpha_one_no_prelimit_is_cn_galerkin():
    prob, u_old, dt = _cn_problem()
    # the unlimited fixed point contracts only like M_L^{-1}(M_L - M_C): many iterations
    u, st = O.cn_step(prob, u_old, dt, tol=1e-14, mode="galerkin", prelimit=False,
                      ksp_atol=1e-15, max_outer=3000)
    assert st["converged"]
    free = ~prob.dir_mask
    lhs = prob.MC @ u / dt + 0.5 * (prob.A @ u)
    rhs = prob.MC @ u_old / dt - 0.5 * (prob.A @ u_old) + prob.f
    scale = np.abs(rhs).max()
    assert np.abs(lhs - rhs)[free].max() < 1e-11 * scale


def test_cn_alpha_zero_is_low_order_cn():
    prob, u_old, dt = _cn_problem()
    u, st = O.cn_step(prob, u_old, dt, tol=1e-14, mode="none", ksp_atol=1e-15)
    B = O.cn_system_matrix(prob, dt)
    rhs = prob.mL / dt * u_old - 0.5 * (prob.AA @ u_old) + prob.f
    rhs[prob.dir_mask] = prob.u_dir[prob.dir_mask]
    ref = spla.spsolve(B.tocsc(), rhs)
    assert np.abs(u - ref).max() < 1e-12
    assert st["outer_its"] == 1       # the low-order system is linear: one correction


@pytest.mark.parametrize("omega", [1.0, 0.7])
def test_cn_zalesak_converged_step(omega):
    prob, u_old, dt = _cn_problem(seed=4)
    tol = 1e-12
    u, st = O.cn_step(prob, u_old, dt, tol=tol, omega=omega, ksp_atol=1e-14, max_outer=400)
    N = prob.mesh.n_nodes
    assert st["converged"] and st["res_final"] < math.sqrt(N) * tol
    free = ~prob.dir_mask
    # Eq. CNZal holds at the returned iterate, with F* recomputed at that iterate
    r = O.cn_fluxes(prob, u, u_old, dt, True)
    ut = u_old - 0.5 * dt * (prob.AA @ u_old - prob.f) / prob.mL
    ut[prob.dir_mask] = 0.0
    alpha, lim = O.zalesak_limiter(prob, r, ut, dt)
    F = O.limited_sum(prob, alpha, r)
    lhs = prob.mL / dt * u + 0.5 * (prob.AA @ u)
    rhs = prob.mL / dt * u_old - 0.5 * (prob.AA @ u_old) + prob.f + F
    assert np.linalg.norm((lhs - rhs)[free]) < math.sqrt(N) * tol * 1.0001
    # conservation and limiter-level bounds
    assert abs(F.sum()) < 1e-14 * np.abs(F).sum()
    M = prob.MC.toarray()
    hi = np.where(M != 0, ut[None, :], -np.inf).max(axis=1) - ut
    lo = np.where(M != 0, ut[None, :], np.inf).min(axis=1) - ut
    inc = dt * F / prob.mL
    assert (inc[free] <= hi[free] + 1e-14).all() and (inc[free] >= lo[free] - 1e-14).all()
    assert st["outer_its"] >= 2


def test_prelimiting_shrinks_and_keeps_sign():
    prob, u_old, dt = _cn_problem(seed=5)
    rng = np.random.default_rng(11)
    u_new = u_old + rng.normal(scale=0.05, size=u_old.shape)
    raw = O.cn_fluxes(prob, u_new, u_old, dt, prelimit=False)
    pre = O.cn_fluxes(prob, u_new, u_old, dt, prelimit=True)
    I, J = prob.pairs
    d = O.entries(prob.D, I, J)
    lim = d * ((u_new + u_old)[J] - (u_new + u_old)[I])
    assert (np.abs(pre) <= np.abs(raw)).all()
    assert (np.abs(pre) <= np.abs(lim) + 0 * lim).all()
    assert (pre * raw >= 0).all() and (pre * lim >= 0).all()
    both = (raw * lim > 0)
    assert (pre[both] != 0).all() and (pre[~both] == 0).all()
    assert np.abs(pre[_mate(prob)] + pre).max() <= 1e-15 * np.abs(pre).max()


def test_prelimiting_saturates_at_twice_the_diffusive_flux():
    """Eq. prelimiting with L = 2: where the raw CN flux and the diffusive flux
    d_ij (ubar_j - ubar_i) at the CN average agree in sign, the prelimited flux is
    the raw flux itself if it is at most twice the diffusive flux in magnitude, and
    exactly twice the diffusive flux otherwise.  The diffusive flux is what
    Eq. flux_002 leaves when the mass term vanishes (dt -> infinity), so it is taken
    from the oracle's own raw flux at dt = inf, not retyped; an oracle with L = 1
    (or with the plain u^n instead of the average) fails."""
    prob, u_old, dt = _cn_problem(seed=5)
    rng = np.random.default_rng(13)
    u_new = u_old + rng.normal(scale=0.05, size=u_old.shape)
    raw = O.cn_fluxes(prob, u_new, u_old, dt, prelimit=False)
    pre = O.cn_fluxes(prob, u_new, u_old, dt, prelimit=True)
    diff = O.cn_fluxes(prob, u_new, u_old, np.inf, prelimit=False)
    same = raw * diff > 0
    big = same & (np.abs(raw) > 2.0 * np.abs(diff))
    small = same & (np.abs(raw) < 2.0 * np.abs(diff))
    assert big.sum() > 50 and small.sum() > 50          # both branches occur
    assert np.array_equal(pre[big], 2.0 * diff[big])
    assert np.array_equal(pre[small], raw[small])
    assert (pre[~same] == 0).all()


# ---------------------------------------------------------------- MC
def _mc_problem(elem="p1", n=9):
    wl = W.stationary_inflow(elem, n)
    mesh = O.structured_mesh(wl.elem, wl.n)
    prob = O.assemble(mesh, wl.eps, wl.b, wl.c, wl.f, wl.dir_mask.astype(bool), wl.u_dir, "mc")
    return prob, wl


@pytest.mark.parametrize("elem", ["p1", "q1"])
def test_mc_fluxes_antisymmetric_and_bar_states_bounded(elem):
    prob, wl = _mc_problem(elem, 7)
    rng = np.random.default_rng(12)
    u = rng.uniform(0, 1, prob.mesh.n_nodes)
    rstar, d = O.mc_limited_fluxes(prob, u)
    mate = _mate(prob)
    assert np.abs(rstar[mate] + rstar).max() <= 1e-15 * np.abs(rstar).max()
    I, J = prob.pairs
    dd = O.entries(prob.D, I, J)
    k_ij = O.entries(prob.K, I, J); k_ji = O.entries(prob.K, J, I)
    M = prob.MC.toarray()
    umax = np.where(M != 0, u[None, :], -np.inf).max(axis=1)
    umin = np.where(M != 0, u[None, :], np.inf).min(axis=1)
    nz = dd != 0
    ubar = 0.5 * (u[I] + u[J]) + k_ij * (u[J] - u[I]) / (2 * dd + (~nz))
    lim_bar = ubar + rstar / (2 * np.abs(dd) + (~nz))
    # The bar state lies between u_i and u_j only where |a_ij|, |a_ji| <= |d_ij|; that
    # holds for every pair with a skew-symmetric convective part (all interior pairs
    # here), not for all boundary pairs.
    ok = nz & (np.abs(k_ij) <= np.abs(dd) * (1 + 1e-12)) & (np.abs(k_ji) <= np.abs(dd) * (1 + 1e-12))
    assert ok.sum() > 0.6 * nz.sum()
    tol = 1e-13
    assert (lim_bar[ok] <= umax[I][ok] + tol).all() and (lim_bar[ok] >= umin[I][ok] - tol).all()
    assert (rstar[~nz] == 0).all()
    # on those pairs |r*| <= |r| with the sign of r (up to roundoff of the bounds)
    r = d["r"]
    eps = 1e-15 * np.abs(r).max()
    assert (np.abs(rstar[ok]) <= np.abs(r[ok]) + eps).all() and (rstar[ok] * r[ok] >= -eps * np.abs(r[ok])).all()
    assert (np.abs(rstar) > 0).sum() > 0 and (np.abs(rstar) < np.abs(r)).sum() > 0


def test_mc_alpha_one_and_zero_limits():
    prob, wl = _mc_problem("p1", 7)
    N = prob.mesh.n_nodes
    dm = prob.dir_mask
    free = ~dm
    for mode in ("galerkin", "none"):
        u, st = O.mc_stationary(prob, tol=1e-13, omega=1.0, mode=mode, ksp="gmres", ksp_atol=1e-15)
        if mode == "galerkin":    # AA u = f + D u  <=>  (K + eps S + c M_L) u = f
            G = (prob.K + prob.eps * prob.S + sp.diags(prob.c * prob.mL)).tolil()
        else:
            G = prob.AA.tolil()
        for i in np.flatnonzero(dm):
            G.rows[i] = [i]; G.data[i] = [1.0]
        rhs = prob.f.copy(); rhs[dm] = prob.u_dir[dm]
        ref = spla.spsolve(G.tocsc(), rhs)
        assert np.abs(u - ref).max() < 1e-10, mode


def test_mc_stationary_converges_within_bounds():
    prob, wl = _mc_problem("p1", 9)
    u, st = O.mc_stationary(prob, tol=1e-10, omega=0.5, ksp="gmres", ksp_atol=1e-13, max_outer=1000)
    N = prob.mesh.n_nodes
    assert st["converged"]
    assert u.min() >= -1e-9 and u.max() <= 1 + 1e-9
    # the limiter is active: the solution differs from the low-order one
    u_lo, _ = O.mc_stationary(prob, tol=1e-12, omega=1.0, mode="none", ksp="gmres", ksp_atol=1e-14)
    assert np.abs(u - u_lo).max() > 1e-3
