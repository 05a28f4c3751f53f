"""Pins for the oracle's explicit SSP + Zalesak FCT stage (Sec. 2.1.2, Sec. 2.1.3).

What fixes the stage without a reference implementation:
  * alpha = 1 reproduces the Galerkin right-hand side, alpha = 0 the low-order
    forward Euler step (the statement after Eq. definition_of_f_i);
  * conservation: sum_i F*_i = 0 (r_ji = -r_ij, alpha_ij = alpha_ji);
  * local bounds: every updated value lies in [min, max] of the predictor over
    its neighbourhood (the purpose of Q^+/- in step 2);
  * Zalesak's factors are the largest admissible ones: where R_i^+ < 1 limits
    all positive fluxes into i, the bound at i is met with equality;
  * constants are preserved; a full rotating run stays in [0, 1].
Bounds, neighbourhoods and predictors are recomputed here from the pinned
matrices, not taken from the oracle."""
import math

import numpy as np
import pytest

from oracle import afc_oracle as O
from paper_2110_15676_gb300 import workloads as W


def _random_problem(elem, n=6, seed=1, c=0.3, eps=1e-3, dir_frac=0.3):
    rng = np.random.default_rng(seed)
    mesh = O.structured_mesh(elem, n)
    N = mesh.n_nodes
    b = W.rotating_b(mesh.xyz) + rng.normal(scale=0.3, size=(N, 3))
    f = rng.uniform(0.0, 1.0, N)
    dm = W.boundary_mask(n).astype(bool) & (rng.uniform(size=N) < 0.5 + dir_frac)
    ud = rng.uniform(0.0, 1.0, N)
    prob = O.assemble(mesh, eps, b, c, f, dm, ud)
    u = rng.uniform(0.0, 1.0, N)
    u[dm] = ud[dm]
    dt = O.cfl_timestep(prob, 0.5)
    return prob, u, dt


def _neighbour_extremes(prob, v):
    """min / max of v over N_i (pattern of M_C, including i), from the dense matrix."""
    M = prob.MC.toarray()
    big = np.where(M != 0.0, v[None, :], -np.inf).max(axis=1)
    small = np.where(M != 0.0, v[None, :], np.inf).min(axis=1)
    return small, big


@pytest.mark.parametrize("elem", ["p1", "q1"])
def test_alpha_one_is_galerkin(elem):
    prob, u, dt = _random_problem(elem)
    free = ~prob.dir_mask
    u_new = O.fe_ssp_stage(prob, u, dt, mode="galerkin")
    A, MC, mL = prob.A, prob.MC, prob.mL
    # Galerkin with the low-order rate: M_L u_new = M_L u + dt (f - A u + (M_L - M_C) udot^L)
    udot = (prob.f - prob.AA @ u) / mL
    udot[prob.dir_mask] = 0.0
    rhs = mL * u + dt * (prob.f - A @ u + mL * udot - MC @ udot)
    assert np.abs(mL * u_new - rhs)[free].max() < 1e-14 * np.abs(rhs).max()
    assert np.array_equal(u_new[prob.dir_mask], prob.u_dir[prob.dir_mask])


@pytest.mark.parametrize("elem", ["p1", "q1"])
def test_alpha_zero_is_low_order(elem):
    prob, u, dt = _random_problem(elem)
    free = ~prob.dir_mask
    u_new = O.fe_ssp_stage(prob, u, dt, mode="none")
    ref = u + dt * (prob.f - prob.AA @ u) / prob.mL
    assert np.abs(u_new - ref)[free].max() < 1e-15 * 4


@pytest.mark.parametrize("elem", ["p1", "q1"])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_zalesak_stage_bounds_conservation_maximality(elem, seed):
    prob, u, dt = _random_problem(elem, seed=seed)
    free = ~prob.dir_mask
    u_new, d = O.fe_ssp_stage(prob, u, dt, want=True)
    I, J = prob.pairs
    # predictor, recomputed from the matrices
    ut = u + dt * (prob.f - prob.AA @ u) / prob.mL
    ut[prob.dir_mask] = prob.u_dir[prob.dir_mask]
    assert np.abs(ut - d["u_tilde"]).max() < 1e-15
    lo, hi = _neighbour_extremes(prob, ut)
    tol = 1e-14
    assert (u_new[free] <= hi[free] + tol).all()
    assert (u_new[free] >= lo[free] - tol).all()
    # conservation of the limited antidiffusive term
    F = d["Fstar"]
    assert abs(F.sum()) < 1e-14 * np.abs(F).sum()
    # antisymmetric fluxes, symmetric correction factors
    key = {(i, j): k for k, (i, j) in enumerate(zip(I, J))}
    mate = np.array([key[(j, i)] for i, j in zip(I, J)])
    r, a = d["r"], d["alpha"]
    # (M_C is symmetric up to the order in which element contributions were summed)
    assert np.abs(r[mate] + r).max() <= 1e-15 * np.abs(r).max()
    nz = np.abs(r) > 1e-12 * np.abs(r).max()
    assert np.abs(a[mate][nz] - a[nz]).max() <= 1e-12
    assert ((a >= 0) & (a <= 1)).all()
    # maximality: where R_i^+ < 1 and every positive flux into i is limited by R_i^+,
    # the upper bound is attained: (dt / m_i) sum_{r_ij > 0} alpha_ij r_ij = max_j ut_j - ut_i
    Rp, Rm = d["Rp"], d["Rm"]
    N = prob.mesh.n_nodes
    pos_sum = np.bincount(I, weights=np.where(r > 0, a * r, 0.0), minlength=N)
    neg_sum = np.bincount(I, weights=np.where(r < 0, a * r, 0.0), minlength=N)
    tight_p = np.ones(N, bool); tight_m = np.ones(N, bool)
    np.logical_and.at(tight_p, I, ~(r > 0) | (a == Rp[I]))
    np.logical_and.at(tight_m, I, ~(r < 0) | (a == Rm[I]))
    sel_p = free & (Rp < 1) & tight_p
    sel_m = free & (Rm < 1) & tight_m
    assert sel_p.sum() + sel_m.sum() > 0
    np.testing.assert_allclose(dt * pos_sum[sel_p] / prob.mL[sel_p], (hi - ut)[sel_p], rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(dt * neg_sum[sel_m] / prob.mL[sel_m], (lo - ut)[sel_m], rtol=1e-12, atol=1e-16)
    # and no factor is smaller than needed: an unlimited node keeps alpha = min of both ends
    assert np.array_equal(a, np.where(r > 0, np.minimum(Rp[I], Rm[J]), np.minimum(Rm[I], Rp[J])))


@pytest.mark.parametrize("elem", ["p1", "q1"])
def test_constants_preserved(elem):
    n = 6
    mesh = O.structured_mesh(elem, n)
    N = mesh.n_nodes
    rng = np.random.default_rng(5)
    b = W.rotating_b(mesh.xyz)
    dm = W.boundary_mask(n).astype(bool)
    prob = O.assemble(mesh, 1e-4, b, 0.0, np.zeros(N), dm, np.full(N, 0.37))
    u = np.full(N, 0.37)
    dt = O.cfl_timestep(prob, 0.9)
    for order in (2, 3):
        v = O.ssp_step(prob, u, dt, order=order)
        assert np.abs(v - 0.37).max() < 1e-15


@pytest.mark.parametrize("order", [2, 3])
def test_rotating_run_stays_in_unit_interval(order):
    wl = W.rotating_transient("p1", 9)
    mesh = O.structured_mesh(wl.elem, wl.n)
    prob = O.assemble(mesh, wl.eps, wl.b, wl.c, wl.f, wl.dir_mask.astype(bool), wl.u_dir)
    dt = O.cfl_timestep(prob, 0.5)
    u = wl.u0.copy()
    for _ in range(20):
        u = O.ssp_step(prob, u, dt, order=order)
        assert u.min() >= -1e-14 and u.max() <= 1 + 1e-14
    assert u.max() > 0.01         # the (diffused) hump is still there


def test_ssp_orders_converge_at_their_rate():
    """Galerkin (alpha = 1) SSP2/SSP3 on a smooth problem: halving dt divides the
    difference to a fine-step solution by ~4 and ~8 (the linear system is smooth)."""
    wl = W.rotating_transient("q1", 7, eps=1e-2)
    mesh = O.structured_mesh(wl.elem, wl.n)
    prob = O.assemble(mesh, wl.eps, wl.b, wl.c, wl.f, wl.dir_mask.astype(bool), wl.u_dir)
    T = 0.05
    def run(order, steps):
        u = wl.u0.copy()
        for _ in range(steps):
            u = O.ssp_step(prob, u, T / steps, order=order, mode="none")
        return u
    for order, rate in ((2, 4.0), (3, 8.0)):
        ref = run(order, 256)
        e1 = np.abs(run(order, 16) - ref).max()
        e2 = np.abs(run(order, 32) - ref).max()
        assert e1 / e2 == pytest.approx(rate, rel=0.2)
