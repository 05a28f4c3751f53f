"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle on
identical seeded inputs.  Sizes span several thread blocks and ragged tails;
edge cases include single-cell grids, anisotropic boxes, element-list meshes
and every limiter mode.  Tolerances: per pass 1e-13 relative to the largest
magnitude of the compared quantity; per time step 1e-10 relative max-norm."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import afc_oracle as O
from paper_2110_15676_gb300 import workloads as W

from pairs import csr_of, gpu_problem, oracle_problem, pair_from_workload, random_workload, relerr

pytestmark = pytest.mark.gpu

PASS_TOL = 1e-13
STEP_TOL = 1e-10


@pytest.fixture(scope="module")
def afc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_15676_gb300 import afc as mod
    return mod


def _matrices(o):
    return {0: o.MC, 1: o.A, 2: o.D, 3: o.AA, 4: o.K, 5: o.S}


# ------------------------------------------------------------------ assembly
@pytest.mark.parametrize("elem", ["p1", "q1"])
@pytest.mark.parametrize("family", ["fct", "mc"])
@pytest.mark.parametrize("n,lo,hi", [((7, 6, 5), (0, 0, 0), (1, 1, 1)), ((2, 2, 2), (0, -1, 0.5), (2, 0.5, 1.25)),
                                     ((9, 3, 4), (0, -1, 0.5), (2, 0.5, 1.25))])
def test_assembly_matches_oracle(afc, elem, family, n, lo, hi):
    wl = random_workload(elem, n, seed=3, lo=lo, hi=hi)
    o, g = pair_from_workload(wl, family)
    for which, M in _matrices(o).items():
        G = csr_of(g, which)
        assert G.shape == M.shape
        if which == 0:   # the pattern is the set of pairs with m_ij != 0
            assert np.array_equal(G.indptr, M.indptr) and np.array_equal(G.indices, M.indices)
        scale = max(np.abs(M.data).max(), 1e-300)
        diff = (G - M).tocsr()
        assert (np.abs(diff.data).max() if diff.nnz else 0.0) <= PASS_TOL * scale * 10, which
    np.testing.assert_allclose(g.lumped_mass(), o.mL, rtol=1e-14)
    info = g.info()
    assert info["nnz"] == o.MC.nnz and info["n_nodes"] == o.mesh.n_nodes


@pytest.mark.parametrize("elem", ["p1", "q1"])
@pytest.mark.parametrize("family", ["fct", "mc"])
def test_nodal_reaction_and_constant_velocity_assembly(afc, elem, family):
    """afc_set_coefficients with a nodal reaction (the Galerkin matrix (c_h phi_j,
    phi_i); lumped in the MC family) and a constant velocity b_const: every matrix
    against the oracle's assembly of the same coefficients."""
    n, lo, hi = (7, 6, 5), (0, -1, 0.5), (2, 0.5, 1.25)
    wl = random_workload(elem, n, seed=31, lo=lo, hi=hi)
    rng = np.random.default_rng(32)
    c_nodal = rng.uniform(0.0, 2.0, wl.n_nodes)
    b_const = np.array([0.3, -0.7, 0.45])
    o = oracle_problem(wl.elem, wl.n, b_const, wl.eps, c_nodal, wl.f, wl.dir_mask, wl.u_dir, family, wl.lo, wl.hi)
    g = gpu_problem(wl.elem, wl.n, b_const, wl.eps, c_nodal, wl.f, wl.dir_mask, wl.u_dir, family, "fp64",
                    wl.lo, wl.hi)
    for which, M in _matrices(o).items():
        G = csr_of(g, which)
        scale = max(np.abs(M.data).max(), 1e-300)
        diff = (G - M).tocsr()
        assert (np.abs(diff.data).max() if diff.nnz else 0.0) <= PASS_TOL * scale * 10, which
    g.close()
    if family == "mc":
        # the stationary MC solve of the inflow problem with the nodal reaction 0.5 + x,
        # which enters AA and the residual lumped
        wl = W.stationary_inflow(elem, 9)
        c_nodal = 0.5 + W.grid_coords(wl.n)[:, 0]
        b_const = np.array([1.0, -0.5, 0.25])
        o = oracle_problem(wl.elem, wl.n, b_const, wl.eps, c_nodal, wl.f, wl.dir_mask, wl.u_dir, "mc")
        g = gpu_problem(wl.elem, wl.n, b_const, wl.eps, c_nodal, wl.f, wl.dir_mask, wl.u_dir, "mc")
        u_ref, st_o = O.mc_stationary(o, tol=1e-12, omega=0.5, ksp="direct", max_outer=3000)
        assert st_o["converged"]
        g.set_solution(wl.u0)
        st = g.solve_stationary(afc.default_opts(limiter=afc.AFC_LIM_MC, fp_tol=1e-12, omega=0.5,
                                                 ksp=afc.AFC_KSP_GMRES, ksp_atol=1e-14, fp_maxit=3000))
        assert st["status"] == afc.AFC_OK
        assert relerr(g.get_solution(), u_ref) < STEP_TOL
        g.close()


def _element_meshes():
    # two tetrahedra sharing a face
    two = (np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1.0]]), np.array([[0, 1, 2, 3], [1, 2, 3, 4]]))
    # the unit cube cut into five tetrahedra (one central, four corner ones)
    cube = np.array([[(k & 1), (k >> 1) & 1, (k >> 2) & 1] for k in range(8)], float)
    five = (cube, np.array([[0, 1, 2, 4], [1, 3, 2, 7], [1, 4, 5, 7], [2, 4, 6, 7], [1, 2, 4, 7]]))
    # a 1 x 1 x 2 block of trilinear cells
    xyz = np.array([[x, y, z] for z in (0, 0.5, 1.0) for y in (0, 1.0) for x in (0, 1.0)])
    two_hex = (xyz, np.array([[0, 1, 2, 3, 4, 5, 6, 7], [4, 5, 6, 7, 8, 9, 10, 11]]))
    return [("p1", *two), ("p1", *five), ("q1", *two_hex)]


@pytest.mark.parametrize("case", range(3))
def test_element_list_meshes(afc, case):
    elem, xyz, conn = _element_meshes()[case]
    N = len(xyz)
    rng = np.random.default_rng(case)
    b = rng.normal(size=(N, 3)); c = 0.4; eps = 0.01; f = rng.uniform(size=N)
    dm = np.zeros(N, np.uint8); dm[0] = 1
    ud = rng.uniform(size=N)
    mesh = O.Mesh(elem, xyz.astype(float), conn.astype(np.int64))
    o = O.assemble(mesh, eps, b, c, f, dm.astype(bool), ud)
    g = afc.Problem.from_elements(elem, xyz, conn)
    g.set_coefficients(eps, b, c, f)
    g.set_dirichlet(dm, ud)
    g.assemble()
    for which, M in _matrices(o).items():
        G = csr_of(g, which)
        assert np.abs((G - M).toarray()).max() <= PASS_TOL * 10 * max(np.abs(M.data).max(), 1e-300)
    # one Zalesak stage from a random state, brute-force sized
    u = rng.uniform(size=N); u[0] = ud[0]
    dt = O.cfl_timestep(o, 0.5)
    ref, d = O.fe_ssp_stage(o, u, dt, want=True)
    g.set_solution(u)
    out = g.fe_stage(dt)
    assert relerr(out["u_new"], ref) < PASS_TOL
    # F*_i is not formed at Dirichlet nodes (their r_ij are not needed, Sec. 2)
    free = ~dm.astype(bool)
    assert np.abs(out["Fstar"] - d["Fstar"])[free].max() <= PASS_TOL * max(np.abs(d["Fstar"]).max(), 1e-300)


# ------------------------------------------------------------------ explicit FCT
@pytest.mark.parametrize("elem,n", [("p1", 9), ("q1", 7), ("p1", (11, 5, 6)), ("q1", (13, 9, 3))])
@pytest.mark.parametrize("limiter", ["zalesak", "galerkin", "none"])
def test_fe_stage_pass_parity(afc, elem, n, limiter):
    wl = random_workload(elem, n, seed=11)
    o, g = pair_from_workload(wl)
    dt = O.cfl_timestep(o, 0.5)
    assert g.cfl_timestep(0.5) == pytest.approx(dt, rel=1e-14)
    ref, d = O.fe_ssp_stage(o, wl.u0, dt, mode=limiter, want=True)
    g.set_solution(wl.u0)
    lim = {"zalesak": afc.AFC_LIM_ZALESAK, "galerkin": afc.AFC_LIM_GALERKIN, "none": afc.AFC_LIM_NONE}[limiter]
    out = g.fe_stage(dt, lim)
    assert relerr(out["u_tilde"], d["u_tilde"]) < PASS_TOL
    free = ~wl.dir_mask.astype(bool)     # F*_i is not formed at Dirichlet nodes
    Fs = max(np.abs(d["Fstar"]).max(), 1e-300)
    assert np.abs(out["Fstar"] - d["Fstar"])[free].max() <= PASS_TOL * Fs * 10
    assert relerr(out["u_new"], ref) < PASS_TOL
    if limiter == "zalesak":
        assert np.abs(out["Rp"] - d["Rp"])[free].max() < 1e-12
        assert np.abs(out["Rm"] - d["Rm"])[free].max() < 1e-12


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("graph", [1, 0])
def test_ssp_rotating_run_parity_and_bounds(afc, order, graph):
    """The small rotating transient (Kuhn P1, 9^3 nodes, CFL 0.5, 20 steps), as one CUDA
    graph per step and as host-issued launches."""
    wl = W.rotating_transient("p1", 9)
    o, g = pair_from_workload(wl)
    dt = O.cfl_timestep(o, 0.5)
    u = wl.u0.copy()
    g.set_solution(u)
    opts = afc.default_opts(scheme=afc.AFC_SSP2 if order == 2 else afc.AFC_SSP3, dt=dt, graph=graph)
    for step in range(20):
        u = O.ssp_step(o, u, dt, order=order)
        st = g.step(opts)
        ug = g.get_solution()
        assert relerr(ug, u) < STEP_TOL, step
        assert ug.min() >= -1e-14 and ug.max() <= 1 + 1e-14
        assert st["umin"] == ug.min() and st["umax"] == ug.max()


def test_constant_state_preserved_on_gpu(afc):
    n = 10
    xyz = W.grid_coords(n)
    N = len(xyz)
    g = gpu_problem("q1", n, W.rotating_b(xyz), 1e-4, 0.0, np.zeros(N), W.boundary_mask(n), np.full(N, 0.37))
    g.set_solution(np.full(N, 0.37))
    dt = g.cfl_timestep(0.9)
    for scheme in (afc.AFC_SSP2, afc.AFC_SSP3):
        g.step(afc.default_opts(scheme=scheme, dt=dt))
        assert np.abs(g.get_solution() - 0.37).max() < 1e-15
    g.step(afc.default_opts(scheme=afc.AFC_CN_NONLINEAR, dt=dt))
    assert np.abs(g.get_solution() - 0.37).max() < 1e-14


# ------------------------------------------------------------------ Crank-Nicolson
@pytest.mark.parametrize("elem,n", [("q1", 9), ("p1", (10, 7, 6))])
@pytest.mark.parametrize("prelimit", [1, 0])
@pytest.mark.parametrize("limiter", ["zalesak", "galerkin", "none"])
def test_cn_limited_sum_parity(afc, elem, n, prelimit, limiter):
    wl = random_workload(elem, n, seed=5)
    o, g = pair_from_workload(wl)
    dt = O.cfl_timestep(o, 1.0)
    rng = np.random.default_rng(9)
    u_old = wl.u0
    u_new = u_old + rng.normal(scale=0.05, size=u_old.shape)
    u_new[wl.dir_mask.astype(bool)] = wl.u_dir[wl.dir_mask.astype(bool)]
    ut = u_old - 0.5 * dt * (o.AA @ u_old - o.f) / o.mL
    ut[o.dir_mask] = o.u_dir[o.dir_mask]
    r = O.cn_fluxes(o, u_new, u_old, dt, bool(prelimit))
    alpha, lim = O.zalesak_limiter(o, r, ut, dt, limiter)
    F = O.limited_sum(o, alpha, r)
    lmode = {"zalesak": afc.AFC_LIM_ZALESAK, "galerkin": afc.AFC_LIM_GALERKIN, "none": afc.AFC_LIM_NONE}[limiter]
    out = g.cn_limited_sum(dt, u_new, u_old, lmode, prelimit)
    assert relerr(out["u_tilde"], ut) < PASS_TOL
    free = ~o.dir_mask
    Fs = max(np.abs(F).max(), 1e-300)
    assert np.abs(out["Fstar"] - F)[free].max() <= PASS_TOL * Fs * 10
    if limiter == "zalesak":
        assert np.abs(out["Rp"] - lim["Rp"])[free].max() < 1e-12
        assert np.abs(out["Rm"] - lim["Rm"])[free].max() < 1e-12


@pytest.mark.parametrize("elem,n", [("q1", 9), ("p1", 8)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("graph", [1, 0])
def test_cn_steps_parity(afc, elem, n, precision, graph):
    """Nonlinear Zal+CN, CFL 1, a few steps; fixed number of corrections per step
    so that both sides do the same work, inner BiCGStab to 1e-14."""
    wl = W.rotating_transient(elem, n)
    o, g = pair_from_workload(wl, precision=precision)
    dt = O.cfl_timestep(o, 1.0)
    u = wl.u0.copy()
    g.set_solution(u)
    mixed = precision == "mixed"
    opts = afc.default_opts(scheme=afc.AFC_CN_NONLINEAR, dt=dt, fp_fixed_its=6, ksp_atol=0.0 if mixed else 1e-14,
                            ksp_rtol=1e-6 if mixed else 0.0,
                            precision=afc.AFC_MIXED if mixed else afc.AFC_FP64, graph=graph)
    for step in range(3):
        u, st_o = O.cn_step(o, u, dt, fixed_iterations=6, ksp_atol=1e-14)
        st = g.step(opts)
        ug = g.get_solution()
        err = relerr(ug, u)
        assert err < (1e-6 if mixed else STEP_TOL), (step, err)
        assert st["outer_its"] == 6


@pytest.mark.parametrize("elem,n", [("q1", 9), ("p1", 8)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("graph", [1, 0])
def test_cn_linear_steps_parity(afc, elem, n, precision, graph):
    """Linear Zal+CN: 4 steps against the oracle's literal linear scheme (direct solve)."""
    wl = W.rotating_transient(elem, n)
    o, g = pair_from_workload(wl, precision=precision)
    dt = O.cfl_timestep(o, 1.0)
    u = wl.u0.copy()
    g.set_solution(u)
    mixed = precision == "mixed"
    opts = afc.default_opts(scheme=afc.AFC_CN_LINEAR, dt=dt, ksp_atol=0.0 if mixed else 1e-14,
                            ksp_rtol=1e-7 if mixed else 0.0,
                            precision=afc.AFC_MIXED if mixed else afc.AFC_FP64, graph=graph)
    for step in range(4):
        u, _ = O.cn_linear_step(o, u, dt)
        st = g.step(opts)
        ug = g.get_solution()
        assert relerr(ug, u) < (1e-6 if mixed else STEP_TOL), step
        assert st["outer_its"] == 1


@pytest.mark.parametrize("elem,n", [("p1", 9), ("q1", 8)])
@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("graph", [1, 0])
def test_transient_mc_steps_parity(afc, elem, n, order, graph):
    """SSP2/SSP3 with the MC limiter (MC family), CFL 0.5, 10 steps."""
    wl = W.rotating_transient(elem, n)
    o, g = pair_from_workload(wl, "mc")
    dt = O.cfl_timestep(o, 0.5)
    u = wl.u0.copy()
    g.set_solution(u)
    opts = afc.default_opts(scheme=afc.AFC_SSP2 if order == 2 else afc.AFC_SSP3, limiter=afc.AFC_LIM_MC, dt=dt,
                            graph=graph)
    for step in range(10):
        u = O.ssp_step(o, u, dt, order=order, mode="mc")
        g.step(opts)
        ug = g.get_solution()
        assert relerr(ug, u) < STEP_TOL, step
        assert ug.min() >= -1e-14 and ug.max() <= 1 + 1e-14


@pytest.mark.parametrize("elem,n", [("p1", 9), ("q1", 8)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("graph", [1, 0])
def test_cn_mc_steps_parity(afc, elem, n, precision, graph):
    """Nonlinear CN with the MC limiter, CFL 1, 3 steps of 6 fixed-point corrections."""
    wl = W.rotating_transient(elem, n)
    o, g = pair_from_workload(wl, "mc", precision=precision)
    dt = O.cfl_timestep(o, 1.0)
    u = wl.u0.copy()
    g.set_solution(u)
    mixed = precision == "mixed"
    opts = afc.default_opts(scheme=afc.AFC_CN_NONLINEAR, limiter=afc.AFC_LIM_MC, dt=dt, fp_fixed_its=6,
                            ksp_atol=0.0 if mixed else 1e-14, ksp_rtol=1e-7 if mixed else 0.0,
                            precision=afc.AFC_MIXED if mixed else afc.AFC_FP64, graph=graph)
    for step in range(3):
        u, _ = O.cn_mc_step(o, u, dt, fixed_iterations=6)
        st = g.step(opts)
        assert relerr(g.get_solution(), u) < (1e-6 if mixed else STEP_TOL), step
        assert st["outer_its"] == 6


def test_transient_mc_stage_parity_and_errors(afc):
    wl = random_workload("q1", (7, 8, 6), seed=44)
    o, g = pair_from_workload(wl, "mc")
    dt = O.cfl_timestep(o, 0.5)
    g.set_solution(wl.u0)
    out = g.fe_stage(dt, afc.AFC_LIM_MC)
    un, info = O.fe_mc_stage(o, wl.u0, dt, want=True)
    free = ~o.dir_mask
    Fs = max(np.abs(info["Fstar"]).max(), 1e-300)
    assert np.abs(out["Fstar"] - info["Fstar"])[free].max() <= PASS_TOL * Fs * 10
    assert relerr(out["u_new"], un) < PASS_TOL * 10
    # transient MC needs the MC family and runs in FP64
    gf = gpu_problem(wl.elem, wl.n, wl.b, wl.eps, wl.c, wl.f, wl.dir_mask, wl.u_dir)
    with pytest.raises(afc.AfcError) as e:
        gf.step(afc.default_opts(scheme=afc.AFC_SSP3, limiter=afc.AFC_LIM_MC, dt=dt))
    assert e.value.status == afc.AFC_E_STATE
    with pytest.raises(afc.AfcError) as e:
        g.step(afc.default_opts(scheme=afc.AFC_SSP3, limiter=afc.AFC_LIM_MC, dt=dt, precision=afc.AFC_MIXED))
    assert e.value.status == afc.AFC_E_INVALID


def test_cn_converged_step_matches_oracle_tolerance(afc):
    wl = W.rotating_transient("q1", 11)
    o, g = pair_from_workload(wl)
    dt = O.cfl_timestep(o, 1.0)
    u_ref, st_o = O.cn_step(o, wl.u0, dt, tol=1e-12, ksp_atol=1e-14, max_outer=200)
    g.set_solution(wl.u0)
    st = g.step(afc.default_opts(scheme=afc.AFC_CN_NONLINEAR, dt=dt, fp_tol=1e-12, ksp_atol=1e-14, fp_maxit=200))
    assert st["status"] == afc.AFC_OK
    assert st["res_final"] < math.sqrt(o.mesh.n_nodes) * 1e-12
    assert relerr(g.get_solution(), u_ref) < STEP_TOL
    assert abs(st["outer_its"] - st_o["outer_its"]) <= 1


# ------------------------------------------------------------------ MC, stationary
@pytest.mark.parametrize("elem,n", [("p1", 9), ("q1", 7), ("p1", (12, 5, 7))])
@pytest.mark.parametrize("limiter", ["mc", "galerkin", "none"])
def test_mc_limited_sum_parity(afc, elem, n, limiter):
    wl = random_workload(elem, n, seed=21)
    o, g = pair_from_workload(wl, "mc")
    rng = np.random.default_rng(4)
    u = rng.uniform(0, 1, o.mesh.n_nodes)
    rstar, d = O.mc_limited_fluxes(o, u, limiter)
    F = O.limited_sum(o, np.ones_like(rstar), rstar)
    lm = {"mc": afc.AFC_LIM_MC, "galerkin": afc.AFC_LIM_GALERKIN, "none": afc.AFC_LIM_NONE}[limiter]
    out = g.mc_limited_sum(u, lm)
    free = ~o.dir_mask
    Fs = max(np.abs(F).max(), 1e-300)
    assert np.abs(out["Fstar"] - F)[free].max() <= PASS_TOL * Fs * 10
    if limiter == "mc":
        assert np.array_equal(out["umax"], d["umax"]) and np.array_equal(out["umin"], d["umin"])


@pytest.mark.parametrize("elem,n", [("p1", 9), ("q1", (8, 7, 6))])
def test_mu_limited_sum_parity(afc, elem, n):
    wl = random_workload(elem, n, seed=22)
    o, g = pair_from_workload(wl, "mc")
    rng = np.random.default_rng(5)
    u = rng.uniform(0, 1, o.mesh.n_nodes)
    rstar, _ = O.mu_limited_fluxes(o, u)
    F = O.limited_sum(o, np.ones_like(rstar), rstar)
    out = g.mc_limited_sum(u, afc.AFC_LIM_MU)
    free = ~o.dir_mask
    assert np.abs(out["Fstar"] - F)[free].max() <= PASS_TOL * max(np.abs(F).max(), 1e-300) * 10


@pytest.mark.parametrize("elem", ["p1", "q1"])
@pytest.mark.parametrize("graph", [1, 0])
def test_mu_stationary_parity(afc, elem, graph):
    wl = W.stationary_inflow(elem, 9)
    o, g = pair_from_workload(wl, "mc")
    u_ref, st_o = O.mc_stationary(o, tol=1e-12, omega=0.5, mode="mu", ksp="direct", max_outer=3000)
    assert st_o["converged"]
    g.set_solution(wl.u0)
    st = g.solve_stationary(afc.default_opts(limiter=afc.AFC_LIM_MU, fp_tol=1e-12, omega=0.5, ksp=afc.AFC_KSP_GMRES,
                                             ksp_atol=1e-14, fp_maxit=3000, graph=graph))
    assert st["status"] == afc.AFC_OK
    assert relerr(g.get_solution(), u_ref) < STEP_TOL


@pytest.mark.parametrize("elem", ["p1", "q1"])
@pytest.mark.parametrize("graph", [1, 0])
def test_mc_stationary_parity(afc, elem, graph):
    wl = W.stationary_inflow(elem, 9)
    o, g = pair_from_workload(wl, "mc")
    u_ref, st_o = O.mc_stationary(o, tol=1e-12, omega=0.5, ksp="gmres", ksp_atol=1e-14, max_outer=1000)
    g.set_solution(wl.u0)
    st = g.solve_stationary(afc.default_opts(limiter=afc.AFC_LIM_MC, fp_tol=1e-12, omega=0.5, ksp=afc.AFC_KSP_GMRES,
                                             ksp_atol=1e-14, fp_maxit=1000, graph=graph))
    assert st["status"] == afc.AFC_OK
    ug = g.get_solution()
    assert relerr(ug, u_ref) < STEP_TOL
    assert ug.min() >= -1e-10 and ug.max() <= 1 + 1e-10


def test_stationary_bicgstab_and_not_converged_status(afc):
    wl = W.stationary_inflow("p1", 9)
    o, g = pair_from_workload(wl, "mc")
    u_ref, _ = O.mc_stationary(o, tol=1e-11, omega=0.5, ksp="bicgstab", ksp_atol=1e-14, max_outer=1000)
    g.set_solution(wl.u0)
    st = g.solve_stationary(afc.default_opts(limiter=afc.AFC_LIM_MC, fp_tol=1e-11, omega=0.5, ksp=afc.AFC_KSP_BICGSTAB,
                                             ksp_atol=1e-14, fp_maxit=1000))
    assert st["status"] == afc.AFC_OK and relerr(g.get_solution(), u_ref) < STEP_TOL
    # an iteration limit that is too small returns the last iterate with AFC_NOT_CONVERGED
    g.set_solution(wl.u0)
    st = g.solve_stationary(afc.default_opts(limiter=afc.AFC_LIM_MC, fp_tol=1e-11, omega=0.5, fp_maxit=3))
    assert st["status"] == afc.AFC_NOT_CONVERGED and st["outer_its"] == 3


@pytest.mark.parametrize("elem", ["p1", "q1"])
@pytest.mark.parametrize("graph", [1, 0])
def test_mc_stationary_mixed_precision(afc, elem, graph):
    """FP32 inner GMRES, float-pair residual and clip: the converged solution within
    1e-6 of the FP64 oracle's, inside [0, 1] up to the solver tolerance."""
    wl = W.stationary_inflow(elem, 9)
    o, g = pair_from_workload(wl, "mc", precision="mixed")
    u_ref, _ = O.mc_stationary(o, tol=1e-10, omega=0.5, ksp="gmres", ksp_atol=1e-14, max_outer=1000)
    g.set_solution(wl.u0)
    st = g.solve_stationary(afc.default_opts(limiter=afc.AFC_LIM_MC, fp_tol=1e-10, omega=0.5, ksp=afc.AFC_KSP_GMRES,
                                             ksp_atol=0.0, ksp_rtol=1e-6, fp_maxit=1000, precision=afc.AFC_MIXED,
                                             graph=graph))
    assert st["status"] == afc.AFC_OK
    ug = g.get_solution()
    assert relerr(ug, u_ref) < 1e-6
    assert ug.min() >= -1e-10 and ug.max() <= 1 + 1e-10


def _pair_sweep_field(kind, o, wl, rng):
    N = o.mesh.n_nodes
    if kind == "uniform":
        u = rng.uniform(0, 1, N)
    elif kind == "front":
        u = W.front_field(o.mesh.xyz, rng)
    elif kind == "exact_floats":      # every value a float: the pairs' low parts are 0
        u = np.float32(rng.uniform(0, 1, N)).astype(np.float64)
        u[1::2] = u[0::2][: len(u[1::2])]                      # many equal neighbours
    else:                             # "wide": magnitudes over 70 decades, both signs
        u = rng.choice([-1.0, 1.0], N) * rng.uniform(1, 10, N) * 10.0 ** rng.uniform(-35, 35, N)
    u[o.dir_mask] = o.u_dir[o.dir_mask]
    return u


@pytest.mark.parametrize("elem,n", [("p1", 9), ("q1", (8, 7, 6)), ("p1", (17, 12, 10))])
@pytest.mark.parametrize("field", ["uniform", "front", "exact_floats", "wide"])
@pytest.mark.parametrize("limiter", ["mc", "galerkin"])
def test_mc_pair_sweep_parity(afc, elem, n, field, limiter):
    """The mixed-precision sweep (float-pair residual and clip, mc_pair.cu) against the
    oracle's residual f + F*(u) - AA u (Sec. 4, Eq. MClimiter), row by row, 0 on
    Dirichlet rows, and against the FP64 sweep of the same problem.  The bound is
    1e-13 of the magnitudes that enter row i (plus 1e-36 absolute, below which float
    pairs hold no digits): |f_i|, |AA_ij u_j|, and for each pair the terms of its two
    clip tests, 2|d_ij| times the bounds of both ends (which reach the neighbours of
    j) and |k_ij|, |k_ji| times |u_i| + |u_j|.  On the O(1) fields that is the row's
    scale; on the field spanning 70 decades it is what a rounding of the clip tests'
    terms can change, in FP64 as in float pairs."""
    wl = random_workload(elem, n, seed=23)
    o, g = pair_from_workload(wl, "mc", precision="mixed")
    rng = np.random.default_rng({"uniform": 1, "front": 2, "exact_floats": 3, "wide": 4}[field])
    u = _pair_sweep_field(field, o, wl, rng)
    lm = afc.AFC_LIM_MC if limiter == "mc" else afc.AFC_LIM_GALERKIN
    g.set_solution(u)
    g.mc_residual_sweep(lm)
    res = g.get_residual()
    rstar, _ = O.mc_limited_fluxes(o, u, limiter)
    F = O.limited_sum(o, np.ones_like(rstar), rstar)
    ro = o.f + F - o.AA @ u
    ro[o.dir_mask] = 0.0
    I, J = o.pairs
    umax, umin = O.mc_bounds(o, u)
    bnd = np.abs(umax) + np.abs(umin)
    d = np.abs(O.entries(o.D, I, J))
    kk = np.abs(O.entries(o.K, I, J)) + np.abs(O.entries(o.K, J, I))
    terms = np.abs(rstar) + 2.0 * d * (bnd[I] + bnd[J]) + kk * (np.abs(u[I]) + np.abs(u[J]))
    rabs = np.zeros(o.mesh.n_nodes)
    np.add.at(rabs, I, terms if limiter == "mc" else np.abs(rstar))
    scale = np.abs(o.f) + abs(o.AA) @ np.abs(u) + rabs
    assert (res[o.dir_mask] == 0).all()
    free = ~o.dir_mask
    assert (np.abs(res - ro)[free] <= PASS_TOL * scale[free] + 1e-36).all()
    # the FP64 sweep of the same problem
    g64 = gpu_problem(wl.elem, wl.n, wl.b, wl.eps, wl.c, wl.f, wl.dir_mask, wl.u_dir, "mc", "fp64", wl.lo, wl.hi)
    g64.set_solution(u)
    g64.mc_residual_sweep(lm)
    r64 = g64.get_residual()
    assert (np.abs(res - r64)[free] <= PASS_TOL * scale[free] + 1e-36).all()
    g.close()
    g64.close()


# ------------------------------------------------------------------ Krylov and SpMV
@pytest.mark.parametrize("system", [0, 1])
@pytest.mark.parametrize("ksp", ["bicgstab", "gmres"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_linear_solves(afc, system, ksp, precision):
    wl = random_workload("q1", (11, 9, 8), seed=2)
    fam = "fct" if system == 1 else "mc"
    o, g = pair_from_workload(wl, fam, precision=precision)
    dt = O.cfl_timestep(o, 1.0)
    B = O.cn_system_matrix(o, dt) if system == 1 else O.stationary_system_matrix(o)
    rng = np.random.default_rng(1)
    rhs = rng.normal(size=o.mesh.n_nodes)
    x_ref = spla.spsolve(B.tocsc(), rhs)
    mixed = precision == "mixed"
    opts = afc.default_opts(ksp=afc.AFC_KSP_GMRES if ksp == "gmres" else afc.AFC_KSP_BICGSTAB,
                            ksp_atol=0.0 if mixed else 1e-12, ksp_rtol=1e-6 if mixed else 0.0, ksp_maxit=2000,
                            precision=afc.AFC_MIXED if mixed else afc.AFC_FP64)
    x, its, res = g.linear_solve(system, rhs, opts, dt)
    assert its > 0
    true_res = np.linalg.norm(rhs - B @ x)
    if mixed:
        assert true_res < 1e-5 * np.linalg.norm(rhs)
    else:
        assert true_res < 2e-12
        assert relerr(x, x_ref) < 1e-10


@pytest.mark.parametrize("restart", [4, 13, 25, 32])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gmres_restart_lengths(afc, restart, precision):
    """GMRES(m) for restart lengths whose Arnoldi steps use every register class of the
    Gram-Schmidt pass (k + 1 up to 4, 8, 12, 16, 20, 24, 32), against a direct solve."""
    wl = random_workload("q1", (11, 9, 8), seed=3)
    o, g = pair_from_workload(wl, "mc", precision=precision)
    B = O.stationary_system_matrix(o)
    rhs = np.random.default_rng(restart).normal(size=o.mesh.n_nodes)
    x_ref = spla.spsolve(B.tocsc(), rhs)
    mixed = precision == "mixed"
    opts = afc.default_opts(ksp=afc.AFC_KSP_GMRES, ksp_atol=0.0 if mixed else 1e-12,
                            ksp_rtol=1e-6 if mixed else 0.0, ksp_maxit=5000, gmres_restart=restart,
                            precision=afc.AFC_MIXED if mixed else afc.AFC_FP64)
    x, its, res = g.linear_solve(0, rhs, opts, 0.0)
    assert its > 0
    true_res = np.linalg.norm(rhs - B @ x)
    if mixed:
        assert true_res < 1e-5 * np.linalg.norm(rhs)
    else:
        assert true_res < 2e-12
        assert relerr(x, x_ref) < 1e-10


def test_low_order_apply(afc):
    wl = random_workload("p1", (13, 11, 7), seed=8)
    o, g = pair_from_workload(wl)
    x = np.random.default_rng(0).normal(size=o.mesh.n_nodes)
    assert relerr(g.apply(afc.AFC_MAT_LOW, x), o.AA @ x) < PASS_TOL
    assert relerr(g.apply(afc.AFC_MAT_MC, x), o.MC @ x) < PASS_TOL


def test_errors_reported(afc):
    wl = random_workload("p1", 5, seed=1)
    g = afc.Problem.structured("p1", 5)
    with pytest.raises(afc.AfcError) as e:
        g.step(afc.default_opts(dt=0.1))
    assert e.value.status == afc.AFC_E_STATE
    g.set_coefficients(wl.eps, wl.b, wl.c, wl.f)
    g.assemble()
    with pytest.raises(afc.AfcError) as e:
        g.step(afc.default_opts(dt=-1.0))
    assert e.value.status == afc.AFC_E_INVALID
    with pytest.raises(afc.AfcError) as e:
        g.solve_stationary(afc.default_opts(limiter=afc.AFC_LIM_MC))
    assert e.value.status == afc.AFC_E_STATE          # MC needs the MC family
    g.set_dirichlet(np.ones(g.N, np.uint8), np.zeros(g.N))
    with pytest.raises(afc.AfcError):
        g.cfl_timestep(0.5)                             # no free node


# ------------------------------------------------------------------ afc_stats: DMP and timing
def test_dmp_violation_and_call_time_reported(afc):
    """afc_stats.dmp_violation = max(0, lo - umin, umax - hi), [lo, hi] the range of the
    call's input state and of the Dirichlet values: at rounding level for Zalesak's
    limiter on discontinuous data (Sec. 2.1.3: the limited stage stays in the local
    bounds), clearly positive for the unlimited Galerkin stage (alpha = 1) on the same
    data, and equal to its definition evaluated on the host from the states."""
    wl = W.rotating_shapes("q1", 17)
    g = gpu_problem(wl.elem, wl.n, wl.b, wl.eps, wl.c, wl.f, wl.dir_mask, wl.u_dir)
    dm = wl.dir_mask.astype(bool)
    dt = g.cfl_timestep(0.5)
    for lim, small in ((afc.AFC_LIM_ZALESAK, True), (afc.AFC_LIM_GALERKIN, False)):
        g.set_solution(wl.u0)
        worst = 0.0
        for step in range(6):
            u_in = g.get_solution()
            st = g.step(afc.default_opts(scheme=afc.AFC_SSP3, limiter=lim, dt=dt))
            u_out = g.get_solution()
            lo = min(u_in.min(), wl.u_dir[dm].min())
            hi = max(u_in.max(), wl.u_dir[dm].max())
            ref = max(0.0, lo - u_out.min(), u_out.max() - hi)
            assert abs(st["dmp_violation"] - ref) <= 1e-15 * max(1.0, ref)
            assert st["t_ms"] > 0.0
            worst = max(worst, st["dmp_violation"])
        if small:
            assert worst <= 1e-14
        else:
            assert worst > 1e-3
    g.close()
