"""Brute force through the C ABI on meshes of one to two cells: the CUDA limiter
passes equal the dense loop-by-loop transcriptions of tests/bruteforce.py for
random states under every Dirichlet mask of a tetrahedron (Zalesak stage: R+/-
and F*) and for every ordering of the nodal values (MC: bounds and F*)."""
import itertools

import numpy as np
import pytest

from oracle import afc_oracle as O
import bruteforce as BF

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def afc():
    from paper_2110_15676_gb300 import afc as A
    return A


def _pair(afc, elem, xyz, conn, mask, family, seed=0):
    rng = np.random.default_rng(seed)
    N = len(xyz)
    b = rng.normal(size=(N, 3)); f = rng.uniform(size=N); ud = rng.uniform(size=N)
    mesh = O.Mesh(elem, xyz.astype(float), conn.astype(np.int64))
    o = O.assemble(mesh, 0.01, b, 0.3, f, np.asarray(mask, bool), ud, family)
    g = afc.Problem.from_elements(elem, xyz, conn)
    g.set_coefficients(0.01, b, 0.3, f)
    g.set_dirichlet(np.asarray(mask, np.uint8), ud)
    g.assemble(afc.AFC_FAMILY_FCT if family == "fct" else afc.AFC_FAMILY_MC)
    return o, g


@pytest.mark.parametrize("case", ["one_tet", "two_tets", "two_hexes"])
def test_zalesak_stage_against_brute_force(afc, case):
    elem, xyz, conn = getattr(BF, case)()
    N = len(xyz)
    masks = list(itertools.product([0, 1], repeat=N)) if N <= 5 else \
        [tuple(np.random.default_rng(k).integers(0, 2, N)) for k in range(12)]
    rng = np.random.default_rng(7)
    for mask in masks:
        o, g = _pair(afc, elem, xyz, conn, mask, "fct")
        dm = np.asarray(mask, bool)
        mC, D, AA = o.MC.toarray(), o.D.toarray(), o.AA.toarray()
        dt = O.cfl_timestep(o, 0.5) if not dm.all() else 0.1
        for _ in range(6):
            u = rng.uniform(size=N)
            u[dm] = o.u_dir[dm]
            udot = (o.f - AA @ u) / o.mL
            udot[dm] = 0.0
            ut = u + dt * udot
            ut[dm] = o.u_dir[dm]
            r = mC * (udot[:, None] - udot[None, :]) + D * (u[None, :] - u[:, None])
            np.fill_diagonal(r, 0.0)
            _, F, Rp, Rm = BF.zalesak(r, mC, o.mL, ut, dt, dm)
            g.set_solution(u)
            out = g.fe_stage(dt)
            scale = max(np.abs(F).max(), 1e-300)
            free = ~dm
            if free.any():
                assert np.abs(out["Fstar"] - F)[free].max() <= 1e-12 * scale
            assert np.abs(out["Rp"] - Rp).max() <= 1e-12 and np.abs(out["Rm"] - Rm).max() <= 1e-12
        g.close()


@pytest.mark.parametrize("case", ["one_tet", "two_tets", "two_hexes"])
def test_mc_limited_sum_against_brute_force(afc, case):
    elem, xyz, conn = getattr(BF, case)()
    N = len(xyz)
    o, g = _pair(afc, elem, xyz, conn, np.zeros(N), "mc", seed=3)
    mC, D, Kc = o.MC.toarray(), o.D.toarray(), o.K.toarray()
    rng = np.random.default_rng(4)
    vals = np.sort(rng.uniform(size=N))
    perms = itertools.permutations(range(N)) if N <= 5 else (rng.permutation(N) for _ in range(200))
    for perm in perms:
        u = vals[list(perm)]
        _, F, umax, umin = BF.mc(u, mC, D, Kc)
        out = g.mc_limited_sum(u, afc.AFC_LIM_MC)
        assert np.array_equal(out["umax"], umax) and np.array_equal(out["umin"], umin)
        assert np.abs(out["Fstar"] - F).max() <= 1e-12 * max(np.abs(F).max(), 1e-300)
    g.close()
