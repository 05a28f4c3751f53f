"""Brute force on meshes of one to two cells: the oracle's vectorised limiters
equal (R+/- and alpha to two units in the last place, F* to 1e-15) the dense
loop-by-loop transcriptions of tests/bruteforce.py over every sign
pattern of the raw fluxes and every Dirichlet mask (Zalesak, one tetrahedron), over
sampled sign patterns and masks on two tetrahedra and two hexahedra (Zalesak), and
over every ordering of the nodal values (MC)."""
import itertools

import numpy as np
import pytest

from oracle import afc_oracle as O
import bruteforce as BF


def _ulps(a, b, n=2):
    """Equal to within n units in the last place: the oracle evaluates Zalesak's
    quotient m Q / (dt P) as (m Q / dt) / P, the transcription as printed, and the two
    roundings may differ in their last bit."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return bool((np.abs(a - b) <= n * np.spacing(np.maximum(np.abs(a), np.abs(b)))).all())


def _problem(elem, xyz, conn, dirichlet, family="fct", seed=0):
    rng = np.random.default_rng(seed)
    N = len(xyz)
    b = rng.normal(size=(N, 3))
    mesh = O.Mesh(elem, xyz.astype(float), conn.astype(np.int64))
    return O.assemble(mesh, 0.01, b, 0.3, rng.uniform(size=N), np.asarray(dirichlet, bool), rng.uniform(size=N),
                      family)


def test_zalesak_every_sign_pattern_and_dirichlet_mask():
    elem, xyz, conn = BF.one_tet()
    N = len(xyz)
    rng = np.random.default_rng(1)
    pairs = [(i, j) for i in range(N) for j in range(i + 1, N)]
    base = _problem(elem, xyz, conn, np.zeros(N))
    mC = base.MC.toarray()
    dt = O.cfl_timestep(base, 0.5)
    u_tilde = rng.uniform(size=N)
    checked = 0
    for mask in itertools.product([0, 1], repeat=N):
        prob = _problem(elem, xyz, conn, mask)
        I, J = prob.pairs
        for signs in itertools.product([-1.0, 0.0, 1.0], repeat=len(pairs)):
            r = np.zeros((N, N))
            for (i, j), sg in zip(pairs, signs):
                r[i, j] = sg * rng.uniform(0.1, 1.0)
                r[j, i] = -r[i, j]
            rd = r[I, J]
            alpha, lim = O.zalesak_limiter(prob, rd, u_tilde, dt, "zalesak")
            F = O.limited_sum(prob, alpha, rd)
            a_bf, F_bf, Rp_bf, Rm_bf = BF.zalesak(r, mC, prob.mL, u_tilde, dt, np.asarray(mask, bool))
            assert _ulps(lim["Rp"], Rp_bf) and _ulps(lim["Rm"], Rm_bf)
            nz = rd != 0.0                  # alpha is irrelevant where r = 0 (reading A11)
            assert _ulps(alpha[nz], a_bf[I, J][nz])
            assert np.abs(F - F_bf).max() <= 1e-15 * max(np.abs(F_bf).max(), 1.0)
            checked += 1
    assert checked == 16 * 729


def _zalesak_case(prob, mC, u_tilde, dt, mask, r):
    I, J = prob.pairs
    rd = r[I, J]
    alpha, lim = O.zalesak_limiter(prob, rd, u_tilde, dt, "zalesak")
    F = O.limited_sum(prob, alpha, rd)
    a_bf, F_bf, Rp_bf, Rm_bf = BF.zalesak(r, mC, prob.mL, u_tilde, dt, np.asarray(mask, bool))
    assert _ulps(lim["Rp"], Rp_bf) and _ulps(lim["Rm"], Rm_bf)
    nz = rd != 0.0                          # alpha is irrelevant where r = 0 (reading A11)
    assert _ulps(alpha[nz], a_bf[I, J][nz])
    assert np.abs(F - F_bf).max() <= 1e-15 * max(np.abs(F_bf).max(), 1.0)


@pytest.mark.parametrize("case,n_masks,n_signs", [("two_tets", 32, 120), ("two_hexes", 10, 60)])
def test_zalesak_sampled_sign_patterns_on_two_cells(case, n_masks, n_signs):
    """Sec. 2.1.3, steps 1-4 on two cells sharing a face: every Dirichlet mask of the
    two tetrahedra (10 seeded masks of the hexahedra) and seeded sign patterns of the
    raw fluxes, including zero fluxes, so that a node's P+/- and Q+/- collect pairs of
    both cells."""
    elem, xyz, conn = getattr(BF, case)()
    N = len(xyz)
    rng = np.random.default_rng(5)
    base = _problem(elem, xyz, conn, np.zeros(N))
    mC = base.MC.toarray()
    pairs = [(i, j) for i in range(N) for j in range(i + 1, N) if mC[i, j] != 0.0]
    dt = O.cfl_timestep(base, 0.5)
    masks = list(itertools.product([0, 1], repeat=N)) if 2 ** N <= n_masks else \
        [tuple(rng.integers(0, 2, N)) for _ in range(n_masks)]
    checked = 0
    for mask in masks:
        prob = _problem(elem, xyz, conn, mask)
        u_tilde = rng.uniform(size=N)
        for _ in range(n_signs):
            signs = rng.choice([-1.0, 0.0, 1.0], size=len(pairs), p=[0.45, 0.1, 0.45])
            r = np.zeros((N, N))
            for (i, j), sg in zip(pairs, signs):
                r[i, j] = sg * rng.uniform(0.1, 1.0)
                r[j, i] = -r[i, j]
            _zalesak_case(prob, mC, u_tilde, dt, mask, r)
            checked += 1
    assert checked == len(masks) * n_signs


def test_mc_every_ordering_of_the_nodal_values():
    for elem, xyz, conn in (BF.one_tet(), BF.two_tets(), BF.two_hexes()):
        N = len(xyz)
        prob = _problem(elem, xyz, conn, np.zeros(N), family="mc", seed=2)
        mC, D, Kc = prob.MC.toarray(), prob.D.toarray(), prob.K.toarray()
        I, J = prob.pairs
        rng = np.random.default_rng(3)
        vals = np.sort(rng.uniform(size=N))
        perms = itertools.permutations(range(N)) if N <= 5 else (rng.permutation(N) for _ in range(400))
        for perm in perms:
            u = vals[list(perm)]
            rs, info = O.mc_limited_fluxes(prob, u, "mc")
            rs_bf, F_bf, umax, umin = BF.mc(u, mC, D, Kc)
            assert np.array_equal(info["umax"], umax) and np.array_equal(info["umin"], umin)
            assert np.abs(rs - rs_bf[I, J]).max() <= 1e-15 * max(np.abs(rs_bf).max(), 1e-300)
