"""Pins for the oracle's mesh and matrices (Sec. 2: M_C, A, M_L, D, AA = A + D).

Each check compares with something the oracle does not compute itself:
exact integrals of polynomials that lie in the finite element space, textbook
stencils of uniform grids, and the algebraic properties the paper states for
D and AA (zero row sums, M-matrix sign pattern)."""
import numpy as np
import pytest

from oracle import afc_oracle as O
from paper_2110_15676_gb300 import workloads as W

BOX_LO = (0.0, -1.0, 0.5)
BOX_HI = (2.0, 0.5, 1.25)


def _box_integral(px, py, pz, lo=BOX_LO, hi=BOX_HI):
    """int over the box of x^px y^py z^pz."""
    out = 1.0
    for p, a, b in zip((px, py, pz), lo, hi):
        out *= (b ** (p + 1) - a ** (p + 1)) / (p + 1)
    return out


def _problem(elem, n=(4, 5, 3), b=(0.3, -0.2, 0.7), eps=1.0, c=0.0, lo=BOX_LO, hi=BOX_HI, fam="fct"):
    mesh = O.structured_mesh(elem, n, lo, hi)
    N = mesh.n_nodes
    bb = np.broadcast_to(np.asarray(b, dtype=float), (N, 3)) if np.ndim(b) == 1 else b
    return O.assemble(mesh, eps, bb, c, np.zeros(N), np.zeros(N, bool), np.zeros(N), fam), mesh


@pytest.mark.parametrize("elem", ["p1", "q1"])
def test_mass_integrates_polynomials_exactly(elem):
    prob, mesh = _problem(elem)
    x, y, z = mesh.xyz.T
    one = np.ones_like(x)
    M = prob.MC
    assert one @ M @ one == pytest.approx(_box_integral(0, 0, 0), rel=1e-13)
    assert x @ M @ y == pytest.approx(_box_integral(1, 1, 0), rel=1e-13)
    assert x @ M @ x == pytest.approx(_box_integral(2, 0, 0), rel=1e-13)
    assert z @ M @ (y + 2 * x) == pytest.approx(_box_integral(0, 1, 1) + 2 * _box_integral(1, 0, 1), rel=1e-13)
    assert prob.mL.sum() == pytest.approx(_box_integral(0, 0, 0), rel=1e-13)
    if elem == "q1":   # x*y and z are both in the trilinear space
        assert (x * y) @ M @ z == pytest.approx(_box_integral(1, 1, 1), rel=1e-13)
        assert (x * y * z) @ M @ (x * y * z) == pytest.approx(_box_integral(2, 2, 2), rel=1e-13)


@pytest.mark.parametrize("elem", ["p1", "q1"])
def test_stiffness_integrates_gradients_exactly(elem):
    prob, mesh = _problem(elem)
    x, y, z = mesh.xyz.T
    S = prob.S
    vol = _box_integral(0, 0, 0)
    assert x @ S @ x == pytest.approx(vol, rel=1e-12)
    assert (x + 2 * y - z) @ S @ (x + 2 * y - z) == pytest.approx(6 * vol, rel=1e-12)
    assert abs(x @ S @ y) < 1e-12 * vol
    assert np.abs(S @ np.ones_like(x)).max() < 1e-13
    if elem == "q1":   # grad(xy) = (y, x, 0)
        assert (x * y) @ S @ (x * y) == pytest.approx(_box_integral(0, 2, 0) + _box_integral(2, 0, 0), rel=1e-12)


@pytest.mark.parametrize("elem", ["p1", "q1"])
def test_convection_orientation_and_exactness(elem):
    """u^T K v = int (b . grad v) u for u, v in the space, b linear (rotating field).
    A transposed K would give int (b . grad u) v, which differs in sign here."""
    mesh = O.structured_mesh(elem, (5, 4, 3), BOX_LO, BOX_HI)
    N = mesh.n_nodes
    b = W.rotating_b(mesh.xyz)
    prob = O.assemble(mesh, 0.0, b, 0.0, np.zeros(N), np.zeros(N, bool), np.zeros(N))
    x, y, z = mesh.xyz.T
    K = prob.K
    # b = (0.5 - y, x - 0.5, 0): (b . grad x) = 0.5 - y, (b . grad y) = x - 0.5
    assert y @ K @ x == pytest.approx(0.5 * _box_integral(0, 1, 0) - _box_integral(0, 2, 0), rel=1e-12)
    assert x @ K @ y == pytest.approx(_box_integral(2, 0, 0) - 0.5 * _box_integral(1, 0, 0), rel=1e-12)
    assert abs(np.ones(N) @ K @ z) < 1e-13
    # row sums of K vanish (K applied to a constant)
    assert np.abs(K @ np.ones(N)).max() < 1e-14


def test_kuhn_p1_laplacian_is_seven_point_stencil():
    h = 0.25
    n = 5
    mesh = O.structured_mesh("p1", n, (0, 0, 0), (1, 1, 1))
    N = mesh.n_nodes
    prob = O.assemble(mesh, 1.0, np.zeros((N, 3)), 0.0, np.zeros(N), np.zeros(N, bool), np.zeros(N))
    S = prob.S.toarray()
    i = 2 + n * (2 + n * 2)             # interior node
    assert S[i, i] == pytest.approx(6 * h, rel=1e-13)
    for off in (1, n, n * n):
        assert S[i, i + off] == pytest.approx(-h, rel=1e-13)
        assert S[i, i - off] == pytest.approx(-h, rel=1e-13)
    # face and body diagonals of the Kuhn split are in the pattern but carry 0
    for off in (1 + n, n + n * n, 1 + n * n, 1 + n + n * n):
        assert prob.MC[i, i + off] != 0.0
        assert abs(S[i, i + off]) < 1e-15 and abs(S[i, i - off]) < 1e-15
    # interior lumped mass is h^3 (24 tetrahedra of volume h^3/6 share the node)
    assert prob.mL[i] == pytest.approx(h ** 3, rel=1e-13)


def test_q1_stencils():
    h = 0.25
    n = 5
    mesh = O.structured_mesh("q1", n, (0, 0, 0), (1, 1, 1))
    N = mesh.n_nodes
    prob = O.assemble(mesh, 1.0, np.zeros((N, 3)), 0.0, np.zeros(N), np.zeros(N, bool), np.zeros(N))
    S = prob.S.toarray(); M = prob.MC.toarray()
    i = 2 + n * (2 + n * 2)
    one_d = {-1: h / 6, 0: 4 * h / 6, 1: h / 6}          # 1D mass stencil
    lap = {0: 8 * h / 3, 1: 0.0, 2: -h / 6, 3: -h / 12}    # by number of nonzero offsets
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                j = i + dx + n * (dy + n * dz)
                assert M[i, j] == pytest.approx(one_d[dx] * one_d[dy] * one_d[dz], rel=1e-13)
                k = abs(dx) + abs(dy) + abs(dz)
                assert S[i, j] == pytest.approx(lap[k], rel=1e-13, abs=1e-15)


@pytest.mark.parametrize("elem", ["p1", "q1"])
@pytest.mark.parametrize("fam", ["fct", "mc"])
def test_upwinding_and_m_matrix(elem, fam):
    mesh = O.structured_mesh(elem, (5, 4, 4), BOX_LO, BOX_HI)
    N = mesh.n_nodes
    rng = np.random.default_rng(0)
    b = W.rotating_b(mesh.xyz) + rng.normal(scale=0.2, size=(N, 3))   # not divergence free
    c = 0.7
    prob = O.assemble(mesh, 1e-3, b, c, np.zeros(N), np.zeros(N, bool), np.zeros(N), fam)
    D = prob.D.toarray()
    A = prob.A.toarray()
    AA = prob.AA.toarray()
    assert np.abs(D - D.T).max() == 0.0                              # symmetric
    assert np.abs(D.sum(axis=1)).max() < 1e-15 * np.abs(D).max() * 30  # zero row sums
    off = ~np.eye(N, dtype=bool)
    assert (D[off] <= 0).all()
    # d_ij is exactly the smallest symmetric correction that removes positive off-diagonals
    Aoff = np.where(off, A, 0.0)
    assert (np.where(off, Aoff + D, 0.0) <= 0).all()
    assert (np.where(off, Aoff.T + D, 0.0) <= 0).all()
    both_nonpos = off & (Aoff <= 0) & (Aoff.T <= 0)
    assert (D[both_nonpos] == 0).all()
    if fam == "fct":
        assert (AA[off] <= 1e-15 * np.abs(AA).max()).all()         # M-matrix sign pattern
    else:
        # MC limits only the convective part (Remark rem:assembling_mc): K + D_K is
        # upwinded; the unlimited diffusion of an anisotropic Q1 grid may be positive
        KD = prob.K.toarray() + D
        assert (KD[off] <= 1e-15 * np.abs(KD).max()).all()
        S = prob.S.toarray()
        assert np.abs(AA - (KD + 1e-3 * S + np.diag(c * prob.mL))).max() < 1e-15 * np.abs(AA).max() * 10
    assert (np.diag(AA) > 0).all()
    # row sums of AA: c m_i (consistent reaction in FCT, lumped in MC: both sum to c m_i)
    assert np.abs(AA.sum(axis=1) - c * prob.mL).max() < 1e-13 * np.abs(AA).max()


@pytest.mark.parametrize("elem", ["p1", "q1"])
def test_nodal_reaction_matrix_closed_forms(elem):
    """The Galerkin reaction term (c_h phi_j, phi_i) with c interpolated from nodal values:
    a constant c gives c M_C, and for c = x, v = y, w = z (all in the FE space)
    1^T R 1 = int x = 1/2 and v^T R w = int x y z = 1/8; the MC system lumps R to its
    row sums (reading A9), so its row sums of AA are int c phi_i."""
    n = 5
    xyz = W.grid_coords(n)
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    mesh = O.structured_mesh(elem, n)
    N = len(xyz)
    b = np.zeros((N, 3))
    dm = np.zeros(N, bool)
    p_const = O.assemble(mesh, 0.0, b, 0.7, np.zeros(N), dm, np.zeros(N))
    p_nodal = O.assemble(mesh, 0.0, b, np.full(N, 0.7), np.zeros(N), dm, np.zeros(N))
    assert abs(p_nodal.A - p_const.A).max() <= 1e-15 * abs(p_const.A).max()
    p_x = O.assemble(mesh, 0.0, b, x, np.zeros(N), dm, np.zeros(N))
    R = p_x.A                                  # eps = 0, b = 0: A = R
    one = np.ones(N)
    assert abs(one @ (R @ one) - 0.5) < 1e-14
    assert abs(y @ (R @ z) - 0.125) < 1e-14
    m_x = O.assemble(mesh, 0.0, b, x, np.zeros(N), dm, np.zeros(N), "mc")
    rs = np.asarray(m_x.AA.sum(axis=1)).ravel()   # K = D = S-part = 0: AA = diag(row sums of R)
    assert np.abs(rs - np.asarray(R.sum(axis=1)).ravel()).max() < 1e-16
    assert abs(rs.sum() - 0.5) < 1e-14
