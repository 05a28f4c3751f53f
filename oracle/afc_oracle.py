"""Plain, slow, FP64 CPU oracle for algebraic flux correction (AFC) of P1/Q1
finite element discretisations of 3D convection-diffusion-reaction equations.

TEST INFRASTRUCTURE ONLY.  This module exists to check the CUDA library.  Only
the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA path: it builds its
own mesh, its own matrices and runs its own loops, in numpy/scipy, in float64.

Every function follows the paper (Jha, Partl, Ahmed, Kuzmin, "An assessment of
solvers for algebraically stabilized discretizations of convection-diffusion-
reaction equations", arXiv 2110.15676) in its own order and notation:

  * Galerkin matrices M_C, A (Sec. 2, Eq. high_order_disc and the entries m_ij,
    a_ij that follow it), lumped mass M_L and discrete upwinding D (Sec. 2),
    low-order operator  AA = A + D (Eq. low_order_disc);
  * raw antidiffusive fluxes r_ij (Eq. r_decomposition), the SSP version with
    the low-order rate (Eq. defn_r_ij_SSP, Eq. lower_time_approx), the
    Crank-Nicolson version (Eq. flux_002) with prelimiting (Eq. prelimiting);
  * Zalesak's limiter (Sec. 2.1.3, steps 1-4);
  * the explicit FE-SSP update (Eq. FE-SSP) and its low-order predictor;
  * the CN predictor (Eq. forward_euler) and the nonlinear CN system (Eq. CNZal);
  * the monolithic convex limiter (Eq. MClimiter, Eq. u_max_min) for the
    stationary problem (Sec. 3.1) with the operator split of Remark
    rem:assembling_mc;
  * the damped fixed-point iteration and stopping rules (Sec. 4, Eq. tol_formula);
  * textbook Jacobi-preconditioned BiCGStab (van der Vorst 1992) and restarted
    GMRES(m) with modified Gram-Schmidt and Givens rotations (Saad & Schultz
    1986), plus a dense direct solve for tiny systems.

Readings of passages the paper leaves open (numbered as in the design notes):
  A2  Q_i^+/- are taken over the sparsity neighbours N_i \\ {i}, not all j.
  A3  The prelimiting argument u is the CN average (u^n + u^{n-1})/2; minmod is
      0 whenever one argument is 0.
  A5  The damped fixed point is u <- u + omega * (AA^{-1}(f + F*(u)) - u),
      solved in defect form.
  A6  Delta t = CFL * min_{i not Dirichlet} m_i / AA_ii.
  A8  MC uses the convective matrix K only for d_ij and the bar states; the
      system matrix is K + D_K + eps*S + c*M_L.
  A9  Reaction in the MC system is lumped (c*M_L).
  A13 The load vector is M_L f_nodal.
  A15 The low-order rate is 0 at Dirichlet nodes (their value does not change).
  A16 An MC flux with d_ij = 0 is limited to 0.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

P1 = "p1"
Q1 = "q1"


# --------------------------------------------------------------------------
# Mesh
# --------------------------------------------------------------------------
@dataclass
class Mesh:
    elem: str                 # "p1" (tetrahedra) or "q1" (trilinear hexahedra)
    xyz: np.ndarray           # (N, 3) node coordinates
    cells: np.ndarray         # (n_cells, 4) or (n_cells, 8) node indices

    @property
    def n_nodes(self) -> int:
        return self.xyz.shape[0]


def structured_mesh(elem: str, n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> Mesh:
    """Uniform box grid with n = (nx, ny, nz) nodes per side, node index
    ix + nx*(iy + ny*iz).  Q1: one hexahedron per cell, local vertex
    k = dx + 2 dy + 4 dz.  P1: each cell cut into the six Kuhn tetrahedra that
    share the diagonal from corner (0,0,0) to corner (1,1,1); tetrahedron for the
    axis order (a, b, c) is {0, e_a, e_a + e_b, e_a + e_b + e_c}."""
    if np.isscalar(n):
        n = (int(n),) * 3
    nx, ny, nz = n
    xs = [np.linspace(lo[d], hi[d], n[d]) for d in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    ix, iy, iz = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), np.arange(nz - 1), indexing="ij")
    ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
    corners = []
    for k in range(8):
        dx, dy, dz = k & 1, (k >> 1) & 1, (k >> 2) & 1
        corners.append((ix + dx) + nx * ((iy + dy) + ny * (iz + dz)))
    corners = np.stack(corners, axis=1)
    if elem == Q1:
        cells = corners
    elif elem == P1:
        tets = []
        for a, b, c in itertools.permutations(range(3)):
            loc = [0, 1 << a, (1 << a) | (1 << b), 7]
            tets.append(corners[:, loc])
        cells = np.concatenate(tets, axis=0)
    else:
        raise ValueError(elem)
    return Mesh(elem, xyz.astype(np.float64), cells.astype(np.int64))


# --------------------------------------------------------------------------
# Element matrices (Sec. 2: m_ij = (phi_j, phi_i),
# a_ij = eps (grad phi_j, grad phi_i) + (b . grad phi_j, phi_i) + (c phi_j, phi_i))
# --------------------------------------------------------------------------
def p1_element_matrices(X, B):
    """X: (E, 4, 3) vertices, B: (E, 4, 3) nodal velocity, for E tetrahedra.
    Exact integrals for the linear basis lambda_k:
    int lambda_i lambda_j = V (1 + delta_ij) / 20, and with b = sum_k b_k lambda_k
    the convection entry is sum_k (b_k . grad lambda_j) V (1 + delta_ik) / 20.
    Returns (E, 4, 4) mass M, stiffness S, convection C with C[e, i, j] = (b.grad phi_j, phi_i)."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, 4, 3)
    B = np.asarray(B, dtype=np.float64).reshape(-1, 4, 3)
    J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)   # columns
    V = np.abs(np.linalg.det(J)) / 6.0
    Jinv = np.linalg.inv(J)
    G = np.zeros((X.shape[0], 4, 3))
    G[:, 1:] = Jinv                   # grad lambda_k = row k of J^{-1}, k = 1..3
    G[:, 0] = -Jinv.sum(axis=1)
    M = V[:, None, None] * (np.ones((4, 4)) + np.eye(4))[None] / 20.0
    S = V[:, None, None] * np.einsum("eid,ejd->eij", G, G)
    BG = np.einsum("ekd,ejd->ekj", B, G)      # BG[e, k, j] = b_k . grad lambda_j
    C = np.einsum("eik,ekj->eij", M, BG)      # C[e, i, j] = sum_k M[i, k] b_k . grad lambda_j
    return M, S, C


def p1_reaction_matrix(X, Cn):
    """(c_h phi_j, phi_i) for c_h = sum_k c_k lambda_k, exactly:
    int lambda_i lambda_j lambda_k = V (1 + d_ij + d_ik + d_jk + 2 d_ijk) / 120
    (the integral of a product of barycentric coordinates, 6 V a! b! c! d! / (a+b+c+d+3)!).
    X: (E, 4, 3) vertices, Cn: (E, 4) nodal reaction.  Returns (E, 4, 4)."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, 4, 3)
    Cn = np.asarray(Cn, dtype=np.float64).reshape(-1, 4)
    J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)
    V = np.abs(np.linalg.det(J)) / 6.0
    d = np.eye(4)
    T = (1.0 + d[:, :, None] + d[:, None, :] + d[None, :, :] + 2.0 * np.einsum("ij,jk->ijk", d, d)) / 120.0
    return V[:, None, None] * np.einsum("ijk,ek->eij", T, Cn)


_GAUSS01 = (0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0))


def q1_reaction_matrix(X, Cn):
    """(c_h phi_j, phi_i) for the trilinear interpolant c_h of the nodal reaction, by
    2x2x2 Gauss quadrature (exact on parallelepipeds: the integrand has degree 3 in
    each reference coordinate).  X: (E, 8, 3), Cn: (E, 8).  Returns (E, 8, 8)."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, 8, 3)
    Cn = np.asarray(Cn, dtype=np.float64).reshape(-1, 8)
    R = np.zeros((X.shape[0], 8, 8))
    bits = np.array([[k & 1, (k >> 1) & 1, (k >> 2) & 1] for k in range(8)], dtype=np.float64)
    for xi in itertools.product(_GAUSS01, repeat=3):
        f1 = [np.where(bits[:, d] == 1, xi[d], 1.0 - xi[d]) for d in range(3)]
        df = [np.where(bits[:, d] == 1, 1.0, -1.0) for d in range(3)]
        phi = f1[0] * f1[1] * f1[2]
        dphi_ref = np.stack([df[0] * f1[1] * f1[2], f1[0] * df[1] * f1[2], f1[0] * f1[1] * df[2]], axis=1)
        J = np.einsum("eka,kd->ead", X, dphi_ref)
        wd = 0.125 * np.abs(np.linalg.det(J))
        cq = Cn @ phi
        R += (wd * cq)[:, None, None] * np.outer(phi, phi)[None]
    return R


def q1_element_matrices(X, B):
    """Trilinear elements on the reference cube [0,1]^3, vertex k = dx + 2dy + 4dz,
    2x2x2 Gauss quadrature (exact on parallelepipeds for mass, stiffness and
    convection with a trilinearly interpolated velocity).  X, B: (E, 8, 3)."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, 8, 3)
    B = np.asarray(B, dtype=np.float64).reshape(-1, 8, 3)
    E = X.shape[0]
    M = np.zeros((E, 8, 8)); S = np.zeros((E, 8, 8)); C = np.zeros((E, 8, 8))
    bits = np.array([[k & 1, (k >> 1) & 1, (k >> 2) & 1] for k in range(8)], dtype=np.float64)
    for xi in itertools.product(_GAUSS01, repeat=3):
        w = 0.125
        f1 = [np.where(bits[:, d] == 1, xi[d], 1.0 - xi[d]) for d in range(3)]
        df = [np.where(bits[:, d] == 1, 1.0, -1.0) for d in range(3)]
        phi = f1[0] * f1[1] * f1[2]                                        # (8,)
        dphi_ref = np.stack([df[0] * f1[1] * f1[2], f1[0] * df[1] * f1[2], f1[0] * f1[1] * df[2]], axis=1)
        J = np.einsum("eka,kd->ead", X, dphi_ref)     # J[e, a, d] = d x_a / d xi_d
        detJ = np.linalg.det(J)
        dphi = np.einsum("kd,eda->eka", dphi_ref, np.linalg.inv(J))   # grad_x phi_k = J^{-T} grad_xi phi_k
        bq = np.einsum("k,eka->ea", phi, B)
        wd = (w * np.abs(detJ))[:, None, None]
        M += wd * np.outer(phi, phi)[None]
        S += wd * np.einsum("eia,eja->eij", dphi, dphi)
        C += wd * np.einsum("i,eja,ea->eij", phi, dphi, bq)      # C[e, i, j] = (b . grad phi_j) phi_i
    return M, S, C


# --------------------------------------------------------------------------
# Problem assembly
# --------------------------------------------------------------------------
@dataclass
class Problem:
    mesh: Mesh
    eps: float
    c: object                     # constant reaction (float) or nodal values (N,)
    b: np.ndarray                 # (N, 3) nodal velocity
    f_nodal: np.ndarray           # (N,)
    dir_mask: np.ndarray          # (N,) bool
    u_dir: np.ndarray             # (N,) Dirichlet values (used where dir_mask)
    limiter_family: str = "fct"   # "fct" (Zalesak) or "mc"
    # assembled quantities
    MC: sp.csr_matrix = None      # consistent mass
    S: sp.csr_matrix = None       # stiffness (grad phi_j, grad phi_i)
    K: sp.csr_matrix = None       # convection (b . grad phi_j, phi_i)
    A: sp.csr_matrix = None       # operator whose off-diagonals define D
    D: sp.csr_matrix = None       # discrete upwinding
    AA: sp.csr_matrix = None      # low-order operator (system operator for MC)
    mL: np.ndarray = None         # lumped mass m_i
    f: np.ndarray = None          # load vector M_L f_nodal (A13)
    pairs: tuple = None           # directed off-diagonal pairs (I, J) with m_IJ != 0
    extra: dict = field(default_factory=dict)


def assemble(mesh: Mesh, eps: float, b, c, f_nodal, dir_mask, u_dir, limiter_family="fct") -> Problem:
    """c: a constant reaction (float) or nodal values (N,), interpolated with the
    element basis; the reaction term is the Galerkin matrix (c phi_j, phi_i) (= c M_C
    for a constant), lumped to its row sums in the MC system (reading A9)."""
    N = mesh.n_nodes
    b = np.broadcast_to(np.asarray(b, dtype=np.float64), (N, 3)).copy()
    f_nodal = np.broadcast_to(np.asarray(f_nodal, dtype=np.float64), (N,)).copy()
    dir_mask = np.asarray(dir_mask, dtype=bool).copy()
    u_dir = np.broadcast_to(np.asarray(u_dir, dtype=np.float64), (N,)).copy()
    elmat = p1_element_matrices if mesh.elem == P1 else q1_element_matrices
    nl = mesh.cells.shape[1]
    cells = mesh.cells
    Me, Se, Ce = elmat(mesh.xyz[cells], b[cells])
    rows = np.repeat(cells, nl, axis=1).ravel()           # row index of entry (e, i, j) is cells[e, i]
    cols = np.tile(cells, (1, nl)).ravel()                # column index is cells[e, j]
    MC = sp.csr_matrix((Me.ravel(), (rows, cols)), shape=(N, N))
    S = sp.csr_matrix((Se.ravel(), (rows, cols)), shape=(N, N))
    K = sp.csr_matrix((Ce.ravel(), (rows, cols)), shape=(N, N))
    for X in (MC, S, K):
        X.sum_duplicates(); X.sort_indices()
    # all three share the element pattern; make the stored patterns identical
    pattern = (abs(MC) + abs(S) + abs(K)).tocsr()
    pattern.data[:] = 1.0
    MC = _on_pattern(MC, pattern); S = _on_pattern(S, pattern); K = _on_pattern(K, pattern)
    mL = np.asarray(MC.sum(axis=1)).ravel()                   # m_i = sum_j m_ij
    if np.ndim(c) == 0:
        R = c * MC
        rL = c * mL
    else:
        cn = np.broadcast_to(np.asarray(c, dtype=np.float64), (N,))
        rmat = p1_reaction_matrix if mesh.elem == P1 else q1_reaction_matrix
        R = sp.csr_matrix((rmat(mesh.xyz[cells], cn[cells]).ravel(), (rows, cols)), shape=(N, N))
        R.sum_duplicates()
        R = _on_pattern(R, pattern)
        rL = np.asarray(R.sum(axis=1)).ravel()
    if limiter_family == "fct":
        A = (eps * S + K + R).tocsr()                         # a_ij of Sec. 2
        D = discrete_upwinding(A)
        AA = (A + D).tocsr()
    elif limiter_family == "mc":
        # Remark rem:assembling_mc with readings A8, A9: flux correction for the
        # eps = 0, c = 0 operator, unlimited diffusion and (lumped) reaction.
        A = K.copy()
        D = discrete_upwinding(K)
        AA = (K + D + eps * S + sp.diags(rL)).tocsr()
    else:
        raise ValueError(limiter_family)
    AA = _on_pattern(AA, pattern)
    I, J = _offdiag_pairs(MC)
    prob = Problem(mesh, eps, c, b, f_nodal, dir_mask, u_dir, limiter_family,
                   MC=MC, S=S, K=K, A=A, D=D, AA=AA, mL=mL, f=mL * f_nodal, pairs=(I, J))
    return prob


def _on_pattern(X, pattern):
    """Return X with exactly the stored pattern of `pattern` (explicit zeros kept)."""
    X = X.tocsr()
    P = pattern.tocoo()
    vals = np.asarray(X[P.row, P.col]).ravel()
    Y = sp.csr_matrix((vals, (P.row, P.col)), shape=X.shape)
    Y.sort_indices()
    return Y


def _offdiag_pairs(MC):
    """Directed pairs (i, j), i != j, with m_ij != 0: the neighbour sets N_i of Eq. u_max_min."""
    C = MC.tocoo()
    keep = (C.row != C.col) & (C.data != 0.0)
    return C.row[keep].astype(np.int64), C.col[keep].astype(np.int64)


def entries(X, I, J):
    return np.asarray(X[I, J]).ravel()


def discrete_upwinding(A):
    """D of Sec. 2: d_ij = -max{a_ij, 0, a_ji} (i != j), d_ii = -sum_{j != i} d_ij."""
    A = A.tocsr()
    C = A.tocoo()
    off = C.row != C.col
    I, Jc = C.row[off], C.col[off]
    aij = C.data[off]
    aji = entries(A, Jc, I)
    dij = -np.maximum(np.maximum(aij, 0.0), aji)
    N = A.shape[0]
    Doff = sp.csr_matrix((dij, (I, Jc)), shape=(N, N))
    diag = -np.asarray(Doff.sum(axis=1)).ravel()
    return (Doff + sp.diags(diag)).tocsr()


def cfl_timestep(prob: Problem, cfl: float) -> float:
    """Reading A6: Delta t = CFL * min over non-Dirichlet i of m_i / AA_ii."""
    diag = prob.AA.diagonal()
    free = ~prob.dir_mask
    return float(cfl * np.min(prob.mL[free] / diag[free]))


# --------------------------------------------------------------------------
# Zalesak's limiter (Sec. 2.1.3)
# --------------------------------------------------------------------------
def zalesak_limiter(prob: Problem, r, u_tilde, dt, mode="zalesak"):
    """r: antidiffusive fluxes r_ij on the directed pairs (I, J).
    mode "zalesak": steps 1-4 of Sec. 2.1.3; "galerkin": alpha = 1; "none": alpha = 0.
    Returns alpha on the pairs and the node arrays P+, P-, Q+, Q-, R+, R-."""
    I, J = prob.pairs
    N = prob.mesh.n_nodes
    # step 1
    Pp = np.bincount(I, weights=np.maximum(r, 0.0), minlength=N)
    Pm = np.bincount(I, weights=np.minimum(r, 0.0), minlength=N)
    # step 2 (reading A2: j over the neighbours N_i \ {i})
    Qp = np.zeros(N); Qm = np.zeros(N)
    np.maximum.at(Qp, I, u_tilde[J] - u_tilde[I])
    np.minimum.at(Qm, I, u_tilde[J] - u_tilde[I])
    # step 3: m_i Q_i / (dt P_i), taken as (m_i Q_i / dt) / P_i so that a subnormal
    # P_i != 0, whose product with dt underflows to 0, cannot make it 0 / 0
    with np.errstate(divide="ignore", invalid="ignore"):
        Rp = np.where(Pp != 0.0, np.minimum(1.0, (prob.mL * Qp / dt) / Pp), 1.0)
        Rm = np.where(Pm != 0.0, np.minimum(1.0, (prob.mL * Qm / dt) / Pm), 1.0)
    Rp[prob.dir_mask] = 1.0
    Rm[prob.dir_mask] = 1.0
    # step 4
    alpha = np.where(r > 0.0, np.minimum(Rp[I], Rm[J]), np.minimum(Rm[I], Rp[J]))
    if mode == "galerkin":
        alpha = np.ones_like(r)
    elif mode == "none":
        alpha = np.zeros_like(r)
    elif mode != "zalesak":
        raise ValueError(mode)
    return alpha, dict(Pp=Pp, Pm=Pm, Qp=Qp, Qm=Qm, Rp=Rp, Rm=Rm)


def limited_sum(prob: Problem, alpha, r):
    """F*_i = sum_{j != i} alpha_ij r_ij (Eq. definition_of_f_i)."""
    I, _ = prob.pairs
    return np.bincount(I, weights=alpha * r, minlength=prob.mesh.n_nodes)


# --------------------------------------------------------------------------
# Explicit SSP schemes with Zalesak FCT (Sec. 2.1.2)
# --------------------------------------------------------------------------
def low_order_rate(prob: Problem, u):
    """Eq. lower_time_approx: udot^L = M_L^{-1}(f - AA u); 0 at Dirichlet nodes (A15)."""
    udot = (prob.f - prob.AA @ u) / prob.mL
    udot[prob.dir_mask] = 0.0
    return udot


def ssp_fluxes(prob: Problem, u, udot):
    """Eq. defn_r_ij_SSP: r_ij = m_ij (udot_i - udot_j) + d_ij (u_j - u_i)."""
    I, J = prob.pairs
    m = entries(prob.MC, I, J)
    d = entries(prob.D, I, J)
    return m * (udot[I] - udot[J]) + d * (u[J] - u[I])


def fe_ssp_stage(prob: Problem, u, dt, mode="zalesak", want=False):
    """One forward-Euler FCT stage, Eq. FE-SSP, with the predictor
    u~ = u + dt M_L^{-1}(f - AA u) constrained to the Dirichlet data."""
    udot = low_order_rate(prob, u)
    u_tilde = u + dt * (prob.f - prob.AA @ u) / prob.mL
    u_tilde[prob.dir_mask] = prob.u_dir[prob.dir_mask]
    r = ssp_fluxes(prob, u, udot)
    alpha, lim = zalesak_limiter(prob, r, u_tilde, dt, mode)
    Fstar = limited_sum(prob, alpha, r)
    u_new = u + dt * (prob.f + Fstar - prob.AA @ u) / prob.mL
    u_new[prob.dir_mask] = prob.u_dir[prob.dir_mask]
    if want:
        return u_new, dict(udot=udot, u_tilde=u_tilde, r=r, alpha=alpha, Fstar=Fstar, **lim)
    return u_new


def fe_mc_stage(prob: Problem, u, dt, want=False):
    """One forward-Euler stage of the transient MC scheme (Sec. 2.2): the fluxes of
    Eq. defn_r_ij_SSP with the low-order rate, limited by Eq. MClimiter with the
    bounds and bar states of the stage input u, F*_i = sum_j r*_ij and
    u_new = u + dt M_L^{-1}(f + F* - AA u), u_D on Dirichlet nodes (MC family)."""
    udot = low_order_rate(prob, u)
    r = ssp_fluxes(prob, u, udot)
    rstar, lim = mc_clip(prob, u, r)
    Fstar = limited_sum(prob, np.ones_like(rstar), rstar)
    u_new = u + dt * (prob.f + Fstar - prob.AA @ u) / prob.mL
    u_new[prob.dir_mask] = prob.u_dir[prob.dir_mask]
    if want:
        return u_new, dict(udot=udot, rstar=rstar, Fstar=Fstar, **lim)
    return u_new


def ssp_step(prob: Problem, u, dt, order=3, mode="zalesak"):
    """order 2: Heun's method as written in Sec. 2.1.2, u^n = (u^{n,0} + u^{n,2}) / 2.
    order 3: the three-stage Shu-Osher SSP scheme (reading A1), each stage one
    forward-Euler FCT update (mode "mc": one forward-Euler MC stage)."""
    if mode == "mc":
        stage = lambda v: fe_mc_stage(prob, v, dt)  # noqa: E731
    else:
        stage = lambda v: fe_ssp_stage(prob, v, dt, mode)  # noqa: E731
    if order == 2:
        u1 = stage(u)
        u2 = stage(u1)
        return 0.5 * (u + u2)
    if order == 3:
        u1 = stage(u)
        u2 = 0.75 * u + 0.25 * stage(u1)
        return u / 3.0 + (2.0 / 3.0) * stage(u2)
    raise ValueError(order)


# --------------------------------------------------------------------------
# Crank-Nicolson FCT (Sec. 2.1.1), nonlinear fixed point (Sec. 4)
# --------------------------------------------------------------------------
def minmod(a, b):
    """Eq. prelimiting: 0 if ab < 0, min if both > 0, max if both < 0 (0 otherwise, A3)."""
    out = np.zeros_like(a)
    pos = (a > 0.0) & (b > 0.0)
    neg = (a < 0.0) & (b < 0.0)
    out[pos] = np.minimum(a[pos], b[pos])
    out[neg] = np.maximum(a[neg], b[neg])
    return out


def cn_fluxes(prob: Problem, u_new, u_old, dt, prelimit=True):
    """Eq. flux_002, then Eq. prelimiting with L = 2 applied to the CN average (A3)."""
    I, J = prob.pairs
    m = entries(prob.MC, I, J)
    d = entries(prob.D, I, J)
    r = (m / dt) * ((u_new[I] - u_old[I]) - (u_new[J] - u_old[J])) \
        + 0.5 * d * ((u_new[J] + u_old[J]) - (u_new[I] + u_old[I]))
    if prelimit:
        ubar = 0.5 * (u_new + u_old)
        r = minmod(r, 2.0 * d * (ubar[J] - ubar[I]))
    return r


def cn_system_matrix(prob: Problem, dt):
    """M_L / dt + AA / 2 with the Dirichlet rows replaced by identity rows."""
    B = (sp.diags(prob.mL / dt) + 0.5 * prob.AA).tolil()
    for i in np.flatnonzero(prob.dir_mask):
        B.rows[i] = [i]; B.data[i] = [1.0]
    return B.tocsr()


def mc_transient_flux_sum(prob: Problem, u):
    """F*_i(u) = sum_j r*_ij(u) of the transient MC scheme (Sec. 2.2): fluxes
    Eq. defn_r_ij_SSP with the low-order rate at u, clipped by Eq. MClimiter."""
    udot = low_order_rate(prob, u)
    rstar, _ = mc_clip(prob, u, ssp_fluxes(prob, u, udot))
    return limited_sum(prob, np.ones_like(rstar), rstar)


def cn_mc_step(prob: Problem, u_old, dt, tol=1e-10, max_outer=100, omega=1.0, ksp="direct", ksp_atol=1e-12,
               ksp_rtol=0.0, ksp_maxit=1000, gmres_restart=20, fixed_iterations=None):
    """One CN step with the MC limiter (Sec. 2.2): Eq. CNZal with
    F* = (F*(u^n) + F*(u^{n-1})) / 2, F*(u) = sum_j r*_ij(u) (mc_transient_flux_sum),
    by the damped fixed point of Sec. 4 from u^{n-1}; MC family.  Returns (u_new, stats)."""
    N = prob.mesh.n_nodes
    dirm = prob.dir_mask
    b0 = prob.mL / dt * u_old - 0.5 * (prob.AA @ u_old) + prob.f
    F_old = mc_transient_flux_sum(prob, u_old)
    Bsys = cn_system_matrix(prob, dt)
    dinv = 1.0 / Bsys.diagonal()
    lu = spla.splu(Bsys.tocsc()) if ksp == "direct" else None
    u = u_old.copy()
    u[dirm] = prob.u_dir[dirm]
    stats = dict(outer_its=0, inner_its=0, res_hist=[])
    for it in range(max_outer + 1):
        Fstar = 0.5 * (mc_transient_flux_sum(prob, u) + F_old)
        res = b0 + Fstar - (prob.mL / dt * u + 0.5 * (prob.AA @ u))
        res[dirm] = 0.0
        R = float(np.linalg.norm(res))
        stats["res_hist"].append(R)
        if fixed_iterations is None:
            if R < math.sqrt(N) * tol or it == max_outer:
                break
        elif it == fixed_iterations:
            break
        if lu is not None:
            delta = lu.solve(res)
        else:
            delta, kst = krylov_solve(Bsys, res, dinv, ksp, ksp_atol, ksp_rtol, ksp_maxit, gmres_restart)
            stats["inner_its"] += kst["its"]
        u = u + omega * delta
        stats["outer_its"] += 1
    stats["res_final"] = stats["res_hist"][-1]
    stats["converged"] = stats["res_final"] < math.sqrt(N) * tol
    return u, stats


def cn_linear_step(prob: Problem, u_old, dt, prelimit=True, mode="zalesak", ksp="direct", ksp_atol=1e-12,
                   ksp_rtol=0.0, ksp_maxit=1000, gmres_restart=20):
    """One step of linear Zal+CN (Sec. 2.1.1, the linearised scheme): u^n in the flux
    formula Eq. flux_002 (and in the prelimiting of reading A3) is replaced by
    2 u~ - u^{n-1}, u~ the predictor Eq. forward_euler, so the fluxes and the factors
    are known before the step and Eq. CNZal becomes one linear system
    (M_L/dt + AA/2) u^n = b0 + F*, Dirichlet rows u^n = u_D.  Returns (u_new, stats)."""
    dirm = prob.dir_mask
    u_tilde = u_old - 0.5 * dt * (prob.AA @ u_old - prob.f) / prob.mL
    u_tilde[dirm] = prob.u_dir[dirm]
    b0 = prob.mL / dt * u_old - 0.5 * (prob.AA @ u_old) + prob.f
    u_approx = 2.0 * u_tilde - u_old
    r = cn_fluxes(prob, u_approx, u_old, dt, prelimit)
    alpha, _ = zalesak_limiter(prob, r, u_tilde, dt, mode)
    Fstar = limited_sum(prob, alpha, r)
    rhs = b0 + Fstar
    rhs[dirm] = prob.u_dir[dirm]
    Bsys = cn_system_matrix(prob, dt)
    if ksp == "direct":
        u = spla.splu(Bsys.tocsc()).solve(rhs)
        its = 0
    else:
        u, kst = krylov_solve(Bsys, rhs, 1.0 / Bsys.diagonal(), ksp, ksp_atol, ksp_rtol, ksp_maxit, gmres_restart)
        its = kst["its"]
    return u, dict(outer_its=1, inner_its=its, Fstar=Fstar, u_tilde=u_tilde)


def cn_step(prob: Problem, u_old, dt, tol=1e-10, max_outer=100, omega=1.0, prelimit=True,
            mode="zalesak", ksp="bicgstab", ksp_atol=1e-12, ksp_rtol=0.0, ksp_maxit=1000,
            gmres_restart=20, fixed_iterations=None):
    """One step of nonlinear Zal+CN: solve Eq. CNZal by the damped fixed point of Sec. 4,
    u <- u + omega * B^{-1} res(u),  res(u) = b0 + F*(u, u_old) - B u,  B = M_L/dt + AA/2,
    stop when ||res||_2 < sqrt(N) tol (Eq. tol_formula).  Q+/- come from the CN predictor
    Eq. forward_euler, which stays fixed for the whole step.  The initial guess is u_old.
    Returns (u_new, stats)."""
    N = prob.mesh.n_nodes
    dirm = prob.dir_mask
    u_tilde = u_old - 0.5 * dt * (prob.AA @ u_old - prob.f) / prob.mL
    u_tilde[dirm] = prob.u_dir[dirm]
    b0 = prob.mL / dt * u_old - 0.5 * (prob.AA @ u_old) + prob.f     # (f^n + f^{n-1})/2 = f
    Bsys = cn_system_matrix(prob, dt)
    dinv = 1.0 / Bsys.diagonal()
    lu = spla.splu(Bsys.tocsc()) if ksp == "direct" else None   # factor once: the matrix is fixed
    u = u_old.copy()
    u[dirm] = prob.u_dir[dirm]
    stats = dict(outer_its=0, inner_its=0, res_hist=[])
    for it in range(max_outer + 1):
        r = cn_fluxes(prob, u, u_old, dt, prelimit)
        alpha, _ = zalesak_limiter(prob, r, u_tilde, dt, mode)
        Fstar = limited_sum(prob, alpha, r)
        res = b0 + Fstar - (prob.mL / dt * u + 0.5 * (prob.AA @ u))
        res[dirm] = 0.0
        R = float(np.linalg.norm(res))
        stats["res_hist"].append(R)
        if fixed_iterations is None:
            if R < math.sqrt(N) * tol or it == max_outer:
                break
        elif it == fixed_iterations:
            break
        if lu is not None:
            delta = lu.solve(res)
        else:
            delta, kst = krylov_solve(Bsys, res, dinv, ksp, ksp_atol, ksp_rtol, ksp_maxit, gmres_restart)
            stats["inner_its"] += kst["its"]
        u = u + omega * delta
        stats["outer_its"] += 1
    stats["res_final"] = stats["res_hist"][-1]
    stats["converged"] = stats["res_final"] < math.sqrt(N) * tol
    return u, stats


# --------------------------------------------------------------------------
# Monolithic convex limiter, stationary problem (Sec. 2.2, Sec. 3.1)
# --------------------------------------------------------------------------
def mc_bounds(prob: Problem, u):
    """Eq. u_max_min over N_i (which contains i)."""
    I, J = prob.pairs
    umax = u.copy(); umin = u.copy()
    np.maximum.at(umax, I, u[J])
    np.minimum.at(umin, I, u[J])
    return umax, umin


def mc_limited_fluxes(prob: Problem, u, mode="mc"):
    """Eq. MClimiter with r_ij = d_ij (u_j - u_i) (Sec. 3.1), bar states
    2 d_ij ubar_ij = d_ij (u_i + u_j) + a_ij (u_j - u_i), a_ij the convective
    entries (A8).  Returns r*_ij on the directed pairs and the bounds."""
    I, J = prob.pairs
    d = entries(prob.D, I, J)
    r = d * (u[J] - u[I])
    if mode == "galerkin":
        return r, {}
    if mode == "none":
        return np.zeros_like(r), {}
    return mc_clip(prob, u, r)


def mc_clip(prob: Problem, u, r):
    """Eq. MClimiter applied to given fluxes r_ij on the directed pairs, with the
    bounds Eq. u_max_min and the bar states of the state u."""
    I, J = prob.pairs
    d = entries(prob.D, I, J)
    aij = entries(prob.K, I, J)
    aji = entries(prob.K, J, I)
    umax, umin = mc_bounds(prob, u)
    rstar = np.zeros_like(r)
    nz = d != 0.0                                        # A16
    dI, uI, uJ = d[nz], u[I[nz]], u[J[nz]]
    ubar_ij = (dI * (uI + uJ) + aij[nz] * (uJ - uI)) / (2.0 * dI)
    ubar_ji = (dI * (uJ + uI) + aji[nz] * (uI - uJ)) / (2.0 * dI)
    rr = r[nz]
    up = np.minimum(rr, np.minimum(2.0 * dI * (ubar_ij - umax[I[nz]]), 2.0 * dI * (umin[J[nz]] - ubar_ji)))
    dn = np.maximum(rr, np.maximum(2.0 * dI * (ubar_ij - umin[I[nz]]), 2.0 * dI * (umax[J[nz]] - ubar_ji)))
    rstar[nz] = np.where(rr > 0.0, up, dn)
    return rstar, dict(umax=umax, umin=umin, r=r)


def mu_limited_fluxes(prob: Problem, u):
    """Monolithic upwind limiter (Sec. 3, MU limiter) on the stationary fluxes
    r_ij = d_ij (u_j - u_i), a_ij the convective entries (A8):
      1. P_i^+/- = sum of r_ij^+/- over the j with a_ji <= a_ij,
      2. Q_i^+ = -sum_j r_ij^-,  Q_i^- = -sum_j r_ij^+  (all neighbours),
      3. R_i^+/- = min{1, Q_i^+/- / P_i^+/-}, 1 at Dirichlet nodes or where P = 0,
      4. for a_ji <= a_ij: alpha_ij = R_i^+ (r_ij > 0), 1 (r_ij = 0), R_i^- (r_ij < 0),
         and alpha_ji = alpha_ij.
    A pair with a_ij = a_ji would be assigned from both ends; it is taken by the
    end with the smaller index, in steps 1 and 4 alike (reading A21).  a_ij and a_ji
    are computed values, so they count as equal within 1e-12 (|a_ij| + |a_ji|):
    pairs that tie exactly in exact arithmetic stay ties after rounding.  Returns
    alpha_ij r_ij on the directed pairs and the factors."""
    I, J = prob.pairs
    d = entries(prob.D, I, J)
    aij = entries(prob.K, I, J)
    aji = entries(prob.K, J, I)
    r = d * (u[J] - u[I])
    N = prob.mesh.n_nodes
    tie = np.abs(aij - aji) <= 1e-12 * (np.abs(aij) + np.abs(aji))
    owns = np.where(tie, I < J, aji < aij)               # i takes the pair (i, j)
    rp = np.maximum(r, 0.0)
    rm = np.minimum(r, 0.0)
    Pp = np.zeros(N); Pm = np.zeros(N); Qp = np.zeros(N); Qm = np.zeros(N)
    np.add.at(Pp, I[owns], rp[owns])
    np.add.at(Pm, I[owns], rm[owns])
    np.add.at(Qp, I, -rm)
    np.add.at(Qm, I, -rp)
    Rp = np.ones(N); Rm = np.ones(N)
    nzp = Pp != 0.0
    nzm = Pm != 0.0
    with np.errstate(over="ignore"):                     # Q / P may exceed the range: R = 1 then
        Rp[nzp] = np.minimum(1.0, Qp[nzp] / Pp[nzp])
        Rm[nzm] = np.minimum(1.0, Qm[nzm] / Pm[nzm])
    Rp[prob.dir_mask] = 1.0
    Rm[prob.dir_mask] = 1.0
    # alpha of the directed pair (i, j) as seen by the pair's owner
    alpha_own = np.where(r > 0.0, Rp[I], np.where(r < 0.0, Rm[I], 1.0))
    # the owner's value for each directed pair: (i, j) owned by i, else by j (the reverse pair)
    order = np.lexsort((J, I))
    key = I.astype(np.int64) * N + J
    rev = np.searchsorted(key[order], J.astype(np.int64) * N + I)
    rev_idx = order[rev]
    alpha = np.where(owns, alpha_own, alpha_own[rev_idx])
    return alpha * r, dict(Pp=Pp, Pm=Pm, Qp=Qp, Qm=Qm, Rp=Rp, Rm=Rm, alpha=alpha, r=r)


def stationary_system_matrix(prob: Problem):
    B = prob.AA.tolil()
    for i in np.flatnonzero(prob.dir_mask):
        B.rows[i] = [i]; B.data[i] = [1.0]
    return B.tocsr()


def mc_stationary(prob: Problem, u0=None, tol=1e-10, max_outer=1000, omega=0.5, mode="mc",
                  ksp="gmres", ksp_atol=1e-12, ksp_rtol=0.0, ksp_maxit=1000, gmres_restart=20,
                  fixed_iterations=None):
    """Sec. 3.1 with the damped fixed point of Sec. 4 (reading A5):
    res = f + F*(u) - AA u, AA delta = res, u <- u + omega delta,
    stop when ||res||_2 < sqrt(N) tol.  ksp = "direct" solves AA delta = res with a
    sparse LU factorisation computed once (AA does not change between iterations)."""
    N = prob.mesh.n_nodes
    dirm = prob.dir_mask
    u = np.zeros(N) if u0 is None else np.array(u0, dtype=np.float64)
    u[dirm] = prob.u_dir[dirm]
    Bsys = stationary_system_matrix(prob)
    dinv = 1.0 / Bsys.diagonal()
    lu = spla.splu(Bsys.tocsc()) if ksp == "direct" else None   # factor once: the matrix is fixed
    stats = dict(outer_its=0, inner_its=0, res_hist=[])
    for it in range(max_outer + 1):
        if mode == "mu":
            rstar, _ = mu_limited_fluxes(prob, u)
        else:
            rstar, _ = mc_limited_fluxes(prob, u, mode)
        Fstar = limited_sum(prob, np.ones_like(rstar), rstar)
        res = prob.f + Fstar - prob.AA @ u
        res[dirm] = 0.0
        R = float(np.linalg.norm(res))
        stats["res_hist"].append(R)
        if fixed_iterations is None:
            if R < math.sqrt(N) * tol or it == max_outer:
                break
        elif it == fixed_iterations:
            break
        if lu is not None:
            delta = lu.solve(res)
        else:
            delta, kst = krylov_solve(Bsys, res, dinv, ksp, ksp_atol, ksp_rtol, ksp_maxit, gmres_restart)
            stats["inner_its"] += kst["its"]
        u = u + omega * delta
        stats["outer_its"] += 1
    stats["res_final"] = stats["res_hist"][-1]
    stats["converged"] = stats["res_final"] < math.sqrt(N) * tol
    return u, stats


# --------------------------------------------------------------------------
# Linear solvers (Sec. 4: rtol = 0, stop when the Euclidean residual norm < atol)
# --------------------------------------------------------------------------
def krylov_solve(B, rhs, dinv, ksp, atol, rtol, maxit, restart):
    if ksp == "bicgstab":
        return bicgstab(B, rhs, dinv, atol, rtol, maxit)
    if ksp == "gmres":
        return gmres(B, rhs, dinv, restart, atol, rtol, maxit)
    if ksp == "direct":
        return dense_solve(B, rhs), dict(its=1)
    raise ValueError(ksp)


def _stop(norm_r, norm_r0, atol, rtol):
    return norm_r < max(atol, rtol * norm_r0)


def bicgstab(B, b, dinv, atol=1e-12, rtol=0.0, maxit=1000):
    """Preconditioned BiCGStab (van der Vorst 1992) with the Jacobi preconditioner
    M^{-1} = diag(dinv) applied to the search directions, x0 = 0.  The stopping test
    uses the true-residual recurrence ||r||_2."""
    x = np.zeros_like(b)
    r = b.copy()
    rhat = r.copy()
    n0 = float(np.linalg.norm(r))
    if _stop(n0, n0, atol, rtol):
        return x, dict(its=0, res=n0)
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b); p = np.zeros_like(b)
    its = 0
    nr = n0
    while its < maxit:
        its += 1
        rho = float(rhat @ r)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        phat = dinv * p
        v = B @ phat
        alpha = rho / float(rhat @ v)
        s = r - alpha * v
        ns = float(np.linalg.norm(s))
        if _stop(ns, n0, atol, rtol):
            x = x + alpha * phat
            nr = ns
            break
        shat = dinv * s
        t = B @ shat
        omega = float(t @ s) / float(t @ t)
        x = x + alpha * phat + omega * shat
        r = s - omega * t
        nr = float(np.linalg.norm(r))
        if _stop(nr, n0, atol, rtol):
            break
        rho_old = rho
    return x, dict(its=its, res=nr)


def gmres(B, b, dinv, m=20, atol=1e-12, rtol=0.0, maxit=1000):
    """Restarted GMRES(m) (Saad & Schultz 1986), right preconditioned with the Jacobi
    preconditioner: B M^{-1} y = b, x = M^{-1} y; modified Gram-Schmidt Arnoldi, Givens
    rotations, x0 = 0.  'its' counts Arnoldi steps (one product with B each)."""
    n = b.shape[0]
    x = np.zeros(n)
    r = b.copy()
    beta = float(np.linalg.norm(r))
    n0 = beta
    its = 0
    if _stop(beta, n0, atol, rtol):
        return x, dict(its=0, res=beta)
    while its < maxit:
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m); sn = np.zeros(m)
        g = np.zeros(m + 1)
        V[0] = r / beta
        g[0] = beta
        k_used = 0
        for k in range(m):
            its += 1
            w = B @ (dinv * V[k])
            for i in range(k + 1):
                H[i, k] = float(w @ V[i])
                w = w - H[i, k] * V[i]
            H[k + 1, k] = float(np.linalg.norm(w))
            if H[k + 1, k] != 0.0:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):                          # apply earlier rotations
                hi, hi1 = H[i, k], H[i + 1, k]
                H[i, k] = cs[i] * hi + sn[i] * hi1
                H[i + 1, k] = -sn[i] * hi + cs[i] * hi1
            denom = math.hypot(H[k, k], H[k + 1, k])
            cs[k] = H[k, k] / denom
            sn[k] = H[k + 1, k] / denom
            H[k, k] = denom
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            k_used = k + 1
            if _stop(abs(g[k + 1]), n0, atol, rtol) or its >= maxit:
                break
        y = np.zeros(k_used)
        for i in range(k_used - 1, -1, -1):             # back substitution
            y[i] = (g[i] - H[i, i + 1:k_used] @ y[i + 1:k_used]) / H[i, i]
        x = x + dinv * (V[:k_used].T @ y)
        r = b - B @ x
        beta = float(np.linalg.norm(r))
        if _stop(beta, n0, atol, rtol):
            break
    return x, dict(its=its, res=beta)


def dense_solve(B, b):
    """Direct solve for tiny systems (Gaussian elimination with partial pivoting)."""
    return np.linalg.solve(B.toarray(), b)


# --------------------------------------------------------------------------
# Error norms of a P1 solution (the L1 and L2 errors the circular convection
# example reports)
# --------------------------------------------------------------------------
def conical_rule(nq: int):
    """Conical product quadrature on the reference tetrahedron (Stroud): Gauss-
    Legendre points s1, s2, s3 in [0, 1], x = s1, y = s2 (1 - s1),
    z = s3 (1 - s1)(1 - s2), weight w1 w2 w3 (1 - s1)^2 (1 - s2).  Returns the
    barycentric coordinates (nq^3, 4) and weights summing to 1/6."""
    g, w = np.polynomial.legendre.leggauss(nq)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    S1, S2, S3 = np.meshgrid(g, g, g, indexing="ij")
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel()
    s1, s2, s3 = S1.ravel(), S2.ravel(), S3.ravel()
    x = s1
    y = s2 * (1.0 - s1)
    z = s3 * (1.0 - s1) * (1.0 - s2)
    W = W * (1.0 - s1) ** 2 * (1.0 - s2)
    lam = np.stack([1.0 - x - y - z, x, y, z], axis=1)
    return lam, W


def p1_error_norms(mesh: Mesh, uh, exact, nq: int = 4, chunk: int = 20000):
    """(||u - u_h||_{L1}, ||u - u_h||_{L2}) over the tetrahedra of `mesh`, u_h the
    piecewise linear interpolant of the nodal values uh and exact(x, y, z) the
    exact solution, by the conical rule with nq^3 points per tetrahedron."""
    if mesh.elem != P1:
        raise ValueError("P1 meshes only")
    lam, W = conical_rule(nq)
    uh = np.asarray(uh, dtype=np.float64)
    e1 = 0.0
    e2 = 0.0
    for s in range(0, len(mesh.cells), chunk):
        c = mesh.cells[s:s + chunk]
        X = mesh.xyz[c]                                          # (E, 4, 3)
        six_vol = np.abs(np.linalg.det(X[:, 1:] - X[:, :1]))    # |det| = 6 V
        P = np.einsum("qk,ekd->eqd", lam, X)
        Uh = np.einsum("qk,ek->eq", lam, uh[c])
        d = np.abs(Uh - exact(P[..., 0], P[..., 1], P[..., 2]))
        e1 += float((d * W[None]).sum(axis=1) @ six_vol)
        e2 += float((d * d * W[None]).sum(axis=1) @ six_vol)
    return e1, math.sqrt(e2)


# --------------------------------------------------------------------------
# L2 error of a Q1 solution on a uniform grid of the unit cube against an
# indicator function (the error the rotating-shapes example reports)
# --------------------------------------------------------------------------
def q1_mass_form(n: int, u):
    """u^T M u for the consistent Q1 mass matrix of the uniform grid of the unit cube
    with n nodes per side: M is the tensor product of the 1D P1 mass matrices
    (h / 6) [2 1; 1 2] per interval, so the form is three 1D products."""
    h = 1.0 / (n - 1)
    U = np.asarray(u, dtype=np.float64).reshape(n, n, n)   # (z, y, x), x fastest

    def m1(V, axis):
        V = np.moveaxis(V, axis, 0)
        W = 4.0 * V
        W[0] -= 2.0 * V[0]
        W[-1] -= 2.0 * V[-1]
        W[1:] += V[:-1]
        W[:-1] += V[1:]
        return np.moveaxis(W * (h / 6.0), 0, axis)

    return float((U * m1(m1(m1(U, 0), 1), 2)).sum())


def q1_indicator_integrals(n: int, u, chi, box, m: int = 4, slab: int = 4):
    """(int u_h chi, int chi^2) over the cells of the uniform Q1 grid in the index box
    `box` = ((x0, x1), (y0, y1), (z0, z1)) of cell indices (outside it chi must
    vanish), u_h the trilinear interpolant of the nodal values u, by the tensor Gauss
    rule with m points per direction in every cell."""
    h = 1.0 / (n - 1)
    g, w = np.polynomial.legendre.leggauss(m)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    Wq = (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel() * h ** 3
    ref = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)          # (Q, 3)
    # trilinear basis at the points, local vertex k = dx + 2 dy + 4 dz
    phi = np.stack([(ref[:, 0] if dx else 1 - ref[:, 0]) * (ref[:, 1] if dy else 1 - ref[:, 1]) *
                    (ref[:, 2] if dz else 1 - ref[:, 2])
                    for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)], axis=1)   # (Q, 8)
    U = np.asarray(u, dtype=np.float64).reshape(n, n, n)
    (x0, x1), (y0, y1), (z0, z1) = box
    cx = np.arange(x0, x1)
    cy = np.arange(y0, y1)
    s_uc = 0.0
    s_c = 0.0
    for za in range(z0, z1, slab):
        cz = np.arange(za, min(za + slab, z1))
        CZ, CY, CX = np.meshgrid(cz, cy, cx, indexing="ij")
        CZ, CY, CX = CZ.ravel(), CY.ravel(), CX.ravel()
        px = (CX[:, None] + ref[None, :, 0]) * h
        py = (CY[:, None] + ref[None, :, 1]) * h
        pz = (CZ[:, None] + ref[None, :, 2]) * h
        C = chi(px, py, pz)                                           # (cells, Q)
        if not C.any():
            continue
        s_c += float((C * C * Wq[None]).sum())
        corner = np.stack([U[CZ + dz, CY + dy, CX + dx] for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)],
                          axis=1)                                     # (cells, 8)
        uq = corner @ phi.T                                           # (cells, Q)
        s_uc += float((uq * C * Wq[None]).sum())
    return s_uc, s_c


def q1_l2_error_indicator(n: int, u, chi, box, m: int = 4):
    """||u_h - chi||_{L2} = sqrt(u^T M u - 2 int u_h chi + int chi^2): the first term
    exact, the other two by the Gauss rule of q1_indicator_integrals (for an
    indicator chi^2 = chi)."""
    uc, c = q1_indicator_integrals(n, u, chi, box, m)
    return math.sqrt(max(q1_mass_form(n, u) - 2.0 * uc + c, 0.0))
