"""Dense, loop-by-loop transcriptions of the limiters for meshes of a few cells.

They take the assembled matrices as dense arrays and follow the paper's steps one
node and one pair at a time, with no vectorisation and no shared code with the
oracle or the CUDA path:

* ``zalesak``: Zalesak's algorithm for given raw fluxes r_ij (Sec. 2.1.3, steps 1-4;
  Q+/- over the sparsity neighbours, reading A2; R = 1 at Dirichlet nodes or where
  P = 0), and the limited sum F*_i = sum_j alpha_ij r_ij.
* ``mc``: the monolithic convex limiter, Eq. MClimiter with the bounds Eq. u_max_min
  and the bar states 2 d_ij ubar_ij = d_ij (u_i + u_j) + a_ij (u_j - u_i), for
  r_ij = d_ij (u_j - u_i) (Sec. 3.1); no flux where d_ij = 0 (reading A16).
"""
import numpy as np


def zalesak(r, mC, mL, u_tilde, dt, dirichlet):
    """r: dense antisymmetric (N, N) raw fluxes on the pattern of mC (0 elsewhere).
    Returns (alpha (N, N), F* (N,), R+ (N,), R- (N,))."""
    N = len(mL)
    nbr = [[j for j in range(N) if j != i and mC[i, j] != 0.0] for i in range(N)]
    Rp = np.ones(N)
    Rm = np.ones(N)
    for i in range(N):
        Pp = 0.0
        Pm = 0.0
        for j in nbr[i]:
            if r[i, j] > 0.0:
                Pp += r[i, j]
            elif r[i, j] < 0.0:
                Pm += r[i, j]
        Qp = 0.0
        Qm = 0.0
        for j in nbr[i]:
            Qp = max(Qp, u_tilde[j] - u_tilde[i])
            Qm = min(Qm, u_tilde[j] - u_tilde[i])
        if dirichlet[i]:
            continue
        if Pp != 0.0:
            Rp[i] = min(1.0, mL[i] * Qp / (dt * Pp))
        if Pm != 0.0:
            Rm[i] = min(1.0, mL[i] * Qm / (dt * Pm))
    alpha = np.zeros((N, N))
    F = np.zeros(N)
    for i in range(N):
        for j in nbr[i]:
            if r[i, j] > 0.0:
                alpha[i, j] = min(Rp[i], Rm[j])
            else:
                alpha[i, j] = min(Rm[i], Rp[j])
            F[i] += alpha[i, j] * r[i, j]
    return alpha, F, Rp, Rm


def mc(u, mC, D, Kc):
    """Limited fluxes r*_ij (dense (N, N)) and F* for the state u; D from Kc."""
    N = len(u)
    nbr = [[j for j in range(N) if j != i and mC[i, j] != 0.0] for i in range(N)]
    umax = np.array([max([u[i]] + [u[j] for j in nbr[i]]) for i in range(N)])
    umin = np.array([min([u[i]] + [u[j] for j in nbr[i]]) for i in range(N)])
    rs = np.zeros((N, N))
    for i in range(N):
        for j in nbr[i]:
            d = D[i, j]
            if d == 0.0:
                continue
            r = d * (u[j] - u[i])
            ub_ij = (d * (u[i] + u[j]) + Kc[i, j] * (u[j] - u[i])) / (2.0 * d)
            ub_ji = (d * (u[j] + u[i]) + Kc[j, i] * (u[i] - u[j])) / (2.0 * d)
            if r > 0.0:
                rs[i, j] = min(r, 2.0 * d * (ub_ij - umax[i]), 2.0 * d * (umin[j] - ub_ji))
            else:
                rs[i, j] = max(r, 2.0 * d * (ub_ij - umin[i]), 2.0 * d * (umax[j] - ub_ji))
    return rs, rs.sum(axis=1), umax, umin


def one_tet():
    return "p1", np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]]), np.array([[0, 1, 2, 3]])


def two_tets():
    return "p1", np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1.0]]), np.array([[0, 1, 2, 3],
                                                                                                   [1, 2, 3, 4]])


def two_hexes():
    xyz = np.array([[x, y, z] for z in (0, 0.5, 1.0) for y in (0, 1.0) for x in (0, 1.0)])
    return "q1", xyz, np.array([[0, 1, 2, 3, 4, 5, 6, 7], [4, 5, 6, 7, 8, 9, 10, 11]])
