"""Build the same problem twice: in the CPU oracle and in the CUDA library.

Both sides get identical inputs from the seeded generators of
paper_2110_15676_gb300.workloads; neither side sees the other's arithmetic."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from oracle import afc_oracle as O
from paper_2110_15676_gb300 import workloads as W


def oracle_problem(elem, n, b, eps, c, f, dir_mask, u_dir, family="fct", lo=(0, 0, 0), hi=(1, 1, 1)):
    mesh = O.structured_mesh(elem, n, lo, hi)
    return O.assemble(mesh, eps, b, c, f, np.asarray(dir_mask, bool), u_dir, family)


def gpu_problem(elem, n, b, eps, c, f, dir_mask, u_dir, family="fct", precision="fp64", lo=(0, 0, 0),
                hi=(1, 1, 1)):
    from paper_2110_15676_gb300 import afc
    P = afc.Problem.structured(elem, n, lo, hi)
    P.set_coefficients(eps, b, c, f)
    P.set_dirichlet(np.asarray(dir_mask, np.uint8), u_dir)
    P.assemble(afc.AFC_FAMILY_FCT if family == "fct" else afc.AFC_FAMILY_MC,
               afc.AFC_FP64 if precision == "fp64" else afc.AFC_MIXED)
    return P


def pair_from_workload(wl: W.Workload, family="fct", precision="fp64"):
    o = oracle_problem(wl.elem, wl.n, wl.b, wl.eps, wl.c, wl.f, wl.dir_mask, wl.u_dir, family, wl.lo, wl.hi)
    g = gpu_problem(wl.elem, wl.n, wl.b, wl.eps, wl.c, wl.f, wl.dir_mask, wl.u_dir, family, precision, wl.lo, wl.hi)
    return o, g


def csr_of(P, which):
    rowptr, col, val = P.export_csr(which)
    N = len(rowptr) - 1
    return sp.csr_matrix((val, col, rowptr), shape=(N, N))


def random_workload(elem, n, seed, family="fct", lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """General small instance: perturbed rotating velocity, reaction, source, mixed Dirichlet set."""
    rng = np.random.default_rng(seed)
    if np.isscalar(n):
        n = (n, n, n)
    xyz = W.grid_coords(n, lo, hi)
    N = len(xyz)
    b = W.rotating_b(xyz) + rng.normal(scale=0.3, size=(N, 3))
    bm = W.boundary_mask(n).astype(bool) & (rng.uniform(size=N) < 0.8)
    ud = rng.uniform(0, 1, N)
    f = rng.uniform(0, 1, N)
    u0 = rng.uniform(0, 1, N)
    u0[bm] = ud[bm]
    return W.Workload(name=f"random_{elem}", elem=elem, n=tuple(n), lo=tuple(lo), hi=tuple(hi), eps=1e-3, c=0.3,
                      b=b, f=f, u0=u0, dir_mask=bm.astype(np.uint8), u_dir=ud)


def relerr(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
