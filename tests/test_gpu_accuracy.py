"""The CUDA path on the paper's circular convection example (stationary, Kuhn P1: MC at
levels 5, 6 and 7, MU at levels 5 and 7): errors equal the oracle's at level 5, are of the
printed order at levels 6 and 7, and decrease with refinement."""
import os

import numpy as np
import pytest

from oracle import afc_oracle as O
from paper_2110_15676_gb300 import workloads as W
from pairs import gpu_problem
from test_oracle_accuracy import printed_errors, stored_oracle

pytestmark = pytest.mark.gpu


def gpu_errors(level, precision, limiter="mc", ksp_rtol=None, fp_tol=1e-13, fp_maxit=6000):
    from paper_2110_15676_gb300 import afc
    n = 2 ** level + 1
    wl = W.circular_convection(n)
    g = gpu_problem(wl.elem, wl.n, wl.b, wl.eps, wl.c, wl.f, wl.dir_mask, wl.u_dir, family="mc",
                    precision=precision)
    g.set_solution(wl.u0)
    mixed = precision == "mixed"
    lim = afc.AFC_LIM_MC if limiter == "mc" else afc.AFC_LIM_MU
    opts = afc.default_opts(limiter=lim, omega=0.5, ksp=afc.AFC_KSP_GMRES, ksp_atol=0.0,
                            ksp_rtol=ksp_rtol or (1e-6 if mixed else 1e-10), fp_tol=fp_tol, fp_maxit=fp_maxit,
                            precision=afc.AFC_MIXED if mixed else afc.AFC_FP64)
    st = g.solve_stationary(opts)
    u = g.get_solution()
    g.close()
    mesh = O.structured_mesh("p1", n)
    e1, e2 = O.p1_error_norms(mesh, u, lambda X, Y, Z: W.circular_exact(X, Y), nq=4 if level <= 5 else 3)
    return st, u, e1, e2


@pytest.mark.parametrize("precision,limiter", [("fp64", "mc"), ("mixed", "mc"), ("mixed", "mu")])
def test_circular_convection_level5_equals_oracle(precision, limiter):
    st, u, e1, e2 = gpu_errors(5, precision, limiter)
    assert st["status"] == 0, st
    s1, s2 = stored_oracle(limiter)[5]
    assert abs(e1 - s1) < 1e-6 * s1 and abs(e2 - s2) < 1e-6 * s2, (e1, e2, s1, s2)
    assert u.min() >= -1e-14 and u.max() <= 1.0 + 1e-14


def test_circular_convection_level6_printed_order_and_convergence():
    ref = printed_errors()
    st6, u6, a1, a2 = gpu_errors(6, "mixed")
    assert st6["status"] == 0, st6
    _, p1, p2 = ref[6]
    assert 0.7 * p1 <= a1 <= 1.3 * p1, a1
    assert 0.7 * p2 <= a2 <= 1.3 * p2, a2
    s1, s2 = stored_oracle()[5]
    assert a1 < s1 and a2 < s2
    assert u6.min() >= -1e-14 and u6.max() <= 1.0 + 1e-14


@pytest.mark.parametrize("limiter", ["mc", "mu"])
def test_circular_convection_level7_printed_order_and_convergence(limiter):
    """Level 7 (129^3 nodes, 12.6 M tetrahedra; the grid of the stationary sweep): the
    printed L1 and L2 errors of the example's table within 30 %, below level 5's.  The
    fixed point stops at 1e-11 (the errors are those of the discretisation, not of the
    stop) with inner GMRES to 1e-2 relative, as the stationary solves of the bench; the
    bounds then hold to that stopping tolerance (the converged-DMP reading of the design
    notes), not to rounding."""
    st, u, a1, a2 = gpu_errors(7, "mixed", limiter, ksp_rtol=1e-2, fp_tol=1e-11, fp_maxit=20000)
    assert st["status"] == 0, st
    _, p1, p2 = printed_errors(limiter)[7]
    assert 0.7 * p1 <= a1 <= 1.3 * p1, (a1, p1)
    assert 0.7 * p2 <= a2 <= 1.3 * p2, (a2, p2)
    s1, s2 = stored_oracle(limiter)[5]
    assert a1 < s1 and a2 < s2
    assert u.min() >= -1e-10 and u.max() <= 1.0 + 1e-10, (u.min(), u.max())
