"""The rotating-shapes accuracy pin (numerical studies, Example "Rotating shapes"):
its initial data and the L2 error the paper reports, on the CPU.  The error norm
||u_h - chi||_{L2} = sqrt(u^T M u - 2 int u_h chi + int chi^2) is pinned on closed
forms (Q1 functions, products of coordinates), the bodies' indicator on their
analytic volumes, and the scheme itself (Zalesak FCT with Heun's SSP2, Sec. 2.1.2)
on its invariants for this problem on a small grid."""
import math
import os

import numpy as np
import pytest

from oracle import afc_oracle as O
from paper_2110_15676_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def printed_rotating_errors():
    """{scheme: L2 error} of the paper's table for the rotating shapes."""
    out = {}
    with open(os.path.join(GOLDEN, "rotating_shapes_errors.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, val = line.split()
            out[name] = float(val)
    return out


def _nodal(n, fn):
    xyz = W.grid_coords(n)
    return fn(xyz[:, 0], xyz[:, 1], xyz[:, 2])


FULL = lambda n: ((0, n - 1),) * 3   # noqa: E731


@pytest.mark.parametrize("n", [3, 6, 9])
def test_mass_form_closed_forms(n):
    assert abs(O.q1_mass_form(n, np.ones(n ** 3)) - 1.0) < 1e-14
    assert abs(O.q1_mass_form(n, _nodal(n, lambda x, y, z: x)) - 1.0 / 3.0) < 1e-14
    # x y is in Q1: int (x y)^2 = 1/9; x + z: int (x + z)^2 = 1/3 + 1/3 + 2/4
    assert abs(O.q1_mass_form(n, _nodal(n, lambda x, y, z: x * y)) - 1.0 / 9.0) < 1e-14
    assert abs(O.q1_mass_form(n, _nodal(n, lambda x, y, z: x + z)) - (2.0 / 3.0 + 0.5)) < 1e-14


@pytest.mark.parametrize("n", [3, 7])
def test_l2_error_on_closed_forms(n):
    xyz = lambda x, y, z: x * y * z   # noqa: E731
    # u_h = I_h(x y z) = x y z exactly (trilinear): error 0
    assert O.q1_l2_error_indicator(n, _nodal(n, xyz), xyz, FULL(n), m=2) < 1e-7
    # against x y z + 1: error 1 (|Omega|)
    e = O.q1_l2_error_indicator(n, _nodal(n, lambda x, y, z: x * y * z + 1.0), xyz, FULL(n), m=2)
    assert abs(e - 1.0) < 1e-13
    # u_h = x, chi = y: int (x - y)^2 = 1/3 + 1/3 - 2/4 = 1/6
    e = O.q1_l2_error_indicator(n, _nodal(n, lambda x, y, z: x), lambda x, y, z: y, FULL(n), m=3)
    assert abs(e * e - 1.0 / 6.0) < 1e-13


def test_bodies_volume_and_interpolant_error_converge():
    chi = W.rotating_bodies
    V = W.ROTATING_BODIES_VOLUME
    errs = []
    for n in (33, 65):
        _, c = O.q1_indicator_integrals(n, np.zeros(n ** 3), chi, FULL(n), m=4)
        assert abs(c - V) < 0.02 * V, (n, c, V)
        u0 = W.rotating_shapes("q1", n).u0
        errs.append(O.q1_l2_error_indicator(n, u0, chi, FULL(n), m=4))
    # the interpolant of a discontinuous function: L2 error ~ h^(1/2)
    assert errs[1] < errs[0] and 1.2 < errs[0] / errs[1] < 1.7, errs


def test_zalesak_ssp2_rotating_shapes_keeps_bounds_on_a_small_grid():
    """Zal+SSP on the rotating shapes at h = 1/16 for a quarter turn: the solution
    stays in [0, 1] to machine precision at every step, as the paper reports for
    every scheme, and the bodies have moved (the error against u0 has grown well
    beyond the interpolant's)."""
    n = 17
    wl = W.rotating_shapes("q1", n)
    mesh = O.structured_mesh(wl.elem, wl.n)
    o = O.assemble(mesh, wl.eps, wl.b, wl.c, wl.f, wl.dir_mask.astype(bool), wl.u_dir)
    dt = 0.016
    u = wl.u0.copy()
    for _ in range(int(round(0.5 * math.pi / dt))):
        u = O.ssp_step(o, u, dt, order=2)
        assert u.min() >= -1e-14 and u.max() <= 1 + 1e-14
    e0 = O.q1_l2_error_indicator(n, wl.u0, W.rotating_bodies, FULL(n))
    e = O.q1_l2_error_indicator(n, u, W.rotating_bodies, FULL(n))
    assert e > 1.3 * e0


def test_printed_rotating_errors_fixture():
    e = printed_rotating_errors()
    assert e["zalesak_ssp"] == 5.76e-2 and e["mc_ssp"] == 5.85e-2 and e["linear_zalesak_cn"] == 5.76e-2
