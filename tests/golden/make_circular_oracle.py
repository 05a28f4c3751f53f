"""Write circular_convection_oracle.txt: the CPU oracle's L1 / L2 errors for the
circular convection example (MC and MU limiters, Kuhn P1 grid, levels 4 and 5).  Calls only
oracle/ (and the input generators); run from the repository root:

    python tests/golden/make_circular_oracle.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import afc_oracle as O  # noqa: E402
from paper_2110_15676_gb300 import workloads as W  # noqa: E402

TOL = 1e-14      # ||res|| < sqrt(N) tol: the fixed point to round-off
OMEGA = 0.5


def solve(level, mode):
    n = 2 ** level + 1
    wl = W.circular_convection(n)
    mesh = O.structured_mesh("p1", n)
    prob = O.assemble(mesh, wl.eps, wl.b, wl.c, wl.f, wl.dir_mask.astype(bool), wl.u_dir, "mc")
    u, st = O.mc_stationary(prob, wl.u0, tol=TOL, max_outer=5000, omega=OMEGA, mode=mode, ksp="direct")
    e1, e2 = O.p1_error_norms(mesh, u, lambda x, y, z: W.circular_exact(x, y), nq=4)
    return n, st["outer_its"], st["res_final"], e1, e2, float(u.min()), float(u.max())


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "circular_convection_oracle.txt")
    lines = ["# CPU oracle (oracle/afc_oracle.py) on the circular convection example, MC and MU limiters,",
             f"# Kuhn P1 grid, damped fixed point omega = {OMEGA} with direct inner solves to",
             f"# ||res|| < sqrt(N) * {TOL}; errors by the conical rule with 4^3 points per tetrahedron.",
             "# Written by tests/golden/make_circular_oracle.py.",
             "# level nodes_per_side limiter fixed_point_its res_final L1 L2 umin umax"]
    for mode in ("mc", "mu"):
        for level in (4, 5):
            n, its, res, e1, e2, mn, mx = solve(level, mode)
            lines.append(f"{level} {n} {mode} {its} {res:.6e} {e1:.12e} {e2:.12e} {mn:.6e} {mx:.6e}")
            print(lines[-1], flush=True)
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
