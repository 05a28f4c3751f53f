"""Seeded synthetic inputs for the AFC hot path.

This module only produces input data: node coordinates of uniform box grids,
nodal velocity fields, initial data, sources and Dirichlet sets.  It holds none
of the method's arithmetic (no matrices, fluxes or limiters), so both the CUDA
library and the CPU oracle can be fed from it.

The workloads mirror the 3D tests of the paper (uniform cube grids, rotating or
constant convection, small diffusion, data in [0, 1]):

* ``rotating_transient``: unit cube, b = (0.5 - y, x - 0.5, 0) (the rotating
  field of the paper's rotating-shapes example), smooth cosine hump of radius
  0.15 centred at (0.5, 0.75, 0.5), f = 0, c = 0, homogeneous Dirichlet data on
  the whole boundary.
* ``stationary_inflow``: unit cube, b = (1, -0.5, 0.25), c = 1, f = 1 on the
  closed cube [0.25, 0.5]^3, Dirichlet data on the inflow faces x = 0, y = 1,
  z = 0 with value 1 where x = 0 and y < 0.5, else 0.
* ``random_transient``: a seeded random instance (node count per side, eps,
  constant unit velocity, hump centre) for batched runs.
* ``rotating_shapes``: the paper's rotating-shapes example (eps = 0, the same
  rotating field, initial data 1 inside a cube, a cone and a hollow cylinder and 0
  elsewhere, ``rotating_bodies``), homogeneous Dirichlet data on the boundary.
* ``circular_convection``: the paper's circular convection example (eps = 0,
  b = (y, -x, 0), exact solution ``circular_exact`` as Dirichlet data on the
  faces y = 1, x = 0, x = 1) on the Kuhn P1 grid.
* ``serving_mix``: a seeded mix of stationary and transient problems of random
  size, element type, eps and c, for a request stream.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

P1 = "p1"
Q1 = "q1"


@dataclass
class Workload:
    name: str
    elem: str
    n: tuple            # nodes per side (nx, ny, nz)
    lo: tuple
    hi: tuple
    eps: float
    c: float
    b: np.ndarray       # (N, 3) nodal velocity
    f: np.ndarray       # (N,) nodal source
    u0: np.ndarray      # (N,) initial data / initial guess
    dir_mask: np.ndarray  # (N,) uint8
    u_dir: np.ndarray   # (N,) Dirichlet values

    @property
    def n_nodes(self) -> int:
        return int(np.prod(self.n))


def grid_coords(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> np.ndarray:
    """(N, 3) node coordinates, node index ix + nx*(iy + ny*iz)."""
    if np.isscalar(n):
        n = (int(n),) * 3
    xs = [np.linspace(lo[d], hi[d], n[d]) for d in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def grid_index(n):
    """Integer (ix, iy, iz) of every node."""
    if np.isscalar(n):
        n = (int(n),) * 3
    iz, iy, ix = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    return ix.ravel(), iy.ravel(), iz.ravel()


def boundary_mask(n) -> np.ndarray:
    if np.isscalar(n):
        n = (int(n),) * 3
    ix, iy, iz = grid_index(n)
    m = (ix == 0) | (ix == n[0] - 1) | (iy == 0) | (iy == n[1] - 1) | (iz == 0) | (iz == n[2] - 1)
    return m.astype(np.uint8)


def cosine_hump(xyz, center=(0.5, 0.75, 0.5), radius=0.15) -> np.ndarray:
    """0.5 (1 + cos(pi r / radius)) for r <= radius, else 0; values in [0, 1]."""
    r = np.linalg.norm(xyz - np.asarray(center)[None, :], axis=1)
    return np.where(r <= radius, 0.5 * (1.0 + np.cos(np.pi * np.minimum(r, radius) / radius)), 0.0)


def rotating_b(xyz) -> np.ndarray:
    return np.stack([0.5 - xyz[:, 1], xyz[:, 0] - 0.5, np.zeros(len(xyz))], axis=1)


def rotating_transient(elem: str, n: int, eps: float = 1e-6) -> Workload:
    xyz = grid_coords(n)
    N = len(xyz)
    return Workload(
        name=f"rotating_{elem}_{n}^3", elem=elem, n=(n, n, n), lo=(0.0,) * 3, hi=(1.0,) * 3,
        eps=eps, c=0.0, b=rotating_b(xyz), f=np.zeros(N), u0=cosine_hump(xyz),
        dir_mask=boundary_mask(n), u_dir=np.zeros(N))


def rotating_bodies(x, y, z) -> np.ndarray:
    """Indicator (1 inside or on the surface, else 0) of the three bodies of the
    rotating-shapes example: the cube of edge 0.25 centred at (0.5, 0.25, 0.5); the
    cone of height 0.5 over the disc of radius 0.125 centred at (0.75, 0.5, 0.25) in
    the plane z = 0.25; the hollow cylinder of inner radius 0.0625, outer radius
    0.125 and height 0.5 over the centre (0.5, 0.75, 0.25)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    cube = (np.abs(x - 0.5) <= 0.125) & (np.abs(y - 0.25) <= 0.125) & (np.abs(z - 0.5) <= 0.125)
    zc = (z >= 0.25) & (z <= 0.75)
    rc = np.hypot(x - 0.75, y - 0.5)
    cone = zc & (rc <= 0.125 * (1.0 - (z - 0.25) / 0.5))
    rh = np.hypot(x - 0.5, y - 0.75)
    hollow = zc & (rh >= 0.0625) & (rh <= 0.125)
    return (cube | cone | hollow).astype(np.float64)


# bounding box of the three bodies, and their total volume:
# 0.25^3 + pi 0.125^2 0.5 / 3 + pi (0.125^2 - 0.0625^2) 0.5
ROTATING_BODIES_BOX = ((0.375, 0.875), (0.125, 0.875), (0.25, 0.75))
ROTATING_BODIES_VOLUME = 0.25 ** 3 + np.pi * 0.125 ** 2 * 0.5 / 3.0 + np.pi * (0.125 ** 2 - 0.0625 ** 2) * 0.5


def rotating_shapes(elem: str, n: int) -> Workload:
    """The rotating-shapes example: unit cube, eps = 0, b = (0.5 - y, x - 0.5, 0),
    c = 0, f = 0, u_D = 0 on the whole boundary, u0 the bodies' indicator at the
    nodes.  One rotation takes t = 2 pi, after which the exact solution is u0 again."""
    xyz = grid_coords(n)
    N = len(xyz)
    return Workload(
        name=f"rotating_shapes_{elem}_{n}^3", elem=elem, n=(n, n, n), lo=(0.0,) * 3, hi=(1.0,) * 3,
        eps=0.0, c=0.0, b=rotating_b(xyz), f=np.zeros(N), u0=rotating_bodies(xyz[:, 0], xyz[:, 1], xyz[:, 2]),
        dir_mask=boundary_mask(n), u_dir=np.zeros(N))


def stationary_inflow(elem: str, n: int, eps: float = 1e-8, c: float = 1.0,
                      b=(1.0, -0.5, 0.25)) -> Workload:
    xyz = grid_coords(n)
    N = len(xyz)
    ix, iy, iz = grid_index(n)
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    # inflow faces for b = (1, -0.5, 0.25): x = 0, y = 1, z = 0 (closed faces)
    inflow = (ix == 0) | (iy == n - 1) | (iz == 0)
    u_dir = np.where((ix == 0) & (y < 0.5), 1.0, 0.0)
    f = np.where((x >= 0.25) & (x <= 0.5) & (y >= 0.25) & (y <= 0.5) & (z >= 0.25) & (z <= 0.5), 1.0, 0.0)
    bb = np.tile(np.asarray(b, dtype=np.float64), (N, 1))
    u0 = np.where(inflow, u_dir, 0.0)
    return Workload(
        name=f"stationary_{elem}_{n}^3", elem=elem, n=(n, n, n), lo=(0.0,) * 3, hi=(1.0,) * 3,
        eps=eps, c=c, b=bb, f=f, u0=u0, dir_mask=inflow.astype(np.uint8), u_dir=u_dir)


def random_transient(rng: np.random.Generator, elem: str = Q1, n_range=(17, 49)) -> Workload:
    n = int(rng.integers(n_range[0], n_range[1] + 1))
    eps = float(10.0 ** rng.uniform(-8.0, -4.0))
    v = rng.normal(size=3)
    v /= np.linalg.norm(v)
    center = rng.uniform(0.3, 0.7, size=3)
    xyz = grid_coords(n)
    N = len(xyz)
    return Workload(
        name=f"random_{elem}_{n}^3", elem=elem, n=(n, n, n), lo=(0.0,) * 3, hi=(1.0,) * 3,
        eps=eps, c=0.0, b=np.tile(v, (N, 1)), f=np.zeros(N), u0=cosine_hump(xyz, center),
        dir_mask=boundary_mask(n), u_dir=np.zeros(N))


def circular_exact(x, y) -> np.ndarray:
    """Exact solution of the circular convection example: with r = sqrt(x^2 + y^2),
    1 on 0.15 <= r <= 0.45, cos^2(10 pi (r - 0.7) / 3) on 0.55 <= r <= 0.85, else 0."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    r = np.sqrt(x * x + y * y)
    u = np.zeros_like(r)
    u[(r >= 0.15) & (r <= 0.45)] = 1.0
    ring = (r >= 0.55) & (r <= 0.85)
    u[ring] = np.cos(10.0 * np.pi * (r[ring] - 0.7) / 3.0) ** 2
    return u


def circular_convection(n: int) -> Workload:
    """The paper's circular convection example on the Kuhn P1 grid with n nodes per
    side: unit cube, eps = 0, b = (y, -x, 0), c = 0, f = 0, Dirichlet data (the exact
    solution) on the faces y = 1, x = 0 and x = 1, homogeneous Neumann elsewhere;
    initial guess 0 with the Dirichlet values."""
    xyz = grid_coords(n)
    N = len(xyz)
    ix, iy, iz = grid_index(n)
    x, y = xyz[:, 0], xyz[:, 1]
    dirm = (iy == n - 1) | (ix == 0) | (ix == n - 1)
    u_dir = circular_exact(x, y)
    b = np.stack([y, -x, np.zeros(N)], axis=1)
    return Workload(
        name=f"circular_p1_{n}^3", elem=P1, n=(n, n, n), lo=(0.0,) * 3, hi=(1.0,) * 3,
        eps=0.0, c=0.0, b=b, f=np.zeros(N), u0=np.where(dirm, u_dir, 0.0),
        dir_mask=dirm.astype(np.uint8), u_dir=u_dir)


def serving_mix(rng: np.random.Generator, count: int, n_range=(17, 97)) -> list:
    """A request stream's problems: each is stationary (the inflow problem above)
    or transient (a random_transient instance) with probability 1/2, on P1 or Q1
    with probability 1/2, with n uniform in n_range, eps log-uniform in
    [1e-8, 1e-4] and c uniform in [0, 1].  Returns (kind, Workload) pairs, kind
    "stationary" or "transient"."""
    out = []
    for _ in range(count):
        kind = "stationary" if rng.uniform() < 0.5 else "transient"
        elem = P1 if rng.uniform() < 0.5 else Q1
        if kind == "stationary":
            n = int(rng.integers(n_range[0], n_range[1] + 1))
            eps = float(10.0 ** rng.uniform(-8.0, -4.0))
            c = float(rng.uniform(0.0, 1.0))
            wl = stationary_inflow(elem, n, eps=eps, c=c)
        else:
            wl = random_transient(rng, elem, n_range)
            wl.c = float(rng.uniform(0.0, 1.0))
        out.append((kind, wl))
    return out


def random_field(rng: np.random.Generator, N: int, lo=0.0, hi=1.0) -> np.ndarray:
    return rng.uniform(lo, hi, size=N)


def front_field(xyz: np.ndarray, rng: np.random.Generator, width=0.03, noise=0.02) -> np.ndarray:
    """A state with the structure limiters act on: a steep smooth front across a
    randomly tilted plane, values in [0, 1], plus small seeded noise (local extrema)."""
    nrm = rng.normal(size=3)
    nrm /= np.linalg.norm(nrm)
    s = (xyz - 0.5) @ nrm
    base = 0.5 * (1.0 + np.tanh(s / width))
    return np.clip(base + noise * rng.uniform(-1.0, 1.0, size=len(xyz)), 0.0, 1.0)
