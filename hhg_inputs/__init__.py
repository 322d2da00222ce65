"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds only *inputs*: macro meshes (vertex coordinates and
tetrahedra with their vertex order), coefficient fields, right-hand sides and
Dirichlet data.  It contains none of the discretisation arithmetic of the
method (no stiffness, no stencils, no refinement); both the CPU oracle and the
CUDA path receive the arrays produced here.

Random nodal fields are defined on a regular (N+1)^3 grid over the bounding
box of the mesh and sampled at node coordinates, so a value depends only on
where a node is, never on how an implementation numbers its nodes.
"""

from __future__ import annotations

import itertools
import math

import numpy as np

# --------------------------------------------------------------------------
# macro meshes
# --------------------------------------------------------------------------

KUHN_PERMS = tuple(itertools.permutations(range(3)))


def unit_tet():
    """One macro tetrahedron (0, e1, e2, e3) in this vertex order."""
    xyz = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    tets = np.array([[0, 1, 2, 3]], dtype=np.int64)
    return xyz, tets


def kuhn_cube(m: int = 1):
    """Unit cube cut into m^3 sub-cubes, each split into 6 Kuhn tetrahedra.

    Every tetrahedron is (c, c+e_a, c+e_a+e_b, c+(1,1,1)) (scaled by 1/m) for a
    permutation (a, b, c) of the axes, listed in that vertex order, so all of
    them share the main diagonal of their sub-cube.  m = 1 gives the 6-macro
    cube; m = 4 gives the 384-macro cube of the elastostatics benchmark
    (Sec. 5.1.2).
    """
    grid = {}
    xyz = []

    def vid(p):
        if p not in grid:
            grid[p] = len(xyz)
            xyz.append([p[0] / m, p[1] / m, p[2] / m])
        return grid[p]

    tets = []
    for cz in range(m):
        for cy in range(m):
            for cx in range(m):
                c = (cx, cy, cz)
                for perm in KUHN_PERMS:
                    p0 = c
                    p1 = list(p0)
                    p1[perm[0]] += 1
                    p2 = list(p1)
                    p2[perm[1]] += 1
                    p3 = (cx + 1, cy + 1, cz + 1)
                    tets.append([vid(tuple(p0)), vid(tuple(p1)), vid(tuple(p2)), vid(p3)])
    return np.array(xyz, dtype=np.float64), np.array(tets, dtype=np.int64)


def kuhn_box(nx: int, ny: int, nz: int):
    """The box (0, nx) x (0, ny) x (0, nz) cut into unit cubes, each split into 6 Kuhn
    tetrahedra as in kuhn_cube (kuhn_box(4, 2, 1) is the foam block of Sec. 5.1.3)."""
    grid = {}
    xyz = []

    def vid(p):
        if p not in grid:
            grid[p] = len(xyz)
            xyz.append([float(p[0]), float(p[1]), float(p[2])])
        return grid[p]

    tets = []
    for cz in range(nz):
        for cy in range(ny):
            for cx in range(nx):
                c = (cx, cy, cz)
                for perm in KUHN_PERMS:
                    p1 = list(c)
                    p1[perm[0]] += 1
                    p2 = list(p1)
                    p2[perm[1]] += 1
                    tets.append([vid(c), vid(tuple(p1)), vid(tuple(p2)), vid((cx + 1, cy + 1, cz + 1))])
    return np.array(xyz, dtype=np.float64), np.array(tets, dtype=np.int64)


def skewed_pair():
    """Two non-degenerate, non-axis-aligned macro tetrahedra sharing one face.

    Used to exercise general affine macro maps and a macro interface whose
    refinement lattices meet at an arbitrary orientation.
    """
    xyz = np.array(
        [
            [0.0, 0.0, 0.0],
            [1.1, 0.1, -0.05],
            [0.2, 0.9, 0.1],
            [0.15, 0.2, 1.05],
            [1.0, 1.0, 0.9],
        ]
    )
    tets = np.array([[0, 1, 2, 3], [4, 3, 2, 1]], dtype=np.int64)
    return xyz, tets


# --------------------------------------------------------------------------
# coefficient fields (functions of coordinates)
# --------------------------------------------------------------------------


def young_sine(x):
    """E(x) = 1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z)."""
    x = np.asarray(x)
    return 1.0 + 0.5 * np.sin(2 * np.pi * x[..., 0]) * np.sin(2 * np.pi * x[..., 1]) * np.sin(
        2 * np.pi * x[..., 2]
    )


def young_cos(x, m: int):
    """E(x) = cos(m pi x y z) + 2, the elastostatics benchmark (Sec. 5.1.2)."""
    x = np.asarray(x)
    return np.cos(m * np.pi * x[..., 0] * x[..., 1] * x[..., 2]) + 2.0


def viscosity_sphere(x, mu_in=1.0, mu_out=1.0e3, radius=0.25, width=0.02):
    """mu = mu_in inside a sphere of the given radius around (1/2,1/2,1/2), mu_out outside,
    blended by a tanh of the given width."""
    x = np.asarray(x)
    r = np.sqrt(((x - 0.5) ** 2).sum(axis=-1))
    return mu_in + (mu_out - mu_in) * 0.5 * (1.0 + np.tanh((r - radius) / width))


def foam_modulus(x, cell=0.5, e_void=1e-2):
    """Stand-in for the foam block's CT-derived Young's modulus (Sec. 5.1.3; the scan is not
    available): material (E = 1) around the Schwarz P surface cos(2 pi x / cell) + cos(2 pi y /
    cell) + cos(2 pi z / cell) = 0, a periodic open-cell structure, and E = e_void in the pores,
    blended by a tanh of the level-set value."""
    x = np.asarray(x, dtype=np.float64)
    w = 2.0 * np.pi / cell
    s = np.cos(w * x[..., 0]) + np.cos(w * x[..., 1]) + np.cos(w * x[..., 2])
    solid = 0.5 * (1.0 - np.tanh((np.abs(s) - 0.8) / 0.2))
    return e_void + (1.0 - e_void) * solid


def plume_temperature(x):
    """Temperature of the stationary plume workload (Sec. 5.2.1): a tilted Gaussian sheet
    around the surface z = 3/10 - (3r/2 + 3/4)(r - 1/2) plus a column exp(-100 r^2) that
    fades out above z of about 0.53 through a logistic factor, with the anisotropic radius
    r^2 = 1.3 (x - 1/2)^2 + 2.7 (y - 1/2)^2 (so no rotational symmetry)."""
    x = np.asarray(x, dtype=np.float64)
    r2 = 1.3 * (x[..., 0] - 0.5) ** 2 + 2.7 * (x[..., 1] - 0.5) ** 2
    r = np.sqrt(r2)
    z = x[..., 2]
    sheet = 0.89 * np.exp(-30.0 * (z + (1.5 * r + 0.75) * (r - 0.5) - 0.3) ** 2 - 10.0 * r2)
    column = 0.98 * np.exp(-100.0 * r2) / (np.exp(17.0 * z - 9.095) + 1.0)
    return sheet + column


def plume_viscosity(x):
    """exp(-theta) of the plume temperature, times 1e-2 above the plane z = 3/4 (a jump that a
    macro mesh with a face on that plane resolves, e.g. kuhn_cube(4))."""
    x = np.asarray(x, dtype=np.float64)
    return np.exp(-plume_temperature(x)) * np.where(x[..., 2] > 0.75, 1e-2, 1.0)


def plume_force(x):
    """Buoyancy body force theta (0, 0, 10) of the plume workload."""
    th = plume_temperature(x)
    f = np.zeros(np.shape(th) + (3,))
    f[..., 2] = 10.0 * th
    return f


def affine_field(x, a0, a):
    x = np.asarray(x)
    return a0 + x @ np.asarray(a)


# --------------------------------------------------------------------------
# seeded grid fields sampled at node coordinates
# --------------------------------------------------------------------------


def grid_index(x, N, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """Nearest (N+1)^3 grid point of each coordinate (the nodes of the meshes used here lie
    exactly on such a grid)."""
    x = np.asarray(x, dtype=np.float64)
    lo = np.asarray(lo)
    hi = np.asarray(hi)
    t = (x - lo) / (hi - lo) * N
    idx = np.rint(t).astype(np.int64)
    if np.any(np.abs(t - idx) > 1e-6) or idx.min() < 0 or idx.max() > N:
        raise ValueError("coordinates are not on the sampling grid")
    return idx


def uniform_grid(N, seed, comps=3, lo=-1.0, hi=1.0):
    """i.i.d. uniform values on an (N+1)^3 grid, shape (N+1, N+1, N+1, comps), indexed [x,y,z]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(N + 1, N + 1, N + 1, comps))


def sample_grid(grid, x):
    N = grid.shape[0] - 1
    idx = grid_index(x, N)
    return grid[idx[..., 0], idx[..., 1], idx[..., 2]]


def lognormal_grid(N, seed, corr=0.1, sigma=1.0):
    """exp of a smoothed Gaussian random field on an (N+1)^3 grid over the unit cube.

    i.i.d. N(0,1) values are convolved separably with a Gaussian kernel whose
    standard deviation is ``corr`` (in domain units, i.e. corr*N grid cells),
    rescaled to standard deviation ``sigma`` and exponentiated.
    """
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((N + 1, N + 1, N + 1))
    s = corr * N
    half = int(math.ceil(4 * s))
    t = np.arange(-half, half + 1, dtype=np.float64)
    ker = np.exp(-0.5 * (t / s) ** 2)
    ker /= ker.sum()
    from scipy.ndimage import convolve1d

    for ax in range(3):
        g = convolve1d(g, ker, axis=ax, mode="reflect")
    g = (g - g.mean()) / g.std() * sigma
    return np.exp(g)


# --------------------------------------------------------------------------
# manufactured solution of the elastostatics benchmark (Sec. 5.1.2)
# --------------------------------------------------------------------------


def u_star(x):
    """u*(x,y,z) = (x^3 y + z^2, x^4 y + 2 z, 3 x + y z^3) / (x y z + 1)."""
    x = np.asarray(x)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    d = X * Y * Z + 1.0
    return np.stack([(X**3 * Y + Z**2) / d, (X**4 * Y + 2 * Z) / d, (3 * X + Y * Z**3) / d], axis=-1)


def lid_velocity(x):
    """Lid-driven cavity data: u = 16 x(1-x) y(1-y) (1,0,0) on z = 1, zero elsewhere."""
    x = np.asarray(x)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    s = np.where(np.abs(Z - 1.0) < 1e-12, 16.0 * X * (1 - X) * Y * (1 - Y), 0.0)
    return np.stack([s, np.zeros_like(s), np.zeros_like(s)], axis=-1)


def node_noise(coords, seed, comps=3, lo=-1.0, hi=1.0):
    """i.i.d. uniform values attached to a set of node coordinates independently of their
    order: the nodes are ranked lexicographically by their coordinates (rounded to 1e-9) and
    the k-th ranked node gets the k-th draw.  Both implementations that hold the same node
    set therefore see the same value at the same node."""
    c = np.rint(np.asarray(coords, dtype=np.float64) * 1e9).astype(np.int64)
    order = np.lexsort(c.T[::-1])
    rng = np.random.default_rng(seed)
    vals = rng.uniform(lo, hi, size=(c.shape[0], comps))
    out = np.empty_like(vals)
    out[order] = vals
    return out if comps > 1 else out[:, 0]
