"""Pins of the boundary traction load oracle (Sec. 5.1.3; no GPU)."""

import numpy as np

import hhg_inputs as hi
from oracle import loads as LD, mesh


def _box(level):
    xyz, tets = hi.kuhn_box(2, 1, 1)
    mm = mesh.MacroMesh.build(xyz, tets)
    return mm, tets, mesh.build_level(mm, level)


def _top_flags(xyz, tets, z):
    flags = np.zeros((len(tets), 4), dtype=np.int32)
    for m, t in enumerate(tets):
        for f in range(4):
            if np.all(np.abs(xyz[[int(t[q]) for q in range(4) if q != f], 2] - z) < 1e-12):
                flags[m, f] = 1
    return flags


def test_boundary_triangles_tile_the_flagged_faces():
    """The refined triangles on the top plane of the 2 x 1 x 1 box cover its area 2 exactly, n^2
    per macro face."""
    for level in (1, 2, 3):
        mm, tets, lv = _box(level)
        flags = _top_flags(mm.xyz, tets, 1.0)
        tri = LD.boundary_triangles(mm, lv, flags)
        X = lv.coords[tri]
        area = 0.5 * np.linalg.norm(np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), axis=1).sum()
        assert abs(area - 2.0) < 1e-12
        assert len(tri) == flags.sum() * 4**level
        assert np.allclose(lv.coords[tri.reshape(-1), 2], 1.0)


def test_load_integrates_affine_traction_exactly():
    """P1 functions are integrated exactly by the P1 mass matrix: for an affine t the total
    load equals int_Gamma t ds in closed form, and the moment sum_i b_i x_i equals
    int_Gamma t x ds for constant t (the P1 interpolant of x is exact)."""
    mm, tets, lv = _box(2)
    flags = _top_flags(mm.xyz, tets, 1.0)
    c = lv.coords
    t = np.stack([1.0 + 0.5 * c[:, 0] - 0.25 * c[:, 1], -2.0 + c[:, 1], 0.3 * c[:, 0]], 1)
    b = LD.traction_load(mm, lv, flags, t)
    # on z = 1, (0,2) x (0,1): int 1 + x/2 - y/4 = 2 + 1 - 0.25; int -2 + y = -4 + 1; int 0.3 x = 0.6
    assert np.allclose(b.sum(axis=0), [2.75, -3.0, 0.6], rtol=0, atol=1e-12)
    t0 = np.tile([0.0, 0.0, -1.0], (lv.num_nodes, 1))
    b0 = LD.traction_load(mm, lv, flags, t0)
    assert np.allclose((b0[:, 2:3] * c).sum(axis=0), [-2.0, -1.0, -2.0], atol=1e-12)  # -int (x, y, 1)
    assert np.all(b0[np.abs(c[:, 2] - 1.0) > 1e-12] == 0.0)


def test_load_is_the_symmetric_boundary_mass_matrix():
    """b = M t with M symmetric and positive definite on the face nodes: b(t1) . t2 = b(t2) . t1
    and b(t) . t > 0."""
    mm, tets, lv = _box(2)
    flags = _top_flags(mm.xyz, tets, 1.0)
    rng = np.random.default_rng(3)
    t1, t2 = rng.normal(size=(2, lv.num_nodes, 3))
    b1 = LD.traction_load(mm, lv, flags, t1)
    b2 = LD.traction_load(mm, lv, flags, t2)
    assert abs((b1 * t2).sum() - (b2 * t1).sum()) < 1e-12
    assert (b1 * t1).sum() > 0


def test_total_force_on_slanted_faces():
    """On the skewed two-macro mesh every boundary face is slanted: a constant traction gives a
    total load of t times the flagged faces' area, computed from the macro vertices."""
    xyz, tets = hi.skewed_pair()
    mm = mesh.MacroMesh.build(xyz, tets)
    lv = mesh.build_level(mm, 3)
    count = {}
    for t in tets:
        for f in range(4):
            key = tuple(sorted(int(t[q]) for q in range(4) if q != f))
            count[key] = count.get(key, 0) + 1
    flags = np.zeros((len(tets), 4), dtype=np.int32)
    area = 0.0
    for m, t in enumerate(tets):
        for f in range(4):
            key = tuple(sorted(int(t[q]) for q in range(4) if q != f))
            if count[key] == 1 and (m + f) % 2 == 0:
                flags[m, f] = 1
                a, b, c = (np.asarray(xyz)[int(t[q])] for q in range(4) if q != f)
                area += 0.5 * np.linalg.norm(np.cross(b - a, c - a))
    assert flags.sum() >= 2
    tval = np.array([0.3, -1.2, 0.7])
    b = LD.traction_load(mm, lv, flags, np.tile(tval, (lv.num_nodes, 1)))
    assert np.allclose(b.sum(axis=0), tval * area, rtol=0, atol=1e-12 * area)
