"""Oracle mesh: uniform refinement of a macro tetrahedral mesh (Sec. 2).

Test infrastructure only (see the package docstring).

Each macro tetrahedron T is refined uniformly ``level`` times; every
refinement splits a tetrahedron into 8 children by Bey's ordered red
refinement (Sec. 2, [bey1995]): with vertices (x0, x1, x2, x3) and edge
midpoints xab, the children are

    (x0,x01,x02,x03) (x01,x1,x12,x13) (x02,x12,x2,x23) (x03,x13,x23,x3)
    (x01,x02,x03,x13) (x01,x02,x12,x13) (x02,x03,x13,x23) (x02,x12,x13,x23)

Vertices are tracked exactly as integer barycentric coordinates with respect
to the four macro vertices (denominator 2^level), so nodes shared by several
macros are identified exactly: a node's key is its set of (global macro
vertex, numerator) pairs.  A node whose key has four non-zero weights lies in
the interior of its macro; every other node lies on the macro skeleton
(faces, edges, vertices of the macro mesh).
"""

from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

# children of Bey's rule as pairs of parent vertex indices (a, a) = vertex a, (a, b) = midpoint
BEY_CHILDREN = (
    ((0, 0), (0, 1), (0, 2), (0, 3)),
    ((0, 1), (1, 1), (1, 2), (1, 3)),
    ((0, 2), (1, 2), (2, 2), (2, 3)),
    ((0, 3), (1, 3), (2, 3), (3, 3)),
    ((0, 1), (0, 2), (0, 3), (1, 3)),
    ((0, 1), (0, 2), (1, 2), (1, 3)),
    ((0, 2), (0, 3), (1, 3), (2, 3)),
    ((0, 2), (1, 2), (1, 3), (2, 3)),
)

EDGES_OF_TET = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
FACES_OF_TET = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))  # face f is opposite local vertex f


def refine_barycentric(level: int) -> np.ndarray:
    """Children of one tetrahedron after ``level`` Bey refinements.

    Returns int64 array (8^level, 4, 4): element, vertex, barycentric weight
    (w.r.t. the 4 macro vertices), with weights summing to 2^level.
    """
    B = np.eye(4, dtype=np.int64)[None]  # (1, 4 vertices, 4 weights)
    for _ in range(level):
        kids = []
        for child in BEY_CHILDREN:
            kids.append(np.stack([B[:, a] + B[:, b] for (a, b) in child], axis=1))
        # order: child-major within each parent is irrelevant; keep parents contiguous
        B = np.stack(kids, axis=1).reshape(-1, 4, 4)
    return B


@dataclass
class MacroMesh:
    xyz: np.ndarray  # (V, 3)
    tets: np.ndarray  # (M, 4) global vertex ids, in refinement order
    dirichlet_faces: set = field(default_factory=set)  # set of sorted vertex triples

    @staticmethod
    def build(xyz, tets, dirichlet_face_flags=None):
        """``dirichlet_face_flags``: optional (M, 4) bool, face f of macro m (opposite its
        local vertex f) is Dirichlet.  Default: every boundary face (one incident macro)."""
        xyz = np.asarray(xyz, dtype=np.float64)
        tets = np.asarray(tets, dtype=np.int64)
        count = {}
        for m, t in enumerate(tets):
            for f in FACES_OF_TET:
                key = tuple(sorted(int(t[v]) for v in f))
                count[key] = count.get(key, 0) + 1
        dfaces = set()
        for m, t in enumerate(tets):
            for fi, f in enumerate(FACES_OF_TET):
                key = tuple(sorted(int(t[v]) for v in f))
                if dirichlet_face_flags is None:
                    if count[key] == 1:
                        dfaces.add(key)
                elif dirichlet_face_flags[m][fi]:
                    dfaces.add(key)
        return MacroMesh(xyz, tets, dfaces)

    def support_is_dirichlet(self, support) -> bool:
        s = set(support)
        return any(s.issubset(f) for f in self.dirichlet_faces)


@dataclass
class Level:
    """One refinement level of the whole macro mesh."""

    level: int
    n: int  # intervals per macro edge, 2^level
    coords: np.ndarray  # (N, 3)
    keys: np.ndarray  # (N, 8) canonical key rows (vid0, w0, ..., vid3, w3)
    skeleton: np.ndarray  # (N,) bool, node lies on the macro skeleton
    dirichlet: np.ndarray  # (N,) bool
    elems: np.ndarray  # (E, 4) node ids in Bey vertex order
    elem_macro: np.ndarray  # (E,)
    elem_local: np.ndarray  # (E, 4, 3) local (i, j, k) of each vertex in its macro
    local_to_node: list  # per macro: dense (n+1)^3 int64 table, -1 outside the macro
    node_macro_local: list  # per node: list of (macro, i, j, k) incidences (filled lazily)

    @property
    def num_nodes(self):
        return self.coords.shape[0]


def _canonical_keys(gv, bary):
    """gv: (4,) global vertex ids; bary: (P, 4) weights -> (P, 8) canonical key rows."""
    BIG = np.iinfo(np.int64).max
    vids = np.where(bary > 0, gv[None, :], BIG)
    order = np.argsort(vids, axis=1, kind="stable")
    v = np.take_along_axis(vids, order, axis=1)
    w = np.take_along_axis(bary, order, axis=1)
    v = np.where(v == BIG, -1, v)
    out = np.empty((bary.shape[0], 8), dtype=np.int64)
    out[:, 0::2] = v
    out[:, 1::2] = w
    return out


def build_level(mm: MacroMesh, level: int) -> Level:
    n = 1 << level
    M = mm.tets.shape[0]
    # all lattice points of the closed macro: (i, j, k), i+j+k <= n
    pts = np.array([(i, j, k) for k in range(n + 1) for j in range(n + 1 - k) for i in range(n + 1 - j - k)],
                   dtype=np.int64)
    bary = np.stack([n - pts.sum(1), pts[:, 0], pts[:, 1], pts[:, 2]], axis=1)
    all_keys = np.concatenate([_canonical_keys(mm.tets[m], bary) for m in range(M)], axis=0)
    ukeys, inverse = np.unique(all_keys, axis=0, return_inverse=True)
    inverse = inverse.reshape(-1)
    P = pts.shape[0]
    local_to_node = []
    for m in range(M):
        tab = -np.ones((n + 1, n + 1, n + 1), dtype=np.int64)
        ids = inverse[m * P:(m + 1) * P]
        tab[pts[:, 0], pts[:, 1], pts[:, 2]] = ids
        local_to_node.append(tab)
    N = ukeys.shape[0]
    # coordinates: sum of weights * macro vertex coordinates / n
    coords = np.zeros((N, 3))
    for c in range(4):
        v = ukeys[:, 2 * c]
        w = ukeys[:, 2 * c + 1]
        ok = v >= 0
        coords[ok] += w[ok, None] * mm.xyz[v[ok]]
    coords /= n
    nnz = (ukeys[:, 1::2] > 0).sum(1)
    skeleton = nnz < 4
    dirichlet = np.zeros(N, dtype=bool)
    for a in np.nonzero(skeleton)[0]:
        support = [int(ukeys[a, 2 * c]) for c in range(4) if ukeys[a, 2 * c + 1] > 0]
        dirichlet[a] = mm.support_is_dirichlet(support)
    # elements
    B = refine_barycentric(level)  # (8^l, 4, 4)
    loc = B[:, :, 1:4]  # (e, 4, 3) local (i, j, k)
    elems, emac, eloc = [], [], []
    for m in range(M):
        tab = local_to_node[m]
        elems.append(tab[loc[..., 0], loc[..., 1], loc[..., 2]])
        emac.append(np.full(loc.shape[0], m, dtype=np.int64))
        eloc.append(loc)
    elems = np.concatenate(elems)
    assert elems.min() >= 0
    return Level(level, n, coords, ukeys, skeleton, dirichlet, elems, np.concatenate(emac),
                 np.concatenate(eloc), local_to_node, None)


def prolongation_parents(mm: MacroMesh, coarse: Level, fine: Level):
    """For every fine node: (a, b) coarse node ids; a == b when the fine node coincides with a
    coarse node, else the fine node is the midpoint of the coarse edge (a, b).

    Derived from the refinement itself: fine vertices are corners or edge midpoints of the
    coarse elements (Bey's rule)."""
    Nf = fine.num_nodes
    par = -np.ones((Nf, 2), dtype=np.int64)
    for m in range(mm.tets.shape[0]):
        ctab = coarse.local_to_node[m]
        ftab = fine.local_to_node[m]
        sel = coarse.elem_macro == m
        cl = coarse.elem_local[sel]  # (e, 4, 3)
        for a in range(4):
            f = ftab[2 * cl[:, a, 0], 2 * cl[:, a, 1], 2 * cl[:, a, 2]]
            c = ctab[cl[:, a, 0], cl[:, a, 1], cl[:, a, 2]]
            par[f, 0] = c
            par[f, 1] = c
        for (a, b) in EDGES_OF_TET:
            mid = cl[:, a] + cl[:, b]
            f = ftab[mid[:, 0], mid[:, 1], mid[:, 2]]
            ca = ctab[cl[:, a, 0], cl[:, a, 1], cl[:, a, 2]]
            cb = ctab[cl[:, b, 0], cl[:, b, 1], cl[:, b, 2]]
            par[f, 0] = np.minimum(ca, cb)
            par[f, 1] = np.maximum(ca, cb)
    assert par.min() >= 0
    return par


def hierarchy(mm: MacroMesh, levels):
    return {l: build_level(mm, l) for l in levels}


def node_incidences(lv: Level):
    """node -> list of (macro, i, j, k)."""
    inc = [[] for _ in range(lv.num_nodes)]
    for m, tab in enumerate(lv.local_to_node):
        ii, jj, kk = np.nonzero(tab >= 0)
        ids = tab[ii, jj, kk]
        for a, i, j, k in zip(ids.tolist(), ii.tolist(), jj.tolist(), kk.tolist()):
            inc[a].append((m, i, j, k))
    return inc


def match_nodes(coords_a, coords_b, tol=1e-9):
    """Permutation p with coords_b[p[i]] == coords_a[i] (nodes of two implementations)."""
    scale = 1e6
    ka = np.rint(np.asarray(coords_a) * scale).astype(np.int64)
    kb = np.rint(np.asarray(coords_b) * scale).astype(np.int64)
    ia = np.lexsort(ka.T[::-1])
    ib = np.lexsort(kb.T[::-1])
    if ka.shape != kb.shape or not np.array_equal(ka[ia], kb[ib]):
        raise ValueError("node sets differ")
    p = np.empty(len(ia), dtype=np.int64)
    p[ia] = ib
    if np.abs(np.asarray(coords_b)[p] - np.asarray(coords_a)).max() > tol:
        raise ValueError("node coordinates differ")
    return p


KUHN_PERMUTATIONS = tuple(itertools.permutations(range(3)))
