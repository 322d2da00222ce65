"""Oracle for the boundary traction (Neumann) load (Sec. 5.1.3).

Test infrastructure only (see the package docstring).

The weak form of the elasticity problem with a traction t on Gamma_N carries the term
int_{Gamma_N} t . v ds.  With t replaced by its P1 interpolant, the load of node i is

    b_i = sum over boundary triangles T of the refined mesh on Gamma_N, T containing i, of
          (|T| / 12) (2 t_i + t_j + t_k)          (j, k the other vertices of T),

the exact P1 mass matrix of each triangle applied to the nodal traction.  The boundary
triangles are found from the refined tetrahedra themselves: faces that belong to exactly
one element and whose three vertices lie on a flagged macro face.
"""

from __future__ import annotations

import numpy as np

from .mesh import Level, MacroMesh


def boundary_triangles(mm: MacroMesh, lv: Level, face_flags):
    """(T, 3) node ids of the refined boundary triangles on the flagged macro faces
    (face_flags: (M, 4), face f of macro m opposite its local vertex f)."""
    flags = np.asarray(face_flags).reshape(-1, 4)
    planes = []
    for m, t in enumerate(mm.tets):
        for f in range(4):
            if flags[m, f]:
                tri = mm.xyz[[int(t[q]) for q in range(4) if q != f]]
                planes.append(tri)
    faces = {}
    for e in lv.elems:
        for f in range(4):
            key = tuple(sorted(int(e[q]) for q in range(4) if q != f))
            faces[key] = faces.get(key, 0) + 1
    out = []
    for key, cnt in faces.items():
        if cnt != 1:
            continue
        X = lv.coords[list(key)]
        for tri in planes:
            a, b, c = tri
            nrm = np.cross(b - a, c - a)
            area2 = np.linalg.norm(nrm)
            if np.abs((X - a) @ nrm).max() > 1e-12 * area2:
                continue
            # barycentric coordinates of the three points in the macro face
            ok = True
            for x in X:
                l1 = np.dot(np.cross(x - a, c - a), nrm) / area2**2
                l2 = np.dot(np.cross(b - a, x - a), nrm) / area2**2
                if l1 < -1e-12 or l2 < -1e-12 or l1 + l2 > 1 + 1e-12:
                    ok = False
                    break
            if ok:
                out.append(key)
                break
    return np.array(out, dtype=np.int64).reshape(-1, 3)


def traction_load(mm: MacroMesh, lv: Level, face_flags, t):
    """(N, 3) load vector b = M_Gamma t on every node (Dirichlet rows included; a solver uses
    the free rows)."""
    t = np.asarray(t, dtype=np.float64).reshape(-1, 3)
    b = np.zeros((lv.num_nodes, 3))
    for tri in boundary_triangles(mm, lv, face_flags):
        X = lv.coords[tri]
        area = 0.5 * np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0]))
        for a in range(3):
            others = [tri[q] for q in range(3) if q != a]
            b[tri[a]] += area / 12.0 * (2.0 * t[tri[a]] + t[others[0]] + t[others[1]])
    return b
