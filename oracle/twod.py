"""Oracle for the 2D variant of the stencil scaling (Sec. 2.1 and Sec. 2.3).

Test infrastructure only (see the package docstring).

One macro triangle (v0, v1, v2) refined uniformly into n^2 triangles (n = 2^level): lattice
points (i, j), i + j <= n, at v0 + (i (v1 - v0) + j (v2 - v0)) / n, numbered row by row,
index j (n + 1) - j (j - 1) / 2 + i; "up" triangles (i, j), (i+1, j), (i, j+1) and "down"
triangles (i+1, j), (i, j+1), (i+1, j+1).  The vector P1 operator of the bilinear form
c_eps (eps(u), eps(v)) + c_div (div u, div v) with a scalar nodal coefficient k:

* nodal integration a_h: every element matrix scaled by the vertex mean kbar^t;
* physical scaling: for every edge (i, j) with its patch of elements P_ij, the block
  khat_ij Shat_ij + R_ij, khat_ij the mean of kbar^t over P_ij, Shat_ij the constant-
  coefficient block, R_ij = 1/2 sum_{t in P_ij} (kbar^t - kbar^{t^m}) a^{a;t}_ij (eq.
  corrtermgeneral, t^m the other element of the patch, a^{a;t} the antisymmetric part
  (a - a^T) / 2 of the element block), and the diagonal block minus the sum of the row's
  off-diagonal blocks;
* unphysical scaling: the same without R.

Only macro-interior rows are scaled; the boundary of the triangle is Dirichlet (identity
rows).  Element matrices are integrated by a 3-point quadrature rule with the P1 gradients
of each triangle.
"""

from __future__ import annotations

import numpy as np

# 3-point rule exact for quadratics (edge midpoints), barycentric weights 1/3
QUAD2 = np.array([[0.5, 0.5, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5]])
QUAD2_W = np.array([1.0, 1.0, 1.0]) / 3.0


def index(n, i, j):
    return j * (n + 1) - j * (j - 1) // 2 + i


class Lattice2D:
    def __init__(self, tri, level):
        self.tri = np.asarray(tri, dtype=np.float64)
        self.n = n = 1 << level
        pts, ij = [], []
        for j in range(n + 1):
            for i in range(n + 1 - j):
                ij.append((i, j))
                pts.append(self.tri[0] + (i * (self.tri[1] - self.tri[0]) + j * (self.tri[2] - self.tri[0])) / n)
        self.ij = np.array(ij)
        self.coords = np.array(pts)
        self.N = len(pts)
        els = []
        for j in range(n):
            for i in range(n - j):
                els.append((index(n, i, j), index(n, i + 1, j), index(n, i, j + 1)))
                if i + j <= n - 2:
                    els.append((index(n, i + 1, j), index(n, i, j + 1), index(n, i + 1, j + 1)))
        self.elems = np.array(els)
        I, J = self.ij[:, 0], self.ij[:, 1]
        self.boundary = (I == 0) | (J == 0) | (I + J == n)


def element_stiffness(X, c_eps, c_div):
    """K[e, a, b, m, l] = a(phi_b e_l, phi_a e_m) on each triangle X[e] (3 x 2 vertices)."""
    E = X.shape[0]
    K = np.zeros((E, 3, 3, 2, 2))
    for e in range(E):
        J = np.stack([X[e, 1] - X[e, 0], X[e, 2] - X[e, 0]], axis=1)  # columns: edge vectors
        area = 0.5 * abs(np.linalg.det(J))
        # gradients of the barycentric functions: rows of [ -1 -1 ; 1 0 ; 0 1 ] J^-1
        G = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]]) @ np.linalg.inv(J)
        for q in range(3):
            w = QUAD2_W[q] * area
            for a in range(3):
                for b in range(3):
                    for m in range(2):
                        for l in range(2):
                            eps = 0.5 * ((m == l) * G[a] @ G[b] + G[a, l] * G[b, m])
                            div = G[b, l] * G[a, m]
                            K[e, a, b, m, l] += w * (c_eps * eps + c_div * div)
    return K


def _blocks(lat, K, kbar):
    """Per element: (a, b) -> global (i, j) and its scaled/unscaled blocks."""
    out = {}
    for e, tri in enumerate(lat.elems):
        for a in range(3):
            for b in range(3):
                out.setdefault((tri[a], tri[b]), []).append(e)
    return out


def operator(lat, K, k, variant="physical"):
    """(2N, 2N) dense matrix (node-major: row 2 i + m) with identity Dirichlet rows."""
    N = lat.N
    k = np.asarray(k, dtype=np.float64)
    kbar = k[lat.elems].mean(axis=1)
    A = np.zeros((2 * N, 2 * N))
    patches = _blocks(lat, K, kbar)
    for i in range(N):
        if lat.boundary[i]:
            A[2 * i:2 * i + 2, 2 * i:2 * i + 2] = np.eye(2)
            continue
        diag = np.zeros((2, 2))
        for (p, q), els in patches.items():
            if p != i or q == i:
                continue
            blocks = []
            for e in els:
                tri = list(lat.elems[e])
                blocks.append(K[e, tri.index(p), tri.index(q)])
            if variant == "nodal":
                S = sum(kbar[e] * B for e, B in zip(els, blocks))
            else:
                S = np.mean([kbar[e] for e in els]) * sum(blocks)
                if variant == "physical":
                    assert len(els) == 2, "an interior row's edge lies in two elements"
                    e0, e1 = els
                    B0, B1 = blocks
                    R = 0.5 * ((kbar[e0] - kbar[e1]) * 0.5 * (B0 - B0.T) + (kbar[e1] - kbar[e0]) * 0.5 * (B1 - B1.T))
                    S = S + R
            A[2 * i:2 * i + 2, 2 * q:2 * q + 2] = S
            diag -= S
        if variant == "nodal":
            diag = np.zeros((2, 2))
            for (p, q), els in patches.items():
                if p == i and q == i:
                    for e in els:
                        tri = list(lat.elems[e])
                        diag += kbar[e] * K[e, tri.index(p), tri.index(p)]
        A[2 * i:2 * i + 2, 2 * i:2 * i + 2] = diag
    return A


def galerkin(lat, K, kfun_quad=None):
    """Constant-coefficient (k = 1) assembled matrix with identity Dirichlet rows."""
    return operator(lat, K, np.ones(lat.N), "nodal")


def apply(A, x):
    """y = A x for a node-major (N, 2) field."""
    return (A @ np.asarray(x, dtype=np.float64).reshape(-1)).reshape(-1, 2)
