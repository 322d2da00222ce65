"""Oracle smoothers, transfers, V-cycle and Krylov solvers (plain FP64, small sizes).

Test infrastructure only (see the package docstring).

Sec. 5 solves with geometric multigrid: matrix-free linear interpolation between
levels, its transpose as restriction, a smoother on every level and a coarse-grid
solve; coarse operators are the scaled-stencil operators of the coarser meshes
with the nodal coefficient evaluated at their nodes (which are fine nodes).  The
smoothers here are point Jacobi, the paper's hybrid Gauss-Seidel, and Chebyshev
semi-iteration on D^-1 A (Saad, Iterative Methods for Sparse Linear Systems, 2nd ed.,
Sec. 12.3), the coarse
solve is a dense direct solve, and CG is the textbook preconditioned conjugate
gradient method (Saad, Alg. 9.1).  Vectors are node-major (N, 3).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.linalg as sla

from . import mesh as M


def free_mask(dirichlet):
    return np.repeat(~np.asarray(dirichlet), 3)


def residual(A, dirichlet, f, x):
    """f - A x on free rows, 0 on Dirichlet rows."""
    r = np.asarray(f, dtype=np.float64).reshape(-1) - A @ np.asarray(x, dtype=np.float64).reshape(-1)
    r[~free_mask(dirichlet)] = 0.0
    return r.reshape(-1, 3)


def point_diagonal(A, dirichlet):
    d = A.diagonal().copy()
    d[~free_mask(dirichlet)] = 1.0
    return d.reshape(-1, 3)


def jacobi(A, dirichlet, f, x, omega, steps):
    """x <- x + omega D^-1 (f - A x), `steps` times (Dirichlet values unchanged)."""
    D = point_diagonal(A, dirichlet)
    x = np.array(x, dtype=np.float64).reshape(-1, 3)
    for _ in range(steps):
        x = x + omega * residual(A, dirichlet, f, x) / D
    return x


def interior_colours(lv: M.Level):
    """Colour of every macro-interior node, 4 (i % 2) + 2 (j % 2) + (k % 2) of its lattice
    coordinates (i, j, k) in its macro; -1 on the macro skeleton.  Every stencil direction
    changes at least one of the three parities, so no two neighbours share a colour."""
    col = -np.ones(lv.num_nodes, dtype=np.int64)
    for tab in lv.local_to_node:
        I, J, K = np.nonzero(tab >= 0)
        ids = tab[I, J, K]
        inner = ~np.asarray(lv.skeleton)[ids]
        col[ids[inner]] = 4 * (I[inner] % 2) + 2 * (J[inner] % 2) + K[inner] % 2
    return col


def hybrid_gauss_seidel(A, dirichlet, skeleton, colours, f, x, omega, steps):
    """Hybrid Gauss-Seidel (Sec. 5: Gauss-Seidel inside the macros, Jacobi-like across their
    interfaces).  One step: x_s += omega D_ss^-1 (f - A x)_s at every free skeleton node at once,
    then for each colour c = 0..7 in turn x_i += D_ii^-1 (f - A x)_i at every macro-interior node
    of colour c, with the x of that moment."""
    D = point_diagonal(A, dirichlet)
    x = np.array(x, dtype=np.float64).reshape(-1, 3)
    skel = np.asarray(skeleton) & ~np.asarray(dirichlet)
    for _ in range(steps):
        r = residual(A, dirichlet, f, x)
        x[skel] += omega * r[skel] / D[skel]
        for c in range(8):
            sel = colours == c
            r = residual(A, dirichlet, f, x)
            x[sel] += r[sel] / D[sel]
    return x


def chebyshev(A, dirichlet, f, x, lam_max, lo, hi, steps):
    """Chebyshev semi-iteration for D^-1 A x = D^-1 f on the interval [lo, hi] * lam_max
    (theta = centre, delta = half width, sigma = theta / delta)."""
    D = point_diagonal(A, dirichlet)
    a, b = lo * lam_max, hi * lam_max
    theta, delta = 0.5 * (b + a), 0.5 * (b - a)
    sigma = theta / delta
    rho = 1.0 / sigma
    x = np.array(x, dtype=np.float64).reshape(-1, 3)
    d = residual(A, dirichlet, f, x) / D / theta
    x = x + d
    for _ in range(steps - 1):
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * residual(A, dirichlet, f, x) / D
        rho = rho_new
        x = x + d
    return x


def prolongation(coarse: M.Level, fine: M.Level, parents):
    """P (fine nodes x coarse nodes) of linear interpolation: weight 1 for a coincident node,
    1/2 for each end of the coarse edge whose midpoint the fine node is."""
    Nf, Nc = fine.num_nodes, coarse.num_nodes
    a, b = parents[:, 0], parents[:, 1]
    same = a == b
    rows = np.concatenate([np.nonzero(same)[0], np.nonzero(~same)[0], np.nonzero(~same)[0]])
    cols = np.concatenate([a[same], a[~same], b[~same]])
    vals = np.concatenate([np.ones(same.sum()), np.full((~same).sum(), 0.5), np.full((~same).sum(), 0.5)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(Nf, Nc))


def prolongate_add(P, xc, xf):
    return np.asarray(xf).reshape(-1, 3) + P @ np.asarray(xc).reshape(-1, 3)


def restrict(P, rf, fine_dirichlet, coarse_dirichlet):
    """P^T rf, with rf taken as 0 on fine Dirichlet nodes and the result 0 on coarse ones."""
    r = np.array(rf, dtype=np.float64).reshape(-1, 3)
    r[np.asarray(fine_dirichlet)] = 0.0
    rc = P.T @ r
    rc[np.asarray(coarse_dirichlet)] = 0.0
    return rc


class Hierarchy:
    """Levels l_min..l_max of one macro mesh with their operators (with Dirichlet rows)."""

    def __init__(self, mm, levels, A_of_level):
        self.mm = mm
        self.lv = {l: M.build_level(mm, l) for l in levels}
        self.levels = sorted(levels)
        self.A = {l: A_of_level(self.lv[l]) for l in levels}
        self.P = {}
        for l in self.levels[1:]:
            par = M.prolongation_parents(mm, self.lv[l - 1], self.lv[l])
            self.P[l] = prolongation(self.lv[l - 1], self.lv[l], par)

    def coarse_solve(self, f):
        l = self.levels[0]
        A, d = self.A[l], self.lv[l].dirichlet
        fr = free_mask(d)
        x = np.zeros(A.shape[0])
        if fr.any():
            Aff = A[fr][:, fr].toarray()
            x[fr] = sla.solve(Aff, np.asarray(f).reshape(-1)[fr])
        return x.reshape(-1, 3)

    def vcycle(self, l, f, x, smoother, pre, post, lam=None, omega=2 / 3, lo=1 / 8, hi=1.1):
        """One V(pre, post) cycle; lam[l] = lambda_max of D^-1 A used by Chebyshev."""
        if l == self.levels[0]:
            return self.coarse_solve(f)
        A, d = self.A[l], self.lv[l].dirichlet

        def smooth(x, steps):
            if steps == 0:
                return x
            if smoother == "jacobi":
                return jacobi(A, d, f, x, omega, steps)
            if smoother == "hybrid_gs":
                lv = self.lv[l]
                return hybrid_gauss_seidel(A, d, lv.skeleton, interior_colours(lv), f, x, omega, steps)
            return chebyshev(A, d, f, x, lam[l], lo, hi, steps)

        x = smooth(x, pre)
        r = residual(A, d, f, x)
        rc = restrict(self.P[l], r, d, self.lv[l - 1].dirichlet)
        ec = self.vcycle(l - 1, rc, np.zeros_like(rc), smoother, pre, post, lam, omega, lo, hi)
        x = prolongate_add(self.P[l], ec, x)
        return smooth(x, post)


def lambda_max_DinvA(A, dirichlet):
    """Largest eigenvalue of D^-1 A on the free DoFs (dense, small sizes)."""
    fr = free_mask(dirichlet)
    Aff = A[fr][:, fr].toarray()
    D = np.diag(Aff)
    Dh = 1.0 / np.sqrt(D)
    return float(np.linalg.eigvalsh(Dh[:, None] * Aff * Dh[None, :]).max())


def direct_solve(A, dirichlet, f, x0):
    """Exact solution with the Dirichlet values of x0 (sparse direct)."""
    import scipy.sparse.linalg as spla

    fr = free_mask(dirichlet)
    x = np.array(x0, dtype=np.float64).reshape(-1)
    Af = A[fr]
    rhs = np.asarray(f).reshape(-1)[fr] - Af[:, ~fr] @ x[~fr]
    x[fr] = spla.spsolve(Af[:, fr].tocsc(), rhs)
    return x.reshape(-1, 3)


def pcg(A, dirichlet, f, x, precond, rtol, max_iter):
    """Preconditioned CG on the free DoFs (Saad, Alg. 9.1); precond(r) -> z."""
    x = np.array(x, dtype=np.float64).reshape(-1, 3)
    r = residual(A, dirichlet, f, x)
    r0 = np.sqrt((r**2).sum())
    z = precond(r)
    p = z.copy()
    rz = (r * z).sum()
    it = 0
    for it in range(1, max_iter + 1):
        q = (A @ p.reshape(-1)).reshape(-1, 3)
        q[np.asarray(dirichlet)] = 0.0
        alpha = rz / (p * q).sum()
        x = x + alpha * p
        r = r - alpha * q
        if np.sqrt((r**2).sum()) <= rtol * r0:
            break
        z = precond(r)
        rzn = (r * z).sum()
        p = z + (rzn / rz) * p
        rz = rzn
    return x, it
