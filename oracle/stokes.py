"""Oracle for the stabilised P1-P1 generalised Stokes operator of Sec. 5.2.

Test infrastructure only (see the package docstring).

    K = [[A(mu), B^T], [B, C]],
    A(mu): the physical-scaling operator of a(u, v) = (2 mu eps(u), eps(v)) (Sec. 2),
    B = -(div u, q),  C = c_l(p, q) = -(h^2/12) (grad p, grad q)   (Sec. 5.2),

with h the mesh size of the level; here h = (6 |T|)^{1/3} / n per macro (the lattice
spacing 1/n on the Kuhn cube).  Unknown ordering: velocity node-major (3N), then the
pressure (N).  Velocity-Dirichlet rows are identity rows; pressure rows are all free.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem
from . import operators as op
from .mesh import Level, MacroMesh


def macro_h(mm: MacroMesh, lv: Level):
    """Stabilisation length per element: (6 |T|)^{1/3} / n of its macro."""
    X = mm.xyz[mm.tets]
    _, volT = fem.p1_geometry(X)
    return (np.cbrt(6.0 * volT) / lv.n)[lv.elem_macro]


def divergence_matrix(lv: Level):
    """B (N x 3N): B[i, 3j+l] = -int phi_i d_l phi_j."""
    Bd = fem.element_divergence(lv.coords[lv.elems])  # (E, a, b, l)
    E = lv.elems.shape[0]
    rows = np.repeat(lv.elems[:, :, None, None], 4, axis=2).repeat(3, axis=3)
    cols = 3 * np.repeat(lv.elems[:, None, :, None], 4, axis=1).repeat(3, axis=3) + np.arange(3)[None, None, None, :]
    N = lv.num_nodes
    return sp.coo_matrix((Bd.reshape(-1), (rows.reshape(-1), cols.reshape(-1))), shape=(N, 3 * N)).tocsr()


def stabilisation_matrix(mm: MacroMesh, lv: Level):
    """C (N x N) = -(h^2/12) (grad p, grad q)."""
    Lap = fem.element_laplace(lv.coords[lv.elems])
    h = macro_h(mm, lv)
    vals = -(h**2 / 12.0)[:, None, None] * Lap
    rows = np.repeat(lv.elems, 4, axis=1).reshape(-1)
    cols = np.tile(lv.elems, (1, 4)).reshape(-1)
    N = lv.num_nodes
    return sp.coo_matrix((vals.reshape(-1), (rows, cols)), shape=(N, N)).tocsr()


def lumped_mass(lv: Level):
    M = fem.element_mass(lv.coords[lv.elems])
    m = np.zeros(lv.num_nodes)
    np.add.at(m, lv.elems.reshape(-1), M.sum(axis=2).reshape(-1))
    return m


def stokes_operator(mm: MacroMesh, lv: Level, mu, variant="physical", khat="patch", iface="symmetric"):
    """(K with Dirichlet velocity rows, K without them)."""
    K_el = fem.element_stiffness(lv.coords[lv.elems], 2.0, 0.0)
    A = op.scaled_operator(lv, K_el, mu, variant, khat=khat, iface=iface)
    B = divergence_matrix(lv)
    C = stabilisation_matrix(mm, lv)
    K = sp.bmat([[A, B.T], [B, C]]).tocsr()
    N = lv.num_nodes
    d = np.zeros(4 * N, dtype=bool)
    dn = np.nonzero(lv.dirichlet)[0]
    for m in range(3):
        d[3 * dn + m] = True
    keep = sp.diags((~d).astype(np.float64))
    Kbc = (keep @ K + sp.diags(d.astype(np.float64))).tocsr()
    return Kbc, K


def pack(u, p):
    return np.concatenate([np.asarray(u).reshape(-1), np.asarray(p).reshape(-1)])


def unpack(x, N):
    return x[:3 * N].reshape(N, 3), x[3 * N:]


def residual(Kbc, dirichlet, f, x):
    """f - K x with 0 on velocity-Dirichlet rows."""
    r = np.asarray(f) - Kbc @ np.asarray(x)
    N = len(dirichlet)
    ru = r[:3 * N].reshape(N, 3)
    ru[np.asarray(dirichlet)] = 0.0
    return r


# ------------------------------------------------------- inexact Uzawa multigrid (Sec. 5.2)
#
# The paper solves its Stokes systems with an all-at-once multigrid whose smoother is an
# inexact Uzawa iteration: a velocity smoothing with the pressure fixed, then a damped
# pressure update with an approximation of the Schur complement S = C - B A^-1 B^T;
# V-cycles with more smoothing steps on coarser levels.  The library's choices, restated
# here one step at a time (vectors (N, 4): velocity node-major, then the pressure):
#   * velocity smoothing: `vsteps` Chebyshev steps on D^-1 A (A the velocity block with
#     Dirichlet identity rows, interval [lo, hi] * lambda_max) for A du = r_u from du = 0, or
#     (smoother "hybrid_gs", the paper's choice in Sec. 5.2.1) `vsteps` hybrid Gauss-Seidel
#     steps with skeleton damping gs_omega;
#   * pressure update: p -= omega (g - B u - C p) / s,  s_i = m_i / mu_i + (-C)_ii
#     (m the lumped mass, a diagonal surrogate of -S);
#   * V-cycle on level l: pre + extra (lmax - l) steps, restriction of the saddle residual
#     (velocity: P^T with Dirichlet rows zeroed; pressure: P^T), recursion from zero,
#     prolongation x += P x_c (both fields), post + extra (lmax - l) steps;
#   * coarsest level: exact solve on the free velocity and all pressure DoFs with
#     beta / N_p added to every pressure-pressure entry (beta = the largest absolute entry),
#     which removes the constant-pressure kernel.


def pack4(x4):
    """(N, 4) node-major (u, v, w, p) -> the packed ordering of stokes_operator."""
    x4 = np.asarray(x4, dtype=np.float64)
    return np.concatenate([x4[:, :3].reshape(-1), x4[:, 3]])


def unpack4(x, N):
    out = np.empty((N, 4))
    out[:, :3] = x[:3 * N].reshape(N, 3)
    out[:, 3] = x[3 * N:]
    return out


def schur_surrogate(mm: MacroMesh, lv: Level, mu):
    """s_i = m_i / mu_i + (-C)_ii."""
    C = stabilisation_matrix(mm, lv)
    return lumped_mass(lv) / np.asarray(mu) - C.diagonal()


class UzawaHierarchy:
    """Levels of one macro mesh with the saddle operator K (velocity-Dirichlet identity
    rows), its velocity block A, the Schur surrogate s, the lumped mass and the linear
    interpolation P between consecutive levels; the viscosity at every level is mu_fun at
    that level's nodes (injection, the nodes of a coarse level being fine nodes)."""

    def __init__(self, mm: MacroMesh, levels, mu_fun):
        from .mesh import build_level, prolongation_parents
        from .solvers import prolongation

        self.mm = mm
        self.levels = sorted(levels)
        self.lv, self.K, self.A, self.s, self.m = {}, {}, {}, {}, {}
        for l in self.levels:
            lv = build_level(mm, l)
            mu = mu_fun(lv.coords)
            Kbc, _ = stokes_operator(mm, lv, mu)
            N = lv.num_nodes
            self.lv[l] = lv
            self.K[l] = Kbc
            self.A[l] = Kbc[:3 * N, :3 * N].tocsr()
            self.s[l] = schur_surrogate(mm, lv, mu)
            self.m[l] = lumped_mass(lv)
        self.P = {}
        for l in self.levels[1:]:
            par = prolongation_parents(mm, self.lv[l - 1], self.lv[l])
            self.P[l] = prolongation(self.lv[l - 1], self.lv[l], par)

    def apply(self, l, x4):
        return unpack4(self.K[l] @ pack4(x4), self.lv[l].num_nodes)

    def residual(self, l, f4, x4):
        r = np.asarray(f4, dtype=np.float64) - self.apply(l, x4)
        r[self.lv[l].dirichlet, :3] = 0.0
        return r

    def dot(self, l, a, b):
        """Inner product over the free velocity DoFs and all pressures."""
        fr = ~self.lv[l].dirichlet
        return float((a[fr, :3] * b[fr, :3]).sum() + (a[:, 3] * b[:, 3]).sum())

    def project_pressure(self, l, x4):
        """Shift the pressure to zero mass-weighted mean."""
        x4 = np.array(x4, dtype=np.float64)
        m = self.m[l]
        x4[:, 3] -= (m * x4[:, 3]).sum() / m.sum()
        return x4

    def coarse_solve(self, f4):
        l = self.levels[0]
        lv = self.lv[l]
        N = lv.num_nodes
        vel = np.repeat(~lv.dirichlet, 3)
        keep = np.concatenate([vel, np.ones(N, dtype=bool)])
        Kd = self.K[l].toarray()[np.ix_(keep, keep)]
        beta = np.abs(Kd).max()
        nv = int(vel.sum())
        Kd[nv:, nv:] += beta / N
        x = np.zeros(4 * N)
        x[keep] = np.linalg.solve(Kd, pack4(f4)[keep])
        return unpack4(x, N)

    def uzawa_step(self, l, f4, x4, lam, vsteps=2, omega=0.5, lo=1 / 8, hi=1.1, smoother="chebyshev",
                   gs_omega=2 / 3):
        from .solvers import chebyshev, hybrid_gauss_seidel, interior_colours

        lv = self.lv[l]
        d = lv.dirichlet
        x4 = np.array(x4, dtype=np.float64)
        r = self.residual(l, f4, x4)
        z = np.zeros((len(d), 3))
        if smoother == "hybrid_gs":
            du = hybrid_gauss_seidel(self.A[l], d, lv.skeleton, interior_colours(lv), r[:, :3], z, gs_omega, vsteps)
        else:
            du = chebyshev(self.A[l], d, r[:, :3], z, lam[l], lo, hi, vsteps)
        x4[:, :3] += du
        r = self.residual(l, f4, x4)
        x4[:, 3] -= omega * r[:, 3] / self.s[l]
        return x4

    def vcycle(self, l, f4, x4, lam, lmax, pre=3, post=3, extra=2, vsteps=2, omega=0.5, lo=1 / 8, hi=1.1,
               smoother="chebyshev", gs_omega=2 / 3):
        """One variable V-cycle on level l (lmax: the finest level, for the extra steps)."""
        from .solvers import restrict

        if l == self.levels[0]:
            return self.coarse_solve(f4)
        x4 = np.array(x4, dtype=np.float64)
        ex = extra * (lmax - l)
        for _ in range(pre + ex):
            x4 = self.uzawa_step(l, f4, x4, lam, vsteps, omega, lo, hi, smoother, gs_omega)
        r = self.residual(l, f4, x4)
        Nc = self.lv[l - 1].num_nodes
        rc = np.zeros((Nc, 4))
        rc[:, :3] = restrict(self.P[l], r[:, :3], self.lv[l].dirichlet, self.lv[l - 1].dirichlet)
        rc[:, 3] = self.P[l].T @ r[:, 3]
        ec = self.vcycle(l - 1, rc, np.zeros((Nc, 4)), lam, lmax, pre, post, extra, vsteps, omega, lo, hi, smoother,
                         gs_omega)
        x4[:, :3] += self.P[l] @ ec[:, :3]
        x4[:, 3] += self.P[l] @ ec[:, 3]
        for _ in range(post + ex):
            x4 = self.uzawa_step(l, f4, x4, lam, vsteps, omega, lo, hi, smoother, gs_omega)
        return x4
