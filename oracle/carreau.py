"""Oracle for the nodal strain rate (Sec. 3) and the Carreau viscosity (Sec. 5.2.2).

Test infrastructure only (see the package docstring).

At every node the velocity components are fitted in the least-squares sense by an
affine polynomial (m = 1) or a quadratic one (m = 2) over the node and its mesh neighbours
(eq. minimization_problem); the fitted gradient gives eps(u) = (grad u + grad u^T)/2, |eps|^2 = eps : eps, and

    mu = eta_inf + (eta0 - eta_inf) (1 + kappa |eps|^2)^r          (eq. carreau).

The fixed-point iteration of Alg. 1 (Sec. 5.2.2) is restated with exact linear solves.
"""

from __future__ import annotations

import numpy as np

from .mesh import Level


def neighbours(lv: Level):
    """node -> sorted array of the nodes sharing an element with it."""
    N = lv.num_nodes
    pairs = np.concatenate([lv.elems[:, [a, b]] for a in range(4) for b in range(4) if a != b])
    pairs = np.unique(pairs, axis=0)
    split = np.searchsorted(pairs[:, 0], np.arange(N + 1))
    return [pairs[split[i]:split[i + 1], 1] for i in range(N)]


# A quadratic fit is used only where the patch determines it: the columns 1, dx/rho and
# dx_a dx_b / rho^2 (rho the patch radius) have a smallest singular value above QUAD_RANK_TOL
# times the largest.  Elsewhere (patches one-sided in some direction, e.g. on the domain
# boundary, where dz^2 and dz agree on the two layers of points) the quadratic terms are not
# determined and would bias the gradient, and the fit is the affine one.  The paper (Sec. 3)
# does not treat such patches.
QUAD_RANK_TOL = 1e-6


def lsq_gradients(lv: Level, u, degree=1):
    """(N, 3, 3) array g[i, c, a] = d u_c / d x_a of the fitted polynomial at node i
    (degree 1: affine; 2: quadratic where the patch determines it, else affine)."""
    u = np.asarray(u).reshape(-1, 3)
    nb = neighbours(lv)
    g = np.zeros((lv.num_nodes, 3, 3))
    for i in range(lv.num_nodes):
        pts = np.concatenate([[i], nb[i]])
        dx = lv.coords[pts] - lv.coords[i]
        rho = np.abs(dx).max()
        y = dx / rho
        cols = [np.ones(len(pts)), y[:, 0], y[:, 1], y[:, 2]]
        if degree == 2:
            quad = cols + [y[:, a] * y[:, b] for a in range(3) for b in range(a, 3)]
            sv = np.linalg.svd(np.stack(quad, axis=1), compute_uv=False)
            if len(pts) >= 10 and sv[-1] > QUAD_RANK_TOL * sv[0]:
                cols = quad
        V = np.stack(cols, axis=1)
        coef, *_ = np.linalg.lstsq(V, u[pts], rcond=None)
        g[i] = coef[1:4].T / rho
    return g


def strain_rate_sq(g):
    e = 0.5 * (g + np.transpose(g, (0, 2, 1)))
    return (e**2).sum(axis=(1, 2))


def carreau(e2, eta0, eta_inf, kappa, r):
    return eta_inf + (eta0 - eta_inf) * (1.0 + kappa * e2) ** r


def viscosity(lv: Level, u, eta0, eta_inf, kappa, r, degree=1):
    return carreau(strain_rate_sq(lsq_gradients(lv, u, degree)), eta0, eta_inf, kappa, r)


# ------------------------------------------------------- fixed-point iteration (Alg. 1)


def saddle_solve(mm, lv: Level, mu, f4, g4):
    """Exact solution of the linearised saddle system (eq. fixpointsystem) for the viscosity
    mu: K(mu) x = f with the velocity-Dirichlet values of g4 and the pressure fixed by a zero
    mass-weighted mean (bordered system [[K, c], [c^T, 0]], c = (0, m), m the lumped mass).
    f4, g4: (N, 4) node-major (u, v, w, p); returns x (N, 4)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    from . import stokes as stk

    N = lv.num_nodes
    Kbc, _ = stk.stokes_operator(mm, lv, mu)
    rhs = stk.pack4(f4)
    d = np.asarray(lv.dirichlet)
    g = np.asarray(g4, dtype=np.float64)
    rhs[:3 * N].reshape(N, 3)[d] = g[d, :3]
    c = np.concatenate([np.zeros(3 * N), stk.lumped_mass(lv)])
    Kb = sp.bmat([[Kbc, sp.csr_matrix(c[:, None])], [sp.csr_matrix(c[None, :]), None]]).tocsc()
    sol = spla.spsolve(Kb, np.concatenate([rhs, [0.0]]))
    return stk.unpack4(sol[:4 * N], N)


def picard(mm, lv: Level, f4, x0, eta0, eta_inf, kappa, r, tol=1e-3, max_picard=40):
    """Alg. 1 (Sec. 5.2.2) with every linear system solved exactly (``saddle_solve``): the
    method's inexact multigrid solves approximate these steps.

        mu^(0) = mu(u^(0));  repeat: x^(n+1) = solve(mu^(n)), mu^(n+1) = mu(u^(n+1)), n += 1
        until max_i |u_i^(n) - u_i^(n-1)|_2 < tol * max_i |u_i^(n)|_2;
        final: x^(n+1) = solve(mu^(n)), mu^(n+1) = mu(u^(n+1)).

    x0 (N, 4) holds u^(0) and the velocity-Dirichlet values.  Returns (x, mu, n, changes)
    with n the number of fixed-point steps before the final solve and changes the relative
    change of each step."""
    x = np.array(x0, dtype=np.float64)
    mu = viscosity(lv, x[:, :3], eta0, eta_inf, kappa, r)
    changes = []
    n = 0
    while n < max_picard:
        prev = x
        x = saddle_solve(mm, lv, mu, f4, x0)
        mu = viscosity(lv, x[:, :3], eta0, eta_inf, kappa, r)
        n += 1
        um = np.linalg.norm(x[:, :3], axis=1).max()
        du = np.linalg.norm(x[:, :3] - prev[:, :3], axis=1).max()
        changes.append(du / um if um > 0 else 0.0)
        if changes[-1] < tol:
            break
    x = saddle_solve(mm, lv, mu, f4, x0)
    mu = viscosity(lv, x[:, :3], eta0, eta_inf, kappa, r)
    return x, mu, n, changes
