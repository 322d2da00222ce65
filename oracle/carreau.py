"""Oracle for the nodal strain rate (Sec. 3) and the Carreau viscosity (Sec. 5.2.2).

Test infrastructure only (see the package docstring).

At every node the velocity components are fitted in the least-squares sense by an
affine polynomial over the node and its mesh neighbours (eq. minimization_problem,
m = 1); the fitted gradient gives eps(u) = (grad u + grad u^T)/2, |eps|^2 = eps : eps, and

    mu = eta_inf + (eta0 - eta_inf) (1 + kappa |eps|^2)^r          (eq. carreau).
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


def lsq_gradients(lv: Level, u, degree=1):
    """(N, 3, 3) array g[i, c, a] = d u_c / d x_a of the fitted polynomial at node i."""
    u = np.asarray(u).reshape(-1, 3)
    nb = neighbours(lv)
    g = np.zeros((lv.num_nodes, 3, 3))
    for i in range(lv.num_nodes):
        pts = np.concatenate([[i], nb[i]])
        dx = lv.coords[pts] - lv.coords[i]
        cols = [np.ones(len(pts)), dx[:, 0], dx[:, 1], dx[:, 2]]
        if degree == 2:
            for a in range(3):
                for b in range(a, 3):
                    cols.append(dx[:, a] * dx[:, b])
        V = np.stack(cols, axis=1)
        coef, *_ = np.linalg.lstsq(V, u[pts], rcond=None)
        g[i] = coef[1:4].T
    return g


def strain_rate_sq(g):
    e = 0.5 * (g + np.transpose(g, (0, 2, 1)))
    return (e**2).sum(axis=(1, 2))


def carreau(e2, eta0, eta_inf, kappa, r):
    return eta_inf + (eta0 - eta_inf) * (1.0 + kappa * e2) ** r


def viscosity(lv: Level, u, eta0, eta_inf, kappa, r):
    return carreau(strain_rate_sq(lsq_gradients(lv, u)), eta0, eta_inf, kappa, r)
