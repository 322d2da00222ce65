"""Oracle element integrals for P1 tetrahedra.

Test infrastructure only (see the package docstring).

All element matrices are integrated by a quadrature rule on each element
(the degree-2 four-point rule with barycentric points (a,b,b,b) and
permutations, a = (5+3 sqrt 5)/20, b = (5-sqrt 5)/20, weights |t|/4), using the
closed-form gradients of the barycentric coordinates.

Index convention for vector-valued blocks (Sec. 2, eq. (macrobilinearform)):
the element block for test vertex a and trial vertex b is

    K[a, b, m, l] = a_t(phi_b e_l, phi_a e_m),

so that (K u)_{a,m} = sum_{b,l} K[a,b,m,l] u_{b,l}: row = test function
(vertex a, component m), column = trial function (vertex b, component l).
With D u = eps(u) or D u = div u (Sec. 2) and the coefficient factored out:

    eps(phi_b e_l) : eps(phi_a e_m) = 1/2 (delta_lm g_a.g_b + (g_a)_l (g_b)_m)
    div(phi_b e_l)  div(phi_a e_m) = (g_b)_l (g_a)_m

with g_a = grad(phi_a).
"""

from __future__ import annotations

import numpy as np

_A = (5.0 + 3.0 * np.sqrt(5.0)) / 20.0
_B = (5.0 - np.sqrt(5.0)) / 20.0
QUAD_BARY = np.array([[_A, _B, _B, _B], [_B, _A, _B, _B], [_B, _B, _A, _B], [_B, _B, _B, _A]])
QUAD_W = np.full(4, 0.25)  # times |t|


def p1_geometry(X):
    """X: (E, 4, 3) vertex coordinates -> (grads (E, 4, 3), volumes (E,))."""
    X = np.asarray(X, dtype=np.float64)
    J = X[:, 1:, :] - X[:, :1, :]  # rows: x_a - x_0
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)  # x - x0 = J^T lam  ->  lam = J^{-T}(x - x0), grad lam_a = Jinv[:, :, a]
    g = np.empty((X.shape[0], 4, 3))
    g[:, 1:, :] = np.transpose(Jinv, (0, 2, 1))
    g[:, 0, :] = -g[:, 1:, :].sum(axis=1)
    return g, np.abs(det) / 6.0


def element_stiffness(X, c_eps: float, c_div: float):
    """K[e, a, b, m, l] of c_eps (eps(u), eps(v)) + c_div (div u, div v) on each element."""
    g, vol = p1_geometry(X)
    E = g.shape[0]
    eye = np.eye(3)
    gg = np.einsum("eai,ebi->eab", g, g)
    eps = 0.5 * (gg[:, :, :, None, None] * eye[None, None, None, :, :]
                 + np.einsum("eal,ebm->eabml", g, g))
    div = np.einsum("ebl,eam->eabml", g, g)
    integrand = c_eps * eps + c_div * div  # constant on the element
    K = np.zeros((E, 4, 4, 3, 3))
    for q in range(QUAD_BARY.shape[0]):
        K += (QUAD_W[q] * vol)[:, None, None, None, None] * integrand
    return K


def elasticity_coefficients(nu: float):
    """a^{E=1} = 1/(1+nu) (eps, eps) + nu/((1+nu)(1-2nu)) (div, div)  (Sec. 5.1.2, eq. (bilinearformE))."""
    return 1.0 / (1.0 + nu), nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


def element_mass(X):
    """Scalar P1 mass matrix M[e, a, b] = int phi_a phi_b by quadrature."""
    _, vol = p1_geometry(X)
    M = np.zeros((X.shape[0], 4, 4))
    for q in range(QUAD_BARY.shape[0]):
        lam = QUAD_BARY[q]
        M += (QUAD_W[q] * vol)[:, None, None] * np.outer(lam, lam)[None]
    return M


def element_laplace(X):
    """Scalar P1 Laplacian L[e, a, b] = int grad phi_a . grad phi_b."""
    g, vol = p1_geometry(X)
    L = np.zeros((X.shape[0], 4, 4))
    for q in range(QUAD_BARY.shape[0]):
        L += (QUAD_W[q] * vol)[:, None, None] * np.einsum("eai,ebi->eab", g, g)
    return L


def element_divergence(X):
    """Bd[e, a, b, l] = -int phi_a d_l phi_b : pressure test vertex a, velocity trial (b, l)."""
    g, vol = p1_geometry(X)
    Bd = np.zeros((X.shape[0], 4, 4, 3))
    for q in range(QUAD_BARY.shape[0]):
        lam = QUAD_BARY[q]
        Bd -= (QUAD_W[q] * vol)[:, None, None, None] * lam[None, :, None, None] * g[:, None, :, :]
    return Bd
