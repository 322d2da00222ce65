"""Pins of the oracle's nodal strain rate and Carreau law (Sec. 3, Sec. 5.2.2; no GPU)."""

import numpy as np

import hhg_inputs as hi
from oracle import carreau as CA, mesh


def _lv(builder, level):
    xyz, tets = builder()
    mm = mesh.MacroMesh.build(xyz, tets)
    return mesh.build_level(mm, level)


def test_affine_velocity_gradient_is_exact():
    for builder in (hi.kuhn_cube, hi.skewed_pair):
        lv = _lv(builder, 2)
        G = np.array([[0.3, -1.2, 0.7], [2.0, 0.1, -0.4], [0.5, 0.5, 1.5]])
        u = lv.coords @ G.T + np.array([1.0, 0.0, -2.0])
        g = CA.lsq_gradients(lv, u)
        assert np.allclose(g, G[None], atol=1e-12)
        e = 0.5 * (G + G.T)
        assert np.allclose(CA.strain_rate_sq(g), (e**2).sum())


def test_quadratic_and_affine_fits_agree_in_macro_interiors():
    """Sec. 3: on the point-symmetric interior patch the quadratic least-squares fit has the
    same gradient at the node as the affine one."""
    lv = _lv(hi.unit_tet, 3)
    u = np.stack([np.sin(3 * lv.coords[:, 0]) * lv.coords[:, 1], lv.coords[:, 2] ** 3,
                  np.cos(lv.coords.sum(1))], 1)
    g1 = CA.lsq_gradients(lv, u, degree=1)
    g2 = CA.lsq_gradients(lv, u, degree=2)
    inner = ~lv.skeleton
    assert np.allclose(g1[inner], g2[inner], atol=1e-12)
    # the unit tetrahedron's skeleton is its boundary: one-sided patches, which do not determine
    # a quadratic fit, so the fit there is the affine one
    assert np.allclose(g1[~inner], g2[~inner], atol=1e-12)


def _quadratic_field(c):
    Q = np.array([[[0.3, 1.0, -0.5], [1.0, 0.2, 0.0], [-0.5, 0.0, 0.7]],
                  [[0.0, 0.4, 0.0], [0.4, -1.0, 0.3], [0.0, 0.3, 0.2]],
                  [[1.0, 0.0, 0.1], [0.0, 0.5, 0.0], [0.1, 0.0, -0.3]]])
    b = np.array([[0.1, 0.2, 0.3], [-0.4, 0.0, 0.5], [0.2, -0.6, 0.1]])
    u = np.stack([np.einsum("na,ab,nb->n", c, Q[q], c) + c @ b[q] for q in range(3)], 1)
    grad = np.stack([2 * c @ Q[q] + b[q] for q in range(3)], 1)
    return u, grad


def test_quadratic_fit_is_exact_for_quadratic_fields_where_determined():
    """m = 2 (eq. minimization_problem) reproduces a quadratic velocity exactly, so its gradient
    is exact at every node whose patch determines the quadratic fit; on the skewed two-macro
    mesh these include interface nodes whose patches are not point-symmetric, where the affine
    fit is not exact.  Where the patch does not determine it (one-sided patches on the domain
    boundary) the fit is the affine one."""
    lv = _lv(hi.skewed_pair, 3)
    u, grad = _quadratic_field(lv.coords)
    g1 = CA.lsq_gradients(lv, u, degree=1)
    g2 = CA.lsq_gradients(lv, u, degree=2)
    e1 = np.abs(g1 - grad).max(axis=(1, 2))
    e2 = np.abs(g2 - grad).max(axis=(1, 2))
    exact2 = e2 < 1e-10 * np.abs(grad).max()
    gained = exact2 & (e1 > 1e-6)
    assert gained.sum() >= 20 and np.all(np.asarray(lv.skeleton)[gained])
    # every node is either quadratic-exact or fitted affinely (the rank rule's fallback)
    assert np.all(exact2 | np.all(np.isclose(g2, g1, rtol=0, atol=1e-12), axis=(1, 2)))
    assert (~exact2).sum() > 0


def test_carreau_law_limits():
    e2 = np.array([0.0, 1e-8, 1.0, 1e12])
    mu = CA.carreau(e2, 140.764, 1.0, 212.2, -0.325)  # the paper's dimensionless parameters
    assert mu[0] == 140.764
    assert np.all(np.diff(mu) < 0)  # shear thinning
    assert abs(mu[-1] - 1.0) < 1e-2 * 140.0


# ---------------------------------------------------------------- Alg. 1 (Sec. 5.2.2)

PAR = dict(eta0=1.0, eta_inf=1e-3, kappa=1.0, r=-0.25)


def _cube(level):
    xyz, tets = hi.kuhn_cube(1)
    mm = mesh.MacroMesh.build(xyz, tets)
    return mm, mesh.build_level(mm, level)


def test_picard_keeps_the_affine_shear_flow():
    """u = (z, 0, 0), p = 0 solves the Carreau-Stokes problem with f = 0 and its own boundary
    values: eps(u) is constant (|eps|^2 = 1/2), so mu is the constant
    eta_inf + (eta0 - eta_inf)(1 + kappa/2)^r (the least-squares fit is exact for affine u),
    div u = 0, and the P1 operator with a constant coefficient annihilates affine fields at
    free nodes.  Started there, Alg. 1 stops after one step with no change; started from the
    boundary values alone, it converges to the same flow."""
    mm, lv = _cube(3)
    N = lv.num_nodes
    ex = np.zeros((N, 4))
    ex[:, 0] = lv.coords[:, 2]
    mu_ex = PAR["eta_inf"] + (PAR["eta0"] - PAR["eta_inf"]) * (1 + PAR["kappa"] / 2) ** PAR["r"]
    f = np.zeros((N, 4))
    x, mu, n, ch = CA.picard(mm, lv, f, ex, **PAR)
    assert n == 1 and ch[0] < 1e-12
    assert np.abs(x[:, :3] - ex[:, :3]).max() < 1e-12 and np.abs(x[:, 3]).max() < 1e-10
    assert np.abs(mu - mu_ex).max() < 1e-12
    x0 = np.zeros((N, 4))
    x0[lv.dirichlet] = ex[lv.dirichlet]
    x, mu, n, ch = CA.picard(mm, lv, f, x0, tol=1e-10, max_picard=60, **PAR)
    assert n > 2 and ch[-1] < 1e-10
    assert np.abs(x - ex).max() < 1e-8
    assert np.abs(mu - mu_ex).max() < 1e-8


def test_picard_constant_viscosity_is_one_stokes_solve():
    """eta0 = eta_inf: mu does not depend on u, so the second step changes nothing (n = 2)
    and the result is the Stokes solution for that viscosity (the saddle system holds with
    it, and not with another)."""
    mm, lv = _cube(3)
    N = lv.num_nodes
    x0 = np.zeros((N, 4))
    x0[:, :3] = hi.lid_velocity(lv.coords)
    x0[~lv.dirichlet] = 0.0
    f = np.zeros((N, 4))
    sols = {}
    for m in (1.0, 3.0):
        x, mu, n, ch = CA.picard(mm, lv, f, x0, eta0=m, eta_inf=m, kappa=1.0, r=-0.25)
        assert n == 2 and ch[1] < 1e-12 and np.all(mu == m)
        sols[m] = x
    assert np.abs(sols[1.0][:, 3]).max() > 1e-2
    # the saddle system holds: free velocity rows and all pressure rows vanish, zero mean
    from oracle import stokes as stk

    for m in (1.0, 3.0):
        Kbc, _ = stk.stokes_operator(mm, lv, np.full(N, m))
        r = stk.residual(Kbc, lv.dirichlet, stk.pack4(f), stk.pack4(sols[m]))
        assert np.abs(r).max() < 1e-12
        assert abs((stk.lumped_mass(lv) * sols[m][:, 3]).sum()) < 1e-14
        Ko, _ = stk.stokes_operator(mm, lv, np.full(N, 4.0 - m))
        assert np.abs(stk.residual(Ko, lv.dirichlet, stk.pack4(f), stk.pack4(sols[m]))).max() > 1e-3
