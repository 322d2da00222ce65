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
    assert np.abs(g1[~inner] - g2[~inner]).max() > 1e-6  # not on the one-sided boundary patches


def test_carreau_law_limits():
    e2 = np.array([0.0, 1e-8, 1.0, 1e12])
    mu = CA.carreau(e2, 140.764, 1.0, 212.2, -0.325)  # the paper's dimensionless parameters
    assert mu[0] == 140.764
    assert np.all(np.diff(mu) < 0)  # shear thinning
    assert abs(mu[-1] - 1.0) < 1e-2 * 140.0
