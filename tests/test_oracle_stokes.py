"""Pins of the oracle's Stokes blocks (Sec. 5.2) by closed forms (no GPU)."""

import numpy as np

import hhg_inputs as hi
from oracle import mesh, stokes as ST


def _lv(builder, level):
    xyz, tets = builder()
    mm = mesh.MacroMesh.build(xyz, tets)
    return mm, mesh.build_level(mm, level)


def test_divergence_of_affine_velocity():
    """(B u)_i = -div(u) int phi_i for affine u, at every node."""
    for builder in (hi.kuhn_cube, hi.skewed_pair):
        mm, lv = _lv(builder, 3)
        G = np.array([[0.3, -1.2, 0.7], [2.0, 0.1, -0.4], [0.5, 0.5, 1.5]])
        u = lv.coords @ G.T + 1.0
        Bu = ST.divergence_matrix(lv) @ u.reshape(-1)
        m = ST.lumped_mass(lv)
        assert np.allclose(Bu, -np.trace(G) * m, atol=1e-14)


def test_gradient_of_affine_pressure_and_stabilisation():
    """(B^T p)_(i,m) = d_m p int phi_i and (C p)_i = 0 for affine p at nodes away from the
    domain boundary; C has zero row sums everywhere."""
    mm, lv = _lv(hi.kuhn_cube, 3)
    g = np.array([0.7, -0.2, 1.3])
    p = lv.coords @ g + 0.5
    B = ST.divergence_matrix(lv)
    C = ST.stabilisation_matrix(mm, lv)
    m = ST.lumped_mass(lv)
    inner = ~lv.dirichlet
    BTp = (B.T @ p).reshape(-1, 3)
    assert np.allclose(BTp[inner], m[inner, None] * g[None, :], atol=1e-14)
    assert np.abs((C @ p)[inner]).max() < 1e-15
    assert np.abs(C @ np.ones(lv.num_nodes)).max() < 1e-16
    # h = 1/n on the Kuhn cube: C = -(h^2/12) L with the P1 Laplacian L
    assert np.allclose(ST.macro_h(mm, lv), 1.0 / lv.n)


def test_saddle_operator_symmetric():
    mm, lv = _lv(hi.skewed_pair, 3)
    mu = 1.0 + lv.coords[:, 0] ** 2
    _, K = ST.stokes_operator(mm, lv, mu)
    assert abs(K - K.T).max() < 1e-15
