"""Pins of the 2D stencil-scaling oracle (Sec. 2.1, Sec. 2.3; no GPU)."""

import numpy as np

from oracle import twod as T

TRIS = [[[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]], [[0.2, 0.1], [1.3, 0.4], [0.5, 1.7]],
        [[-0.4, 0.3], [0.9, -0.6], [0.7, 1.1]]]
NU = 0.3
CE, CD = 1.0 / (1.0 + NU), NU / ((1.0 + NU) * (1.0 - 2.0 * NU))


def _k(c):
    return 1.0 + 0.5 * np.sin(3 * c[:, 0]) * np.cos(2 * c[:, 1])


def test_antisymmetric_part_is_geometry_independent():
    """Sec. 2.3: the antisymmetric part of every element block between two vertices is
    [[0, -g], [g, 0]] with |g| independent of the triangle's shape.  With a^a = (a - a^T)/2
    the eps form gives |g| = 1/8 (the paper prints 1/4: the factor discussed for 3D), and
    the div form gives -2 times the eps form's value (the paper: the same with a flipped sign)."""
    for tri in TRIS:
        lat = T.Lattice2D(tri, 2)
        X = lat.coords[lat.elems]
        Ke = T.element_stiffness(X, 1.0, 0.0)
        Kd = T.element_stiffness(X, 0.0, 1.0)
        for e in range(len(lat.elems)):
            for a in range(3):
                for b in range(3):
                    if a == b:
                        continue
                    ae = 0.5 * (Ke[e, a, b] - Ke[e, a, b].T)
                    ad = 0.5 * (Kd[e, a, b] - Kd[e, a, b].T)
                    assert abs(ae[0, 0]) < 1e-14 and abs(ae[0, 1] + ae[1, 0]) < 1e-14
                    assert abs(abs(ae[1, 0]) - 0.125) < 1e-13
                    assert abs(ad[1, 0] + 2.0 * ae[1, 0]) < 1e-13


def test_correction_closed_form():
    """eq. correction2d: the physical-scaling block minus the unphysical one is the correction
    (kbar^t - kbar^{t^m}) a^{a;t} = +-(1/3)(k_p - k_{p^m}) / 8 [[0, -1], [1, 0]] for the eps form:
    1/24 of the coefficient difference across the edge (the paper: 1/12)."""
    lat = T.Lattice2D(TRIS[1], 3)
    K = T.element_stiffness(lat.coords[lat.elems], 1.0, 0.0)
    k = _k(lat.coords)
    R = T.operator(lat, K, k, "physical") - T.operator(lat, K, k, "unphysical")
    n = lat.n
    checked = 0
    for i in np.nonzero(~lat.boundary)[0]:
        a, b = lat.ij[i]
        # the edge to (a + 1, b): its elements' third vertices are (a, b + 1) and (a + 1, b - 1)
        j = T.index(n, a + 1, b)
        p, pm = T.index(n, a, b + 1), T.index(n, a + 1, b - 1)
        blk = R[2 * i:2 * i + 2, 2 * j:2 * j + 2]
        assert abs(blk[0, 0]) < 1e-14 and abs(blk[0, 1] + blk[1, 0]) < 1e-14
        assert abs(abs(blk[1, 0]) - abs(k[p] - k[pm]) / 24.0) < 1e-13
        checked += 1
    assert checked > 10


def test_constant_coefficient_forms_equal_galerkin():
    for tri in TRIS:
        lat = T.Lattice2D(tri, 3)
        K = T.element_stiffness(lat.coords[lat.elems], CE, CD)
        G = T.galerkin(lat, K)
        for v in ("physical", "unphysical", "nodal"):
            A = T.operator(lat, K, 2.5 * np.ones(lat.N), v)
            inn = np.repeat(~lat.boundary, 2)
            assert np.abs((A - 2.5 * G)[inn]).max() < 1e-12 * np.abs(G).max()


def test_lemma_affine_coefficient_2d():
    """Lemma 2.1 in 2D: for affine k the physical scaling equals nodal integration on the
    interior rows; the unphysical scaling does not."""
    for tri in TRIS:
        lat = T.Lattice2D(tri, 3)
        K = T.element_stiffness(lat.coords[lat.elems], CE, CD)
        c = lat.coords
        k = 1.0 + 0.3 * c[:, 0] - 0.2 * c[:, 1]
        inn = np.repeat(~lat.boundary, 2)
        P, N, U = (T.operator(lat, K, k, v) for v in ("physical", "nodal", "unphysical"))
        assert np.abs((P - N)[inn]).max() < 1e-12 * np.abs(N).max()
        assert np.abs((U - N)[inn]).max() > 1e-5 * np.abs(N).max()


def test_symmetry_and_rigid_modes_2d():
    lat = T.Lattice2D(TRIS[1], 3)
    K = T.element_stiffness(lat.coords[lat.elems], CE, CD)
    c = lat.coords
    A = T.operator(lat, K, _k(c), "physical")
    inn = np.repeat(~lat.boundary, 2)
    Ai = A[np.ix_(inn, inn)]
    assert np.abs(Ai - Ai.T).max() < 1e-13 * np.abs(Ai).max()
    for r in (np.tile([1.0, 0.0], (lat.N, 1)), np.tile([0.0, 1.0], (lat.N, 1)), np.stack([-c[:, 1], c[:, 0]], 1)):
        assert np.abs(T.apply(A, r)[~lat.boundary]).max() < 1e-12 * np.abs(A).max()


def test_element_matrices_integrate_the_energy_of_affine_fields():
    """For u = G x + b the strain is constant, so sum_e u_e^T K_e u_e equals the area of the macro
    triangle times c_eps eps:eps + c_div (tr eps)^2 in closed form (no quadrature involved)."""
    rng = np.random.default_rng(4)
    for tri in TRIS:
        lat = T.Lattice2D(tri, 2)
        K = T.element_stiffness(lat.coords[lat.elems], CE, CD)
        G = rng.normal(size=(2, 2))
        u = lat.coords @ G.T + rng.normal(size=2)
        ue = u[lat.elems]  # (E, 3, 2)
        energy = np.einsum("eam,eabml,ebl->", ue, K, ue)
        eps = 0.5 * (G + G.T)
        t = np.asarray(tri, dtype=np.float64)
        area = 0.5 * abs(np.linalg.det(np.stack([t[1] - t[0], t[2] - t[0]], 1)))
        want = area * (CE * (eps**2).sum() + CD * np.trace(eps) ** 2)
        assert abs(energy - want) < 1e-12 * abs(want)
