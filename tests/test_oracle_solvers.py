"""Pins of the oracle's smoothers, transfers and solvers (no GPU)."""

import numpy as np
import scipy.sparse as sp

import hhg_inputs as hi
from oracle import fem, mesh, operators as op, solvers as S


def _hier(builder, levels, kfun):
    xyz, tets = builder()
    mm = mesh.MacroMesh.build(xyz, tets)
    ce, cd = fem.elasticity_coefficients(0.3)

    def A_of(lv):
        K = fem.element_stiffness(lv.coords[lv.elems], ce, cd)
        return op.with_dirichlet_rows(op.scaled_operator(lv, K, kfun(lv.coords)), lv.dirichlet)

    return S.Hierarchy(mm, levels, A_of)


def test_prolongation_reproduces_affine_fields():
    """Linear interpolation is exact for functions that are affine on every macro."""
    for builder in (hi.kuhn_cube, hi.skewed_pair, hi.unit_tet):
        H = _hier(builder, [2, 3], lambda c: np.ones(len(c)))
        B = np.array([[0.3, -1.2, 0.7], [2.0, 0.1, -0.4], [0.5, 0.5, 1.5]])
        u = lambda c: c @ B.T + np.array([1.0, -2.0, 0.25])
        uc, uf = u(H.lv[2].coords), u(H.lv[3].coords)
        assert np.abs(S.prolongate_add(H.P[3], uc, np.zeros_like(uf)) - uf).max() < 1e-13


def test_restriction_is_transpose_of_prolongation():
    H = _hier(hi.kuhn_cube, [2, 3], lambda c: np.ones(len(c)))
    rng = np.random.default_rng(0)
    lc, lf = H.lv[2], H.lv[3]
    rf = rng.normal(size=(lf.num_nodes, 3))
    rf[lf.dirichlet] = 0.0
    ec = rng.normal(size=(lc.num_nodes, 3))
    ec[lc.dirichlet] = 0.0
    lhs = (S.restrict(H.P[3], rf, lf.dirichlet, lc.dirichlet) * ec).sum()
    rhs = (rf * S.prolongate_add(H.P[3], ec, np.zeros_like(rf))).sum()
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def test_chebyshev_matches_polynomial_closed_form():
    """On a diagonal system (D^-1 A = diag(lambda)) k Chebyshev steps multiply each error
    component by T_k((theta - lambda)/delta) / T_k(theta/delta)."""
    lam = np.linspace(0.05, 1.9, 30)
    A = sp.diags(np.repeat(lam, 3))  # D = A, so D^-1 A = I ... use a scaled diagonal instead
    d = np.repeat(np.linspace(1.0, 3.0, 30), 3)
    A = sp.diags(d * np.repeat(lam, 3)).tocsr()
    # point diagonal of A is d*lam, so D^-1 A = I; build a non-trivial D^-1 A via a 2x2-free
    # construction: scale the operator but keep the diagonal fixed is impossible for a
    # diagonal matrix, so test the recurrence on D^-1 A = I with a wide interval instead.
    dirichlet = np.zeros(30, dtype=bool)
    f = np.zeros((30, 3))
    x0 = np.random.default_rng(1).normal(size=(30, 3))
    k, lo, hi, lmax = 4, 0.2, 1.6, 1.0
    x = S.chebyshev(A, dirichlet, f, x0, lmax, lo, hi, k)
    a, b = lo * lmax, hi * lmax
    theta, delta = (a + b) / 2, (b - a) / 2
    Tk = lambda t: np.cosh(k * np.arccosh(t)) if abs(t) >= 1 else np.cos(k * np.arccos(t))
    factor = Tk((theta - 1.0) / delta) / Tk(theta / delta)
    assert np.allclose(x, factor * x0, rtol=1e-12, atol=1e-14)


def test_chebyshev_error_polynomial_on_full_spectrum():
    """Same closed form per eigencomponent for a symmetric D^-1 A with a spread spectrum:
    A = D^{1/2} Q diag(mu) Q^T D^{1/2} with unit diagonal blocks folded into D."""
    rng = np.random.default_rng(3)
    n = 24
    mu = np.linspace(0.1, 2.0, n)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    B = Q @ np.diag(mu) @ Q.T
    s = np.sqrt(np.diag(B))
    C = B / np.outer(s, s)  # unit diagonal, same eigenvectors up to scaling
    mu_c, V = np.linalg.eigh(C)
    A = sp.csr_matrix(np.kron(C, np.eye(3)))
    dirichlet = np.zeros(n, dtype=bool)
    f = np.zeros((n, 3))
    x0 = rng.normal(size=(n, 3))
    k, lo, hi, lmax = 3, 1 / 30, 1.1, mu_c.max()
    x = S.chebyshev(A, dirichlet, f, x0, lmax, lo, hi, k)
    a, b = lo * lmax, hi * lmax
    theta, delta = (a + b) / 2, (b - a) / 2
    Tk = lambda t: np.where(np.abs(t) >= 1, np.cosh(k * np.arccosh(np.maximum(np.abs(t), 1.0))) * np.sign(t) ** k,
                            np.cos(k * np.arccos(np.clip(t, -1, 1))))
    g = Tk((theta - mu_c) / delta) / Tk(np.array(theta / delta))
    want = V @ (g[:, None] * (V.T @ x0))
    assert np.allclose(x, want, atol=1e-12)


def test_pcg_matches_direct_solve():
    H = _hier(hi.kuhn_cube, [3], lambda c: 1.0 + c[:, 0] * c[:, 1])
    lv, A = H.lv[3], H.A[3]
    f = hi.node_noise(lv.coords, seed=1)
    x0 = np.zeros_like(f)
    D = S.point_diagonal(A, lv.dirichlet)
    x, it = S.pcg(A, lv.dirichlet, f, x0, lambda r: r / D, 1e-12, 500)
    xd = S.direct_solve(A, lv.dirichlet, f, x0)
    assert np.abs(x - xd).max() < 1e-9 * np.abs(xd).max()


def test_vcycle_contracts():
    """V(2,2) Chebyshev cycles (interval [lambda/8, 1.1 lambda]) reduce the residual by a
    level-independent factor (< 0.35 over the first three cycles)."""
    H = _hier(hi.kuhn_cube, [2, 3, 4], lambda c: 1.0 + 0.5 * np.sin(3 * c[:, 0]) * np.cos(2 * c[:, 1]))
    lam = {l: S.lambda_max_DinvA(H.A[l], H.lv[l].dirichlet) for l in (3, 4)}
    for l in (3, 4):
        lv, A = H.lv[l], H.A[l]
        f = hi.node_noise(lv.coords, seed=2)
        f[lv.dirichlet] = 0.0
        x = np.zeros_like(f)
        r0 = np.linalg.norm(S.residual(A, lv.dirichlet, f, x))
        for _ in range(3):
            x = H.vcycle(l, f, x, "chebyshev", 2, 2, lam)
        r3 = np.linalg.norm(S.residual(A, lv.dirichlet, f, x))
        assert (r3 / r0) ** (1 / 3) < 0.35


def test_colouring_separates_neighbours():
    """No two macro-interior nodes of one colour share an element (so a colour pass of the
    hybrid Gauss-Seidel smoother is independent of its order), and all eight colours occur."""
    for builder, level in ((hi.kuhn_cube, 3), (hi.skewed_pair, 3)):
        xyz, tets = builder()
        lv = mesh.build_level(mesh.MacroMesh.build(xyz, tets), level)
        col = S.interior_colours(lv)
        assert set(col[~lv.skeleton].tolist()) == set(range(8)) and np.all(col[lv.skeleton] == -1)
        E = lv.elems
        for a in range(4):
            for b in range(a + 1, 4):
                ca, cb = col[E[:, a]], col[E[:, b]]
                assert not np.any((ca >= 0) & (ca == cb))


def test_hybrid_gauss_seidel_is_gauss_seidel_inside_a_macro():
    """On the single unit macro tetrahedron every free node is macro-interior, so one hybrid
    step is the Gauss-Seidel step x + M^-1 (f - A x) with M = D + L: D the point diagonal, L the
    couplings to the nodes of earlier colours (the nodes taken colour by colour; the three
    components of a node are updated together, so their coupling stays on the right-hand side).
    Here M is assembled from A and the triangular system solved directly; and the step lowers
    the energy norm of the error."""
    H = _hier(hi.unit_tet, [3], lambda c: 1.0 + 0.5 * np.sin(3 * c[:, 0]) * np.cos(2 * c[:, 1]))
    lv, A = H.lv[3], H.A[3]
    d = lv.dirichlet
    col = S.interior_colours(lv)
    assert not np.any(lv.skeleton & ~d)
    f = hi.node_noise(lv.coords, seed=3)
    f[d] = 0.0
    x0 = hi.node_noise(lv.coords, seed=4)
    x0[d] = 0.0
    x1 = S.hybrid_gauss_seidel(A, d, lv.skeleton, col, f, x0, 0.7, 1)
    free = np.nonzero(~d)[0]
    order = free[np.argsort(col[free], kind="stable")]
    dofs = (3 * order[:, None] + np.arange(3)[None, :]).reshape(-1)
    Aff = A.tocsr()[dofs][:, dofs].tocoo()
    cdof = np.repeat(col[order], 3)
    lower = cdof[Aff.row] > cdof[Aff.col]
    diag = Aff.row == Aff.col
    sel = lower | diag
    M = sp.coo_matrix((Aff.data[sel], (Aff.row[sel], Aff.col[sel])), shape=Aff.shape).tocsr()
    r = (f.reshape(-1) - A @ x0.reshape(-1))[dofs]
    want = x0.reshape(-1).copy()
    want[dofs] += sp.linalg.spsolve_triangular(M, r, lower=True)
    assert np.abs(x1.reshape(-1) - want).max() < 1e-12 * np.abs(want).max()
    xs = S.direct_solve(A, d, f, np.zeros_like(f))
    en = lambda x: float((x - xs).reshape(-1) @ (A @ (x - xs).reshape(-1)))
    assert en(x1) < en(x0)


def test_hybrid_gs_vcycles_contract():
    """Stationary V(3,3) cycles with the hybrid Gauss-Seidel smoother (the paper's solver,
    Sec. 5) on the 6-macro cube reduce the residual by a level-independent factor."""
    H = _hier(hi.kuhn_cube, [2, 3, 4], lambda c: 1.0 + 0.5 * np.sin(3 * c[:, 0]) * np.cos(2 * c[:, 1]))
    for l in (3, 4):
        lv, A = H.lv[l], H.A[l]
        f = hi.node_noise(lv.coords, seed=2)
        f[lv.dirichlet] = 0.0
        x = np.zeros_like(f)
        r0 = np.linalg.norm(S.residual(A, lv.dirichlet, f, x))
        for _ in range(3):
            x = H.vcycle(l, f, x, "hybrid_gs", 3, 3, omega=2 / 3)
        r3 = np.linalg.norm(S.residual(A, lv.dirichlet, f, x))
        assert (r3 / r0) ** (1 / 3) < 0.3


def test_hybrid_gauss_seidel_skeleton_step_is_jacobi():
    """Across the macro interfaces the step is Jacobi-like (Sec. 5): on the 6-macro cube the
    free skeleton nodes move by exactly omega D^-1 (f - A x) of the old iterate, and the
    macro-interior nodes by a Gauss-Seidel step that differs from the Jacobi one."""
    H = _hier(hi.kuhn_cube, [3], lambda c: 1.0 + c[:, 0] * c[:, 2])
    lv, A = H.lv[3], H.A[3]
    d = lv.dirichlet
    f = hi.node_noise(lv.coords, seed=5)
    f[d] = 0.0
    x0 = hi.node_noise(lv.coords, seed=6)
    x0[d] = 0.0
    x1 = S.hybrid_gauss_seidel(A, d, lv.skeleton, S.interior_colours(lv), f, x0, 0.6, 1)
    jac = x0 + 0.6 * S.residual(A, d, f, x0) / S.point_diagonal(A, d)
    skel = lv.skeleton & ~d
    inner = ~lv.skeleton
    assert skel.any() and np.abs(x1[skel] - jac[skel]).max() < 1e-14 * np.abs(jac).max()
    assert np.abs(x1[inner] - (x0 + S.residual(A, d, f, x0) / S.point_diagonal(A, d))[inner]).max() > 1e-3
    assert np.array_equal(x1[d], x0[d])
