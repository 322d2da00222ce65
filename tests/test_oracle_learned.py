"""Pins of the conv-net oracle used to check the learned preconditioner's kernels (no GPU)."""

import numpy as np

from oracle import learned as LN


def test_delta_kernel_is_a_shift():
    rng = np.random.default_rng(0)
    a = rng.normal(size=(1, 4, 5, 6, 2))
    W = np.zeros((27, 2, 2))
    t = LN.offsets().index((1, 0, -1))
    W[t] = np.eye(2)
    out = LN.conv(a, W)
    want = np.zeros_like(a)
    want[:, :-1, :, 1:, :] = a[:, 1:, :, :-1, :]
    assert np.array_equal(out, want)


def test_transpose_is_adjoint():
    rng = np.random.default_rng(1)
    a = rng.normal(size=(2, 5, 4, 6, 3))
    g = rng.normal(size=(2, 5, 4, 6, 2))
    W = rng.normal(size=(27, 3, 2))
    lhs = (LN.conv(a, W) * g).sum()
    rhs = (a * LN.conv_transpose_input(g, W)).sum()
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    dW = LN.conv_weight_grad(a, g)
    eps = rng.normal(size=W.shape)
    assert abs((dW * eps).sum() - (LN.conv(a, eps) * g).sum()) < 1e-10 * abs((dW * eps).sum())


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 4, 4, 5, LN.CIN))
    tgt = rng.normal(size=(2, 4, 4, 5, 3))
    Ws, bs = LN.init_params(3)
    Ws = [W + 0.05 * rng.normal(size=W.shape) for W in Ws]
    bs = [0.1 * rng.normal(size=b.shape) for b in bs]
    loss, dWs, dbs = LN.loss_and_grads(x, tgt, Ws, bs, round_bf16=False)
    h = 1e-6
    for l in range(LN.NLAYERS):
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in Ws[l].shape)
            if l == 0 and idx[1] >= LN.CIN:
                continue
            Wp = [W.copy() for W in Ws]
            Wp[l][idx] += h
            Wm = [W.copy() for W in Ws]
            Wm[l][idx] -= h
            fd = (LN.loss_and_grads(x, tgt, Wp, bs, False)[0] - LN.loss_and_grads(x, tgt, Wm, bs, False)[0]) / (2 * h)
            assert abs(fd - dWs[l][idx]) <= 1e-6 * max(1.0, abs(fd)), (l, idx, fd, dWs[l][idx])
        o = int(rng.integers(0, 3 if l == LN.NLAYERS - 1 else LN.C))
        bp = [b.copy() for b in bs]
        bp[l][o] += h
        bm = [b.copy() for b in bs]
        bm[l][o] -= h
        fd = (LN.loss_and_grads(x, tgt, Ws, bp, False)[0] - LN.loss_and_grads(x, tgt, Ws, bm, False)[0]) / (2 * h)
        assert abs(fd - dbs[l][o]) <= 1e-6 * max(1.0, abs(fd))


def test_bf16_rounding():
    v = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 65504.0])
    r = LN.bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125
    assert abs(r[3] + 3.140625) < 1e-12


def _cube_problem(level):
    import hhg_inputs as hi
    from oracle import fem, mesh, operators as op, solvers as S

    xyz, tets = hi.kuhn_cube()
    mm = mesh.MacroMesh.build(xyz, tets)
    ce, cd = fem.elasticity_coefficients(0.3)
    kf = lambda c: hi.young_sine(c)

    def A_of(lv):
        K = fem.element_stiffness(lv.coords[lv.elems], ce, cd)
        return op.with_dirichlet_rows(op.scaled_operator(lv, K, kf(lv.coords)), lv.dirichlet)

    H = S.Hierarchy(mm, list(range(2, level + 1)), A_of)
    lam = {l: S.lambda_max_DinvA(H.A[l], H.lv[l].dirichlet) for l in range(3, level + 1)}
    lv = H.lv[level]
    vox, dims = LN.grid_index(lv.coords, 1.0 / 2**level)
    vc = lambda r: H.vcycle(level, r, np.zeros_like(r), "chebyshev", 2, 2, lam)
    return H, lv, vox, dims, kf(lv.coords), vc


def test_grid_index_is_a_bijection_onto_the_cube_lattice():
    H, lv, vox, dims, k, vc = _cube_problem(3)
    assert dims == (9, 9, 9)
    flat = (vox[:, 0] * 9 + vox[:, 1]) * 9 + vox[:, 2]
    assert np.array_equal(np.sort(flat), np.arange(729))


def test_combination_never_loses_to_the_vcycle():
    """(a, b) minimise the energy norm of the error over span{z0, c}: any other point of
    that plane -- the V-cycle step alone (b = 0) included -- leaves a larger error."""
    import hhg_inputs as hi

    H, lv, vox, dims, k, vc = _cube_problem(3)
    A = H.A[3]
    fr = ~lv.dirichlet
    e = hi.node_noise(lv.coords, seed=5)
    e[~fr] = 0.0
    r = (A @ e.reshape(-1)).reshape(-1, 3)
    r[~fr] = 0.0
    v = vc(r)
    Ws, bs = LN.init_params(7)
    z, w, c = LN.correction(A, lv.dirichlet, vox, dims, k, r, v, Ws, bs)
    assert np.abs(c).max() > 0 and w != 0

    def energy(zz):
        d = (e - zz).reshape(-1)
        return float(d @ (A @ d))

    best = energy(z)
    z0, _ = LN._scaled_step(A, lv.dirichlet, r, v)
    rng = np.random.default_rng(0)
    for _ in range(6):
        da, db = rng.normal(size=2) * 0.05
        assert energy(z + da * z0 + db * c * np.abs(z0).max() / np.abs(c).max()) > best
    assert best <= energy(z0) <= energy(v) * (1 + 1e-12)


def test_features_are_scale_invariant_and_pairs_consistent():
    import hhg_inputs as hi

    H, lv, vox, dims, k, vc = _cube_problem(3)
    A = H.A[3]
    fr = ~lv.dirichlet
    e = hi.node_noise(lv.coords, seed=6)
    e[~fr] = 0.0
    X, T, e1 = LN.training_pair(A, lv.dirichlet, vox, dims, k, e, vc)
    X2, T2, _ = LN.training_pair(A, lv.dirichlet, vox, dims, k, 3.0 * e, vc)
    assert np.allclose(X, X2, rtol=1e-12, atol=1e-14) and np.allclose(T, T2, rtol=1e-12, atol=1e-14)
    # the target is D e1 / s and the residual channels are A e1 / s with the same s
    Dg = A.diagonal().reshape(-1, 3)
    t = T[0, vox[:, 0], vox[:, 1], vox[:, 2]]
    r1 = X[0, vox[:, 0], vox[:, 1], vox[:, 2], :3]
    s = (Dg[fr] * e1[fr])[0, 0] / t[fr][0, 0]
    Ae1 = (A @ e1.reshape(-1)).reshape(-1, 3)
    assert np.allclose(r1[fr] * s, Ae1[fr], rtol=1e-10, atol=1e-12 * np.abs(Ae1).max())
    # s is the RMS of D z0 over the free DoFs: the z0 channels have unit mean square
    z0c = X[0, vox[fr, 0], vox[fr, 1], vox[fr, 2], 3:6]
    assert abs((z0c**2).mean() - 1.0) < 1e-12


def test_coarse_mode_without_coarsening_is_the_fine_mode():
    import hhg_inputs as hi

    H, lv, vox, dims, k, vc = _cube_problem(3)
    A = H.A[3]
    r = hi.node_noise(lv.coords, seed=8)
    r[lv.dirichlet] = 0.0
    v = vc(r)
    Ws, bs = LN.init_params(3)
    z, w, c = LN.correction(A, lv.dirichlet, vox, dims, k, r, v, Ws, bs)
    zc, wc, cc = LN.coarse_correction(H, 3, 0, vox, dims, k, r, v, Ws, bs)
    assert np.array_equal(z, zc) and w == wc and np.array_equal(c, cc)


def test_coarse_mode_inputs_and_combination():
    """Injection picks the coincident fine node; the coarse correction, prolongated, still
    never loses to the V-cycle step in the energy norm."""
    import hhg_inputs as hi

    H, lv, vox, dims, k, vc = _cube_problem(3)
    idx = LN._inject_index(H, 3)
    assert np.array_equal(H.lv[3].coords[idx], H.lv[2].coords)
    A = H.A[3]
    e = hi.node_noise(lv.coords, seed=9)
    e[lv.dirichlet] = 0.0
    r = (A @ e.reshape(-1)).reshape(-1, 3)
    r[lv.dirichlet] = 0.0
    v = vc(r)
    vox_c, dims_c = LN.grid_index(H.lv[2].coords, 1.0 / 4)
    k_c = hi.young_sine(H.lv[2].coords)
    Ws, bs = LN.init_params(4)
    z, w, c = LN.coarse_correction(H, 3, 1, vox_c, dims_c, k_c, r, v, Ws, bs)
    assert np.abs(c).max() > 0 and not c[lv.dirichlet].any()

    def energy(zz):
        d = (e - zz).reshape(-1)
        return float(d @ (A @ d))

    z0, _ = LN._scaled_step(A, lv.dirichlet, r, v)
    assert energy(z) <= energy(z0) * (1 + 1e-12)
    # the pair's target is D_c e1 / s at the injected nodes
    X, T, e1 = LN.coarse_training_pair(H, 3, 1, vox_c, dims_c, k_c, e, vc)
    Dc = LN._point_diag(H, 2)
    t = T[0, vox_c[:, 0], vox_c[:, 1], vox_c[:, 2]]
    fr = ~H.lv[2].dirichlet
    ratio = (Dc * e1[idx])[fr] / t[fr]
    assert np.allclose(ratio, ratio.flat[0], rtol=1e-10)
