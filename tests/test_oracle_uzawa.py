"""Pins of the inexact Uzawa multigrid oracle (Sec. 5.2) and of the Stokes variant of the
learned-preconditioner oracle (no GPU).

The Uzawa cycle is pinned to an independent formulation: the saddle system bordered by
the mass-weighted zero-mean pressure constraint, solved by a sparse direct method.  The
learned Stokes combination is pinned to a least-squares solve of the same 2x2 problem."""

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import hhg_inputs as hi
from oracle import learned as LN, mesh, solvers as S, stokes as ST


def _mu(c):
    return hi.viscosity_sphere(c, mu_in=1.0, mu_out=10.0, radius=0.3, width=0.1)


@pytest.fixture(scope="module")
def hier3():
    xyz, tets = hi.kuhn_cube()
    H = ST.UzawaHierarchy(mesh.MacroMesh.build(xyz, tets), [2, 3], _mu)
    lam = {3: S.lambda_max_DinvA(H.A[3], H.lv[3].dirichlet)}
    return H, lam


def _rhs(H, l, seed):
    lv = H.lv[l]
    f = np.zeros((lv.num_nodes, 4))
    f[:, :3] = hi.node_noise(lv.coords, seed)
    f[:, 3] = hi.node_noise(lv.coords, seed + 1, comps=1).reshape(-1)
    f[lv.dirichlet, :3] = 0.0
    return f


def _bordered_solve(H, l, f):
    """Zero-mean-pressure solution of K x = f (f_p summing to zero), by a sparse direct
    solve of [[K_ff, b], [b^T, 0]] with b the lumped mass on the pressure rows."""
    lv = H.lv[l]
    N = lv.num_nodes
    keep = np.concatenate([np.repeat(~lv.dirichlet, 3), np.ones(N, dtype=bool)])
    Kf = H.K[l][keep][:, keep]
    b = np.zeros(Kf.shape[0])
    b[-N:] = H.m[l]
    M = sp.bmat([[Kf, sp.csr_matrix(b[:, None])], [sp.csr_matrix(b[None, :]), None]]).tocsc()
    sol = spla.spsolve(M, np.concatenate([ST.pack4(f)[keep], [0.0]]))
    x = np.zeros(4 * N)
    x[keep] = sol[:-1]
    return ST.unpack4(x, N)


def test_coarsest_level_solve_is_exact(hier3):
    H, _ = hier3
    f = _rhs(H, 2, 3)
    f[:, 3] -= f[:, 3].mean()  # orthogonal to the constant-pressure kernel
    x = H.coarse_solve(f)
    r = H.residual(2, f, x)
    assert np.abs(r).max() <= 1e-10 * np.abs(f).max()
    want = _bordered_solve(H, 2, f)
    assert np.abs(H.project_pressure(2, x) - want).max() <= 1e-9 * np.abs(want).max()


def test_uzawa_vcycles_converge_to_the_saddle_solution(hier3):
    H, lam = hier3
    f = _rhs(H, 3, 7)
    f[:, 3] -= f[:, 3].mean()
    want = _bordered_solve(H, 3, f)
    x = np.zeros_like(f)
    norms = [np.linalg.norm(H.residual(3, f, x))]
    for _ in range(30):
        x = H.vcycle(3, f, x, lam, 3)
        norms.append(np.linalg.norm(H.residual(3, f, x)))
    rates = np.array(norms[1:]) / np.array(norms[:-1])
    assert rates.max() < 0.9 and rates[5:].max() < 0.6, rates
    assert np.abs(H.project_pressure(3, x) - want).max() <= 1e-6 * np.abs(want).max()


def test_uzawa_step_without_pressure_relaxation_only_smooths_the_velocity(hier3):
    H, lam = hier3
    f = _rhs(H, 3, 11)
    x0 = np.zeros_like(f)
    x0[:, 3] = hi.node_noise(H.lv[3].coords, 12, comps=1).reshape(-1)
    x1 = H.uzawa_step(3, f, x0, lam, vsteps=2, omega=0.0)
    assert np.array_equal(x1[:, 3], x0[:, 3])
    # the velocity correction is the Chebyshev smoother of A du = r_u from du = 0
    r = H.residual(3, f, x0)
    du = S.chebyshev(H.A[3], H.lv[3].dirichlet, r[:, :3], np.zeros_like(r[:, :3]), lam[3], 1 / 8, 1.1, 2)
    assert np.allclose(x1[:, :3], du, rtol=0, atol=1e-14 * np.abs(du).max())


def test_uzawa_with_hybrid_gauss_seidel_converges_to_the_saddle_solution(hier3):
    """The paper's solver settings (Sec. 5.2.1): hybrid Gauss-Seidel velocity smoothing, one
    step per Uzawa step, pressure relaxation 0.3, V(3,3) cycles; the iterates reach the
    bordered direct solution."""
    H, lam = hier3
    f = _rhs(H, 3, 13)
    f[:, 3] -= f[:, 3].mean()
    want = _bordered_solve(H, 3, f)
    x = np.zeros_like(f)
    norms = [np.linalg.norm(H.residual(3, f, x))]
    for _ in range(40):
        x = H.vcycle(3, f, x, lam, 3, vsteps=1, omega=0.3, smoother="hybrid_gs")
        norms.append(np.linalg.norm(H.residual(3, f, x)))
    rates = np.array(norms[1:]) / np.array(norms[:-1])
    assert rates[1:].max() < 0.7, rates  # the first cycle may raise the mixed velocity-pressure norm
    assert np.abs(H.project_pressure(3, x) - want).max() <= 1e-6 * np.abs(want).max()


def test_hybrid_gauss_seidel_uzawa_step_smooths_then_relaxes_the_pressure(hier3):
    """With the pressure fixed the velocity correction is the hybrid Gauss-Seidel step on
    A du = r_u from du = 0; the pressure then moves by -omega (g - B u - C p) / s."""
    H, lam = hier3
    lv = H.lv[3]
    f = _rhs(H, 3, 17)
    x0 = np.zeros_like(f)
    x0[:, 3] = hi.node_noise(lv.coords, 18, comps=1).reshape(-1)
    x1 = H.uzawa_step(3, f, x0, lam, vsteps=1, omega=0.3, smoother="hybrid_gs")
    r = H.residual(3, f, x0)
    du = S.hybrid_gauss_seidel(H.A[3], lv.dirichlet, lv.skeleton, S.interior_colours(lv), r[:, :3],
                               np.zeros_like(r[:, :3]), 2 / 3, 1)
    assert np.allclose(x1[:, :3], du, rtol=0, atol=1e-14 * np.abs(du).max())
    xu = x0.copy()
    xu[:, :3] = du
    rp = H.residual(3, f, xu)[:, 3]
    assert np.allclose(x1[:, 3], x0[:, 3] - 0.3 * rp / H.s[3], rtol=0, atol=1e-13 * np.abs(x0[:, 3]).max())


def _grid(H, l):
    return LN.grid_index(H.lv[l].coords, 1.0 / 2**l)


def _random_net(seed):
    rng = np.random.default_rng(seed)
    Ws, bs = LN.init_params(seed, LN.STOKES_CIN, LN.STOKES_COUT)
    Ws = [LN.bf16(W + 0.05 * rng.normal(size=W.shape) * (W != 0)) for W in Ws]
    bs = [0.05 * rng.normal(size=b.shape) for b in bs]
    bs[-1][LN.STOKES_COUT:] = 0.0
    return Ws, bs


def test_stokes_combination_is_the_residual_least_squares_step(hier3):
    H, lam = hier3
    l = 3
    d = H.lv[l].dirichlet
    vox, dims = _grid(H, l)
    r = _rhs(H, l, 21)
    v = H.vcycle(l, r, np.zeros_like(r), lam, l)
    Ws, bs = _random_net(5)
    k = _mu(H.lv[l].coords)
    z, w, c = LN.stokes_correction(H, l, vox, dims, k, r, v, Ws, bs)
    z0, Kz0 = LN._stokes_step(H, l, r, v)
    on = np.ones(r.shape, dtype=bool)
    on[d, :3] = False
    Kc = H.apply(l, c)
    Amat = np.stack([Kz0[on], Kc[on]], axis=1)
    (a, b), *_ = np.linalg.lstsq(Amat, r[on], rcond=None)
    assert np.allclose(z, a * z0 + b * c, rtol=0, atol=1e-10 * np.abs(z).max())
    assert abs(w - b / a) <= 1e-9 * max(1.0, abs(w))
    rz = np.linalg.norm(H.residual(l, r, z)[on])
    rz0 = np.linalg.norm(H.residual(l, r, z0)[on])
    assert rz <= rz0 * (1 + 1e-12)


def test_stokes_pair_is_consistent(hier3):
    H, lam = hier3
    l = 3
    lv = H.lv[l]
    d = lv.dirichlet
    vox, dims = _grid(H, l)
    e = _rhs(H, l, 31)
    k = _mu(lv.coords)
    X, T, e1 = LN.stokes_training_pair(H, l, vox, dims, k, e, lambda r: H.vcycle(l, r, np.zeros_like(r), lam, l))
    assert abs((H.m[l] * e1[:, 3]).sum()) <= 1e-12 * np.abs(e1[:, 3]).sum()
    on = np.ones(e.shape, dtype=bool)
    on[d, :3] = False
    Xv = X[0, vox[:, 0], vox[:, 1], vox[:, 2]]
    Tv = T[0, vox[:, 0], vox[:, 1], vox[:, 2]]
    D = LN.stokes_diag(H, l)
    r1 = H.residual(l, np.zeros_like(e1), -e1)
    # the D z0 / s channels have unit RMS over the free velocity DoFs and over the pressures
    # (definition of s and s_p); r1 / s and the targets D e1 / s share those scales
    for comps in ([0, 1, 2], [3]):
        m = on[:, comps]
        assert abs(np.sqrt((Xv[:, [4 + c for c in comps]][m] ** 2).mean()) - 1.0) < 1e-12
        scale = np.linalg.norm(Xv[:, comps][m]) / np.linalg.norm(r1[:, comps][m])
        assert np.allclose(Tv[:, comps][m] / scale, (D * e1)[:, comps][m], rtol=1e-10,
                           atol=1e-12 * np.abs(D * e1)[:, comps].max())
        assert np.allclose(Xv[:, comps][m] / scale, r1[:, comps][m], rtol=1e-10,
                           atol=1e-12 * np.abs(Xv[:, comps]).max() / scale)
    assert np.allclose(Xv[:, 8], np.log(k) - np.log(k).mean())
