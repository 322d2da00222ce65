"""Smoothers, transfers, V-cycle and solvers of the CUDA library against the FP64 oracle.

Tolerances: FP64 kernels 1e-11 relative to the largest entry (a few sweeps of
rounding); solves are checked by the oracle's own residual of the returned solution
(<= rtol, with 1% slack for the difference between the recursive and true residual)
and, where stated, against a sparse direct solve.
"""

import numpy as np
import pytest

import hhg_inputs as hi
from oracle import fem, mesh, operators as op, solvers as S
from paper_1908_08666_gb300 import binding as B

from hhg_gpu import NU, Ctx, Pair, kfun_smooth as _kfun  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cube4():
    p = Pair(hi.kuhn_cube, 4)
    B.hhg_mg_setup(p.ctx.h)
    yield p
    p.close()


@pytest.fixture(scope="module")
def skew4():
    p = Pair(hi.skewed_pair, 4)
    B.hhg_mg_setup(p.ctx.h)
    yield p
    p.close()


@pytest.mark.parametrize("name", ["cube4", "skew4"])
def test_diagonal_and_transfers(name, request):
    p = request.getfixturevalue(name)
    t = p.ctx.torch
    for l in (3, 4):
        lv = p.H.lv[l]
        d = t.empty(3 * B.hhg_num_nodes(p.ctx.h, l)[0], dtype=t.float64, device="cuda")
        B.hhg_diagonal(p.ctx.h, l, B.F64, d)
        want = S.point_diagonal(p.H.A[l], lv.dirichlet)
        assert np.abs(p.from_lib(l, d) - want).max() <= 1e-13 * np.abs(want).max()
        # prolongation and restriction between l-1 and l
        lc = p.H.lv[l - 1]
        xc = hi.node_noise(lc.coords, seed=11)
        xc[lc.dirichlet] = 0.0
        xf = hi.node_noise(lv.coords, seed=12)
        xcd, xfd = p.to_lib(l - 1, xc, t.float64), p.to_lib(l, xf, t.float64)
        B.hhg_prolongate_add(p.ctx.h, l, B.F64, xcd, xfd)
        want = S.prolongate_add(p.H.P[l], xc, xf)
        assert np.abs(p.from_lib(l, xfd) - want).max() <= 1e-14 * np.abs(want).max()
        rf = hi.node_noise(lv.coords, seed=13)
        rf[lv.dirichlet] = 0.0
        rc = t.empty(3 * B.hhg_num_nodes(p.ctx.h, l - 1)[0], dtype=t.float64, device="cuda")
        B.hhg_restrict(p.ctx.h, l, B.F64, p.to_lib(l, rf, t.float64), rc)
        want = S.restrict(p.H.P[l], rf, lv.dirichlet, lc.dirichlet)
        assert np.abs(p.from_lib(l - 1, rc) - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("name", ["cube4", "skew4"])
def test_hybrid_gauss_seidel_smoother_and_vcycle(name, request):
    """The paper's smoother (Sec. 5): hybrid Gauss-Seidel steps (skeleton Jacobi with weight
    omega, then eight colour passes over the macro interiors) and a V(3,3) cycle with it,
    against oracle.solvers.hybrid_gauss_seidel (FP64 to 1e-11, FP32 to 2e-5)."""
    p = request.getfixturevalue(name)
    t = p.ctx.torch
    h = p.ctx.h
    l = 4
    lv, A = p.H.lv[l], p.H.A[l]
    col = S.interior_colours(lv)
    f = hi.node_noise(lv.coords, seed=31)
    x0 = hi.node_noise(lv.coords, seed=32)
    try:
        B.hhg_set_mg_params(h, smoother=B.SMOOTH_HYBRID_GS, omega=0.6, pre=3, post=3)
        for steps in (1, 2):
            want = S.hybrid_gauss_seidel(A, lv.dirichlet, lv.skeleton, col, f, x0, 0.6, steps)
            x = p.to_lib(l, x0, t.float64)
            B.hhg_smooth(h, l, B.F64, steps, p.to_lib(l, f, t.float64), x)
            assert np.abs(p.from_lib(l, x) - want).max() <= 1e-11 * np.abs(want).max()
            x32 = p.to_lib(l, x0, t.float32)
            B.hhg_smooth(h, l, B.F32, steps, p.to_lib(l, f, t.float32), x32)
            assert np.abs(p.from_lib(l, x32) - want).max() <= 2e-5 * np.abs(want).max()
        f2 = f.copy()
        f2[lv.dirichlet] = 0.0
        x = t.zeros(3 * B.hhg_num_nodes(h, l)[0], dtype=t.float64, device="cuda")
        B.hhg_vcycle(h, l, B.F64, p.to_lib(l, f2, t.float64), x)
        want = p.H.vcycle(l, f2, np.zeros_like(f2), "hybrid_gs", 3, 3, omega=0.6)
        assert np.abs(p.from_lib(l, x) - want).max() <= 1e-10 * np.abs(want).max()
    finally:
        B.hhg_set_mg_params(h)


def test_lambda_estimate(cube4):
    p = cube4
    for l in (3, 4):
        exact = S.lambda_max_DinvA(p.H.A[l], p.H.lv[l].dirichlet)
        est = B.hhg_get_lambda_max(p.ctx.h, l)
        assert 0.9 * exact <= est <= exact * (1 + 1e-9)


@pytest.mark.parametrize("name", ["cube4", "skew4"])
def test_smoothers_and_vcycle(name, request):
    p = request.getfixturevalue(name)
    t = p.ctx.torch
    h = p.ctx.h
    l = 4
    lv, A = p.H.lv[l], p.H.A[l]
    lam = {q: S.lambda_max_DinvA(p.H.A[q], p.H.lv[q].dirichlet) for q in (3, 4)}
    for q in (3, 4):
        B.hhg_set_lambda_max(h, q, lam[q])
    f = hi.node_noise(lv.coords, seed=21)
    x0 = hi.node_noise(lv.coords, seed=22)
    try:
        # Jacobi
        B.hhg_set_mg_params(h, smoother=B.SMOOTH_JACOBI, omega=0.6)
        x = p.to_lib(l, x0, t.float64)
        B.hhg_smooth(h, l, B.F64, 3, p.to_lib(l, f, t.float64), x)
        want = S.jacobi(A, lv.dirichlet, f, x0, 0.6, 3)
        assert np.abs(p.from_lib(l, x) - want).max() <= 1e-11 * np.abs(want).max()
        # Chebyshev (3 and 4 steps: odd and even numbers of buffer swaps)
        B.hhg_set_mg_params(h, smoother=B.SMOOTH_CHEBYSHEV)
        for steps in (3, 4):
            x = p.to_lib(l, x0, t.float64)
            B.hhg_smooth(h, l, B.F64, steps, p.to_lib(l, f, t.float64), x)
            want = S.chebyshev(A, lv.dirichlet, f, x0, lam[l], 1 / 8, 1.1, steps)
            assert np.abs(p.from_lib(l, x) - want).max() <= 1e-11 * np.abs(want).max()
            x32 = p.to_lib(l, x0, t.float32)
            B.hhg_smooth(h, l, B.F32, steps, p.to_lib(l, f, t.float32), x32)
            assert np.abs(p.from_lib(l, x32) - want).max() <= 2e-5 * np.abs(want).max()
        # one V(2,2) cycle from zero
        f2 = f.copy()
        f2[lv.dirichlet] = 0.0
        x = t.zeros(3 * B.hhg_num_nodes(h, l)[0], dtype=t.float64, device="cuda")
        B.hhg_vcycle(h, l, B.F64, p.to_lib(l, f2, t.float64), x)
        want = p.H.vcycle(l, f2, np.zeros_like(f2), "chebyshev", 2, 2, lam)
        assert np.abs(p.from_lib(l, x) - want).max() <= 1e-10 * np.abs(want).max()
    finally:
        B.hhg_set_mg_params(h)


@pytest.fixture(scope="module")
def cube5():
    p = Pair(hi.kuhn_cube, 5)
    B.hhg_mg_setup(p.ctx.h)
    yield p
    p.close()


@pytest.mark.parametrize("method,dt,rtol", [
    (B.SOLVE_PCG_JACOBI, B.F64, 1e-10),
    (B.SOLVE_MG_CG, B.F64, 1e-8),
    (B.SOLVE_IR_MG_CG, B.F64, 1e-8),
    (B.SOLVE_MG, B.F64, 1e-8),
    (B.SOLVE_MG_CG, B.F32, 1e-5),
])
def test_solvers_cube_level5(cube5, method, dt, rtol):
    """Checked by the oracle's residual of the returned solution (the comparison with a
    direct solve is the unit-tetrahedron test's: a sparse LU of the level-5 cube takes
    minutes)."""
    p = cube5
    t = p.ctx.torch
    h = p.ctx.h
    l = 5
    lv, A = p.H.lv[l], p.H.A[l]
    f = hi.node_noise(lv.coords, seed=31)
    g = np.zeros_like(f)
    g[lv.dirichlet] = hi.node_noise(lv.coords, seed=32)[lv.dirichlet] * 0.1  # non-zero Dirichlet data
    tdt = t.float64 if dt == B.F64 else t.float32
    x = p.to_lib(l, g, tdt)
    rep = B.hhg_solve(h, p.to_lib(l, f, tdt), x, method=method, level=l, dt=dt, rtol=rtol, max_iter=500)
    assert rep["converged"]
    xs = p.from_lib(l, x)
    assert np.array_equal(xs[lv.dirichlet], p.from_lib(l, p.to_lib(l, g, tdt))[lv.dirichlet])
    r0 = np.linalg.norm(S.residual(A, lv.dirichlet, f, g))
    r = np.linalg.norm(S.residual(A, lv.dirichlet, f, xs))
    slack = 1.01 if dt == B.F64 else 20.0
    assert r <= slack * rtol * r0, (r / r0, rep)
    if method == B.SOLVE_IR_MG_CG:
        assert rep["inner_iterations"] >= rep["iterations"] >= 1


def test_jacobi_pcg_unit_tet_level5():
    """The 1-macro configuration: Jacobi-PCG to 1e-10 agrees with a direct solve."""
    p = Pair(hi.unit_tet, 5, kfun=lambda c: hi.young_sine(c))
    try:
        t = p.ctx.torch
        l = 5
        lv, A = p.H.lv[l], p.H.A[l]
        f = hi.node_noise(lv.coords, seed=1)
        x = t.zeros(3 * B.hhg_num_nodes(p.ctx.h, l)[0], dtype=t.float64, device="cuda")
        rep = B.hhg_solve(p.ctx.h, p.to_lib(l, f, t.float64), x, method=B.SOLVE_PCG_JACOBI, level=l, dt=B.F64,
                          rtol=1e-10, max_iter=2000)
        xd = S.direct_solve(A, lv.dirichlet, f, np.zeros_like(f))
        assert np.abs(p.from_lib(l, x) - xd).max() <= 1e-7 * np.abs(xd).max(), rep
    finally:
        p.close()


def test_full_size_ir_solve_cube_level7():
    """The benchmark configuration (6-macro cube, level 7, lognormal E, f ~ U[-1, 1]):
    FP64 iterative refinement around FP32 MG-CG reaches an FP64 relative residual of 1e-8;
    sampled residual rows are recomputed by the single-row oracle from the returned x."""
    from oracle import rows
    from hhg_gpu import torch_cuda

    torch = torch_cuda()
    xyz, tets = hi.kuhn_cube(1)
    level = 7
    N = 1 << level
    kgrid = hi.lognormal_grid(N, seed=2)
    fgrid = hi.uniform_grid(N, seed=3)
    kf = lambda c: hi.sample_grid(kgrid[..., None], c)[:, 0]
    ctx = Ctx(xyz, tets, level, dict(nu=NU))
    try:
        h = ctx.h
        ctx.set_k(kf(ctx.coords_u))
        B.hhg_mg_setup(h)
        f = ctx.to_lib(hi.sample_grid(fgrid, ctx.coords_u), torch.float64, 3)
        x = torch.zeros_like(f)
        rep = B.hhg_solve(h, f, x, method=B.SOLVE_IR_MG_CG, level=level, dt=B.F64, rtol=1e-8, max_iter=20,
                          inner_rtol=1e-3, inner_max_iter=50)
        assert rep["converged"] and rep["rel_residual"] <= 1e-8
        r = torch.empty_like(f)
        r2 = B.hhg_residual(h, level, B.F64, f, x, r, want_norm=True)
        assert np.sqrt(r2) <= 1.01e-8 * rep["residual0"]
        # sampled rows: oracle residual from the GPU solution
        xu = ctx.from_lib(x, 3)
        ru = ctx.from_lib(r, 3)
        key = np.rint(ctx.coords_u * N).astype(np.int64)
        grid_x = np.zeros((N + 1, N + 1, N + 1, 3))
        grid_x[key[:, 0], key[:, 1], key[:, 2]] = xu
        xf = lambda c: hi.sample_grid(grid_x, c)
        ce, cd = fem.elasticity_coefficients(NU)
        mm = mesh.MacroMesh.build(xyz, tets)
        rng = np.random.default_rng(5)
        first = np.full(ctx.U, -1, dtype=np.int64)
        first[ctx.e2u[::-1]] = np.arange(ctx.E)[::-1]
        nt = ctx.E // 6
        fu = hi.sample_grid(fgrid, ctx.coords_u)
        for u in rng.choice(np.nonzero(~ctx.udir)[0], 16, replace=False):
            m, loc = divmod(int(first[u]), nt)
            from test_gpu_parity import _decode
            ax, _ = rows.row(mm, level, m, _decode(N, loc), kf, xf, ce, cd)
            r_or = fu[u] - ax
            assert np.abs(r_or - ru[u]).max() <= 1e-9 * np.abs(fu[u]).max()
    finally:
        ctx.close()


@pytest.mark.parametrize("coarsest", [0, 1])
def test_coarser_hierarchies_on_a_48_macro_mesh(coarsest):
    """Hierarchies that start below level 2 (hhg_set_coarsest_level): on the 48-macro cube the
    coarsest levels 0 and 1 hold only skeleton nodes (vertices, and edge midpoints at level 1),
    where the level-2 hierarchy's direct solve would take 7 x 7 x 7 x 3 free DoFs.  The
    transfers and the operator of every level, one V(2,2) Chebyshev cycle and an MG-CG solve
    equal the oracle's hierarchy on the same levels."""
    p = Pair(lambda: hi.kuhn_cube(2), 3, coarsest=coarsest)
    try:
        t = p.ctx.torch
        h = p.ctx.h
        B.hhg_mg_setup(h)
        lam = {q: S.lambda_max_DinvA(p.H.A[q], p.H.lv[q].dirichlet) for q in range(coarsest + 1, 4)}
        for q, v in lam.items():
            B.hhg_set_lambda_max(h, q, v)
        for l in range(coarsest, 4):
            lv = p.H.lv[l]
            x = hi.node_noise(lv.coords, seed=30 + l)
            y = t.empty(3 * B.hhg_num_nodes(h, l)[0], dtype=t.float64, device="cuda")
            B.hhg_apply(h, l, B.F64, p.to_lib(l, x, t.float64), y)
            want = op.apply(p.H.A[l], x)
            assert np.abs(p.from_lib(l, y) - want).max() <= 1e-12 * np.abs(want).max(), l
            if l == coarsest:
                continue
            lc = p.H.lv[l - 1]
            xc = hi.node_noise(lc.coords, seed=40 + l)
            xc[lc.dirichlet] = 0.0
            xf = hi.node_noise(lv.coords, seed=50 + l)
            xfd = p.to_lib(l, xf, t.float64)
            B.hhg_prolongate_add(h, l, B.F64, p.to_lib(l - 1, xc, t.float64), xfd)
            want = S.prolongate_add(p.H.P[l], xc, xf)
            assert np.abs(p.from_lib(l, xfd) - want).max() <= 1e-14 * np.abs(want).max(), l
            rf = hi.node_noise(lv.coords, seed=60 + l)
            rf[lv.dirichlet] = 0.0
            rc = t.empty(3 * B.hhg_num_nodes(h, l - 1)[0], dtype=t.float64, device="cuda")
            B.hhg_restrict(h, l, B.F64, p.to_lib(l, rf, t.float64), rc)
            want = S.restrict(p.H.P[l], rf, lv.dirichlet, lc.dirichlet)
            assert np.abs(p.from_lib(l - 1, rc) - want).max() <= 1e-13 * np.abs(want).max(), l
        lv = p.H.lv[3]
        f = hi.node_noise(lv.coords, seed=71)
        f[lv.dirichlet] = 0.0
        x = t.zeros(3 * B.hhg_num_nodes(h, 3)[0], dtype=t.float64, device="cuda")
        fd = p.to_lib(3, f, t.float64)
        B.hhg_vcycle(h, 3, B.F64, fd, x)
        want = p.H.vcycle(3, f, np.zeros_like(f), "chebyshev", 2, 2, lam)
        assert np.abs(p.from_lib(3, x) - want).max() <= 1e-10 * np.abs(want).max()
        x.zero_()
        rep = B.hhg_solve(h, fd, x, method=B.SOLVE_MG_CG, level=3, dt=B.F64, rtol=1e-8, max_iter=100)
        r = S.residual(p.H.A[3], lv.dirichlet, f, p.from_lib(3, x))
        assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(f), rep
    finally:
        p.close()


def test_coarsest_level_must_precede_refinement():
    t = pytest.importorskip("torch")
    xyz, tets = hi.kuhn_cube(1)
    h = B.hhg_create(0, t.cuda.current_stream().cuda_stream)
    try:
        B.hhg_set_macro_mesh(h, xyz, tets)
        with pytest.raises(B.HhgError):
            B.hhg_set_coarsest_level(h, 10)
        B.hhg_set_coarsest_level(h, 1)
        with pytest.raises(B.HhgError):
            B.hhg_refine(h, 0)
        B.hhg_refine(h, 3)
        with pytest.raises(B.HhgError) as ei:
            B.hhg_set_coarsest_level(h, 0)
        assert ei.value.status == 8  # HHG_ERR_STATE
        assert B.hhg_num_nodes(h, 1)[1] == 3**3
    finally:
        B.hhg_destroy(h)
