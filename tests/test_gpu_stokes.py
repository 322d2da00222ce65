"""Stokes saddle operator and MINRES solves of the CUDA library against the FP64 oracle."""

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import hhg_inputs as hi
from oracle import mesh, stokes as ST
from paper_1908_08666_gb300 import binding as B

from hhg_gpu import Ctx

pytestmark = pytest.mark.gpu

FP32_C = 64 * 2.0**-24


def _mu(c):
    return hi.viscosity_sphere(c, mu_in=1.0, mu_out=10.0, radius=0.3, width=0.1)


def _setup(builder, level):
    xyz, tets = builder()
    mm = mesh.MacroMesh.build(xyz, tets)
    lv = mesh.build_level(mm, level)
    Kbc, K = ST.stokes_operator(mm, lv, _mu(lv.coords))
    ctx = Ctx(xyz, tets, level, dict(kind=B.STOKES))
    perm = mesh.match_nodes(lv.coords, ctx.coords_u)
    ctx.set_k(_mu(ctx.coords_u))
    return mm, lv, Kbc, K, ctx, perm


def _to_u(perm, u, p):
    out = np.empty((len(p), 4))
    out[perm, :3] = u
    out[perm, 3] = p
    return out


# interior kernel 0: automatic (all macros in one launch at these sizes); 2: one launch per macro
@pytest.mark.parametrize("builder,level,kernel", [(hi.kuhn_cube, 4, 0), (hi.kuhn_cube, 4, 2), (hi.skewed_pair, 3, 0)],
                         ids=["cube_l4", "cube_l4_per_macro", "skewed_l3"])
def test_stokes_apply_residual_parity(builder, level, kernel):
    mm, lv, Kbc, K, ctx, perm = _setup(builder, level)
    try:
        t = ctx.torch
        B.hhg_set_interior_kernel(ctx.h, kernel)
        N = lv.num_nodes
        xu, xp = hi.node_noise(lv.coords, 5), hi.node_noise(lv.coords, 6, comps=1)
        fu, fp = hi.node_noise(lv.coords, 7), hi.node_noise(lv.coords, 8, comps=1)
        x_or, f_or = ST.pack(xu, xp), ST.pack(fu, fp)
        y_or = Kbc @ x_or
        r_or = ST.residual(Kbc, lv.dirichlet, f_or, x_or)
        # row scale for the FP32 bound: sum_j |K_ij| |x_j| + |f_i|
        scale = abs(Kbc) @ np.abs(x_or) + np.abs(f_or)
        for dt, tdt in ((B.F64, t.float64), (B.F32, t.float32)):
            x = ctx.to_lib(_to_u(perm, xu, xp), tdt, 4)
            f = ctx.to_lib(_to_u(perm, fu, fp), tdt, 4)
            y = t.empty_like(x)
            r = t.empty_like(x)
            B.hhg_stokes_apply(ctx.h, level, dt, x, y)
            n2 = B.hhg_stokes_residual(ctx.h, level, dt, f, x, r, want_norm=True)
            yg = ctx.from_lib(y, 4)[perm]
            rg = ctx.from_lib(r, 4)[perm]
            yg = ST.pack(yg[:, :3], yg[:, 3])
            rg = ST.pack(rg[:, :3], rg[:, 3])
            if dt == B.F64:
                assert np.abs(yg - y_or).max() <= 1e-12 * np.abs(y_or).max()
                assert np.abs(rg - r_or).max() <= 1e-12 * np.abs(r_or).max()
                assert abs(n2 - (r_or**2).sum()) <= 1e-11 * (r_or**2).sum()
            else:
                assert np.all(np.abs(yg - y_or) <= FP32_C * scale)
                assert np.all(np.abs(rg - r_or) <= FP32_C * scale)
    finally:
        ctx.close()


def _direct(mm, lv, Kbc, f):
    """Solution with the mass-weighted zero-mean pressure (bordered system)."""
    N = lv.num_nodes
    m = ST.lumped_mass(lv)
    c = np.concatenate([np.zeros(3 * N), m])
    A = sp.bmat([[Kbc, sp.csr_matrix(c[:, None])], [sp.csr_matrix(c[None, :]), None]]).tocsc()
    sol = spla.spsolve(A, np.concatenate([f, [0.0]]))
    return sol[:-1]


@pytest.fixture(scope="module")
def cube4_solve():
    """Stokes level-4 cube: GPU context, oracle operator, right-hand side and the direct
    solution (computed once for all solver methods)."""
    level = 4
    mm, lv, Kbc, K, ctx, perm = _setup(hi.kuhn_cube, level)
    N = lv.num_nodes
    fu = hi.node_noise(lv.coords, 9)
    fu[lv.dirichlet] = 0.0
    f_or = ST.pack(fu, np.zeros(N))
    B.hhg_mg_setup(ctx.h)
    xd = _direct(mm, lv, Kbc, f_or)
    yield dict(level=level, lv=lv, Kbc=Kbc, ctx=ctx, perm=perm, fu=fu, f_or=f_or, xd=xd)
    ctx.close()


@pytest.mark.parametrize("method", [B.SOLVE_STOKES_MINRES, B.SOLVE_STOKES_IR_MINRES, B.SOLVE_STOKES_UZAWA,
                                    B.SOLVE_STOKES_IR_UZAWA])
def test_stokes_minres_solve(cube4_solve, method):
    d = cube4_solve
    ctx, lv, perm, level = d["ctx"], d["lv"], d["perm"], d["level"]
    t = ctx.torch
    N = lv.num_nodes
    f = ctx.to_lib(_to_u(perm, d["fu"], np.zeros(N)), t.float64, 4)
    x = t.zeros_like(f)
    rep = B.hhg_solve(ctx.h, f, x, method=method, level=level, dt=B.F64, rtol=1e-8, max_iter=400,
                      inner_rtol=1e-3, inner_max_iter=200)
    xg = ctx.from_lib(x, 4)[perm]
    x_g = ST.pack(xg[:, :3], xg[:, 3])
    r = ST.residual(d["Kbc"], lv.dirichlet, d["f_or"], x_g)
    assert np.linalg.norm(r) <= 2e-8 * np.linalg.norm(d["f_or"]), rep
    xd = d["xd"]
    assert np.abs(x_g - xd).max() <= 1e-5 * np.abs(xd).max(), rep
    assert abs((ST.lumped_mass(lv) * x_g[3 * N:]).sum()) <= 1e-10 * np.abs(x_g[3 * N:]).sum()


@pytest.mark.parametrize("builder,level,coarsest", [(hi.kuhn_cube, 4, 2), (lambda: hi.kuhn_cube(2), 3, 1)],
                         ids=["cube_l4", "cube2_l3_coarsest1"])
def test_uzawa_with_hybrid_gauss_seidel_matches_oracle(builder, level, coarsest):
    """The paper's Stokes solver settings (Sec. 5.2.1): inexact Uzawa with hybrid Gauss-Seidel
    velocity smoothing (one step per Uzawa step), pressure relaxation 0.3 and variable V(3,3)
    cycles with two more steps per coarser level.  One cycle from zero in FP64 equals the
    oracle's cycle; the stationary iteration then reaches a relative residual of 1e-8 (the
    oracle's cycles contract by about 0.7 each on the 6-macro cube: about 50 cycles).  Also on
    the 48-macro cube with the coarsest level 1 (hhg_set_coarsest_level), whose direct
    saddle solve holds the edge midpoints and macro vertices only."""
    xyz, tets = builder()
    H = ST.UzawaHierarchy(mesh.MacroMesh.build(xyz, tets), list(range(coarsest, level + 1)), _mu)
    lv = H.lv[level]
    N = lv.num_nodes
    ctx = Ctx(xyz, tets, level, dict(kind=B.STOKES), coarsest=coarsest)
    try:
        t = ctx.torch
        perm = mesh.match_nodes(lv.coords, ctx.coords_u)
        ctx.set_k(_mu(ctx.coords_u))
        B.hhg_set_mg_params(ctx.h, smoother=B.SMOOTH_HYBRID_GS, uzawa_pre=3, uzawa_post=3, uzawa_extra=2,
                            uzawa_vsteps=1, uzawa_omega=0.3)
        B.hhg_mg_setup(ctx.h)
        f = np.zeros((N, 4))
        f[:, :3] = hi.node_noise(lv.coords, 21)
        f[:, 3] = hi.node_noise(lv.coords, 22, comps=1).reshape(-1)
        f[:, 3] -= f[:, 3].mean()  # orthogonal to the constant-pressure kernel
        f[lv.dirichlet, :3] = 0.0
        want = H.project_pressure(level, H.vcycle(level, f, np.zeros_like(f), {}, level, vsteps=1, omega=0.3,
                                                  smoother="hybrid_gs"))
        fd = ctx.to_lib(_to_u(perm, f[:, :3], f[:, 3]), t.float64, 4)
        x = t.zeros_like(fd)
        rep = B.hhg_solve(ctx.h, fd, x, method=B.SOLVE_STOKES_UZAWA, level=level, dt=B.F64, rtol=1e-14, max_iter=1,
                          allow_not_converged=True)
        assert rep["iterations"] == 1
        got = ctx.from_lib(x, 4)[perm]
        assert np.abs(got[:, :3] - want[:, :3]).max() <= 1e-9 * np.abs(want[:, :3]).max()
        assert np.abs(got[:, 3] - want[:, 3]).max() <= 1e-9 * np.abs(want[:, 3]).max()
        x.zero_()
        rep = B.hhg_solve(ctx.h, fd, x, method=B.SOLVE_STOKES_UZAWA, level=level, dt=B.F64, rtol=1e-8,
                          max_iter=100)
        assert rep["converged"], rep
    finally:
        B.hhg_set_mg_params(ctx.h)
        ctx.close()
