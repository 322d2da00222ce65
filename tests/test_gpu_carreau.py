"""Carreau viscosity from the nodal least-squares strain rate and the Picard iteration (Alg. 1)."""

import numpy as np
import pytest

import hhg_inputs as hi
from oracle import carreau as CA, mesh
from paper_1908_08666_gb300 import binding as B

from hhg_gpu import Ctx

pytestmark = pytest.mark.gpu

PAR = dict(eta0=1.0, eta_inf=1e-3, kappa=1.0, r=-0.25)


def _u(c):
    return np.stack([np.sin(2 * c[:, 0]) * c[:, 1] ** 2, np.cos(c[:, 1] + 2 * c[:, 2]), c[:, 0] * c[:, 2] ** 2], 1)


@pytest.mark.parametrize("builder,level,degree", [(hi.kuhn_cube, 4, 1), (hi.skewed_pair, 3, 1), (hi.skewed_pair, 3, 2),
                                                  (hi.skewed_pair, 4, 2), (lambda: hi.kuhn_cube(2), 3, 2)],
                         ids=["cube_l4", "skewed_l3", "skewed_l3_quadratic", "skewed_l4_quadratic",
                              "cube2_l3_quadratic"])
def test_carreau_viscosity_parity(builder, level, degree):
    """Affine (m = 1) and quadratic (m = 2, where the patch determines it) least-squares
    strain rates (Sec. 3) against the oracle's; the quadratic fit differs from the affine one
    at the skewed mesh's interface nodes."""
    xyz, tets = builder()
    lv = mesh.build_level(mesh.MacroMesh.build(xyz, tets), level)
    ctx = Ctx(xyz, tets, level, dict(kind=B.STOKES))
    try:
        t = ctx.torch
        B.hhg_set_strain_fit(ctx.h, degree)
        perm = mesh.match_nodes(lv.coords, ctx.coords_u)
        u = ctx.to_lib(_u(ctx.coords_u), t.float64, 3)
        mu = t.empty(ctx.E, dtype=t.float64, device="cuda")
        B.hhg_carreau_viscosity(ctx.h, level, u, mu, **PAR)
        got = ctx.from_lib(mu, 1)[perm, 0]
        want = CA.viscosity(lv, _u(lv.coords), **PAR, degree=degree)
        assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max()
        if degree == 2 and builder is hi.skewed_pair:
            other = CA.viscosity(lv, _u(lv.coords), **PAR, degree=1)
            assert np.abs(other - want).max() > 1e-8 * np.abs(want).max()
        full = mu.cpu().numpy()
        assert np.array_equal(full, ctx.from_lib(mu, 1)[ctx.e2u, 0])
    finally:
        ctx.close()


def test_picard_lid_driven_cavity():
    """Alg. 1 on the 6-macro cube, level 4, lid velocity 16x(1-x)y(1-y) on z = 1: the
    fixed-point iteration stops on the relative change criterion, the final relative
    residual reaches 1e-3, and the viscosity lies in [eta_inf, eta0] and is below eta0
    where the fluid is sheared."""
    xyz, tets = hi.kuhn_cube(1)
    level = 4
    ctx = Ctx(xyz, tets, level, dict(kind=B.STOKES))
    try:
        t = ctx.torch
        ctx.set_k(np.ones(ctx.U))
        x0 = np.zeros((ctx.U, 4))
        x0[:, :3] = hi.lid_velocity(ctx.coords_u)
        x = ctx.to_lib(x0, t.float64, 4)
        f = t.zeros_like(x)
        rep = B.hhg_picard(ctx.h, f, x, level, picard_tol=1e-3, max_picard=40, step_rtol=1e-2, step_max_iter=200,
                           final_rtol=1e-3, **PAR)
        assert rep["converged"] and rep["final_rel_residual"] <= 1e-3, rep
        assert PAR["eta_inf"] <= rep["mu_min"] <= rep["mu_max"] <= PAR["eta0"] + 1e-12
        assert rep["mu_min"] < 0.9
        xs = ctx.from_lib(x, 4)
        assert np.allclose(xs[ctx.udir, :3], x0[ctx.udir, :3])
    finally:
        ctx.close()


def test_picard_parity_with_exact_steps():
    """Alg. 1 on the 6-macro cube, level 3, lid velocity on z = 1 and a seeded body force,
    with each fixed-point step solved to 1e-11 (FP64 refinement): the GPU's fixed-point
    count, final velocity, pressure and viscosity equal those of the oracle's Alg. 1 with
    exact sparse solves (oracle.carreau.picard).  The oracle's change sequence keeps a
    margin of 20% from the stopping threshold, so the count is not decided by rounding."""
    from oracle import carreau as CA

    xyz, tets = hi.kuhn_cube(1)
    level = 3
    mm = mesh.MacroMesh.build(xyz, tets)
    lv = mesh.build_level(mm, level)
    N = lv.num_nodes

    def setup(coords, dirichlet):
        x0 = np.zeros((len(coords), 4))
        x0[:, :3] = hi.lid_velocity(coords)
        x0[~dirichlet] = 0.0
        f = np.zeros((len(coords), 4))
        f[:, :3] = 20.0 * hi.node_noise(coords, seed=7)
        f[dirichlet, :3] = 0.0
        return x0, f

    x0o, fo = setup(lv.coords, lv.dirichlet)
    tol = 1e-3
    xo, muo, no, ch = CA.picard(mm, lv, fo, x0o, tol=tol, **PAR)
    assert all(abs(c / tol - 1.0) > 0.2 for c in ch)
    ctx = Ctx(xyz, tets, level, dict(kind=B.STOKES))
    try:
        t = ctx.torch
        perm = mesh.match_nodes(lv.coords, ctx.coords_u)
        assert np.array_equal(ctx.udir[perm], lv.dirichlet)
        ctx.set_k(np.ones(ctx.U))
        x0, f = setup(ctx.coords_u, ctx.udir)
        x = ctx.to_lib(x0, t.float64, 4)
        fd = ctx.to_lib(f, t.float64, 4)
        rep = B.hhg_picard(ctx.h, fd, x, level, picard_tol=tol, max_picard=40, step_rtol=1e-11,
                           step_max_iter=400, final_rtol=1e-11, **PAR)
        assert rep["picard_iterations"] == no, (rep, ch)
        xg = ctx.from_lib(x, 4)[perm]
        # the viscosity left as the coefficient is mu(u) of the final velocity
        mu_d = t.empty(ctx.E, dtype=t.float64, device="cuda")
        B.hhg_carreau_viscosity(ctx.h, level, x, mu_d, **PAR)
        mug = ctx.from_lib(mu_d, 1)[perm, 0]
        eu = np.abs(xg[:, :3] - xo[:, :3]).max() / np.abs(xo[:, :3]).max()
        ep = np.abs(xg[:, 3] - xo[:, 3]).max() / np.abs(xo[:, 3]).max()
        em = np.abs(mug - muo).max() / np.abs(muo).max()
        assert eu < 1e-7 and ep < 1e-7 and em < 1e-7, (eu, ep, em)
        assert abs(rep["mu_min"] - muo.min()) < 1e-7 and abs(rep["mu_max"] - muo.max()) < 1e-7
    finally:
        ctx.close()
