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


@pytest.mark.parametrize("builder,level", [(hi.kuhn_cube, 4), (hi.skewed_pair, 3)], ids=["cube_l4", "skewed_l3"])
def test_carreau_viscosity_parity(builder, level):
    xyz, tets = builder()
    lv = mesh.build_level(mesh.MacroMesh.build(xyz, tets), level)
    ctx = Ctx(xyz, tets, level, dict(kind=B.STOKES))
    try:
        t = ctx.torch
        perm = mesh.match_nodes(lv.coords, ctx.coords_u)
        u = ctx.to_lib(_u(ctx.coords_u), t.float64, 3)
        mu = t.empty(ctx.E, dtype=t.float64, device="cuda")
        B.hhg_carreau_viscosity(ctx.h, level, u, mu, **PAR)
        got = ctx.from_lib(mu, 1)[perm, 0]
        want = CA.viscosity(lv, _u(lv.coords), **PAR)
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
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
