"""Boundary traction (Neumann) load of the CUDA library against the oracle (Sec. 5.1.3), and a
clamped block under a top-plane traction solved by multigrid against a sparse direct solve."""

import numpy as np
import pytest

import hhg_inputs as hi
from oracle import fem, loads as LD, mesh, operators as op, solvers as S
from paper_1908_08666_gb300 import binding as B

from hhg_gpu import Ctx

pytestmark = pytest.mark.gpu


def _flags(xyz, tets, axis, value):
    flags = np.zeros((len(tets), 4), dtype=np.int32)
    for m, t in enumerate(tets):
        for f in range(4):
            if np.all(np.abs(xyz[[int(t[q]) for q in range(4) if q != f], axis] - value) < 1e-12):
                flags[m, f] = 1
    return flags


def _setup(level, traction_faces):
    xyz, tets = hi.kuhn_box(2, 1, 1)
    dflags = _flags(xyz, tets, 2, 0.0)  # clamped bottom; every other boundary face is natural
    tflags = np.zeros_like(dflags)
    for axis, value in traction_faces:
        tflags |= _flags(xyz, tets, axis, value)
    mm = mesh.MacroMesh.build(xyz, tets, dflags.astype(bool))
    lv = mesh.build_level(mm, level)
    ctx = Ctx(xyz, tets, level, dict(nu=0.3), dirichlet_face_flags=dflags)
    perm = mesh.match_nodes(lv.coords, ctx.coords_u)
    assert np.array_equal(ctx.udir[perm], lv.dirichlet)
    return xyz, tets, mm, lv, ctx, perm, tflags


@pytest.mark.parametrize("level", [2, 3])
def test_traction_load_parity(level):
    """Top plane, the x = 2 side and the y = 0 side carry an affine-plus-sine traction (macro
    faces of several types); the load equals the oracle's on every free row and every copy."""
    xyz, tets, mm, lv, ctx, perm, tflags = _setup(level, [(2, 1.0), (0, 2.0), (1, 0.0)])
    try:
        t_ = ctx.torch
        c = lv.coords
        tr = np.stack([np.sin(2 * c[:, 0]) + c[:, 1], -1.0 + 0.5 * c[:, 2], c[:, 0] * c[:, 1]], 1)
        want = LD.traction_load(mm, lv, tflags, tr)
        free = ~lv.dirichlet
        tu = np.empty_like(tr)
        tu[perm] = tr
        for dt, tdt, tol in ((B.F64, t_.float64, 1e-13), (B.F32, t_.float32, 1e-6)):
            td = ctx.to_lib(tu, tdt, 3)
            f = t_.zeros_like(td)
            B.hhg_traction_load(ctx.h, level, dt, tflags, td, f)
            got = ctx.from_lib(f, 3)[perm]
            assert np.abs(got[free] - want[free]).max() <= tol * np.abs(want).max()
            assert np.all(got[~free] == 0.0)
            full = f.double().cpu().numpy().reshape(3, ctx.E).T
            assert np.array_equal(full, ctx.from_lib(f, 3)[ctx.e2u])
        # a face shared by two macros cannot carry a traction
        keys = [[tuple(sorted(int(v) for v in np.delete(t, f))) for f in range(4)] for t in tets]
        count = {}
        for row in keys:
            for k in row:
                count[k] = count.get(k, 0) + 1
        mi, fi = next((m, q) for m in range(len(tets)) for q in range(4) if count[keys[m][q]] == 2)
        bad = np.zeros_like(tflags)
        bad[mi, fi] = 1
        with pytest.raises(B.HhgError):
            B.hhg_traction_load(ctx.h, level, B.F64, bad, td, f)
    finally:
        ctx.close()


def test_clamped_block_under_top_traction():
    """The foam setup's boundary conditions (Sec. 5.1.3) on a 2 x 1 x 1 block: clamped at z = 0,
    traction (0, 0, -1) on z = 1, the other faces free; MG-CG reaches 1e-10 and the displacement
    equals the oracle's sparse direct solve of the same system."""
    level = 3
    xyz, tets, mm, lv, ctx, perm, tflags = _setup(level, [(2, 1.0)])
    try:
        t_ = ctx.torch
        kf = lambda c: 1.0 + 0.5 * np.cos(3 * c[:, 0]) * np.sin(2 * c[:, 1] + c[:, 2])
        ctx.set_k(kf(ctx.coords_u))
        tr = np.tile([0.0, 0.0, -1.0], (lv.num_nodes, 1))
        ce, cd = fem.elasticity_coefficients(0.3)
        K = fem.element_stiffness(lv.coords[lv.elems], ce, cd)
        A = op.with_dirichlet_rows(op.scaled_operator(lv, K, kf(lv.coords)), lv.dirichlet)
        b = LD.traction_load(mm, lv, tflags, tr)
        b[lv.dirichlet] = 0.0
        want = S.direct_solve(A, lv.dirichlet, b, np.zeros_like(b))
        tu = np.empty_like(tr)
        tu[perm] = tr
        f = t_.zeros(3 * ctx.E, dtype=t_.float64, device="cuda")
        B.hhg_traction_load(ctx.h, level, B.F64, tflags, ctx.to_lib(tu, t_.float64, 3), f)
        B.hhg_mg_setup(ctx.h)
        x = t_.zeros_like(f)
        rep = B.hhg_solve(ctx.h, f, x, method=B.SOLVE_MG_CG, level=level, dt=B.F64, rtol=1e-10, max_iter=100)
        got = ctx.from_lib(x, 3)[perm]
        assert np.abs(got - want).max() <= 1e-8 * np.abs(want).max(), rep
        assert want[:, 2].min() < 0  # the block is pressed down
    finally:
        ctx.close()
