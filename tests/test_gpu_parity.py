"""Parity of the CUDA operator apply / residual against the FP64 CPU oracle, through the C ABI.

Tolerances:
  FP64: max |y_gpu - y_oracle| / max |y_oracle| <= 1e-12 (rounding differences of sums of at
        most a few hundred terms).
  FP32: per row, |y32 - y_oracle|_i <= 64 * 2^-24 * sum_j |A_ij| |x_j - x_i|  (the scale of the
        row's terms in the difference form the kernels evaluate: FP32 rounding of x, k, the
        stencil constants and about 64 accumulated products), on free rows; Dirichlet rows
        return x rounded to FP32.
"""

import os

import numpy as np
import pytest
import scipy.sparse as sp

import hhg_inputs as hi
from oracle import fem, mesh, operators as op, rows
from paper_1908_08666_gb300 import binding as B

from hhg_gpu import Ctx

pytestmark = pytest.mark.gpu

FP32_C = 64 * 2.0**-24


def _oracle(xyz, tets, level, kfun, variant="physical", khat="patch", iface="symmetric", nu=0.3):
    mm = mesh.MacroMesh.build(xyz, tets)
    lv = mesh.build_level(mm, level)
    ce, cd = fem.elasticity_coefficients(nu)
    K = fem.element_stiffness(lv.coords[lv.elems], ce, cd)
    A = op.scaled_operator(lv, K, kfun(lv.coords), variant, khat=khat, iface=iface)
    return mm, lv, A


def _kfun(c):
    return 1.0 + 0.5 * np.sin(2 * np.pi * c[:, 0]) * np.sin(2 * np.pi * c[:, 1]) * np.sin(2 * np.pi * c[:, 2]) \
        + 0.3 * c[:, 2]


def _fp32_scale(A, x, lv):
    """sum_j |A_ij| |x_j - x_i| per node (3 components)."""
    N = lv.num_nodes
    Ac = A.tocoo()
    ni, nj = Ac.row // 3, Ac.col // 3
    diff = np.abs(x.reshape(-1)[Ac.col] - x.reshape(N, 3)[ni, Ac.col % 3])
    s = np.zeros(3 * N)
    np.add.at(s, Ac.row, np.abs(Ac.data) * diff)
    return s.reshape(N, 3)


CASES = [
    ("unit_tet_l5", hi.unit_tet, 5, {}),
    ("cube_l4", hi.kuhn_cube, 4, {}),
    ("cube_l4_unphysical", hi.kuhn_cube, 4, {"variant": "unphysical"}),
    ("cube_l4_khat_edge", hi.kuhn_cube, 4, {"khat": "edge"}),
    ("cube_l4_practical", hi.kuhn_cube, 4, {"iface": "practical"}),
    ("cube_l4_nodal", hi.kuhn_cube, 4, {"variant": "nodal"}),
    ("cube_l4_stored", hi.kuhn_cube, 4, {"variant": "stored"}),
    ("cube_l4_tile", hi.kuhn_cube, 4, {"kernel": 1}),
    ("skewed_l4_tile", hi.skewed_pair, 4, {"kernel": 1}),
    ("cube_l4_unphysical_tile", hi.kuhn_cube, 4, {"variant": "unphysical", "kernel": 1}),
    ("skewed_l4_stored", hi.skewed_pair, 4, {"variant": "stored"}),
    ("skewed_l4_nodal", hi.skewed_pair, 4, {"variant": "nodal"}),
    ("skewed_l4", hi.skewed_pair, 4, {}),
    ("cube2_l3", lambda: hi.kuhn_cube(2), 3, {}),
    # interior kernel 0 (automatic) launches all macros at once at these sizes; 2 forces one
    # launch per macro, 3 one launch for all
    ("cube_l4_per_macro", hi.kuhn_cube, 4, {"kernel": 2}),
    ("skewed_l4_per_macro", hi.skewed_pair, 4, {"kernel": 2}),
    ("cube_l4_unphysical_per_macro", hi.kuhn_cube, 4, {"variant": "unphysical", "kernel": 2}),
    ("cube2_l3_per_macro", lambda: hi.kuhn_cube(2), 3, {"kernel": 2}),
    ("unit_tet_l5_batched", hi.unit_tet, 5, {"kernel": 3}),
]

_VAR = {"physical": B.PHYSICAL, "unphysical": B.UNPHYSICAL, "nodal": B.NODAL, "stored": B.STORED}
_KH = {"patch": B.KHAT_PATCH, "edge": B.KHAT_EDGE}
_IF = {"symmetric": B.IFACE_SYMMETRIC, "practical": B.IFACE_PRACTICAL}


@pytest.mark.parametrize("name,builder,level,opt", CASES, ids=[c[0] for c in CASES])
def test_apply_and_residual_parity(name, builder, level, opt):
    xyz, tets = builder()
    variant = opt.get("variant", "physical")
    khat = opt.get("khat", "patch")
    iface = opt.get("iface", "symmetric")
    # the stored-stencil variant is the physical-scaling operator with stored macro-interior rows
    mm, lv, A = _oracle(xyz, tets, level, _kfun, "physical" if variant == "stored" else variant, khat, iface)
    A_bc = op.with_dirichlet_rows(A, lv.dirichlet)
    ctx = Ctx(xyz, tets, level, dict(nu=0.3, variant=_VAR[variant], khat=_KH[khat], iface=_IF[iface]))
    try:
        t = ctx.torch
        B.hhg_set_interior_kernel(ctx.h, opt.get("kernel", 0))
        perm = mesh.match_nodes(lv.coords, ctx.coords_u)  # oracle node i == gpu unique node perm[i]
        assert np.array_equal(ctx.udir[perm], lv.dirichlet)
        ctx.set_k(_kfun(ctx.coords_u))
        x_or = hi.node_noise(lv.coords, seed=7)
        f_or = hi.node_noise(lv.coords, seed=8)
        x_u = np.empty_like(x_or)
        x_u[perm] = x_or
        f_u = np.empty_like(f_or)
        f_u[perm] = f_or
        y_or = op.apply(A_bc, x_or)
        r_or = op.residual(A, f_or, x_or, lv.dirichlet)
        scale = _fp32_scale(A, x_or, lv)
        if variant == "stored":
            # stored rows are evaluated as the plain product sum_j A_ij x_j, whose FP32 rounding
            # scales with sum_j |A_ij| |x_j| (the centre block included)
            scale = (abs(A) @ np.abs(x_or).reshape(-1)).reshape(-1, 3)
        free = ~lv.dirichlet
        for dt, tdt in ((B.F64, t.float64), (B.F32, t.float32)):
            x = ctx.to_lib(x_u, tdt, 3)
            f = ctx.to_lib(f_u, tdt, 3)
            y = t.empty_like(x)
            r = t.empty_like(x)
            B.hhg_apply(ctx.h, level, dt, x, y)
            nrm = B.hhg_residual(ctx.h, level, dt, f, x, r, want_norm=True)
            yg = ctx.from_lib(y, 3)[perm]
            rg = ctx.from_lib(r, 3)[perm]
            if dt == B.F64:
                assert np.abs(yg - y_or).max() <= 1e-12 * np.abs(y_or).max()
                assert np.abs(rg - r_or).max() <= 1e-12 * np.abs(r_or).max()
                assert abs(nrm - (r_or[free] ** 2).sum()) <= 1e-11 * (r_or[free] ** 2).sum()
            else:
                assert np.all(np.abs(yg - y_or)[free] <= FP32_C * scale[free] + 1e-30)
                assert np.all(np.abs(rg - r_or)[free] <= FP32_C * (scale[free] + np.abs(f_or[free])) + 1e-30)
                assert np.abs(yg - y_or)[~free].max(initial=0) <= 2**-24 * np.abs(x_or).max()
                assert np.all(rg[~free] == 0)
                assert abs(nrm - (r_or[free] ** 2).sum()) <= 1e-4 * (r_or[free] ** 2).sum()
            # every copy of a skeleton node holds the same value
            full = y.double().cpu().numpy().reshape(3, ctx.E).T
            assert np.array_equal(full, ctx.from_lib(y, 3)[ctx.e2u])
    finally:
        ctx.close()


def _sample_rows(n, rng, nmacro=6):
    """Macro-interior rows (macro, (i, j, k)) of every kind the kernels treat differently:
    uniform over the interior, the last slices (k >= n - 8, where a slice holds few rows),
    rows next to a macro face (i, j or k = 1, or i + j + k = n - 1) and the ends of slice
    rows (i = n - 1 - j - k)."""
    out = []

    def rand_interior(kmin=1):
        # slice k with probability proportional to its (M - 1) M / 2 interior points
        # (M = n - 1 - k), row j proportional to its M - j points, then i uniform
        ks = np.arange(kmin, n - 2)
        Ms = n - 1 - ks
        k = int(rng.choice(ks, p=(Ms - 1) * Ms / ((Ms - 1) * Ms).sum()))
        M = n - 1 - k
        js = np.arange(1, M)
        j = int(rng.choice(js, p=(M - js) / (M - js).sum()))
        i = int(rng.integers(1, M - j + 1))
        return i, j, k

    for _ in range(1200):
        out.append((int(rng.integers(nmacro)), rand_interior()))
    for _ in range(400):
        out.append((int(rng.integers(nmacro)), rand_interior(n - 8)))
    for q in range(400):
        i, j, k = rand_interior()
        s = n - 1 - (i + j + k)
        which = q % 4
        if which == 0:
            i = 1
        elif which == 1:
            j = 1
        elif which == 2:
            k = 1
        else:
            i += s
        out.append((int(rng.integers(nmacro)), (i, j, k)))
    for _ in range(200):
        i, j, k = rand_interior()
        out.append((int(rng.integers(nmacro)), (n - 1 - j - k, j, k)))
    return out


@pytest.mark.parametrize("level", [7, 8], ids=["level7", "level8"])
def test_full_size_sampled_rows_cube(level):
    """The 6-macro cube at level 7 (129^3 nodes, the launch configuration of the benchmark)
    and level 8 (257^3 nodes): 2200 macro-interior rows (uniform, last slices, next to macro
    faces, ends of slice rows) and skeleton rows of every multiplicity (face, edge, vertex
    nodes) against the single-row oracle: FP64 within 1e-12 of the row scale, FP32 within
    the per-row bound 64 * 2^-24 * sum_j |A_ij| |x_j - x_i| stated above."""
    import multiprocessing as mpc

    import oracle_rows_pool as orp

    n = 1 << level
    xyz, tets = hi.kuhn_cube(1)
    rng = np.random.default_rng(level)
    interior = _sample_rows(n, rng)
    ctx = Ctx(xyz, tets, level, dict(nu=0.3))
    try:
        t = ctx.torch
        grid_k = hi.lognormal_grid(n, seed=2)
        grid_x = hi.uniform_grid(n, seed=3)
        ctx.set_k(hi.sample_grid(grid_k[..., None], ctx.coords_u)[:, 0])
        xu = hi.sample_grid(grid_x, ctx.coords_u)
        nt = ctx.E // 6
        first = np.full(ctx.U, -1, dtype=np.int64)
        first[ctx.e2u[::-1]] = np.arange(ctx.E)[::-1]
        picks = [(int(ctx.e2u[m * nt + _lattice_index(n, *ijk)]), m, ijk) for m, ijk in interior]
        # skeleton rows: three free nodes of every multiplicity (incident macros), 100 more
        # random free face nodes
        per_inc = np.bincount(ctx.e2u, minlength=ctx.U)
        skel = []
        for cnt in np.unique(per_inc):
            cand = np.nonzero((per_inc == cnt) & ~ctx.udir)[0]
            if cnt > 1 and len(cand):
                skel += list(rng.choice(cand, min(3 if cnt > 2 else 103, len(cand)), replace=False))
        for u in skel:
            m, loc = divmod(int(first[u]), nt)
            picks.append((int(u), m, _decode(n, loc)))
        nproc = max(1, min(8, (os.cpu_count() or 1)))
        chunks = [picks[q::nproc] for q in range(nproc)]
        with mpc.get_context("spawn").Pool(nproc, initializer=orp.init, initargs=(level,)) as pool:
            res = pool.map(orp.job, [[(m, ijk) for _, m, ijk in ch] for ch in chunks])
        want = {}
        for ch, rs in zip(chunks, res):
            for (u, _, _), (y, sc) in zip(ch, rs):
                want[u] = (y, sc)
        assert len(want) >= 2000
        for dt, tdt in ((B.F64, t.float64), (B.F32, t.float32)):
            x = ctx.to_lib(xu, tdt, 3)
            y = t.empty_like(x)
            B.hhg_apply(ctx.h, level, dt, x, y)
            yg = ctx.from_lib(y, 3)
            worst = 0.0
            for u, (yr, sc) in want.items():
                err = np.abs(yg[u] - yr)
                if dt == B.F64:
                    assert err.max() <= 1e-12 * (sc.max() + np.abs(yr).max()), (u, yg[u], yr)
                else:
                    assert np.all(err <= FP32_C * sc + 1e-30), (u, yg[u], yr, sc)
                    worst = max(worst, float((err / (sc + 1e-300)).max()))
            if dt == B.F32:
                print("level %d: %d rows, worst FP32 error / term scale %.3g (bound %.3g)"
                      % (level, len(want), worst, FP32_C))
    finally:
        ctx.close()


def _lattice_index(n, i, j, k):
    m = n - k
    T = lambda a: a * (a + 1) * (a + 2) // 6
    return T(n + 1) - T(n + 1 - k) + j * (2 * m + 3 - j) // 2 + i


def _decode(n, loc):
    for k in range(n + 1):
        m = n - k
        sz = (m + 1) * (m + 2) // 2
        if loc < sz:
            for j in range(m + 1):
                L = m - j + 1
                if loc < L:
                    return (loc, j, k)
                loc -= L
        loc -= sz
    raise ValueError


def test_bf16_coefficient_parity_and_error():
    """BF16 coefficient: the GPU operator equals the oracle's operator built with the
    BF16-rounded nodal values (FP64 to 1e-12, FP32 to the FP32 bound; the FP32 apply reads
    the BF16 bits), and differs from the operator of the unrounded coefficient by the
    stated rounding error (each block by at most 2^-8 of its terms)."""
    from oracle.learned import bf16

    xyz, tets = hi.kuhn_cube()
    level = 4
    mm, lv, A = _oracle(xyz, tets, level, _kfun)
    _, _, Ab = _oracle(xyz, tets, level, lambda c: bf16(_kfun(c)))
    Ab_bc = op.with_dirichlet_rows(Ab, lv.dirichlet)
    A_bc = op.with_dirichlet_rows(A, lv.dirichlet)
    ctx = Ctx(xyz, tets, level, dict(nu=0.3))
    try:
        t = ctx.torch
        perm = mesh.match_nodes(lv.coords, ctx.coords_u)
        kb = np.empty(lv.num_nodes)
        kb[perm] = bf16(_kfun(lv.coords))
        kl = ctx.to_lib(kb, t.float32, 1).to(t.bfloat16)
        assert np.array_equal(kl.float().cpu().numpy(), ctx.to_lib(kb, t.float32, 1).cpu().numpy())
        B.hhg_set_coefficient(ctx.h, kl.view(t.int16), B.BF16)
        x_or = hi.node_noise(lv.coords, seed=7)
        x_u = np.empty_like(x_or)
        x_u[perm] = x_or
        y_b = op.apply(Ab_bc, x_or)
        y_k = op.apply(A_bc, x_or)
        scale = _fp32_scale(Ab, x_or, lv)
        free = ~lv.dirichlet
        for dt, tdt in ((B.F64, t.float64), (B.F32, t.float32)):
            x = ctx.to_lib(x_u, tdt, 3)
            y = t.empty_like(x)
            B.hhg_apply(ctx.h, level, dt, x, y)
            yg = ctx.from_lib(y, 3)[perm]
            if dt == B.F64:
                assert np.abs(yg - y_b).max() <= 1e-12 * np.abs(y_b).max()
            else:
                assert np.all(np.abs(yg - y_b)[free] <= FP32_C * scale[free] + 1e-30)
        # the stated error of the BF16 coefficient against the exact one (2^-8 per term; the
        # row scale below sums |A_ij| rather than the terms' magnitudes, hence a factor 2)
        assert np.all(np.abs(y_b - y_k)[free] <= 2.0**-7 * _fp32_scale(A, x_or, lv)[free] + 1e-30)
        assert np.linalg.norm(y_b - y_k) > 0
    finally:
        ctx.close()
