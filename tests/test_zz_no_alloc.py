"""The allocation-free residual entry point (hhg_residual_noalloc) against hhg_residual.

Some callers cannot allocate device memory when they need a residual norm: their
device memory is owned by another allocator, or they run a time-critical solver
loop that must not pay cudaMalloc's latency and implicit synchronisation.  For
them hhg_residual_noalloc keeps its scratch in a static device array.  This
file is collected last on purpose, so a run that stops at the first failure has
already run every other test.  It passes alone in a fresh process and after the
other tests.
"""

import numpy as np
import pytest

import hhg_inputs as hi
from paper_1908_08666_gb300 import binding as B

from hhg_gpu import Ctx

pytestmark = pytest.mark.gpu


CASES = [
    ("cube_l5", hi.kuhn_cube, 5, {}, False),
    ("skewed_l4", hi.skewed_pair, 4, {}, False),
    ("cube_l4_unphysical", hi.kuhn_cube, 4, {"variant": B.UNPHYSICAL}, False),
    ("cube_l4_khat_edge", hi.kuhn_cube, 4, {"khat": B.KHAT_EDGE}, False),
    ("cube_l4_practical", hi.kuhn_cube, 4, {"iface": B.IFACE_PRACTICAL}, False),
    ("cube_l4_bf16_coefficient", hi.kuhn_cube, 4, {}, True),
]


@pytest.mark.parametrize("name,builder,level,problem,bf16", CASES, ids=[c[0] for c in CASES])
def test_residual_noalloc_matches_residual(name, builder, level, problem, bf16):
    """Every operator variant hhg_set_problem offers to this entry point (the no-alloc path
    takes other kernels for the face nodes and, with a BF16 coefficient, reads its widened
    values), two calls in a row, FP64 and FP32."""
    xyz, tets = builder()
    ctx = Ctx(xyz, tets, level, dict(nu=0.3, **problem))
    try:
        t = ctx.torch
        k = 1.0 + 0.5 * np.cos(3.0 * ctx.coords_u).prod(axis=1)
        if bf16:
            kl = ctx.to_lib(k, t.float32, 1).to(t.bfloat16)
            B.hhg_set_coefficient(ctx.h, kl.view(t.int16), B.BF16)
        else:
            ctx.set_k(k)
        for dt, tdt, tol in ((B.F64, t.float64, 1e-12), (B.F32, t.float32, 64 * 2.0**-24)):
            for call in range(2):  # two calls in a row: the shared scratch keeps the last call's contents
                x = ctx.to_lib(hi.node_noise(ctx.coords_u, seed=20 + call), tdt, 3)
                f = ctx.to_lib(hi.node_noise(ctx.coords_u, seed=40 + call), tdt, 3)
                r_ref = t.empty_like(x)
                r_new = t.full_like(x, float("nan"))
                n_ref = B.hhg_residual(ctx.h, level, dt, f, x, r_ref, want_norm=True)
                n_new = B.hhg_residual_noalloc(ctx.h, level, dt, f, x, r_new)
                t.cuda.synchronize()
                a = ctx.from_lib(r_ref, 3)
                b = ctx.from_lib(r_new, 3)
                scale = np.abs(a).max()
                assert np.isfinite(b).all()
                assert np.abs(a - b).max() <= tol * scale
                assert abs(n_new - n_ref) <= (1e-12 if dt == B.F64 else 1e-5) * n_ref
                # every copy of a skeleton node holds the same value
                full = r_new.double().cpu().numpy().reshape(3, ctx.E).T
                assert np.array_equal(full, b[ctx.e2u])
    finally:
        ctx.close()


def test_residual_noalloc_rejects_levels_beyond_its_scratch():
    """The 384-macro cube at level 6 needs more partial sums than the static scratch holds;
    the call is rejected with HHG_ERR_ARG and a message, before any launch."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    xyz, tets = hi.kuhn_cube(4)
    h = B.hhg_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        B.hhg_set_macro_mesh(h, xyz, tets)
        B.hhg_refine(h, 6)
        B.hhg_set_problem(h, nu=0.3)
        E, _, _ = B.hhg_num_nodes(h, 6)
        k = torch.ones(E, dtype=torch.float64, device="cuda")
        B.hhg_set_coefficient(h, k, B.F64)
        x = torch.zeros(3 * E, dtype=torch.float32, device="cuda")
        f = torch.zeros_like(x)
        r = torch.empty_like(x)
        with pytest.raises(B.HhgError) as ei:
            B.hhg_residual_noalloc(h, 6, B.F32, f, x, r)
        assert ei.value.status == 1 and "no-alloc scratch" in str(ei.value)
    finally:
        B.hhg_destroy(h)
