"""Learned preconditioner on the GPU against the oracle (oracle/learned.py).

Tolerances.  The network runs with BF16 activations and weights and FP32 accumulation;
the oracle rounds the same tensors to BF16 but accumulates in FP64, so a hidden
activation can land one BF16 step (2^-8 relative) away where the two sums straddle a
rounding boundary.  The backward pass stores its gradient tensors in BF16 while the
oracle keeps them in FP64 (about 2^-9 relative per layer).  Hence: forward outputs to
1e-2 of their largest magnitude, gradients to 2e-2 in norm per layer (the stated
tolerance for BF16 gradients), FP32 multigrid quantities to 1e-4.
"""

import numpy as np
import pytest

import hhg_inputs as hi
from oracle import learned as LN, solvers as S
from paper_1908_08666_gb300 import binding as B

from hhg_gpu import Ctx, Pair, torch_cuda

pytestmark = pytest.mark.gpu


def _params(seed, cout=LN.COUT):
    """Oracle initialisation perturbed so that every layer (biases included) matters."""
    rng = np.random.default_rng(seed)
    Ws, bs = LN.init_params(seed, 2 * cout + 1, cout)
    Ws = [LN.bf16(W + 0.02 * rng.normal(size=W.shape) * (W != 0)) for W in Ws]
    Ws[-1][:, :, cout:] = 0.0
    bs = [0.05 * rng.normal(size=b.shape) for b in bs]
    bs[-1][cout:] = 0.0
    return Ws, bs


def _flat(Ws, bs):
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in zip(Ws, bs)]).astype(np.float32)


def _unflat(p):
    L = 27 * 16 * 16 + 16
    return ([p[l * L:l * L + 6912].reshape(27, 16, 16) for l in range(4)],
            [p[l * L + 6912:(l + 1) * L] for l in range(4)])


@pytest.fixture(scope="module")
def ctx():
    xyz, tets = hi.unit_tet()
    c = Ctx(xyz, tets, 3)
    yield c
    c.close()


def test_param_layout_roundtrip(ctx):
    Ws, bs = _params(1)
    p = _flat(Ws, bs)
    assert p.size == B.hhg_learn_num_params()
    B.hhg_learn_set_params(ctx.h, p)
    q = B.hhg_learn_get_params(ctx.h)
    assert np.array_equal(p, q)
    B.hhg_learn_init(ctx.h, 5)
    q = B.hhg_learn_get_params(ctx.h)
    Wq, bq = _unflat(q)
    assert np.array_equal(LN.bf16(q), q)  # BF16 values
    assert not Wq[0][:, LN.CIN:, :].any() and not Wq[3][:, :, LN.COUT:].any()
    assert all(not b.any() for b in bq)
    assert abs(Wq[1].std() - np.sqrt(2.0 / (27 * 16))) < 0.1 * np.sqrt(2.0 / (27 * 16))


@pytest.mark.parametrize("cout", [3, 4], ids=["elasticity", "stokes"])
@pytest.mark.parametrize("kernel", [0, 1, 2], ids=["mma_sync", "tcgen05", "tma_tcgen05"])
@pytest.mark.parametrize("shape", [(2, 5, 6, 19), (1, 3, 4, 16), (1, 1, 1, 1), (1, 9, 7, 40)])
def test_forward_matches_oracle(ctx, shape, kernel, cout):
    t = ctx.torch
    B.hhg_learn_set_conv_kernel(ctx.h, kernel)
    Bn, D, H, W = shape
    cin = 2 * cout + 1
    rng = np.random.default_rng(sum(shape))
    Ws, bs = _params(2, cout)
    B.hhg_learn_set_params(ctx.h, _flat(Ws, bs))
    x = rng.normal(size=(Bn, D, H, W, cin)).astype(np.float32)
    out = t.empty((Bn, D, H, W, cout), dtype=t.float32, device="cuda")
    B.hhg_learn_forward(ctx.h, ctx.dev(x, t.float32), cin, Bn, D, H, W, out, cout)
    t.cuda.synchronize()
    want, _ = LN.forward(x.astype(np.float64), Ws, bs, cout=cout)
    got = out.cpu().numpy().astype(np.float64)
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-2 * scale
    assert np.linalg.norm(got - want) <= 3e-3 * np.linalg.norm(want)


@pytest.mark.parametrize("cout", [3, 4], ids=["elasticity", "stokes"])
@pytest.mark.parametrize("kernel", [0, 1, 2], ids=["mma_sync", "tcgen05", "tma_tcgen05"])
@pytest.mark.parametrize("shape", [(2, 6, 5, 21), (1, 4, 4, 16)])
def test_gradients_match_oracle(ctx, shape, kernel, cout):
    t = ctx.torch
    B.hhg_learn_set_conv_kernel(ctx.h, kernel)
    Bn, D, H, W = shape
    cin = 2 * cout + 1
    rng = np.random.default_rng(10 + sum(shape))
    Ws, bs = _params(3, cout)
    B.hhg_learn_set_params(ctx.h, _flat(Ws, bs))
    x = rng.normal(size=(Bn, D, H, W, cin)).astype(np.float32)
    tgt = rng.normal(size=(Bn, D, H, W, cout)).astype(np.float32)
    loss, g = B.hhg_learn_loss_grad(ctx.h, ctx.dev(x, t.float32), cin, ctx.dev(tgt, t.float32), Bn, D, H, W, cout)
    wl, dWs, dbs = LN.loss_and_grads(x.astype(np.float64), tgt.astype(np.float64), Ws, bs, cout=cout)
    assert abs(loss - wl) <= 1e-3 * wl
    gW, gb = _unflat(g.astype(np.float64))
    for l in range(4):
        assert np.linalg.norm(gW[l] - dWs[l]) <= 2e-2 * np.linalg.norm(dWs[l]), l
        assert np.linalg.norm(gb[l] - dbs[l]) <= 2e-2 * np.linalg.norm(dbs[l]) + 1e-12, l
    # structural zeros: unused input channels of layer 0, unused outputs of the last layer
    assert not gW[0][:, cin:, :].any() and not gW[3][:, :, cout:].any() and not gb[3][cout:].any()


@pytest.fixture(scope="module")
def cube4():
    p = Pair(hi.kuhn_cube, 4, kfun=hi.young_sine)
    h = p.ctx.h
    B.hhg_mg_setup(h)
    lam = {q: S.lambda_max_DinvA(p.H.A[q], p.H.lv[q].dirichlet) for q in (3, 4)}
    for q in (3, 4):
        B.hhg_set_lambda_max(h, q, lam[q])
    p.lam = lam
    p.vox, p.dims = LN.grid_index(p.H.lv[4].coords, 1.0 / 16)
    yield p
    p.close()


def test_tcgen05_wait_runout_reports_timeout_and_keeps_the_context(ctx):
    """Fault handling without a fault: with the tensor-core convolution's wait for its MMAs
    bounded to zero polls, the wait runs out in every block; each block records the error,
    still waits (with the default bound) for the MMAs it issued before freeing their tensor
    memory, skips its epilogue and returns.  The call fails with HHG_ERR_TIMEOUT and the
    context falls back to kernel 0; with the default bound restored, the tensor-core kernel
    gives the oracle's result again in the same context."""
    t = ctx.torch
    Ws, bs = _params(2, 3)
    B.hhg_learn_set_params(ctx.h, _flat(Ws, bs))
    Bn, D, H, W = 1, 3, 4, 16
    x = np.random.default_rng(7).normal(size=(Bn, D, H, W, 7)).astype(np.float32)
    xd = ctx.dev(x, t.float32)
    out = t.empty((Bn, D, H, W, 3), dtype=t.float32, device="cuda")
    B.hhg_learn_set_conv_kernel(ctx.h, 1)
    B.hhg_learn_set_conv_wait(ctx.h, 0)
    try:
        with pytest.raises(B.HhgError) as ei:
            B.hhg_learn_forward(ctx.h, xd, 7, Bn, D, H, W, out, 3)
        assert ei.value.status == 7 and "timed out" in str(ei.value)
    finally:
        B.hhg_learn_set_conv_wait(ctx.h, -1)
    B.hhg_learn_set_conv_kernel(ctx.h, 1)
    B.hhg_learn_forward(ctx.h, xd, 7, Bn, D, H, W, out, 3)
    t.cuda.synchronize()
    want, _ = LN.forward(x.astype(np.float64), Ws, bs, cout=3)
    got = out.cpu().numpy().astype(np.float64)
    assert np.abs(got - want).max() <= 1e-2 * np.abs(want).max()


def test_grid_of_the_cube(cube4):
    B.hhg_learn_set_conv_kernel(cube4.ctx.h, 0)
    dims, nfree = B.hhg_learn_grid(cube4.ctx.h, 4)
    assert dims == (17, 17, 17) and nfree == 15**3


def test_training_pairs_match_oracle(cube4):
    p = cube4
    t = p.ctx.torch
    h = p.ctx.h
    l = 4
    lv, A = p.H.lv[l], p.H.A[l]
    D, H, W = p.dims
    e0 = np.random.default_rng(4).uniform(-1, 1, size=(D, H, W, 3)).astype(np.float32)
    B.hhg_learn_reserve_pairs(h, l, 4)
    assert B.hhg_learn_collect(h, l, p.ctx.dev(e0, t.float32), 2) == 2
    e = e0[p.vox[:, 0], p.vox[:, 1], p.vox[:, 2]].astype(np.float64)
    e[lv.dirichlet] = 0.0
    vc = lambda r: p.H.vcycle(l, r, np.zeros_like(r), "chebyshev", 2, 2, p.lam)
    k = hi.young_sine(lv.coords)
    for j in range(2):
        X, T, e = LN.training_pair(A, lv.dirichlet, p.vox, p.dims, k, e, vc)
        xg, tg = B.hhg_learn_get_pair(h, j, p.dims)
        assert np.allclose(xg, X[0], rtol=2.0**-7, atol=1e-4 * np.abs(X).max()), j
        assert np.abs(tg - T[0]).max() <= 1e-4 * np.abs(T).max(), j


def test_precondition_matches_oracle(cube4):
    p = cube4
    t = p.ctx.torch
    h = p.ctx.h
    l = 4
    lv, A = p.H.lv[l], p.H.A[l]
    Ws, bs = _params(4)
    B.hhg_learn_set_params(h, _flat(Ws, bs))
    r = hi.node_noise(lv.coords, seed=41)
    r[lv.dirichlet] = 0.0
    rd = p.to_lib(l, r, t.float32)
    z0d = t.empty_like(rd)
    zd = t.empty_like(rd)
    assert B.hhg_learn_precondition(h, l, 0, rd, z0d) == 0.0
    alpha = B.hhg_learn_precondition(h, l, 1, rd, zd)
    v = p.H.vcycle(l, r, np.zeros_like(r), "chebyshev", 2, 2, p.lam)
    z, w_or, c = LN.correction(A, lv.dirichlet, p.vox, p.dims, hi.young_sine(lv.coords), r, v, Ws, bs)
    vg, zg = p.from_lib(l, z0d), p.from_lib(l, zd)
    assert np.abs(vg - v).max() <= 1e-4 * np.abs(v).max()
    assert abs(alpha - w_or) <= 3e-2 * abs(w_or)
    z0, _ = LN._scaled_step(A, lv.dirichlet, r, v)
    bc = z - z0 * (z * z0).sum() / (z0 * z0).sum()  # the part of z off the V-cycle direction
    assert np.abs(zg - z).max() <= 3e-2 * np.abs(bc).max() + 1e-4 * np.abs(z).max()
    st = B.hhg_learn_stats(h, reset=True)
    assert st["applications"] == 1 and st["fallbacks"] == 0 and st["gain_mean"] >= -1e-6


def _coarse_grid(p, lc):
    vox_c, dims_c = LN.grid_index(p.H.lv[lc].coords, 1.0 / 2**lc)
    return vox_c, dims_c, hi.young_sine(p.H.lv[lc].coords)


def test_coarse_mode_pairs_match_oracle(cube4):
    """Coarse-grid mode (network one level below the solve): the pairs live on the level-3
    grid, restricted residual and injected z0 / error."""
    p = cube4
    t = p.ctx.torch
    h = p.ctx.h
    l = 4
    lv, A = p.H.lv[l], p.H.A[l]
    vox_c, dims_c, k_c = _coarse_grid(p, 3)
    D, H, W = p.dims
    e0 = np.random.default_rng(14).uniform(-1, 1, size=(D, H, W, 3)).astype(np.float32)
    B.hhg_learn_set_coarsening(h, 1)
    try:
        B.hhg_learn_reserve_pairs(h, l, 4)
        assert B.hhg_learn_collect(h, l, p.ctx.dev(e0, t.float32), 2) == 2
        e = e0[p.vox[:, 0], p.vox[:, 1], p.vox[:, 2]].astype(np.float64)
        e[lv.dirichlet] = 0.0
        vc = lambda r: p.H.vcycle(l, r, np.zeros_like(r), "chebyshev", 2, 2, p.lam)
        for j in range(2):
            X, T, e = LN.coarse_training_pair(p.H, l, 1, vox_c, dims_c, k_c, e, vc)
            xg, tg = B.hhg_learn_get_pair(h, j, dims_c)
            assert np.allclose(xg, X[0], rtol=2.0**-7, atol=1e-4 * np.abs(X).max()), j
            assert np.abs(tg - T[0]).max() <= 1e-4 * np.abs(T).max(), j
    finally:
        B.hhg_learn_set_coarsening(h, 0)


def test_coarse_mode_precondition_matches_oracle(cube4):
    p = cube4
    t = p.ctx.torch
    h = p.ctx.h
    l = 4
    lv, A = p.H.lv[l], p.H.A[l]
    vox_c, dims_c, k_c = _coarse_grid(p, 3)
    Ws, bs = _params(5)
    B.hhg_learn_set_params(h, _flat(Ws, bs))
    r = hi.node_noise(lv.coords, seed=43)
    r[lv.dirichlet] = 0.0
    rd = p.to_lib(l, r, t.float32)
    zd = t.empty_like(rd)
    B.hhg_learn_set_coarsening(h, 1)
    try:
        alpha = B.hhg_learn_precondition(h, l, 1, rd, zd)
    finally:
        B.hhg_learn_set_coarsening(h, 0)
    v = p.H.vcycle(l, r, np.zeros_like(r), "chebyshev", 2, 2, p.lam)
    z, w_or, c = LN.coarse_correction(p.H, l, 1, vox_c, dims_c, k_c, r, v, Ws, bs)
    assert abs(alpha - w_or) <= 3e-2 * abs(w_or)
    zg = p.from_lib(l, zd)
    z0, _ = LN._scaled_step(A, lv.dirichlet, r, v)
    bc = z - z0 * (z * z0).sum() / (z0 * z0).sum()
    assert np.abs(zg - z).max() <= 3e-2 * np.abs(bc).max() + 1e-4 * np.abs(z).max()


def test_precondition_never_worse_than_the_vcycle(cube4):
    """Energy norm of the error after one application, with and without the network
    (random weights: the line search must keep the step no worse)."""
    p = cube4
    t = p.ctx.torch
    h = p.ctx.h
    l = 4
    lv, A = p.H.lv[l], p.H.A[l]
    B.hhg_learn_init(h, 9)
    for seed in (1, 2, 3):
        e = hi.node_noise(lv.coords, seed=50 + seed)
        e[lv.dirichlet] = 0.0
        r = (A @ e.reshape(-1)).reshape(-1, 3)
        r[lv.dirichlet] = 0.0
        rd = p.to_lib(l, r, t.float32)
        zs = []
        for use in (0, 1):
            zd = t.empty_like(rd)
            B.hhg_learn_precondition(h, l, use, rd, zd)
            d = (e - p.from_lib(l, zd)).reshape(-1)
            zs.append(float(d @ (A @ d)))
        assert zs[1] <= zs[0] * (1 + 1e-5)


def test_learned_solver_reaches_tolerance(cube4):
    p = cube4
    t = p.ctx.torch
    h = p.ctx.h
    l = 4
    lv, A = p.H.lv[l], p.H.A[l]
    B.hhg_learn_init(h, 11)
    f = hi.node_noise(lv.coords, seed=61)
    for method in (B.SOLVE_IR_FCG, B.SOLVE_IR_FCG_LEARNED):
        x = p.to_lib(l, np.zeros_like(f), t.float64)
        rep = B.hhg_solve(h, p.to_lib(l, f, t.float64), x, method=method, level=l, rtol=1e-8, max_iter=20,
                          inner_rtol=1e-3, inner_max_iter=50)
        assert rep["converged"]
        res = np.linalg.norm(S.residual(A, lv.dirichlet, f, p.from_lib(l, x)))
        assert res <= 1.01e-8 * np.linalg.norm(S.residual(A, lv.dirichlet, f, np.zeros_like(f)))


def test_learned_needs_lattice_mesh():
    xyz, tets = hi.skewed_pair()
    c = Ctx(xyz, tets, 3)
    try:
        c.set_k(np.ones(c.U))
        with pytest.raises(B.HhgError) as ei:
            B.hhg_learn_grid(c.h, 3)
        assert ei.value.status == 4
    finally:
        c.close()


def test_training_reduces_the_loss():
    torch_cuda()
    p = Pair(hi.kuhn_cube, 4, kfun=hi.young_sine)
    try:
        t = p.ctx.torch
        h = p.ctx.h
        B.hhg_mg_setup(h)
        dims, _ = B.hhg_learn_grid(h, 4)
        B.hhg_learn_reserve_pairs(h, 4, 8)
        for s in range(4):
            e0 = np.random.default_rng(70 + s).uniform(-1, 1, size=dims + (3,)).astype(np.float32)
            B.hhg_learn_collect(h, 4, p.ctx.dev(e0, t.float32), 2)
        B.hhg_learn_init(h, 1)
        rep = B.hhg_learn_train(h, steps=200, batch=4, crop=12, lr=3e-3, seed=3)
        assert rep["pairs"] == 8
        assert rep["loss_last"] < 0.7 * rep["loss_first"], rep
        # deterministic: the same seed from the same start gives the same parameters
        p1 = B.hhg_learn_get_params(h)
        B.hhg_learn_init(h, 1)
        B.hhg_learn_train(h, steps=200, batch=4, crop=12, lr=3e-3, seed=3)
        assert np.array_equal(p1, B.hhg_learn_get_params(h))
    finally:
        p.close()


def test_trained_network_gains_over_the_plain_vcycle():
    """What training buys: a network trained on level-5 CG error pairs (8 lognormal
    coefficient fields, seeds 100..107) and applied at level 6 to an unseen field (seed 2)
    adds energy reduction on top of the V-cycle and saves flexible-CG iterations against
    the same solver with the V-cycle alone; an untrained network does neither."""
    torch_cuda()
    tr = Ctx(*hi.kuhn_cube(), 5)
    try:
        t = tr.torch
        B.hhg_learn_reserve_pairs(tr.h, 5, 192)
        for s in range(8):
            tr.set_k(hi.sample_grid(hi.lognormal_grid(32, 100 + s), tr.coords_u))
            B.hhg_mg_setup(tr.h)
            for q in range(4):
                f = np.random.default_rng(1000 * s + q).uniform(-1, 1, size=(tr.U, 3))
                f[tr.udir] = 0.0
                B.hhg_learn_collect_cg(tr.h, 5, tr.to_lib(f, t.float32, 3), 6)
        B.hhg_learn_init(tr.h, 1)
        rep = B.hhg_learn_train(tr.h, steps=1500, batch=8, crop=24, lr=2e-3, seed=2)
        assert rep["pairs"] == 192 and rep["loss_last"] < 0.6 * rep["loss_first"], rep
        params = B.hhg_learn_get_params(tr.h)
    finally:
        tr.close()
    ev = Ctx(*hi.kuhn_cube(), 6)
    try:
        t = ev.torch
        ev.set_k(hi.sample_grid(hi.lognormal_grid(64, 2), ev.coords_u))
        B.hhg_mg_setup(ev.h)
        f = hi.node_noise(ev.coords_u, seed=300)
        f[ev.udir] = 0.0
        fd = ev.to_lib(f, t.float64, 3)
        out = {}
        for label, method, p in (("plain", B.SOLVE_IR_FCG, None), ("untrained", B.SOLVE_IR_FCG_LEARNED, "init"),
                                 ("trained", B.SOLVE_IR_FCG_LEARNED, params)):
            if p is not None:
                B.hhg_learn_init(ev.h, 1) if isinstance(p, str) else B.hhg_learn_set_params(ev.h, p)
            x = t.zeros_like(fd)
            B.hhg_learn_stats(ev.h, reset=True)
            r = B.hhg_solve(ev.h, fd, x, method=method, level=6, rtol=1e-8, max_iter=30, inner_rtol=1e-3,
                            inner_max_iter=100)
            out[label] = (r, B.hhg_learn_stats(ev.h))
        assert all(r["converged"] for r, _ in out.values())
        assert out["trained"][1]["gain_mean"] > 0.005 > out["untrained"][1]["gain_mean"], out
        assert out["trained"][0]["inner_iterations"] < out["plain"][0]["inner_iterations"], out
    finally:
        ev.close()


def test_coarse_mode_trained_network_gains():
    """Coarse-grid mode: a network trained on level-5 CG error pairs stored one level down
    (8 lognormal fields) and applied one level below a level-6 solve on an unseen field
    adds energy reduction over the V-cycle that an untrained network does not."""
    torch_cuda()
    tr = Ctx(*hi.kuhn_cube(), 5)
    try:
        t = tr.torch
        B.hhg_learn_set_coarsening(tr.h, 1)
        B.hhg_learn_reserve_pairs(tr.h, 5, 64)
        for s in range(8):
            tr.set_k(hi.sample_grid(hi.lognormal_grid(32, 100 + s), tr.coords_u))
            B.hhg_mg_setup(tr.h)
            for q in range(2):
                f = np.random.default_rng(1000 * s + q).uniform(-1, 1, size=(tr.U, 3))
                f[tr.udir] = 0.0
                B.hhg_learn_collect_cg(tr.h, 5, tr.to_lib(f, t.float32, 3), 4)
        B.hhg_learn_init(tr.h, 1)
        rep = B.hhg_learn_train(tr.h, steps=800, batch=8, crop=16, lr=2e-3, seed=2)
        assert rep["pairs"] == 64 and rep["loss_last"] < 0.8 * rep["loss_first"], rep
        params = B.hhg_learn_get_params(tr.h)
    finally:
        tr.close()
    ev = Ctx(*hi.kuhn_cube(), 6)
    try:
        t = ev.torch
        ev.set_k(hi.sample_grid(hi.lognormal_grid(64, 2), ev.coords_u))
        B.hhg_mg_setup(ev.h)
        B.hhg_learn_set_coarsening(ev.h, 1)
        f = hi.node_noise(ev.coords_u, seed=300)
        f[ev.udir] = 0.0
        fd = ev.to_lib(f, t.float64, 3)
        gains = {}
        for label in ("untrained", "trained"):
            B.hhg_learn_init(ev.h, 1) if label == "untrained" else B.hhg_learn_set_params(ev.h, params)
            x = t.zeros_like(fd)
            B.hhg_learn_stats(ev.h, reset=True)
            r = B.hhg_solve(ev.h, fd, x, method=B.SOLVE_IR_FCG_LEARNED, level=6, rtol=1e-8, max_iter=30,
                            inner_rtol=1e-3, inner_max_iter=100)
            assert r["converged"], r
            gains[label] = B.hhg_learn_stats(ev.h)["gain_mean"]
        assert gains["trained"] > 0.002 and gains["trained"] > gains["untrained"], gains
    finally:
        ev.close()
