"""Learned preconditioner for Stokes on the GPU against the oracle: the inexact Uzawa
V-cycle it builds on, its training pairs, one application with a random network, the
residual-norm guarantee, and the flexible-GCR solvers with and without the network.

Tolerances as for elasticity: FP32 multigrid quantities to 1e-4 of their largest
magnitude, BF16 features to 2^-7 relative, the network's combination weight and the
part of z along the network's correction to 3e-2 (BF16 network, FP32 inner products)."""

import numpy as np
import pytest

import hhg_inputs as hi
from oracle import learned as LN, mesh, solvers as S, stokes as ST
from paper_1908_08666_gb300 import binding as B

from hhg_gpu import Ctx, torch_cuda

pytestmark = pytest.mark.gpu

LEVEL = 4


def _mu(c):
    return hi.viscosity_sphere(c, mu_in=1.0, mu_out=10.0, radius=0.3, width=0.1)


class StokesPair:
    def __init__(self, level):
        torch_cuda()
        xyz, tets = hi.kuhn_cube()
        self.H = ST.UzawaHierarchy(mesh.MacroMesh.build(xyz, tets), list(range(2, level + 1)), _mu)
        self.lam = {q: S.lambda_max_DinvA(self.H.A[q], self.H.lv[q].dirichlet) for q in range(3, level + 1)}
        self.ctx = Ctx(xyz, tets, level, dict(kind=B.STOKES))
        self.ctx.set_k(_mu(self.ctx.coords_u))
        B.hhg_mg_setup(self.ctx.h)
        for q, v in self.lam.items():
            B.hhg_set_lambda_max(self.ctx.h, q, v)
        self.level = level
        self.perm = mesh.match_nodes(self.H.lv[level].coords, self.ctx.coords_u)
        self.vox, self.dims = LN.grid_index(self.H.lv[level].coords, 1.0 / 2**level)
        self.k = _mu(self.H.lv[level].coords)

    def to_lib(self, x4, dtype):
        u = np.empty_like(x4)
        u[self.perm] = x4
        return self.ctx.to_lib(u, dtype, 4)

    def from_lib(self, field):
        return self.ctx.from_lib(field, 4)[self.perm]

    def noise(self, seed):
        lv = self.H.lv[self.level]
        x = np.zeros((lv.num_nodes, 4))
        x[:, :3] = hi.node_noise(lv.coords, seed)
        x[:, 3] = hi.node_noise(lv.coords, seed + 1, comps=1).reshape(-1)
        x[lv.dirichlet, :3] = 0.0
        return x

    def mg(self, r):
        return self.H.vcycle(self.level, r, np.zeros_like(r), self.lam, self.level)

    def close(self):
        self.ctx.close()


@pytest.fixture(scope="module")
def sp4():
    p = StokesPair(LEVEL)
    yield p
    p.close()


def _random_net(seed):
    rng = np.random.default_rng(seed)
    Ws, bs = LN.init_params(seed, LN.STOKES_CIN, LN.STOKES_COUT)
    Ws = [LN.bf16(W + 0.02 * rng.normal(size=W.shape) * (W != 0)) for W in Ws]
    bs = [0.05 * rng.normal(size=b.shape) for b in bs]
    bs[-1][LN.STOKES_COUT:] = 0.0
    flat = np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in zip(Ws, bs)]).astype(np.float32)
    return Ws, bs, flat


def test_channels(sp4):
    assert B.hhg_learn_channels(sp4.ctx.h) == (9, 4)


def test_uzawa_vcycle_matches_oracle(sp4):
    p = sp4
    t = p.ctx.torch
    r = p.noise(3)
    rd = p.to_lib(r, t.float32)
    zd = t.empty_like(rd)
    assert B.hhg_learn_precondition(p.ctx.h, p.level, 0, rd, zd) == 0.0
    want = p.mg(r)
    got = p.from_lib(zd)
    assert np.abs(got[:, :3] - want[:, :3]).max() <= 1e-4 * np.abs(want[:, :3]).max()
    assert np.abs(got[:, 3] - want[:, 3]).max() <= 1e-4 * np.abs(want[:, 3]).max()


def test_stokes_training_pairs_match_oracle(sp4):
    p = sp4
    t = p.ctx.torch
    h = p.ctx.h
    D, H, W = p.dims
    e0 = np.random.default_rng(4).uniform(-1, 1, size=(D, H, W, 4)).astype(np.float32)
    B.hhg_learn_reserve_pairs(h, p.level, 4)
    assert B.hhg_learn_collect(h, p.level, p.ctx.dev(e0, t.float32), 2) == 2
    e = e0[p.vox[:, 0], p.vox[:, 1], p.vox[:, 2]].astype(np.float64)
    e[p.H.lv[p.level].dirichlet, :3] = 0.0
    for j in range(2):
        X, T, e = LN.stokes_training_pair(p.H, p.level, p.vox, p.dims, p.k, e, p.mg)
        xg, tg = B.hhg_learn_get_pair(h, j, p.dims, nc=4)
        assert np.allclose(xg, X[0], rtol=2.0**-7, atol=1e-4 * np.abs(X).max()), j
        assert np.abs(tg - T[0]).max() <= 1e-4 * np.abs(T).max(), j


def test_stokes_precondition_matches_oracle(sp4):
    p = sp4
    t = p.ctx.torch
    h = p.ctx.h
    Ws, bs, flat = _random_net(4)
    B.hhg_learn_set_params(h, flat)
    r = p.noise(41)
    rd = p.to_lib(r, t.float32)
    zd = t.empty_like(rd)
    B.hhg_learn_stats(h, reset=True)
    alpha = B.hhg_learn_precondition(h, p.level, 1, rd, zd)
    v = p.mg(r)
    z, w_or, c = LN.stokes_correction(p.H, p.level, p.vox, p.dims, p.k, r, v, Ws, bs)
    assert abs(alpha - w_or) <= 3e-2 * abs(w_or)
    zg = p.from_lib(zd)
    z0, _ = LN._stokes_step(p.H, p.level, r, v)
    bc = z - z0 * (z * z0).sum() / (z0 * z0).sum()  # the part of z off the multigrid direction
    assert np.abs(zg - z).max() <= 3e-2 * np.abs(bc).max() + 1e-4 * np.abs(z).max()
    st = B.hhg_learn_stats(h, reset=True)
    assert st["applications"] == 1 and st["fallbacks"] == 0 and st["gain_mean"] >= -1e-6


def test_stokes_precondition_never_worse_than_the_cycle(sp4):
    """Residual norm after one application, with and without the network (initial
    weights: the least-squares combination must keep the step no worse)."""
    p = sp4
    t = p.ctx.torch
    h = p.ctx.h
    l = p.level
    B.hhg_learn_init(h, 9)
    for seed in (1, 2, 3):
        r = p.noise(50 + 2 * seed)
        rd = p.to_lib(r, t.float32)
        norms = []
        for use in (0, 1):
            zd = t.empty_like(rd)
            B.hhg_learn_precondition(h, l, use, rd, zd)
            rr = p.H.residual(l, r, p.from_lib(zd))
            norms.append(np.sqrt(p.H.dot(l, rr, rr)))
        assert norms[1] <= norms[0] * (1 + 1e-5)


@pytest.mark.parametrize("method", [B.SOLVE_STOKES_IR_FGCR, B.SOLVE_STOKES_IR_FGCR_LEARNED], ids=["fgcr", "learned"])
def test_stokes_fgcr_solvers_reach_tolerance(sp4, method):
    p = sp4
    t = p.ctx.torch
    h = p.ctx.h
    l = p.level
    B.hhg_learn_init(h, 11)
    f = p.noise(61)
    f[:, 3] -= f[:, 3].mean()  # consistent with the constant-pressure kernel
    x = p.to_lib(np.zeros_like(f), t.float64)
    rep = B.hhg_solve(h, p.to_lib(f, t.float64), x, method=method, level=l, rtol=1e-8, max_iter=20, inner_rtol=1e-3,
                      inner_max_iter=60)
    assert rep["converged"], rep
    xg = p.from_lib(x)
    res = p.H.residual(l, f, xg)
    assert np.sqrt(p.H.dot(l, res, res)) <= 1.01e-8 * np.sqrt(p.H.dot(l, f, f)), rep
    assert abs((p.H.m[l] * xg[:, 3]).sum()) <= 1e-10 * np.abs(xg[:, 3]).sum()


def test_stokes_training_reduces_the_loss(sp4):
    p = sp4
    t = p.ctx.torch
    h = p.ctx.h
    B.hhg_learn_reserve_pairs(h, p.level, 16)
    for s in range(4):
        f = p.noise(80 + 2 * s)
        f[:, 3] -= f[:, 3].mean()
        B.hhg_learn_collect_cg(h, p.level, p.to_lib(f, t.float32), 4)
    B.hhg_learn_init(h, 1)
    rep = B.hhg_learn_train(h, steps=200, batch=4, crop=12, lr=3e-3, seed=3)
    assert rep["pairs"] == 16
    assert rep["loss_last"] < 0.8 * rep["loss_first"], rep
