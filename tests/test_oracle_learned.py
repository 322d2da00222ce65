"""Pins of the conv-net oracle used to check the learned preconditioner's kernels (no GPU)."""

import numpy as np

from oracle import learned as LN


def test_delta_kernel_is_a_shift():
    rng = np.random.default_rng(0)
    a = rng.normal(size=(1, 4, 5, 6, 2))
    W = np.zeros((27, 2, 2))
    t = LN.offsets().index((1, 0, -1))
    W[t] = np.eye(2)
    out = LN.conv(a, W)
    want = np.zeros_like(a)
    want[:, :-1, :, 1:, :] = a[:, 1:, :, :-1, :]
    assert np.array_equal(out, want)


def test_transpose_is_adjoint():
    rng = np.random.default_rng(1)
    a = rng.normal(size=(2, 5, 4, 6, 3))
    g = rng.normal(size=(2, 5, 4, 6, 2))
    W = rng.normal(size=(27, 3, 2))
    lhs = (LN.conv(a, W) * g).sum()
    rhs = (a * LN.conv_transpose_input(g, W)).sum()
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    dW = LN.conv_weight_grad(a, g)
    eps = rng.normal(size=W.shape)
    assert abs((dW * eps).sum() - (LN.conv(a, eps) * g).sum()) < 1e-10 * abs((dW * eps).sum())


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 4, 4, 5, 4))
    tgt = rng.normal(size=(2, 4, 4, 5, 3))
    Ws, bs = LN.init_params(3)
    Ws = [W + 0.05 * rng.normal(size=W.shape) for W in Ws]
    bs = [0.1 * rng.normal(size=b.shape) for b in bs]
    loss, dWs, dbs = LN.loss_and_grads(x, tgt, Ws, bs, round_bf16=False)
    h = 1e-6
    for l in range(LN.NLAYERS):
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in Ws[l].shape)
            if l == 0 and idx[1] >= LN.CIN:
                continue
            Wp = [W.copy() for W in Ws]
            Wp[l][idx] += h
            Wm = [W.copy() for W in Ws]
            Wm[l][idx] -= h
            fd = (LN.loss_and_grads(x, tgt, Wp, bs, False)[0] - LN.loss_and_grads(x, tgt, Wm, bs, False)[0]) / (2 * h)
            assert abs(fd - dWs[l][idx]) <= 1e-6 * max(1.0, abs(fd)), (l, idx, fd, dWs[l][idx])
        o = int(rng.integers(0, 3 if l == LN.NLAYERS - 1 else LN.C))
        bp = [b.copy() for b in bs]
        bp[l][o] += h
        bm = [b.copy() for b in bs]
        bm[l][o] -= h
        fd = (LN.loss_and_grads(x, tgt, Ws, bp, False)[0] - LN.loss_and_grads(x, tgt, Ws, bm, False)[0]) / (2 * h)
        assert abs(fd - dbs[l][o]) <= 1e-6 * max(1.0, abs(fd))


def test_bf16_rounding():
    v = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 65504.0])
    r = LN.bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125
    assert abs(r[3] + 3.140625) < 1e-12
