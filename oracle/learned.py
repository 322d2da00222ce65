"""Oracle for the learned preconditioner: its convolutional network (plain numpy, FP64 with
BF16 rounding where the GPU stores BF16) and the preconditioner application around it.

Test infrastructure only (see the package docstring).  The network is not part of the
paper; this module defines what the GPU kernels compute so that their forward pass,
gradients, training pairs and preconditioner application can be checked.

Network: 4 layers of 3x3x3 convolutions on a channels-last grid (z, y, x, c) with zero
padding, 16 hidden channels, ReLU after the first three layers:

    a_0 = bf16(input)   (CIN = 7 channels, padded with zeros to 16)
    z_l = conv(a_{l-1}, W_l) + b_l,   a_l = bf16(relu(z_l))  (l = 1..3),   out = z_4[..., :3]

conv(a, W)[v, o] = sum_{t, i} a[v + off(t), i] W[t, i, o], tap t = (dz+1)*9 + (dy+1)*3 + (dx+1),
offsets dz, dy, dx in {-1, 0, 1}.  Weights are BF16 values (W[t, i, o], 27 x 16 x 16),
biases FP32.  Loss: mean over the batch, voxels and the 3 output channels of
(out - target)^2.

Preconditioner application for a residual r (vectors node-major (N, 3), FP64):
v = V-cycle(r), z0 = a0 v with a0 = (v, r) / (v, A v), r1 = r - A z0, D = point
diagonal, s = RMS of D z0 over the free DoFs; input features per grid voxel of a free
node: r1/s, D z0/s, log k - mean log k (the last also at Dirichlet nodes); correction
c = s out / D on free nodes; z = a z0 + b c with (a, b) minimising the energy norm
(e - z, A (e - z)) of the error e = A^-1 r (the 2x2 normal equations need only r).
Training pair from an error e: z0 as above for r = A e, e1 = e - z0, r1 = A e1,
target D e1 / s.

Coarse-grid mode (``coarse_*``, elasticity): the network runs q levels below the solve's
level l.  Its inputs are r1 restricted q times (P^T with Dirichlet rows zeroed, as in the
V-cycle) and z0 injected (coarse nodes are fine nodes), with that level's point diagonal
and log k; its correction s out / D is prolongated q times (P) and then combined as
above.  Its training target is D e1 / s with e1 injected to the coarse level.

Stokes (``stokes_*``; vectors (N, 4): velocity, then pressure; K the saddle operator with
velocity-Dirichlet identity rows, v = one inexact Uzawa V-cycle of the residual): the
same with 4 components, CIN = 9 input channels (r1/s, D z0/s, log mu) and 4 outputs,
where D is the velocity point diagonal and, for the pressure, the Schur surrogate
m_i / mu_i + (-C)_ii; the velocity channels and targets are scaled by s, the RMS of
D z0 over the free velocity DoFs, the pressure ones by s_p, the RMS of D z0 over the
pressures (the two diagonals differ by orders of magnitude); z0 = v unscaled (the Uzawa cycle is a convergent iteration by itself); and, K
being indefinite, the residual norm replaces the energy norm: (a, b) minimise
|r - K (a z0 + b c)|_2.  The training error e1 = e - z0 has its pressure shifted to zero
mass-weighted mean.
"""

from __future__ import annotations

import numpy as np

C = 16
NLAYERS = 4
CIN, COUT = 7, 3


def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    u = ((u + rounding) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def offsets():
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def conv(a, W):
    """a: (B, D, H, X, Cin), W: (27, Cin, Cout) -> (B, D, H, X, Cout), zero padding."""
    B, D, H, X, _ = a.shape
    p = np.pad(a, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    out = np.zeros((B, D, H, X, W.shape[2]))
    for t, (dz, dy, dx) in enumerate(offsets()):
        sl = p[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + X, :]
        out += sl @ W[t]
    return out


def conv_transpose_input(g, W):
    """Gradient of conv w.r.t. its input: sum over taps of g shifted back times W^T."""
    B, D, H, X, _ = g.shape
    p = np.pad(g, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    out = np.zeros((B, D, H, X, W.shape[1]))
    for t, (dz, dy, dx) in enumerate(offsets()):
        sl = p[:, 1 - dz:1 - dz + D, 1 - dy:1 - dy + H, 1 - dx:1 - dx + X, :]
        out += sl @ W[t].T
    return out


def conv_weight_grad(a, g):
    """dL/dW[t, i, o] = sum_v a[v + off(t), i] g[v, o]."""
    B, D, H, X, Cin = a.shape
    p = np.pad(a, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    dW = np.zeros((27, Cin, g.shape[-1]))
    for t, (dz, dy, dx) in enumerate(offsets()):
        sl = p[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + X, :]
        dW[t] = np.einsum("bzyxi,bzyxo->io", sl, g)
    return dW


def init_params(seed, cin0=CIN, cout=COUT):
    """He-style initialisation (BF16-rounded weights, zero biases)."""
    rng = np.random.default_rng(seed)
    Ws, bs = [], []
    for l in range(NLAYERS):
        cin = cin0 if l == 0 else C
        W = np.zeros((27, C, C))
        W[:, :cin, :] = rng.normal(size=(27, cin, C)) * np.sqrt(2.0 / (27 * cin))
        if l == NLAYERS - 1:
            W[:, :, cout:] = 0.0
            W *= 0.1
        Ws.append(bf16(W))
        bs.append(np.zeros(C))
    return Ws, bs


def forward(x, Ws, bs, round_bf16=True, cout=COUT):
    """x: (B, D, H, X, cin <= 16) -> (out (B, D, H, X, cout), activations)."""
    rnd = bf16 if round_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    a = np.zeros(x.shape[:4] + (C,))
    a[..., :x.shape[-1]] = rnd(x)
    acts = [a]
    for l in range(NLAYERS):
        z = conv(acts[-1], Ws[l]) + bs[l]
        if l < NLAYERS - 1:
            acts.append(rnd(np.maximum(z, 0.0)))
        else:
            out = z
    return out[..., :cout], acts


def loss_and_grads(x, target, Ws, bs, round_bf16=True, cout=COUT):
    """MSE loss and its gradients w.r.t. all weights and biases (the BF16 rounding of the
    activations is treated as identity in the backward pass, as on the GPU)."""
    out, acts = forward(x, Ws, bs, round_bf16, cout)
    n = out.size
    diff = out - target
    loss = float((diff**2).sum() / n)
    g = np.zeros(out.shape[:4] + (C,))
    g[..., :cout] = 2.0 * diff / n
    dWs, dbs = [None] * NLAYERS, [None] * NLAYERS
    for l in reversed(range(NLAYERS)):
        dWs[l] = conv_weight_grad(acts[l], g)
        dbs[l] = g.sum(axis=(0, 1, 2, 3))
        if l > 0:
            g = conv_transpose_input(g, Ws[l]) * (acts[l] > 0)
    return loss, dWs, dbs


def grid_index(coords, h):
    """(z, y, x) voxel of every node of an axis-aligned lattice with spacing h and dims."""
    lo = coords.min(axis=0)
    ijk = np.rint((coords - lo) / h).astype(np.int64)
    assert np.allclose(lo + ijk * h, coords, atol=1e-9)
    dims = tuple(int(v) for v in ijk.max(axis=0)[::-1] + 1)  # (D, H, W) = (nz, ny, nx)
    return ijk[:, ::-1], dims


def _dot_free(a, b, dirichlet):
    fr = ~np.asarray(dirichlet)
    return float((a[fr] * b[fr]).sum())


def features(vox, dims, dirichlet, k, r1, z0, D):
    """Input grid (1, D, H, W, CIN) and the scale s (see the module docstring)."""
    fr = ~np.asarray(dirichlet)
    s2 = ((D[fr] * z0[fr]) ** 2).sum() / (3.0 * max(fr.sum(), 1))
    s = np.sqrt(s2) if s2 > 0 else 1.0
    X = np.zeros((1,) + dims + (CIN,))
    lk = np.log(k)
    lk = lk - lk.mean()
    X[0, vox[:, 0], vox[:, 1], vox[:, 2], 6] = lk
    f = np.zeros((len(k), 6))
    f[:, :3] = r1 / s
    f[:, 3:] = D * z0 / s
    f[~fr] = 0.0
    X[0, vox[fr, 0], vox[fr, 1], vox[fr, 2], :6] = f[fr]
    return X, s


def _scaled_step(A, dirichlet, r, v):
    """Energy-optimal multiple a0 v of the V-cycle output v for the residual r, and A a0 v."""
    Av = (A @ v.reshape(-1)).reshape(-1, 3)
    den = _dot_free(v, Av, dirichlet)
    a0 = _dot_free(v, r, dirichlet) / den if den > 0 else 1.0
    return a0 * v, a0 * Av


def _combine(A, dirichlet, r, z0, Az0, c):
    """z = a z0 + b c minimising the energy norm of the error A^-1 r - z, and b / a."""
    Ac = (A @ c.reshape(-1)).reshape(-1, 3)
    M = np.array([[_dot_free(z0, Az0, dirichlet), _dot_free(c, Az0, dirichlet)],
                  [_dot_free(c, Az0, dirichlet), _dot_free(c, Ac, dirichlet)]])
    rhs = np.array([_dot_free(z0, r, dirichlet), _dot_free(c, r, dirichlet)])
    a, b = np.linalg.solve(M, rhs)
    return a * z0 + b * c, b / a


def correction(A, dirichlet, vox, dims, k, r, v, Ws, bs):
    """(z, b/a, c): the learned preconditioner's output for residual r given v = V-cycle(r):
    z0 = a0 v, c from the network, z = a z0 + b c minimising the energy norm of the error
    over span{z0, c}."""
    fr = ~np.asarray(dirichlet)
    Dg = A.diagonal().reshape(-1, 3).copy()
    Dg[~fr] = 1.0
    z0, Az0 = _scaled_step(A, dirichlet, r, v)
    r1 = r - Az0
    r1[~fr] = 0.0
    X, s = features(vox, dims, dirichlet, k, r1, z0, Dg)
    out, _ = forward(X, Ws, bs)
    c = s * out[0, vox[:, 0], vox[:, 1], vox[:, 2], :] / Dg
    c[~fr] = 0.0
    z, w = _combine(A, dirichlet, r, z0, Az0, c)
    return z, w, c


def _inject_index(H, lev):
    """Index in level lev of every node of level lev - 1 (coarse nodes are fine nodes)."""
    key = lambda c: tuple(np.rint(np.asarray(c) * 2.0**(lev + 2)).astype(np.int64))
    fine = {key(c): i for i, c in enumerate(H.lv[lev].coords)}
    return np.array([fine[key(c)] for c in H.lv[lev - 1].coords], dtype=np.int64)


def coarse_inputs(H, l, q, r1, z0, e1=None):
    """r1 restricted and z0, e1 injected from level l to level l - q (H: a multigrid
    hierarchy with levels, operators A and prolongations P)."""
    from .solvers import restrict

    for lev in range(l, l - q, -1):
        idx = _inject_index(H, lev)
        r1 = restrict(H.P[lev], r1, H.lv[lev].dirichlet, H.lv[lev - 1].dirichlet)
        z0 = np.asarray(z0)[idx]
        e1 = None if e1 is None else np.asarray(e1)[idx]
    return r1, z0, e1


def _point_diag(H, lev):
    D = H.A[lev].diagonal().reshape(-1, 3).copy()
    D[H.lv[lev].dirichlet] = 1.0
    return D


def coarse_correction(H, l, q, vox_c, dims_c, k_c, r, v, Ws, bs):
    """(z, b/a, c) of the coarse-grid mode for residual r given v = V-cycle(r) at level l;
    vox_c, dims_c, k_c: the node grid and coefficient of level l - q."""
    A, d = H.A[l], H.lv[l].dirichlet
    lc = l - q
    dc = H.lv[lc].dirichlet
    z0, Az0 = _scaled_step(A, d, r, v)
    r1 = r - Az0
    r1[d] = 0.0
    r1c, z0c, _ = coarse_inputs(H, l, q, r1, z0)
    Dc = _point_diag(H, lc)
    X, s = features(vox_c, dims_c, dc, k_c, r1c, z0c, Dc)
    out, _ = forward(X, Ws, bs)
    c = s * out[0, vox_c[:, 0], vox_c[:, 1], vox_c[:, 2], :] / Dc
    c[dc] = 0.0
    for lev in range(lc + 1, l + 1):
        c = H.P[lev] @ c
    z, w = _combine(A, d, r, z0, Az0, c)
    return z, w, c


def coarse_training_pair(H, l, q, vox_c, dims_c, k_c, e, vcycle):
    """(inputs, target, e1) of one multigrid step from the error e at level l, with the
    pair on the node grid of level l - q."""
    A, d = H.A[l], H.lv[l].dirichlet
    lc = l - q
    dc = H.lv[lc].dirichlet
    r = (A @ e.reshape(-1)).reshape(-1, 3)
    r[d] = 0.0
    z0, _ = _scaled_step(A, d, r, vcycle(r))
    e1 = e - z0
    r1 = (A @ e1.reshape(-1)).reshape(-1, 3)
    r1[d] = 0.0
    r1c, z0c, e1c = coarse_inputs(H, l, q, r1, z0, e1)
    Dc = _point_diag(H, lc)
    X, s = features(vox_c, dims_c, dc, k_c, r1c, z0c, Dc)
    T = np.zeros((1,) + dims_c + (COUT,))
    fr = ~np.asarray(dc)
    T[0, vox_c[fr, 0], vox_c[fr, 1], vox_c[fr, 2], :] = (Dc * e1c / s)[fr]
    return X, T, e1


def training_pair(A, dirichlet, vox, dims, k, e, vcycle):
    """(inputs (1, D, H, W, CIN), target (1, D, H, W, 3), e1) of one multigrid step from error e."""
    fr = ~np.asarray(dirichlet)
    Dg = A.diagonal().reshape(-1, 3).copy()
    Dg[~fr] = 1.0
    r = (A @ e.reshape(-1)).reshape(-1, 3)
    r[~fr] = 0.0
    z0, _ = _scaled_step(A, dirichlet, r, vcycle(r))
    e1 = e - z0
    r1 = (A @ e1.reshape(-1)).reshape(-1, 3)
    r1[~fr] = 0.0
    X, s = features(vox, dims, dirichlet, k, r1, z0, Dg)
    T = np.zeros((1,) + dims + (COUT,))
    T[0, vox[fr, 0], vox[fr, 1], vox[fr, 2], :] = (Dg * e1 / s)[fr]
    return X, T, e1


# ------------------------------------------------------------------------------ Stokes

STOKES_CIN, STOKES_COUT = 9, 4


def stokes_diag(H, l):
    """(N, 4) diagonal D of the features: velocity point diagonal of A (1 on Dirichlet
    rows), then the Schur surrogate."""
    N = H.lv[l].num_nodes
    D = np.empty((N, 4))
    D[:, :3] = H.A[l].diagonal().reshape(N, 3)
    D[H.lv[l].dirichlet, :3] = 1.0
    D[:, 3] = H.s[l]
    return D


def stokes_features(vox, dims, dirichlet, k, r1, z0, D):
    """Input grid (1, D, H, W, 9) and the per-component scales (N, 4) (s on the velocity
    components, s_p on the pressure) for (N, 4) fields r1, z0, D."""
    d = np.asarray(dirichlet)
    on = np.ones(z0.shape, dtype=bool)
    on[d, :3] = False
    w = D * z0

    def rms(v):
        s2 = (v**2).sum() / max(v.size, 1)
        return np.sqrt(s2) if s2 > 0 else 1.0

    sc = np.empty(z0.shape)
    sc[:, :3] = rms(w[:, :3][on[:, :3]])
    sc[:, 3] = rms(w[:, 3])
    X = np.zeros((1,) + dims + (STOKES_CIN,))
    lk = np.log(k)
    X[0, vox[:, 0], vox[:, 1], vox[:, 2], 8] = lk - lk.mean()
    f = np.zeros((len(k), 8))
    f[:, :4] = np.where(on, r1 / sc, 0.0)
    f[:, 4:] = np.where(on, w / sc, 0.0)
    X[0, vox[:, 0], vox[:, 1], vox[:, 2], :8] = f
    return X, sc


def _stokes_step(H, l, r, v):
    """The Stokes multigrid step z0 = v (unscaled) and K z0."""
    return np.array(v, dtype=np.float64), H.apply(l, v)


def stokes_correction(H, l, vox, dims, k, r, v, Ws, bs):
    """(z, b/a, c) of the Stokes learned preconditioner for residual r given v = MG(r):
    z0 = a0 v, c from the network, z = a z0 + b c minimising |r - K z|_2."""
    d = H.lv[l].dirichlet
    D = stokes_diag(H, l)
    z0, Kz0 = _stokes_step(H, l, r, v)
    r1 = r - Kz0
    r1[d, :3] = 0.0
    X, s = stokes_features(vox, dims, d, k, r1, z0, D)
    out, _ = forward(X, Ws, bs, cout=STOKES_COUT)
    c = s * out[0, vox[:, 0], vox[:, 1], vox[:, 2], :] / D
    c[d, :3] = 0.0
    Kc = H.apply(l, c)
    M = np.array([[H.dot(l, Kz0, Kz0), H.dot(l, Kc, Kz0)], [H.dot(l, Kc, Kz0), H.dot(l, Kc, Kc)]])
    rhs = np.array([H.dot(l, Kz0, r), H.dot(l, Kc, r)])
    a, b = np.linalg.solve(M, rhs)
    return a * z0 + b * c, b / a, c


def stokes_training_pair(H, l, vox, dims, k, e, mg):
    """(inputs (1, D, H, W, 9), target (1, D, H, W, 4), e1) of one multigrid step from the
    error e ((N, 4), zero velocity on Dirichlet nodes); mg(r) = one V-cycle from zero."""
    d = H.lv[l].dirichlet
    D = stokes_diag(H, l)
    r = H.residual(l, np.zeros_like(e), -e)  # K e with zero velocity-Dirichlet rows
    z0, _ = _stokes_step(H, l, r, mg(r))
    e1 = H.project_pressure(l, e - z0)
    r1 = H.residual(l, np.zeros_like(e1), -e1)
    X, s = stokes_features(vox, dims, d, k, r1, z0, D)
    on = np.ones(e.shape, dtype=bool)
    on[d, :3] = False
    T = np.zeros((1,) + dims + (STOKES_COUT,))
    T[0, vox[:, 0], vox[:, 1], vox[:, 2], :] = np.where(on, D * e1 / s, 0.0)
    return X, T, e1
