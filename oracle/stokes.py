"""Oracle for the stabilised P1-P1 generalised Stokes operator of Sec. 5.2.

Test infrastructure only (see the package docstring).

    K = [[A(mu), B^T], [B, C]],
    A(mu): the physical-scaling operator of a(u, v) = (2 mu eps(u), eps(v)) (Sec. 2),
    B = -(div u, q),  C = c_l(p, q) = -(h^2/12) (grad p, grad q)   (Sec. 5.2),

with h the mesh size of the level; here h = (6 |T|)^{1/3} / n per macro (the lattice
spacing 1/n on the Kuhn cube).  Unknown ordering: velocity node-major (3N), then the
pressure (N).  Velocity-Dirichlet rows are identity rows; pressure rows are all free.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem
from . import operators as op
from .mesh import Level, MacroMesh


def macro_h(mm: MacroMesh, lv: Level):
    """Stabilisation length per element: (6 |T|)^{1/3} / n of its macro."""
    X = mm.xyz[mm.tets]
    _, volT = fem.p1_geometry(X)
    return (np.cbrt(6.0 * volT) / lv.n)[lv.elem_macro]


def divergence_matrix(lv: Level):
    """B (N x 3N): B[i, 3j+l] = -int phi_i d_l phi_j."""
    Bd = fem.element_divergence(lv.coords[lv.elems])  # (E, a, b, l)
    E = lv.elems.shape[0]
    rows = np.repeat(lv.elems[:, :, None, None], 4, axis=2).repeat(3, axis=3)
    cols = 3 * np.repeat(lv.elems[:, None, :, None], 4, axis=1).repeat(3, axis=3) + np.arange(3)[None, None, None, :]
    N = lv.num_nodes
    return sp.coo_matrix((Bd.reshape(-1), (rows.reshape(-1), cols.reshape(-1))), shape=(N, 3 * N)).tocsr()


def stabilisation_matrix(mm: MacroMesh, lv: Level):
    """C (N x N) = -(h^2/12) (grad p, grad q)."""
    Lap = fem.element_laplace(lv.coords[lv.elems])
    h = macro_h(mm, lv)
    vals = -(h**2 / 12.0)[:, None, None] * Lap
    rows = np.repeat(lv.elems, 4, axis=1).reshape(-1)
    cols = np.tile(lv.elems, (1, 4)).reshape(-1)
    N = lv.num_nodes
    return sp.coo_matrix((vals.reshape(-1), (rows, cols)), shape=(N, N)).tocsr()


def lumped_mass(lv: Level):
    M = fem.element_mass(lv.coords[lv.elems])
    m = np.zeros(lv.num_nodes)
    np.add.at(m, lv.elems.reshape(-1), M.sum(axis=2).reshape(-1))
    return m


def stokes_operator(mm: MacroMesh, lv: Level, mu, variant="physical", khat="patch", iface="symmetric"):
    """(K with Dirichlet velocity rows, K without them)."""
    K_el = fem.element_stiffness(lv.coords[lv.elems], 2.0, 0.0)
    A = op.scaled_operator(lv, K_el, mu, variant, khat=khat, iface=iface)
    B = divergence_matrix(lv)
    C = stabilisation_matrix(mm, lv)
    K = sp.bmat([[A, B.T], [B, C]]).tocsr()
    N = lv.num_nodes
    d = np.zeros(4 * N, dtype=bool)
    dn = np.nonzero(lv.dirichlet)[0]
    for m in range(3):
        d[3 * dn + m] = True
    keep = sp.diags((~d).astype(np.float64))
    Kbc = (keep @ K + sp.diags(d.astype(np.float64))).tocsr()
    return Kbc, K


def pack(u, p):
    return np.concatenate([np.asarray(u).reshape(-1), np.asarray(p).reshape(-1)])


def unpack(x, N):
    return x[:3 * N].reshape(N, 3), x[3 * N:]


def residual(Kbc, dirichlet, f, x):
    """f - K x with 0 on velocity-Dirichlet rows."""
    r = np.asarray(f) - Kbc @ np.asarray(x)
    N = len(dirichlet)
    ru = r[:3 * N].reshape(N, 3)
    ru[np.asarray(dirichlet)] = 0.0
    return r
