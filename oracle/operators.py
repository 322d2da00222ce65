"""Oracle global operators, built from the definitions of Sec. 2 as sparse FP64 matrices.

Test infrastructure only (see the package docstring).

Matrices act on node-major vectors: DoF 3*i+m is component m of node i.
Row = test function, column = trial function (see ``fem``).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem
from .mesh import EDGES_OF_TET, Level, MacroMesh

PAIRS = tuple((a, b) for a in range(4) for b in range(4) if a != b)


def element_coords(mm: MacroMesh, lv: Level):
    return lv.coords[lv.elems]


def kbar(lv: Level, k):
    """Element mean of the nodal coefficient, eq. (nodalquad)."""
    return np.asarray(k, dtype=np.float64)[lv.elems].mean(axis=1)


def _blocks_to_csr(rows, cols, blocks, N):
    """rows/cols: (P,) node ids, blocks: (P, 3, 3) [m, l] -> (3N x 3N) CSR, duplicates summed."""
    m = np.arange(3)
    R = (3 * rows[:, None, None] + m[None, :, None]).repeat(3, axis=2)
    C = (3 * cols[:, None, None] + m[None, None, :]).repeat(3, axis=1)
    A = sp.coo_matrix((blocks.reshape(-1), (R.reshape(-1), C.reshape(-1))), shape=(3 * N, 3 * N))
    return A.tocsr()


def nodal_integration(lv: Level, Kel, k):
    """a_h: sum over elements of kbar^t times the element stiffness, eq. (nodalintegration)."""
    kb = kbar(lv, k)
    rows = np.repeat(lv.elems, 4, axis=1).reshape(-1)
    cols = np.tile(lv.elems, (1, 4)).reshape(-1)
    blocks = (kb[:, None, None, None, None] * Kel).reshape(-1, 3, 3)
    return _blocks_to_csr(rows, cols, blocks, lv.num_nodes)


def _reflected_elements(lv: Level, E_idx, a, b):
    """Element t^m: point reflection of element t through the midpoint of its edge (a, b)
    (Sec. 2, proof of Lemma 2.1: grad phi_i^t = -grad phi_j^{t^m}).  Returns element ids,
    -1 where the reflected element is not an element of the same macro."""
    loc = lv.elem_local[E_idx]  # (P, 4, 3)
    mac = lv.elem_macro[E_idx]
    refl = loc[np.arange(len(E_idx)), a][:, None, :] + loc[np.arange(len(E_idx)), b][:, None, :] - loc
    n = lv.n
    inside = (refl.min(axis=(1, 2)) >= 0) & (refl.sum(axis=2).max(axis=1) <= n)
    nodes = -np.ones((len(E_idx), 4), dtype=np.int64)
    for m in np.unique(mac):
        sel = (mac == m) & inside
        tab = lv.local_to_node[m]
        r = refl[sel]
        nodes[sel] = tab[r[..., 0], r[..., 1], r[..., 2]]
    # element lookup by (macro, sorted vertex set)
    ekey = np.concatenate([lv.elem_macro[:, None], np.sort(lv.elems, axis=1)], axis=1)
    qkey = np.concatenate([mac[:, None], np.sort(nodes, axis=1)], axis=1)
    order = np.lexsort(ekey.T[::-1])
    sk = ekey[order]
    # binary search row-wise via structured view
    dt = np.dtype([("f%d" % i, np.int64) for i in range(5)])
    skv = np.ascontiguousarray(sk).view(dt).reshape(-1)
    qv = np.ascontiguousarray(qkey).view(dt).reshape(-1)
    pos = np.searchsorted(skv, qv)
    pos = np.minimum(pos, len(skv) - 1)
    found = (skv[pos] == qv) & inside
    out = np.where(found, order[pos], -1)
    return out


def scaled_operator(lv: Level, Kel, k, variant="physical", khat="patch", iface="symmetric",
                    skeleton_diag="zero_row_sum"):
    """Physical (\\hat a_h) or unphysical (\\tilde a_h) stencil scaling (Sec. 2).

    For an edge (i, j) inside macro T the block is

        S_ij = khat_ij * Shat_ij + R_ij,
        Shat_ij = sum_{t in patch} sym(K^t_ij),                       eq. (stiffcontribution)
        khat_ij = mean over the patch of kbar^t (eq. (patchmean)) or (k_i + k_j)/2 (Remark),
        R_ij = 1/2 sum_{t in patch} (kbar^t - kbar^{t^m}) antisym(K^t_ij), eq. (corrtermgeneral)

    (R = 0 for the unphysical variant).  A macro-interior row i has the centre block
    S_ii = -sum_{j != i} S_ij (zero row sum, Lemma 2.1).

    Interface rows (Sec. 2.2):
      iface="symmetric": the off-diagonal pair (i, j) uses a_h when both nodes lie on the macro
                         skeleton, the scaled block otherwise.  The diagonal block of a skeleton
                         row is either a_h(i, i) (skeleton_diag="nodal", the literal reading of
                         the case x_i = x_j on the skeleton) or minus the sum of the row's
                         off-diagonal blocks (skeleton_diag="zero_row_sum", which keeps
                         translations in the kernel of every row; it is a symmetric block
                         because the antisymmetric parts of a_h and of the scaled blocks agree).
      iface="practical": every row of a skeleton node is the a_h row.
    variant="nodal" returns a_h itself.
    """
    N = lv.num_nodes
    k = np.asarray(k, dtype=np.float64)
    kb = kbar(lv, k)
    A_nodal = nodal_integration(lv, Kel, k)
    if variant == "nodal":
        return A_nodal
    E = lv.elems.shape[0]
    # one record per (element, ordered local pair a != b)
    recE = np.repeat(np.arange(E), len(PAIRS))
    ra = np.tile(np.array([p[0] for p in PAIRS]), E)
    rb = np.tile(np.array([p[1] for p in PAIRS]), E)
    ri = lv.elems[recE, ra]
    rj = lv.elems[recE, rb]
    rmac = lv.elem_macro[recE]
    blk = Kel[recE, ra, rb]  # (P, 3, 3) [m, l]
    sym = 0.5 * (blk + np.transpose(blk, (0, 2, 1)))
    anti = 0.5 * (blk - np.transpose(blk, (0, 2, 1)))
    # patch = elements of macro T containing both i and j
    gkey = np.stack([rmac, ri, rj], axis=1)
    ug, gid = np.unique(gkey, axis=0, return_inverse=True)
    gid = gid.reshape(-1)
    G = ug.shape[0]
    cnt = np.bincount(gid, minlength=G).astype(np.float64)
    Shat = np.zeros((G, 3, 3))
    np.add.at(Shat, gid, sym)
    if khat == "patch":
        kh = np.bincount(gid, weights=kb[recE], minlength=G) / cnt
    elif khat == "edge":
        kh = 0.5 * (k[ug[:, 1]] + k[ug[:, 2]])
    else:
        raise ValueError(khat)
    gi, gj = ug[:, 1], ug[:, 2]
    skel = lv.skeleton
    if iface == "symmetric":
        use_scaled = ~(skel[gi] & skel[gj])
    elif iface == "practical":
        use_scaled = ~skel[gi]
    else:
        raise ValueError(iface)
    R = np.zeros((G, 3, 3))
    if variant == "physical":
        need = use_scaled[gid]
        tm = -np.ones(len(recE), dtype=np.int64)
        tm[need] = _reflected_elements(lv, recE[need], ra[need], rb[need])
        if np.any(tm[need] < 0):
            raise AssertionError("a reflected element is missing for a scaled pair")
        contrib = np.zeros_like(anti)
        contrib[need] = 0.5 * (kb[recE[need]] - kb[tm[need]])[:, None, None] * anti[need]
        np.add.at(R, gid, contrib)
    elif variant != "unphysical":
        raise ValueError(variant)
    S = kh[:, None, None] * Shat + R
    # assemble: scaled pairs from S, the rest from a_h
    rows = gi[use_scaled]
    cols = gj[use_scaled]
    blocks = S[use_scaled]
    A_scaled_off = _blocks_to_csr(rows, cols, blocks, N)
    # centre blocks of macro-interior rows: -sum_j S_ij
    interior = ~skel
    centre = np.zeros((N, 3, 3))
    np.add.at(centre, gi[use_scaled & interior[gi]], S[use_scaled & interior[gi]])
    centre = -centre
    cid = np.nonzero(interior)[0]
    A_centre = _blocks_to_csr(cid, cid, centre[cid], N)
    # a_h entries for the remaining pairs and for skeleton diagonals
    An = A_nodal.tocoo()
    ni, nj = An.row // 3, An.col // 3
    if iface == "symmetric":
        keep = skel[ni] & skel[nj]
        if skeleton_diag == "zero_row_sum":
            keep &= ni != nj
        elif skeleton_diag != "nodal":
            raise ValueError(skeleton_diag)
    else:
        keep = skel[ni]
    A_rest = sp.coo_matrix((An.data[keep], (An.row[keep], An.col[keep])), shape=An.shape).tocsr()
    A = (A_scaled_off + A_centre + A_rest).tocsr()
    if iface == "symmetric" and skeleton_diag == "zero_row_sum":
        # centre block of skeleton rows: minus the sum of all off-diagonal blocks of the row
        sid = np.nonzero(skel)[0]
        C = A.tocoo()
        ci, cj = C.row // 3, C.col // 3
        sel = skel[ci] & (ci != cj)
        cen = np.zeros((N, 3, 3))
        np.add.at(cen, (ci[sel], C.row[sel] % 3, C.col[sel] % 3), C.data[sel])
        A = (A + _blocks_to_csr(sid, sid, -cen[sid], N)).tocsr()
    return A


def edge_blocks(A, i, j):
    """3x3 block (row node i, column node j) of a node-major operator."""
    return A[3 * i:3 * i + 3, 3 * j:3 * j + 3].toarray()


def with_dirichlet_rows(A, dirichlet_nodes):
    """Rows of Dirichlet DoFs replaced by identity rows (columns kept): y = A x on free rows,
    y = x on Dirichlet rows."""
    d = np.zeros(A.shape[0], dtype=bool)
    dn = np.nonzero(dirichlet_nodes)[0]
    for m in range(3):
        d[3 * dn + m] = True
    A = A.tocsr().copy()
    keep = sp.diags((~d).astype(np.float64))
    return (keep @ A + sp.diags(d.astype(np.float64))).tocsr()


def apply(A_bc, x):
    """y = A x with the Dirichlet rows of A_bc (see ``with_dirichlet_rows``); x node-major (N, 3)."""
    return (A_bc @ np.asarray(x).reshape(-1)).reshape(-1, 3)


def residual(A, f, x, dirichlet_nodes):
    """r = f - A x on free rows, 0 on Dirichlet rows (eq. (residuallinalg))."""
    r = (np.asarray(f).reshape(-1) - A @ np.asarray(x).reshape(-1)).reshape(-1, 3)
    r[np.asarray(dirichlet_nodes)] = 0.0
    return r


def macro_stiffness(mm: MacroMesh, lv: Level, c_eps, c_div):
    return fem.element_stiffness(lv.coords[lv.elems], c_eps, c_div)


def edge_count_stats(lv: Level):
    """Per node: set of neighbours; per edge: number of elements containing it."""
    cnt = {}
    for (a, b) in EDGES_OF_TET:
        i = np.minimum(lv.elems[:, a], lv.elems[:, b])
        j = np.maximum(lv.elems[:, a], lv.elems[:, b])
        for p in zip(i.tolist(), j.tolist()):
            cnt[p] = cnt.get(p, 0) + 1
    return cnt
