"""Oracle: one row of an operator at any refinement level, by local refinement.

Test infrastructure only (see the package docstring).

For a node p the row (A x)_p needs only the elements that contain p.  They are
found by refining each macro that contains p with Bey's rule, keeping at every
level only the children whose closure contains p; after ``level`` steps the
survivors are exactly the (up to 24 in a macro interior) elements around p.
The row is then built from the same definitions as ``operators`` (Sec. 2):
patch means, reflected elements, the correction R, and the interface rules.
This makes full-size rows checkable one at a time.
"""

from __future__ import annotations

import numpy as np

from . import fem
from .mesh import BEY_CHILDREN, MacroMesh


def _key(gv, bary):
    return tuple(sorted((int(gv[c]), int(bary[c])) for c in range(4) if bary[c] > 0))


def elements_around(mm: MacroMesh, level: int, macro: int, local_ijk):
    """All elements (over all macros) containing the node given by its local lattice
    coordinates in ``macro``.  Returns list of (macro, (4,4) int bary at denominator 2^level)."""
    n = 1 << level
    i, j, k = local_ijk
    gv = mm.tets[macro]
    q_bary = np.array([n - i - j - k, i, j, k], dtype=np.int64)
    key = _key(gv, q_bary)
    weight = dict(key)
    out = []
    for m, tv in enumerate(mm.tets):
        if not set(weight).issubset(set(int(v) for v in tv)):
            continue
        q = np.array([weight.get(int(v), 0) for v in tv], dtype=np.float64)  # bary in macro m
        elems = [np.eye(4, dtype=np.int64)]
        for l in range(level):
            nxt = []
            for B in elems:
                for child in BEY_CHILDREN:
                    C = np.stack([B[a] + B[b] for (a, b) in child])
                    # closure test: q * 2^{l+1} / n  =  lam^T C  with lam >= 0
                    target = q * (2 ** (l + 1)) / n
                    lam = np.linalg.solve(C.T.astype(np.float64), target)
                    if lam.min() >= -1e-9:
                        nxt.append(C)
            elems = nxt
        for B in elems:
            out.append((m, B))
    return out, key


def row(mm: MacroMesh, level: int, macro: int, local_ijk, kfun, xfun, c_eps, c_div,
        variant="physical", khat="patch", iface="symmetric", skeleton_diag="zero_row_sum",
        want_scale=False):
    """(A x)_p for the node p = (macro, local_ijk); kfun(coords)->k, xfun(coords)->(.,3).
    Returns (y, key); with want_scale also the row's term scale
    s_m = sum_{j != p} sum_l |A_pj[m, l]| |x_j[l] - x_p[l]| (the magnitude of the terms of the
    difference form sum_j A_pj (x_j - x_p), for rounding bounds)."""
    n = 1 << level
    elems, pkey = elements_around(mm, level, macro, local_ijk)
    keys = []  # per element: list of 4 node keys
    X = np.zeros((len(elems), 4, 3))
    for e, (m, B) in enumerate(elems):
        gv = mm.tets[m]
        keys.append([_key(gv, B[a]) for a in range(4)])
        X[e] = (B.astype(np.float64) @ mm.xyz[gv]) / n
    K = fem.element_stiffness(X, c_eps, c_div)
    node_pos = {}
    for e in range(len(elems)):
        for a in range(4):
            node_pos[keys[e][a]] = X[e, a]
    allkeys = list(node_pos)
    coords = np.array([node_pos[kk] for kk in allkeys])
    kval = dict(zip(allkeys, np.asarray(kfun(coords), dtype=np.float64).reshape(-1)))
    xval = dict(zip(allkeys, np.asarray(xfun(coords), dtype=np.float64).reshape(-1, 3)))
    kb = np.array([np.mean([kval[kk] for kk in keys[e]]) for e in range(len(elems))])

    def skeleton(kk):
        return len(kk) < 4

    p_skel = skeleton(pkey)
    # local index of p in each element
    ia = [keys[e].index(pkey) for e in range(len(elems))]
    neigh = sorted({kk for e in range(len(elems)) for kk in keys[e] if kk != pkey})
    blocks = {}
    for j in neigh:
        ejs = [e for e in range(len(elems)) if j in keys[e]]
        a_h = sum(kb[e] * K[e, ia[e], keys[e].index(j)] for e in ejs)
        if variant == "nodal":
            blocks[j] = a_h
            continue
        if iface == "symmetric":
            scaled = not (p_skel and skeleton(j))
        else:
            scaled = not p_skel
        if not scaled:
            blocks[j] = a_h
            continue
        # patch inside the macro that contains the edge (all of ejs lie in one macro here)
        macs = {elems[e][0] for e in ejs}
        assert len(macs) == 1
        Shat = np.zeros((3, 3))
        R = np.zeros((3, 3))
        ksum = 0.0
        for e in ejs:
            blk = K[e, ia[e], keys[e].index(j)]
            Shat += 0.5 * (blk + blk.T)
            ksum += kb[e]
            if variant == "physical":
                # reflected element: vertex set {x_p + x_j - v}
                pj = np.array(node_pos[pkey]) + np.array(node_pos[j])
                refl = {tuple(np.round(pj - X[e, a], 12)) for a in range(4)}
                em = [f for f in ejs if {tuple(np.round(X[f, a], 12)) for a in range(4)} == refl]
                assert len(em) == 1, "reflected element missing"
                R += 0.5 * (kb[e] - kb[em[0]]) * 0.5 * (blk - blk.T)
        if khat == "patch":
            kh = ksum / len(ejs)
        else:
            kh = 0.5 * (kval[pkey] + kval[j])
        blocks[j] = kh * Shat + R
    if variant == "nodal" or (p_skel and (iface == "practical" or skeleton_diag == "nodal")):
        centre = sum(kb[e] * K[e, ia[e], ia[e]] for e in range(len(elems)))
    else:
        centre = -sum(blocks.values())
    y = centre @ xval[pkey]
    for j, b in blocks.items():
        y = y + b @ xval[j]
    if want_scale:
        sc = np.zeros(3)
        for j, b in blocks.items():
            sc += np.abs(b) @ np.abs(xval[j] - xval[pkey])
        return y, pkey, sc
    return y, pkey
