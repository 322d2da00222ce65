"""Pins of the CPU oracle against facts the paper and the mathematics fix (no GPU).

Each test names the passage it follows.  None of them compares the oracle with
itself: they check closed forms, invariants the paper proves, brute-force
identities, and the numbers the paper prints.
"""

import itertools
import json
import math
import os

import numpy as np
import pytest

import hhg_inputs as hi
from oracle import fem, mesh, operators as op, rows

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _level(builder, level):
    xyz, tets = builder()
    mm = mesh.MacroMesh.build(xyz, tets)
    return mm, mesh.build_level(mm, level)


# ---------------------------------------------------------------- mesh (Sec. 2, Sec. 5.1.1)


def test_refinement_counts_match_paper_storage_figures():
    """Sec. 5.1.1: 128 intervals per macro edge -> 1.09e6 DoFs per macro, 8.4 MiB per vector
    and 2.8 MiB for k (doubles), and 500,062,500 inner-loop executions = 500 x 3 macros x
    interior nodes."""
    gold = json.load(open(os.path.join(GOLD, "paper_counts.json")))
    mm, lv = _level(hi.unit_tet, 7)
    N = lv.num_nodes
    interior = int((~lv.skeleton).sum())
    assert abs(3 * N / gold["dofs_per_macro"]["value"] - 1) < 0.01
    assert abs(24 * N / 2**20 / gold["vector_storage_per_macro_MiB"]["value"] - 1) < 0.01
    assert abs(8 * N / 2**20 / gold["coefficient_storage_per_macro_MiB"]["value"] - 1) < 0.01
    assert 500 * 3 * interior == gold["inner_loop_executions_per_rank"]["value"]
    assert lv.elems.shape[0] == 8**7


def test_cube_is_conforming_lattice():
    """6 Kuhn macros refined l times give the (n+1)^3 lattice; element volumes fill the cube."""
    for level in (1, 2, 3):
        mm, lv = _level(hi.kuhn_cube, level)
        n = 1 << level
        assert lv.num_nodes == (n + 1) ** 3
        _, vol = fem.p1_geometry(lv.coords[lv.elems])
        assert abs(vol.sum() - 1.0) < 1e-12
        assert np.allclose(vol, 1.0 / (6 * n**3))
        g = np.rint(lv.coords * n).astype(int)
        assert len({tuple(r) for r in g}) == (n + 1) ** 3


def test_interior_stencil_structure():
    """Sec. 2 / Sec. 2.4 / Sec. 4.1: an interior node has 14 neighbours, 24 elements (8 of each
    congruence class); 8 'red' edges lie in 6 elements and 6 edges in 4 elements."""
    gold = json.load(open(os.path.join(GOLD, "paper_counts.json")))
    for builder in (hi.unit_tet, hi.skewed_pair):
        mm, lv = _level(builder, 3)
        cnt = op.edge_count_stats(lv)
        inner = np.nonzero(~lv.skeleton)[0]
        for p in inner[:: max(1, len(inner) // 7)]:
            els = np.nonzero((lv.elems == p).any(1))[0]
            assert len(els) == 24
            nb = set(lv.elems[els].reshape(-1).tolist()) - {int(p)}
            assert len(nb) == gold["neighbours"]["value"]
            val = sorted(cnt[(min(p, q), max(p, q))] for q in nb)
            assert val.count(6) == gold["elements_per_edge"]["red_edges"]
            assert val.count(4) == gold["elements_per_edge"]["other_edges"]
            # congruence classes: shapes up to translation and point reflection
            X = lv.coords[lv.elems[els]]
            shapes = {}
            for e in range(len(els)):
                E = X[e] - X[e].mean(0)
                d = np.sort(np.round(np.linalg.norm(E[:, None] - E[None], axis=2).reshape(-1), 9))
                shapes.setdefault(tuple(d), 0)
                shapes[tuple(d)] += 1
            if builder is hi.unit_tet:
                assert sorted(shapes.values()) == [8, 8, 8]


# ---------------------------------------------------------------- element integrals


def _rand_tets(count, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(count, 4, 3))
    _, vol = fem.p1_geometry(X)
    return X[vol > 0.05]


def test_element_stiffness_energy_of_affine_fields():
    """For u = B x + c, v = C x + d: a_t(u, v) = |t| (c_eps sym(B):sym(C) + c_div tr B tr C)."""
    X = _rand_tets(40, 1)
    rng = np.random.default_rng(2)
    ce, cd = 0.7, 1.9
    K = fem.element_stiffness(X, ce, cd)
    _, vol = fem.p1_geometry(X)
    for e in range(X.shape[0]):
        B, C = rng.normal(size=(3, 3)), rng.normal(size=(3, 3))
        u = X[e] @ B.T + rng.normal(size=3)
        v = X[e] @ C.T + rng.normal(size=3)
        got = np.einsum("am,abml,bl->", v, K[e], u)
        sB, sC = 0.5 * (B + B.T), 0.5 * (C + C.T)
        want = vol[e] * (ce * (sB * sC).sum() + cd * np.trace(B) * np.trace(C))
        assert abs(got - want) < 1e-12 * max(1, abs(want))


def test_element_stiffness_rigid_modes():
    """Translations and rotations have eps = 0 and div = 0: they are in the kernel."""
    X = _rand_tets(20, 3)
    K = fem.element_stiffness(X, 1.0, 1.0)
    for e in range(X.shape[0]):
        modes = [np.tile(np.eye(3)[c], (4, 1)) for c in range(3)]
        for w in np.eye(3):
            modes.append(np.cross(w, X[e]))
        for u in modes:
            assert np.abs(np.einsum("abml,bl->am", K[e], u)).max() < 1e-12


def test_antisymmetric_part_closed_form_up_to_factor():
    """Sec. 2.4, eq. (localcorr3d) gives the antisymmetric part as (x_p - x_q)/12 in cross-product
    form.  With a^{a} = (a - a^T)/2 (eq. (symmmantisymm)) the eps-form value is (x_p - x_q)/24
    and the div form gives -2 times it (the paper's 'same values, flipped sign' is off by the
    factor 2 its gamma/beta/delta = a_lm - a_ml definition introduces)."""
    X = _rand_tets(30, 4)
    signs = set()
    for ce, cd, scale in ((1.0, 0.0, 1 / 24), (0.0, 1.0, -1 / 12)):
        K = fem.element_stiffness(X, ce, cd)
        for e in range(X.shape[0]):
            anti = 0.5 * (K[e, 0, 1] - K[e, 0, 1].T)
            d = X[e, 2] - X[e, 3]
            cross = np.array([[0, -d[2], d[1]], [d[2], 0, -d[0]], [-d[1], d[0], 0]])
            det = np.linalg.det(X[e, 1:] - X[e, 0])
            assert np.allclose(anti, np.sign(det) * scale * cross, atol=1e-12) or np.allclose(
                anti, -np.sign(det) * scale * cross, atol=1e-12)
            signs.add(np.sign(anti[0, 1] / cross[0, 1]) * np.sign(det) * np.sign(scale))
    assert len(signs) == 1


# ---------------------------------------------------------------- operators (Sec. 2)


@pytest.fixture(scope="module")
def cube3():
    mm, lv = _level(hi.kuhn_cube, 3)
    ce, cd = fem.elasticity_coefficients(0.3)
    K = fem.element_stiffness(lv.coords[lv.elems], ce, cd)
    return mm, lv, K


@pytest.fixture(scope="module")
def skew3():
    mm, lv = _level(hi.skewed_pair, 3)
    ce, cd = fem.elasticity_coefficients(0.3)
    K = fem.element_stiffness(lv.coords[lv.elems], ce, cd)
    return mm, lv, K


def test_constant_coefficient_all_forms_equal_galerkin(cube3):
    """Sec. 2: for constant k the scaled stencils reproduce the exact Galerkin matrix."""
    mm, lv, K = cube3
    k = np.full(lv.num_nodes, 2.5)
    A1 = op.nodal_integration(lv, K, np.ones(lv.num_nodes))
    for var in ("physical", "unphysical", "nodal"):
        A = op.scaled_operator(lv, K, k, var)
        assert abs(A - 2.5 * A1).max() < 1e-13


@pytest.mark.parametrize("fixture", ["cube3", "skew3"])
def test_lemma_affine_coefficient(fixture, request):
    """Lemma 2.1: for k affine on each edge patch, physical scaling equals nodal integration;
    unphysical scaling does not."""
    mm, lv, K = request.getfixturevalue(fixture)
    k = hi.affine_field(lv.coords, 2.0, [0.7, -0.4, 0.9])
    An = op.nodal_integration(lv, K, k)
    Ap = op.scaled_operator(lv, K, k, "physical")
    Au = op.scaled_operator(lv, K, k, "unphysical")
    scale = abs(An).max()
    assert abs(Ap - An).max() < 1e-14 * 10 * scale
    assert abs(Au - An).max() > 1e-4 * scale


@pytest.mark.parametrize("fixture", ["cube3", "skew3"])
def test_edge_mean_khat_equals_patch_mean_for_affine_coefficient(fixture, request):
    """Remark after Sec. 2.2 (khat = (k_i + k_j)/2) against eq. (patchmean): the patch of an
    edge inside a macro is point-symmetric about the edge midpoint (t -> t^m maps it onto
    itself), so for an affine k the mean of the element means kbar^t is k at the midpoint,
    i.e. (k_i + k_j)/2.  The two khat rules then give the same operator in both variants; for
    a non-affine k they differ."""
    mm, lv, K = request.getfixturevalue(fixture)
    k = hi.affine_field(lv.coords, 2.0, [0.7, -0.4, 0.9])
    scale = abs(op.nodal_integration(lv, K, k)).max()
    for var in ("physical", "unphysical"):
        Ap = op.scaled_operator(lv, K, k, var, khat="patch")
        Ae = op.scaled_operator(lv, K, k, var, khat="edge")
        assert abs(Ap - Ae).max() < 1e-13 * scale
    rng = np.random.default_rng(17)
    kr = rng.uniform(0.5, 3.0, lv.num_nodes)
    assert abs(op.scaled_operator(lv, K, kr, khat="patch") - op.scaled_operator(lv, K, kr, khat="edge")).max() \
        > 1e-4 * scale


@pytest.mark.parametrize("fixture", ["cube3", "skew3"])
def test_practical_interface_rule_pins(fixture, request):
    """Sec. 2.2, practical interface rows (every skeleton row is the a_h row): for constant k
    the whole operator is the Galerkin matrix (both a_h and the scaled blocks reproduce it,
    Sec. 2); for affine k it is nodal integration everywhere (Lemma 2.1 on the macro-interior
    rows, a_h on the skeleton rows)."""
    mm, lv, K = request.getfixturevalue(fixture)
    G = op.nodal_integration(lv, K, np.ones(lv.num_nodes))
    A = op.scaled_operator(lv, K, np.full(lv.num_nodes, 1.7), iface="practical")
    assert abs(A - 1.7 * G).max() < 1e-13 * abs(G).max()
    k = hi.affine_field(lv.coords, 2.0, [0.3, 0.5, -0.2])
    An = op.nodal_integration(lv, K, k)
    for khat in ("patch", "edge"):
        Ap = op.scaled_operator(lv, K, k, iface="practical", khat=khat)
        assert abs(Ap - An).max() < 1e-13 * abs(An).max()
    # the unphysical variant keeps the interior rows away from a_h (the pin can fail)
    Au = op.scaled_operator(lv, K, k, "unphysical", iface="practical")
    assert abs(Au - An).max() > 1e-4 * abs(An).max()


def test_correction_is_antisymmetric_part_of_nodal_blocks(skew3):
    """eq. (corrtermgeneral): R_ij = 1/2 sum (kbar^t - kbar^{t^m}) antisym(a^t_ij) equals the
    antisymmetric part of the nodal-integration block, since the reflection pairs the patch; so
    sum_j R_ij = 0 for every macro-interior row."""
    mm, lv, K = skew3
    rng = np.random.default_rng(5)
    k = rng.uniform(0.5, 3.0, lv.num_nodes)
    An = op.nodal_integration(lv, K, k)
    Ap = op.scaled_operator(lv, K, k, "physical")
    Au = op.scaled_operator(lv, K, k, "unphysical")
    inner = np.nonzero(~lv.skeleton)[0]
    for i in inner[:40]:
        Rsum = np.zeros((3, 3))
        cols = np.unique(Ap[3 * i].indices // 3)
        for j in cols:
            if j == i:
                continue
            Bp, Bn, Bu = (op.edge_blocks(M, i, j) for M in (Ap, An, Au))
            assert np.allclose(0.5 * (Bp - Bp.T), 0.5 * (Bn - Bn.T), atol=1e-15)
            R = Bp - Bu
            assert np.allclose(R, -R.T, atol=1e-15)
            Rsum += R
        assert np.abs(Rsum).max() < 1e-15


def test_symmetry_and_rigid_modes(skew3):
    """Sec. 2.2: the symmetric interface definition gives a symmetric matrix; the zero row sum
    (Lemma 2.1) keeps translations in the kernel of every row for any k; rotations are in the
    kernel only when k is affine (then the form equals nodal integration, which annihilates
    every rigid mode)."""
    mm, lv, K = skew3
    rng = np.random.default_rng(7)
    krand = rng.uniform(0.5, 3.0, lv.num_nodes)
    kaff = hi.affine_field(lv.coords, 2.0, [0.3, 0.5, -0.2])
    Ar = op.scaled_operator(lv, K, krand, "physical", iface="symmetric")
    Aa = op.scaled_operator(lv, K, kaff, "physical", iface="symmetric")
    Ap = op.scaled_operator(lv, K, krand, "physical", iface="practical")
    assert abs(Ar - Ar.T).max() < 1e-15
    assert abs(Ap - Ap.T).max() > 1e-6
    trans = [np.tile(np.eye(3)[c], (lv.num_nodes, 1)) for c in range(3)]
    rots = [np.cross(w, lv.coords) for w in np.eye(3)]
    for u in trans:
        assert np.abs(Ar @ u.reshape(-1)).max() < 1e-13
    for u in trans + rots:
        assert np.abs(Aa @ u.reshape(-1)).max() < 1e-13
    assert max(np.abs(Ar @ u.reshape(-1)).max() for u in rots) > 1e-5


def test_quadratic_patch_test_on_cube_lattice(cube3):
    """On the translation- and point-symmetric cube lattice, the P1 stencil with constant k is
    exact for quadratics: (A u)_i = h^3 * (-div sigma(u)) at every interior node (the local
    truncation error of a centrally symmetric stencil vanishes on quadratics)."""
    mm, lv, K = cube3
    ce, cd = fem.elasticity_coefficients(0.3)
    A = op.scaled_operator(lv, K, np.ones(lv.num_nodes), "physical")
    rng = np.random.default_rng(11)
    Q = rng.normal(size=(3, 3, 3))
    Q = 0.5 * (Q + np.transpose(Q, (0, 2, 1)))  # u_m = x^T Q_m x
    u = np.einsum("ni,mij,nj->nm", lv.coords, Q, lv.coords)
    # grad u_m = 2 Q_m x ; -div sigma = -(ce * (lap u + grad div u)/2 + cd grad div u)
    lap = 2 * np.trace(Q, axis1=1, axis2=2)  # per component m
    graddiv = 2 * np.array([sum(Q[j, j, m] for j in range(3)) for m in range(3)])
    f = -(ce * 0.5 * (lap + graddiv) + cd * graddiv)
    h = 1.0 / lv.n
    y = (A @ u.reshape(-1)).reshape(-1, 3)
    free = ~lv.dirichlet
    assert np.allclose(y[free], h**3 * f[None, :], rtol=0, atol=1e-13)


# ---------------------------------------------------------------- row oracle


def test_row_oracle_equals_assembled_rows(skew3):
    """Rows built by local refinement equal the rows of the global assembly, for all variants."""
    mm, lv, K = skew3
    ce, cd = fem.elasticity_coefficients(0.3)
    kf = lambda c: 1 + 0.5 * np.sin(3 * c[:, 0]) * np.cos(2 * c[:, 1]) + c[:, 2] ** 2
    xf = lambda c: np.stack([np.sin(c[:, 0] + c[:, 1]), c[:, 2] ** 2 - c[:, 0], np.cos(2 * c[:, 1])], 1)
    inc = mesh.node_incidences(lv)
    rng = np.random.default_rng(1)
    picks = rng.choice(lv.num_nodes, 12, replace=False)
    for var, iface in (("physical", "symmetric"), ("physical", "practical"), ("unphysical", "symmetric"),
                       ("nodal", "symmetric")):
        A = op.scaled_operator(lv, K, kf(lv.coords), var, iface=iface)
        y = (A @ xf(lv.coords).reshape(-1)).reshape(-1, 3)
        for a in picks:
            m, i, j, kk = inc[a][0]
            yr, _ = rows.row(mm, 3, m, (i, j, kk), kf, xf, ce, cd, var, iface=iface)
            assert np.abs(yr - y[a]).max() < 1e-14 * 10


# ---------------------------------------------------------------- elastostatics benchmark (Sec. 5.1.2)


def _elastostatics_error(level_paper, m, variant):
    sympy = pytest.importorskip("sympy")
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    nu = 0.34
    X, Y, Z = sympy.symbols("x y z")
    u = sympy.Matrix([(X**3 * Y + Z**2), (X**4 * Y + 2 * Z), (3 * X + Y * Z**3)]) / (X * Y * Z + 1)
    E = sympy.cos(m * sympy.pi * X * Y * Z) + 2
    g = u.jacobian([X, Y, Z])
    eps = (g + g.T) / 2
    sig = E * (eps / (1 + nu) + nu / ((1 + nu) * (1 - 2 * nu)) * eps.trace() * sympy.eye(3))
    f = -sympy.Matrix([sum(sympy.diff(sig[i, j], [X, Y, Z][j]) for j in range(3)) for i in range(3)])
    ffun = sympy.lambdify((X, Y, Z), list(f), "numpy")

    level = level_paper + 2  # 2^(l+2) intervals per macro edge of the 6-macro cube
    mm, lv = _level(hi.kuhn_cube, level)
    ce, cd = fem.elasticity_coefficients(nu)
    Xe = lv.coords[lv.elems]
    K = fem.element_stiffness(Xe, ce, cd)
    A = op.scaled_operator(lv, K, hi.young_cos(lv.coords, m), variant)
    fv = np.stack([np.broadcast_to(c, lv.num_nodes) for c in ffun(*lv.coords.T)], 1)
    Me = fem.element_mass(Xe)
    r = np.repeat(lv.elems, 4, axis=1).reshape(-1)
    c = np.tile(lv.elems, (1, 4)).reshape(-1)
    M = sp.coo_matrix((Me.reshape(-1), (r, c)), shape=(lv.num_nodes,) * 2).tocsr()
    b = (M @ fv).reshape(-1)  # load vector M I_h f
    d = np.repeat(lv.dirichlet, 3)
    fr = ~d
    x = np.zeros(3 * lv.num_nodes)
    x[d] = hi.u_star(lv.coords).reshape(-1)[d]
    Aff = A[fr][:, fr]
    x[fr] = spla.spsolve(Aff.tocsc(), b[fr] - A[fr][:, d] @ x[d])
    # discrete L2 error on the 256-interval lattice of the interpolants (Sec. 5.1.2)
    n = lv.n
    ug = np.zeros((n + 1,) * 3 + (3,))
    gi = np.rint(lv.coords * n).astype(int)
    ug[gi[:, 0], gi[:, 1], gi[:, 2]] = x.reshape(-1, 3)
    NL = 256
    a = np.arange(NL + 1) / NL
    err2 = 0.0
    for zi in range(0, NL + 1):
        P = np.stack(np.meshgrid(a, a, [a[zi]], indexing="ij"), -1).reshape(-1, 3)
        t = P * n
        cell = np.minimum(np.floor(t).astype(np.int64), n - 1)
        s = t - cell
        order = np.argsort(-s, axis=1, kind="stable")
        ss = np.take_along_axis(s, order, axis=1)
        w = np.stack([1 - ss[:, 0], ss[:, 0] - ss[:, 1], ss[:, 1] - ss[:, 2], ss[:, 2]], 1)
        v = cell.copy()
        val = w[:, :1] * ug[v[:, 0], v[:, 1], v[:, 2]]
        for q in range(3):
            v[np.arange(len(v)), order[:, q]] += 1
            val += w[:, q + 1:q + 2] * ug[v[:, 0], v[:, 1], v[:, 2]]
        err2 += ((val - hi.u_star(P)) ** 2).sum()
    return math.sqrt(err2 / NL**3)


@pytest.mark.slow
def test_elastostatics_benchmark_convergence():
    """Sec. 5.1.2: O(h^2) in the discrete L2 norm for nodal integration and physical scaling
    (eoc 1.94/1.97 in the paper), physical within 1% of nodal for m = 1 and within 15% for
    m = 8, unphysical scaling far off for m = 8.

    The paper does not state the orientation of its Kuhn split or how the load vector was
    formed; with the split and load (M I_h f) used here the errors differ from the printed
    ones by up to about 30% (reflecting the split changes them by a factor up to 1.7 at
    these levels), so magnitudes are checked to a factor 1.6, and the rates and the
    physical/nodal ratios tightly."""
    gold = json.load(open(os.path.join(GOLD, "elastostatics_table.json")))
    e = {}
    for m in (1, 8):
        for var in ("nodal", "physical", "unphysical"):
            e[(m, var)] = [_elastostatics_error(l, m, var) for l in (1, 2)]
    for m in (1, 8):
        for var in ("nodal", "physical"):
            paper = gold["errors"]["m%d" % m][var][:2]
            for got, want in zip(e[(m, var)], paper):
                assert want / 1.6 < got < want * 1.6, (m, var, got, want)
            eoc = math.log2(e[(m, var)][0] / e[(m, var)][1])
            assert 1.85 < eoc < 2.1, (m, var, eoc)
    assert abs(e[(1, "physical")][1] / e[(1, "nodal")][1] - 1) < 0.02
    assert abs(e[(8, "physical")][1] / e[(8, "nodal")][1] - 1) < 0.15
    assert e[(8, "unphysical")][1] > 1.5 * e[(8, "physical")][1]
