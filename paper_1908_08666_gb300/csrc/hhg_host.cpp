// libhhgs host side: context, macro mesh, refinement levels, skeleton
// (interface) bookkeeping, per-macro stencil precomputation in FP64, and the
// C ABI declared in include/hhg.h.
//
// Stencil precomputation (Sec. 2, Lemma 2.1; Sec. 2.4, eq. correctionterm3D):
// inside a macro the refined mesh is the affine image of the Freudenthal
// lattice, so every interior node sees the same 24 elements of 6 shapes (one
// per Kuhn permutation).  For each of the 14 stencil directions d the patch
// of the edge (0, d) is the set of elements containing both end points;
//   Shat_d = sum_{t in patch} sym(K^t_{0d})                        (eq. stiffcontribution)
//   R_d    = 1/2 sum_t (kbar^t - kbar^{t^m}) antisym(K^t_{0d})      (eq. corrtermgeneral)
// with t^m the point reflection of t through the edge midpoint.  Writing
// kbar^t - kbar^{t^m} as a combination of nodal k values turns R_d into
// sum_c (k_{r_c} - k_{r_c^m}) C_{d,c} over the ring pairs of the edge; the
// axial vectors of the antisymmetric C_{d,c} are what the kernels store.
// Everything here is derived from the element stiffness matrices, computed
// from the closed-form P1 gradients.
#include "hhg_ctx.h"

namespace {

// element stiffness K[a][b][m][l] = |t| (c_eps eps(phi_b e_l):eps(phi_a e_m) + c_div div(phi_b e_l) div(phi_a e_m))
void element_stiffness(const Vec3d v[4], double c_eps, double c_div, double K[4][4][9]) {
  double J[3][3];
  for (int r = 0; r < 3; ++r) {
    J[r][0] = (r == 0 ? v[1].x : r == 1 ? v[2].x : v[3].x) - v[0].x;
    J[r][1] = (r == 0 ? v[1].y : r == 1 ? v[2].y : v[3].y) - v[0].y;
    J[r][2] = (r == 0 ? v[1].z : r == 1 ? v[2].z : v[3].z) - v[0].z;
  }
  const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  if (std::fabs(det) < 1e-300) THROW(HHG_ERR_ARG, "degenerate element");
  // inverse of J; gradient of barycentric a (a=1..3) = column a-1 of J^{-1}
  double inv[3][3];
  inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  double g[4][3];
  for (int a = 1; a < 4; ++a)
    for (int c = 0; c < 3; ++c) g[a][c] = inv[c][a - 1];
  for (int c = 0; c < 3; ++c) g[0][c] = -(g[1][c] + g[2][c] + g[3][c]);
  const double vol = std::fabs(det) / 6.0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      const double gg = g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2];
      for (int m = 0; m < 3; ++m)
        for (int l = 0; l < 3; ++l) {
          const double eps = 0.5 * ((l == m ? gg : 0.0) + g[a][l] * g[b][m]);
          const double dv = g[b][l] * g[a][m];
          K[a][b][m * 3 + l] = vol * (c_eps * eps + c_div * dv);
        }
    }
}

struct MacroGeom {
  Vec3d v[4];
  Vec3d kuhn_to_x(double X, double Y, double Z, int n) const {
    // x = v0 + (X (v1-v0) + Y (v2-v1) + Z (v3-v2)) / n
    Vec3d r;
    r.x = v[0].x + (X * (v[1].x - v[0].x) + Y * (v[2].x - v[1].x) + Z * (v[3].x - v[2].x)) / n;
    r.y = v[0].y + (X * (v[1].y - v[0].y) + Y * (v[2].y - v[1].y) + Z * (v[3].y - v[2].y)) / n;
    r.z = v[0].z + (X * (v[1].z - v[0].z) + Y * (v[2].z - v[1].z) + Z * (v[3].z - v[2].z)) / n;
    return r;
  }
};

void kuhn_vertices(int p, int P[4][3]) {
  int a0, a1, a2;
  kuhn_perm(p, a0, a1, a2);
  for (int v = 0; v < 4; ++v)
    for (int c = 0; c < 3; ++c) P[v][c] = (v == 3) ? 1 : 0;
  P[1][a0] = 1;
  P[2][a0] = 1;
  P[2][a1] = 1;
}

// Kuhn coordinates of stencil direction d
void dir_kuhn(int d, int out[3]) {
  const int di = dir_di(d), dj = dir_dj(d), dk = dir_dk(d);
  out[0] = di + dj + dk;
  out[1] = dj + dk;
  out[2] = dk;
}

int dir_from_kuhn(const int v[3]) {
  for (int d = 0; d < NDIR; ++d) {
    int w[3];
    dir_kuhn(d, w);
    if (w[0] == v[0] && w[1] == v[1] && w[2] == v[2]) return d;
  }
  return -1;
}

// Per-macro constants at intervals n: element stiffness of the 6 Kuhn element
// types and the interior stencil (Shat and the correction axial vectors).
// P1 gradients and volume of one element
void element_gradients(const Vec3d v[4], double g[4][3], double& vol) {
  double K[4][4][9];
  element_stiffness(v, 1.0, 0.0, K);  // validates the element
  double J[3][3];
  const Vec3d* w[3] = {&v[1], &v[2], &v[3]};
  for (int r = 0; r < 3; ++r) {
    J[r][0] = w[r]->x - v[0].x;
    J[r][1] = w[r]->y - v[0].y;
    J[r][2] = w[r]->z - v[0].z;
  }
  const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  // columns of J^{-1} = gradients of barycentrics 1..3 (cofactor formula)
  const double c00 = (J[1][1] * J[2][2] - J[1][2] * J[2][1]), c01 = (J[0][2] * J[2][1] - J[0][1] * J[2][2]),
               c02 = (J[0][1] * J[1][2] - J[0][2] * J[1][1]);
  const double c10 = (J[1][2] * J[2][0] - J[1][0] * J[2][2]), c11 = (J[0][0] * J[2][2] - J[0][2] * J[2][0]),
               c12 = (J[0][2] * J[1][0] - J[0][0] * J[1][2]);
  const double c20 = (J[1][0] * J[2][1] - J[1][1] * J[2][0]), c21 = (J[0][1] * J[2][0] - J[0][0] * J[2][1]),
               c22 = (J[0][0] * J[1][1] - J[0][1] * J[1][0]);
  const double inv[3][3] = {{c00 / det, c01 / det, c02 / det}, {c10 / det, c11 / det, c12 / det},
                            {c20 / det, c21 / det, c22 / det}};
  for (int a = 1; a < 4; ++a)
    for (int c = 0; c < 3; ++c) g[a][c] = inv[c][a - 1];
  for (int c = 0; c < 3; ++c) g[0][c] = -(g[1][c] + g[2][c] + g[3][c]);
  vol = std::fabs(det) / 6.0;
}

void macro_constants(const MacroGeom& G, int n, double c_eps, double c_div, MacroConsts<double>& out) {
  double KE[6][4][4][9];
  double BD[6][4][4][3], LC[6][4][4];
  // stabilisation length of the macro's refined mesh: h = (6 |T|)^{1/3} / n (the lattice
  // spacing 1/n on the Kuhn cube)
  double hT;
  {
    Vec3d v[4] = {G.v[0], G.v[1], G.v[2], G.v[3]};
    double g[4][3], volT;
    element_gradients(v, g, volT);
    hT = std::cbrt(6.0 * volT) / n;
  }
  for (int p = 0; p < 6; ++p) {
    int P[4][3];
    kuhn_vertices(p, P);
    Vec3d v[4];
    for (int a = 0; a < 4; ++a) v[a] = G.kuhn_to_x(P[a][0], P[a][1], P[a][2], n);
    element_stiffness(v, c_eps, c_div, KE[p]);
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        for (int q = 0; q < 9; ++q) out.ke[p][a][b][q] = KE[p][a][b][q];
    double g[4][3], vol;
    element_gradients(v, g, vol);
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        for (int l = 0; l < 3; ++l) BD[p][a][b][l] = -0.25 * vol * g[b][l];
        LC[p][a][b] = -(hT * hT / 12.0) * vol * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]);
        for (int l = 0; l < 3; ++l) out.bd[p][a][b][l] = BD[p][a][b][l];
        out.lc[p][a][b] = LC[p][a][b];
      }
  }
  // patches of the 14 directions
  for (int d = 0; d < NDIR; ++d) {
    int dk[3];
    dir_kuhn(d, dk);
    double Sh[9] = {0};
    // coefficient matrix of k at each neighbour offset (index = direction, 14 = centre)
    double C[NDIR + 1][9];
    double wk[NDIR + 1];
    std::memset(C, 0, sizeof(C));
    std::memset(wk, 0, sizeof(wk));
    int count = 0;
    struct PatchEl {
      int p, a, b;
      int c[3];
    };
    std::vector<PatchEl> patch;
    for (int p = 0; p < 6; ++p) {
      int P[4][3];
      kuhn_vertices(p, P);
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          if (a == b) continue;
          if (P[b][0] - P[a][0] == dk[0] && P[b][1] - P[a][1] == dk[1] && P[b][2] - P[a][2] == dk[2]) {
            PatchEl e;
            e.p = p;
            e.a = a;
            e.b = b;
            for (int c = 0; c < 3; ++c) e.c[c] = -P[a][c];
            patch.push_back(e);
          }
        }
    }
    count = (int)patch.size();
    if (count != (dir_red(d) ? 6 : 4)) THROW(HHG_ERR_STATE, "patch of direction %d has %d elements", d, count);
    auto node_of = [&](const int off[3]) -> int {
      if (off[0] == 0 && off[1] == 0 && off[2] == 0) return NDIR;
      return dir_from_kuhn(off);
    };
    for (int l = 0; l < 3; ++l) {
      out.st.B[d][l] = 0;
      out.st.G[d][l] = 0;
    }
    out.st.C[d] = 0;
    for (const PatchEl& e : patch) {
      for (int l = 0; l < 3; ++l) {
        out.st.B[d][l] += BD[e.p][e.a][e.b][l];
        out.st.G[d][l] += BD[e.p][e.b][e.a][l];
      }
      out.st.C[d] += LC[e.p][e.a][e.b];
    }
    for (const PatchEl& e : patch) {
      const double* K = KE[e.p][e.a][e.b];
      for (int m = 0; m < 3; ++m)
        for (int l = 0; l < 3; ++l) Sh[m * 3 + l] += 0.5 * (K[m * 3 + l] + K[l * 3 + m]);
      int P[4][3];
      kuhn_vertices(e.p, P);
      // vertices of t and of its reflection t^m (d - v)
      for (int v = 0; v < 4; ++v) {
        int off[3] = {e.c[0] + P[v][0], e.c[1] + P[v][1], e.c[2] + P[v][2]};
        int ref[3] = {dk[0] - off[0], dk[1] - off[1], dk[2] - off[2]};
        const int iv = node_of(off), ir = node_of(ref);
        if (iv < 0 || ir < 0) THROW(HHG_ERR_STATE, "patch vertex is not a stencil neighbour");
        wk[iv] += 0.25 / count;
        for (int m = 0; m < 3; ++m)
          for (int l = 0; l < 3; ++l) {
            const double an = 0.5 * (K[m * 3 + l] - K[l * 3 + m]);
            C[iv][m * 3 + l] += 0.5 * 0.25 * an;
            C[ir][m * 3 + l] -= 0.5 * 0.25 * an;
          }
      }
    }
    // checks: Shat symmetric, khat weights, ring structure, pair antisymmetry
    for (int m = 0; m < 3; ++m)
      for (int l = 0; l < 3; ++l) {
        double full = 0;
        for (const PatchEl& e : patch) full += KE[e.p][e.a][e.b][m * 3 + l];
        if (std::fabs(full - Sh[m * 3 + l]) > 1e-12 * (1 + std::fabs(full)))
          THROW(HHG_ERR_STATE, "reference stencil of direction %d is not symmetric", d);
      }
    const double wr = dir_red(d) ? 1.0 / 12.0 : 0.125;
    double cmax = 0;
    for (int q = 0; q <= NDIR; ++q)
      for (int r = 0; r < 9; ++r) cmax = std::max(cmax, std::fabs(C[q][r]));
    for (int q = 0; q <= NDIR; ++q) {
      bool ring = false;
      for (int c = 0; c < ring_count(d); ++c) ring |= (q == ring_a(d, c) || q == ring_b(d, c));
      const double want = (q == NDIR || q == d) ? 0.25 : (ring ? wr : 0.0);
      if (std::fabs(wk[q] - want) > 1e-14) THROW(HHG_ERR_STATE, "patch-mean weight mismatch (dir %d)", d);
      if (!ring) {
        for (int r = 0; r < 9; ++r)
          if (std::fabs(C[q][r]) > 1e-12 * cmax) THROW(HHG_ERR_STATE, "correction outside the ring (dir %d)", d);
      }
    }
    for (int c = 0; c < 3; ++c) {
      for (int r = 0; r < 3; ++r) out.st.s[d][c][r] = 0;
      if (c >= ring_count(d)) continue;
      const double* A = C[ring_a(d, c)];
      const double* B = C[ring_b(d, c)];
      for (int r = 0; r < 9; ++r)
        if (std::fabs(A[r] + B[r]) > 1e-12 * (cmax + 1e-300))
          THROW(HHG_ERR_STATE, "ring pair is not antisymmetric (dir %d)", d);
      // axial vector of A: [a]_x = [[0,-a3,a2],[a3,0,-a1],[-a2,a1,0]]
      out.st.s[d][c][0] = A[7];
      out.st.s[d][c][1] = A[2];
      out.st.s[d][c][2] = A[3];
    }
    // The stencil is point-symmetric: the correction stencils of d and -d are equal
    // (the ring pairs of -d are those of d through the neighbour i - d, swapped, and the
    // block of the edge (i, i - d) is the transpose of that of (i - d, i)).  The kernels use
    // s[d] for both directions.
    if (d >= 7)
      for (int c = 0; c < ring_count(d); ++c)
        for (int r = 0; r < 3; ++r)
          if (std::fabs(out.st.s[d][c][r] - out.st.s[d - 7][c][r]) > 1e-13 * (cmax + 1e-300))
            THROW(HHG_ERR_STATE, "correction stencils of directions %d and %d differ", d - 7, d);
    if (d < 7) {
      out.st.S[d][0] = Sh[0];
      out.st.S[d][1] = Sh[4];
      out.st.S[d][2] = Sh[8];
      out.st.S[d][3] = Sh[1];
      out.st.S[d][4] = Sh[2];
      out.st.S[d][5] = Sh[5];
    } else {
      const double* S = out.st.S[d - 7];
      const double want[6] = {Sh[0], Sh[4], Sh[8], Sh[1], Sh[2], Sh[5]};
      for (int r = 0; r < 6; ++r)
        if (std::fabs(S[r] - want[r]) > 1e-12 * (1 + std::fabs(want[r])))
          THROW(HHG_ERR_STATE, "Shat(-d) != Shat(d) for direction %d", d);
    }
  }
}

// the centre terms of B, B^T and C at a macro-interior node, from the 24 elements around it
void check_stokes_row_sums(const MacroConsts<double>& mc) {
  double b0[3] = {0, 0, 0}, c0 = 0, scale = 0;
  for (int p = 0; p < 6; ++p)
    for (int a = 0; a < 4; ++a) {
      for (int l = 0; l < 3; ++l) b0[l] += mc.bd[p][a][a][l];
      c0 += mc.lc[p][a][a];
    }
  double sb[3] = {b0[0], b0[1], b0[2]}, sg[3] = {b0[0], b0[1], b0[2]}, sc = c0;
  for (int d = 0; d < NDIR; ++d) {
    for (int l = 0; l < 3; ++l) {
      sb[l] += mc.st.B[d][l];
      sg[l] += mc.st.G[d][l];
      scale = std::max(scale, std::fabs(mc.st.B[d][l]));
    }
    sc += mc.st.C[d];
  }
  for (int l = 0; l < 3; ++l)
    if (std::fabs(sb[l]) > 1e-12 * scale || std::fabs(sg[l]) > 1e-12 * scale || std::fabs(b0[l]) > 1e-12 * scale)
      THROW(HHG_ERR_STATE, "Stokes divergence stencil has a non-zero row sum");
  if (std::fabs(sc) > 1e-12 * (std::fabs(c0) + 1e-300)) THROW(HHG_ERR_STATE, "stabilisation row sum");
}

template <typename T>
MacroConsts<T> cast_consts(const MacroConsts<double>& c) {
  MacroConsts<T> o;
  const double* s = (const double*)&c;
  T* d = (T*)&o;
  static_assert(sizeof(MacroConsts<double>) / sizeof(double) == sizeof(MacroConsts<T>) / sizeof(T), "layout");
  for (size_t q = 0; q < sizeof(MacroConsts<double>) / sizeof(double); ++q) d[q] = (T)s[q];
  return o;
}



void build_level(hhg_ctx* c, int level) {
  auto L = std::make_unique<LevelHost>();
  const int n = 1 << level;
  const int M = (int)c->tets.size();
  L->level = level;
  L->n = n;
  L->nt = lattice_size(n);
  L->entries = L->nt * M;
  // tiles
  for (int k = 1; k <= n - 3; ++k)
    for (int j0 = 1; j0 <= n - 2 - k; j0 += TILE_J)
      for (int i0 = 1; i0 <= n - 1 - k - j0; i0 += TILE_I) L->tiles_int.push_back((k << 20) | (j0 << 10) | i0);
  for (int k = 0; k <= n; ++k)
    for (int j0 = 0; j0 <= n - k; j0 += TILE_J)
      for (int i0 = 0; i0 <= n - k - j0; i0 += TILE_I) L->tiles_all.push_back((k << 20) | (j0 << 10) | i0);
  // pairs of neighbouring interior points (i, i + 1) of slice k, row by row, in chunks of
  // INTERIOR_BLOCK: floor(M^2 / 4) pairs per slice (M = n - 1 - k)
  for (int k = 1; k <= n - 3; ++k) {
    const int M = n - 1 - k;
    const int count = M * M / 4;
    for (int start = 0; start < count; start += INTERIOR_BLOCK) L->tiles_pair.push_back((k << 20) | start);
  }
  // boxes of TILE3_I x TILE3_J x TILE3_K lattice points (i, j, k) with at least one
  // macro-interior point, for the shared-memory tile kernel
  for (int k0 = 1; k0 <= n - 3; k0 += TILE3_K)
    for (int j0 = 1; j0 <= n - 2 - k0; j0 += TILE3_J)
      for (int i0 = 1; i0 <= n - 1 - k0 - j0; i0 += TILE3_I) L->tiles3.push_back((k0 << 20) | (j0 << 10) | i0);
  // hybrid Gauss-Seidel colour chunks: for colour (ci, cj, ck) the rows j = cj (mod 2) of the
  // slices k = ck (mod 2), split into chunks of 32 points i = ci (mod 2)
  for (int col = 0; col < 8; ++col) {
    const int ci = col >> 2, cj = (col >> 1) & 1, ck = col & 1;
    L->gs_ptr[col] = (int32_t)L->gs_chunks.size();
    for (int k = 1; k <= n - 3; ++k) {
      if ((k & 1) != ck) continue;
      for (int j = 1; j <= n - 2 - k; ++j) {
        if ((j & 1) != cj) continue;
        const int last = n - 1 - j - k;
        for (int i0 = ci ? 1 : 2; i0 <= last; i0 += 64) L->gs_chunks.push_back((k << 20) | (j << 10) | i0);
      }
    }
  }
  L->gs_ptr[8] = (int32_t)L->gs_chunks.size();
  // interior points of slice k, enumerated row by row (j = 1..M-1, i = 1..M-j, M = n-1-k),
  // in chunks of INTERIOR_BLOCK
  for (int k = 1; k <= n - 3; ++k) {
    const int M = n - 1 - k;
    const int count = (M - 1) * M / 2;
    for (int start = 0; start < count; start += INTERIOR_BLOCK) L->tiles_lin.push_back((k << 20) | start);
  }
  // skeleton nodes
  std::unordered_map<std::array<int64_t, 3>, int32_t, KeyHash> skel_id;
  std::vector<std::vector<SkelInc>> incs;
  L->entry_to_unique.assign(L->entries, -1);
  int64_t nint = 0;
  for (int m = 0; m < M; ++m)
    for (int k = 0; k <= n; ++k)
      for (int j = 0; j <= n - k; ++j)
        for (int i = 0; i <= n - k - j; ++i) {
          const int64_t e = (int64_t)m * L->nt + lattice_index(n, i, j, k);
          if (lattice_interior(n, i, j, k)) {
            L->entry_to_unique[e] = nint++;
            continue;
          }
          const int64_t w[4] = {n - i - j - k, i, j, k};
          std::vector<std::pair<int64_t, int64_t>> kv;
          for (int q = 0; q < 4; ++q)
            if (w[q] > 0) kv.push_back({c->tets[m][q], w[q]});
          std::sort(kv.begin(), kv.end());
          std::array<int64_t, 3> key = {-1, -1, -1};
          for (size_t q = 0; q < kv.size(); ++q) key[q] = kv[q].first * 4096 + kv[q].second;
          auto it = skel_id.find(key);
          int32_t sid;
          if (it == skel_id.end()) {
            sid = (int32_t)incs.size();
            skel_id.emplace(key, sid);
            incs.emplace_back();
            L->skel_key.push_back(key);
            // Dirichlet if the node's support lies in a Dirichlet face
            bool dir = false;
            if (kv.size() == 3) {
              dir = c->dir_faces.count({kv[0].first, kv[1].first, kv[2].first}) > 0;
            } else if (kv.size() == 2) {
              dir = c->dir_edges.count({kv[0].first, kv[1].first}) > 0;
            } else {
              dir = c->dir_verts.count(kv[0].first) > 0;
            }
            L->skel_dir.push_back(dir ? 1 : 0);
            L->skel_support.push_back((int8_t)kv.size());
          } else {
            sid = it->second;
          }
          SkelInc I;
          I.macro = m;
          I.i = (int16_t)i;
          I.j = (int16_t)j;
          I.k = (int16_t)k;
          I.pad = 0;
          incs[sid].push_back(I);
        }
  const int64_t nskel = (int64_t)incs.size();
  L->skel_ptr.assign(nskel + 1, 0);
  for (int64_t s = 0; s < nskel; ++s) L->skel_ptr[s + 1] = L->skel_ptr[s] + (int32_t)incs[s].size();
  L->skel_inc.reserve(L->skel_ptr[nskel]);
  for (auto& v : incs)
    for (auto& I : v) L->skel_inc.push_back(I);
  L->nunique = nint + nskel;
  L->unique_first.assign(L->nunique, -1);
  L->unique_dir.assign(L->nunique, 0);
  L->mask.assign(L->entries, 0);
  for (int64_t e = 0; e < L->entries; ++e) {
    const int64_t u = L->entry_to_unique[e];
    if (u >= 0) {
      L->unique_first[u] = e;
      L->mask[e] = 1;
    }
  }
  for (int64_t s = 0; s < nskel; ++s) {
    const int64_t u = nint + s;
    for (int q = L->skel_ptr[s]; q < L->skel_ptr[s + 1]; ++q) {
      const SkelInc& I = L->skel_inc[q];
      const int64_t e = (int64_t)I.macro * L->nt + lattice_index(n, I.i, I.j, I.k);
      L->entry_to_unique[e] = u;
      if (q == L->skel_ptr[s]) {
        L->unique_first[u] = e;
        L->mask[e] = L->skel_dir[s] ? 0 : 1;
      }
    }
    L->unique_dir[u] = L->skel_dir[s];
  }
  for (const SkelInc& I : L->skel_inc) L->skel_entries.push_back((int64_t)I.macro * L->nt + lattice_index(n, I.i, I.j, I.k));
  L->nfree = L->nunique;
  for (int64_t s = 0; s < nskel; ++s) L->nfree -= L->skel_dir[s];
  L->mask_own.assign(L->entries, 0);
  for (int64_t u = 0; u < L->nunique; ++u) L->mask_own[L->unique_first[u]] = 1;
  // lumped mass (sum over the elements around a node of |t|/4); all elements of a macro
  // have the volume |T| / n^3
  {
    std::vector<double> volt(M);
    for (int m = 0; m < M; ++m) {
      Vec3d v[4];
      for (int q = 0; q < 4; ++q) v[q] = c->xyz[c->tets[m][q]];
      double g[4][3], vol;
      element_gradients(v, g, vol);
      volt[m] = vol / ((double)n * n * n);
    }
    auto elements_inside = [&](int i, int j, int k) {
      int cnt = 0;
      const int X = i + j + k, Y = j + k, Z = k;
      for (int p = 0; p < 6; ++p) {
        int P[4][3];
        kuhn_vertices(p, P);
        for (int av = 0; av < 4; ++av) {
          bool ok = true;
          for (int v = 0; v < 4 && ok; ++v) {
            const int VX = X - P[av][0] + P[v][0], VY = Y - P[av][1] + P[v][1], VZ = Z - P[av][2] + P[v][2];
            ok = 0 <= VZ && VZ <= VY && VY <= VX && VX <= n;
          }
          cnt += ok;
        }
      }
      return cnt;
    };
    std::vector<double> mu(L->nunique, 0.0);
    for (int m = 0; m < M; ++m)
      for (int64_t q = 0; q < L->nt; ++q) {
        const int64_t e = (int64_t)m * L->nt + q;
        const int64_t u = L->entry_to_unique[e];
        if (u < nint) mu[u] = 6.0 * volt[m];
      }
    for (int64_t s = 0; s < nskel; ++s)
      for (int q = L->skel_ptr[s]; q < L->skel_ptr[s + 1]; ++q) {
        const SkelInc& I = L->skel_inc[q];
        mu[nint + s] += 0.25 * volt[I.macro] * elements_inside(I.i, I.j, I.k);
      }
    L->lumped.resize(L->entries);
    for (int64_t e = 0; e < L->entries; ++e) L->lumped[e] = mu[L->entry_to_unique[e]];
  }
  // skeleton split for the kernels: free face-interior nodes, free edge/vertex nodes and
  // Dirichlet nodes; and the same face/edge-vertex split including Dirichlet nodes
  auto add_face = [&](int64_t s, std::vector<int32_t>& nodes, std::vector<FaceItem>& items) {
    const int32_t fid = (int32_t)nodes.size();
    nodes.push_back((int32_t)s);
    for (int q = L->skel_ptr[s]; q < L->skel_ptr[s + 1]; ++q) {
      const SkelInc& I = L->skel_inc[q];
      const int w[4] = {n - I.i - I.j - I.k, I.i, I.j, I.k};
      int f = -1, zeros = 0;
      for (int cc = 0; cc < 4; ++cc)
        if (w[cc] == 0) {
          f = cc;
          ++zeros;
        }
      if (zeros != 1) THROW(HHG_ERR_STATE, "face node with %d zero barycentric weights", zeros);
      FaceItem it;
      it.macro = I.macro;
      it.node = fid;
      it.i = I.i;
      it.j = I.j;
      it.k = I.k;
      it.f = (int16_t)f;
      items.push_back(it);
    }
  };
  std::vector<int64_t> free_face;
  for (int64_t s = 0; s < nskel; ++s) {
    if (L->skel_dir[s])
      L->dir_nodes.push_back((int32_t)s);
    else if (L->skel_support[s] == 3)
      free_face.push_back(s);
    else
      L->ev_nodes.push_back((int32_t)s);
    if (L->skel_support[s] == 3)
      add_face(s, L->face_nodes_all, L->face_items_all);
    else
      L->ev_all.push_back((int32_t)s);
  }
  // free face nodes ordered by their incidences (macro and face type of each), so that the
  // lanes of a warp of the face-row kernel take the same face types
  {
    auto face_type = [&](const SkelInc& I) {
      return (I.i + I.j + I.k == n) ? 0 : (I.i == 0) ? 1 : (I.j == 0) ? 2 : 3;
    };
    auto key = [&](int64_t s) {
      std::array<int64_t, 5> kk{};
      const int b0 = L->skel_ptr[s], b1 = L->skel_ptr[s + 1];
      for (int q = 0; q < 2; ++q) {
        if (b0 + q < b1) {
          kk[2 * q] = L->skel_inc[b0 + q].macro;
          kk[2 * q + 1] = face_type(L->skel_inc[b0 + q]);
        } else {
          kk[2 * q] = -1;
        }
      }
      kk[4] = s;
      return kk;
    };
    std::sort(free_face.begin(), free_face.end(), [&](int64_t a, int64_t b) { return key(a) < key(b); });
    for (int64_t s : free_face) add_face(s, L->face_nodes, L->face_items);
  }
  // group the face items by macro and face type so that the lanes of a warp share the
  // candidate set (the unrolled candidate loop then does not diverge)
  auto item_order = [](const FaceItem& a, const FaceItem& b) {
    if (a.macro != b.macro) return a.macro < b.macro;
    if (a.f != b.f) return a.f < b.f;
    if (a.k != b.k) return a.k < b.k;
    if (a.j != b.j) return a.j < b.j;
    return a.i < b.i;
  };
  std::stable_sort(L->face_items.begin(), L->face_items.end(), item_order);
  std::stable_sort(L->face_items_all.begin(), L->face_items_all.end(), item_order);
  // candidate elements around a face-interior point that lie inside the macro (per face
  // type); checked against every face item of this level
  auto cand_inside = [](int nn, int i, int j, int k, int bit) {
    const int p = bit >> 2, av = bit & 3;
    int P[4][3];
    kuhn_vertices(p, P);
    const int X = i + j + k, Y = j + k, Z = k;
    for (int v = 0; v < 4; ++v) {
      const int VX = X - P[av][0] + P[v][0], VY = Y - P[av][1] + P[v][1], VZ = Z - P[av][2] + P[v][2];
      if (!(0 <= VZ && VZ <= VY && VY <= VX && VX <= nn)) return false;
    }
    return true;
  };
  {
    const int nn = 16;
    const int rep[4][3] = {{5, 5, 6}, {0, 5, 5}, {5, 0, 5}, {5, 5, 0}};
    for (int f = 0; f < 4; ++f) {
      L->face_mask[f] = 0;
      for (int bit = 0; bit < 24; ++bit)
        if (cand_inside(nn, rep[f][0], rep[f][1], rep[f][2], bit)) L->face_mask[f] |= 1u << bit;
    }
    for (const FaceItem& it : L->face_items_all)
      for (int bit = 0; bit < 24; ++bit)
        if (cand_inside(n, it.i, it.j, it.k, bit) != (((L->face_mask[it.f] >> bit) & 1u) != 0))
          THROW(HHG_ERR_STATE, "face candidate mask mismatch");
  }
  for (int64_t e = 0; e < L->entries; ++e)
    if (L->entry_to_unique[e] < 0) THROW(HHG_ERR_STATE, "entry without node");
  c->levels[level] = std::move(L);
}

// restriction lists: coarse level lc, fine level lc+1
void build_restriction(hhg_ctx* c, int lc) {
  LevelHost& C = *c->levels[lc];
  LevelHost& F = *c->levels[lc + 1];
  const int nf = F.n;
  const int64_t nskel = (int64_t)C.skel_dir.size();
  C.rptr.assign(nskel + 1, 0);
  C.rent.clear();
  C.rw.clear();
  for (int64_t s = 0; s < nskel; ++s) {
    std::map<int64_t, std::pair<int64_t, double>> fine;  // unique fine node -> (entry, weight)
    if (!C.skel_dir[s]) {
      for (int q = C.skel_ptr[s]; q < C.skel_ptr[s + 1]; ++q) {
        const SkelInc& I = C.skel_inc[q];
        const int fi = 2 * I.i, fj = 2 * I.j, fk = 2 * I.k;
        for (int d = -1; d < NDIR; ++d) {
          const int qi = fi + (d < 0 ? 0 : dir_di(d)), qj = fj + (d < 0 ? 0 : dir_dj(d)),
                    qk = fk + (d < 0 ? 0 : dir_dk(d));
          if (!lattice_inside(nf, qi, qj, qk)) continue;
          const int64_t e = (int64_t)I.macro * F.nt + lattice_index(nf, qi, qj, qk);
          const int64_t u = F.entry_to_unique[e];
          if (F.unique_dir[u]) continue;
          fine.emplace(u, std::make_pair(e, d < 0 ? 1.0 : 0.5));
        }
      }
    }
    for (auto& kv : fine) {
      C.rent.push_back(kv.second.first);
      C.rw.push_back(kv.second.second);
    }
    C.rptr[s + 1] = (int32_t)C.rent.size();
  }
}

void upload_level(hhg_ctx* c, LevelHost& L) {
  upload(L.d_tiles_int, L.tiles_int);
  upload(L.d_tiles_all, L.tiles_all);
  upload(L.d_tiles_lin, L.tiles_lin);
  upload(L.d_tiles_pair, L.tiles_pair);
  upload(L.d_tiles3, L.tiles3);
  upload(L.d_gs_chunks, L.gs_chunks);
  upload(L.d_skel_entries, L.skel_entries);
  upload(L.d_skel_ptr, L.skel_ptr);
  upload(L.d_skel_inc, L.skel_inc);
  upload(L.d_skel_dir, L.skel_dir);
  upload(L.d_mask, L.mask);
  upload(L.d_mask_own, L.mask_own);
  {
    std::vector<double> im(L.entries);
    std::vector<float> im32(L.entries);
    for (int64_t e = 0; e < L.entries; ++e) {
      im[e] = 1.0 / L.lumped[e];
      im32[e] = (float)im[e];
    }
    upload(L.d_invm64, im);
    upload(L.d_invm32, im32);
    std::vector<float> m32(L.lumped.begin(), L.lumped.end());
    upload(L.d_mass64, L.lumped);
    upload(L.d_mass32, m32);
  }
  upload(L.d_face_items, L.face_items);
  upload(L.d_face_items_all, L.face_items_all);
  upload(L.d_face_nodes_all, L.face_nodes_all);
  upload(L.d_ev_all, L.ev_all);
  upload(L.d_face_nodes, L.face_nodes);
  upload(L.d_ev_nodes, L.ev_nodes);
  upload(L.d_dir_nodes, L.dir_nodes);
  CK(L.d_acc32.alloc(std::max<size_t>(1, L.face_nodes_all.size()) * 8 * sizeof(float)));
  CK(L.d_acc64.alloc(std::max<size_t>(1, L.face_nodes_all.size()) * 8 * sizeof(double)));
  CK(cudaMemset(L.d_acc32.p, 0, L.d_acc32.bytes));
  CK(cudaMemset(L.d_acc64.p, 0, L.d_acc64.bytes));
  upload(L.d_first, L.unique_first);
  upload(L.d_e2u, L.entry_to_unique);
  if (!L.rptr.empty()) {
    upload(L.d_rptr, L.rptr);
    upload(L.d_rent, L.rent);
    upload(L.d_rw64, L.rw);
    std::vector<float> rw32(L.rw.begin(), L.rw.end());
    upload(L.d_rw32, rw32);
  }
  CK(L.d_k64.alloc(L.entries * sizeof(double)));
  CK(L.d_k32.alloc(L.entries * sizeof(float)));
  LevelDev& D = L.dev;
  D.n = L.n;
  D.nmacro = (int)c->tets.size();
  D.nt = L.nt;
  D.entries = L.entries;
  D.ntiles_int = (int32_t)L.tiles_int.size();
  D.ntiles_all = (int32_t)L.tiles_all.size();
  D.tiles_int = L.d_tiles_int.as<int32_t>();
  D.tiles_all = L.d_tiles_all.as<int32_t>();
  D.ntiles_lin = (int32_t)L.tiles_lin.size();
  D.tiles_lin = L.d_tiles_lin.as<int32_t>();
  D.ntiles_pair = (int32_t)L.tiles_pair.size();
  D.tiles_pair = L.d_tiles_pair.as<int32_t>();
  D.ntiles3 = (int32_t)L.tiles3.size();
  D.tiles3 = L.d_tiles3.as<int32_t>();
  for (int q = 0; q < 9; ++q) D.gs_ptr[q] = L.gs_ptr[q];
  D.gs_chunks = L.d_gs_chunks.as<int32_t>();
  D.nskel_entries = (int64_t)L.skel_entries.size();
  D.skel_entries = L.d_skel_entries.as<int64_t>();
  D.nskel = (int32_t)L.skel_dir.size();
  D.skel_ptr = L.d_skel_ptr.as<int32_t>();
  D.skel_inc = L.d_skel_inc.as<SkelInc>();
  D.skel_dir = L.d_skel_dir.as<int8_t>();
  D.mask = L.d_mask.as<uint8_t>();
  D.nface_items = (int32_t)L.face_items.size();
  D.nface_nodes = (int32_t)L.face_nodes.size();
  D.nev = (int32_t)L.ev_nodes.size();
  D.ndir = (int32_t)L.dir_nodes.size();
  D.face_items = L.d_face_items.as<FaceItem>();
  D.face_nodes = L.d_face_nodes.as<int32_t>();
  D.ev_nodes = L.d_ev_nodes.as<int32_t>();
  D.dir_nodes = L.d_dir_nodes.as<int32_t>();
  for (int f = 0; f < 4; ++f) D.face_mask[f] = L.face_mask[f];
  D.nface_items_all = (int32_t)L.face_items_all.size();
  D.nface_nodes_all = (int32_t)L.face_nodes_all.size();
  D.nev_all = (int32_t)L.ev_all.size();
  D.face_items_all = L.d_face_items_all.as<FaceItem>();
  D.face_nodes_all = L.d_face_nodes_all.as<int32_t>();
  D.ev_all = L.d_ev_all.as<int32_t>();
  D.acc32 = L.d_acc32.as<float>();
  D.acc64 = L.d_acc64.as<double>();
}

}  // namespace


// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

hhg_status hhg_create(hhg_ctx** out, int device, void* stream) {
  if (!out) return HHG_ERR_ARG;
  *out = nullptr;
  hhg_ctx* c = nullptr;
  try {
    c = new hhg_ctx();
  } catch (...) {
    return HHG_ERR_OOM;
  }
  c->device = device;
  c->stream = (cudaStream_t)stream;
  hhg_status st = guard(c, [&] {
    CK(c->scalar.alloc(64 * sizeof(double)));
    CK(cudaMallocHost((void**)&c->pinned, 64 * sizeof(double)));
    CK(upload_direction_tables());
  });
  if (st != HHG_OK) {
    delete c;
    return st;
  }
  *out = c;
  return HHG_OK;
}

hhg_status hhg_destroy(hhg_ctx* c) {
  if (!c) return HHG_ERR_ARG;
  cudaSetDevice(c->device);
  delete c;
  return HHG_OK;
}

const char* hhg_last_error(hhg_ctx* c) { return c ? c->err.c_str() : "null context"; }

hhg_status hhg_set_timeout(hhg_ctx* c, int64_t ms) {
  return guard(c, [&] {
    if (ms <= 0) THROW(HHG_ERR_ARG, "timeout must be positive");
    c->timeout_ms = ms;
  });
}

hhg_status hhg_set_macro_mesh(hhg_ctx* c, const double* xyz, int64_t nverts, const int64_t* tets, int64_t ntets,
                              const int32_t* dflags) {
  return guard(c, [&] {
    if (!xyz || !tets || nverts < 4 || ntets < 1) THROW(HHG_ERR_ARG, "empty mesh");
    if (nverts >= (1LL << 40)) THROW(HHG_ERR_ARG, "too many vertices");
    c->xyz.resize(nverts);
    for (int64_t v = 0; v < nverts; ++v) c->xyz[v] = {xyz[3 * v], xyz[3 * v + 1], xyz[3 * v + 2]};
    c->tets.resize(ntets);
    std::map<std::array<int64_t, 3>, int> fcount;
    for (int64_t t = 0; t < ntets; ++t) {
      for (int q = 0; q < 4; ++q) {
        const int64_t v = tets[4 * t + q];
        if (v < 0 || v >= nverts) THROW(HHG_ERR_ARG, "tet %lld has bad vertex id", (long long)t);
        c->tets[t][q] = v;
      }
      MacroGeom G;
      for (int q = 0; q < 4; ++q) G.v[q] = c->xyz[c->tets[t][q]];
      double K[4][4][9];
      element_stiffness(G.v, 1.0, 0.0, K);  // throws on degenerate tets
      for (int f = 0; f < 4; ++f) {
        std::array<int64_t, 3> key;
        int r = 0;
        for (int q = 0; q < 4; ++q)
          if (q != f) key[r++] = c->tets[t][q];
        std::sort(key.begin(), key.end());
        fcount[key]++;
      }
    }
    c->dir_faces.clear();
    c->dir_edges.clear();
    c->dir_verts.clear();
    for (int64_t t = 0; t < ntets; ++t)
      for (int f = 0; f < 4; ++f) {
        std::array<int64_t, 3> key;
        int r = 0;
        for (int q = 0; q < 4; ++q)
          if (q != f) key[r++] = c->tets[t][q];
        std::sort(key.begin(), key.end());
        const bool dir = dflags ? dflags[4 * t + f] != 0 : fcount[key] == 1;
        if (dir) c->dir_faces.insert(key);
      }
    for (const auto& f : c->dir_faces) {
      c->dir_edges.insert({f[0], f[1]});
      c->dir_edges.insert({f[0], f[2]});
      c->dir_edges.insert({f[1], f[2]});
      for (int q = 0; q < 3; ++q) c->dir_verts.insert(f[q]);
    }
    c->have_mesh = true;
    c->levels.clear();
    c->level_max = -1;
    c->level_min = 2;
    c->have_problem = false;
    c->have_coeff = false;
  });
}

hhg_status hhg_traction_load(hhg_ctx* c, int level, hhg_dtype dt, const int32_t* face_flags, const void* t_dev,
                             void* f_dev) {
  return guard(c, [&] {
    LevelHost& L = c->lv(level);
    if (!face_flags || !t_dev || !f_dev) THROW(HHG_ERR_ARG, "null argument");
    if (dt != HHG_F64 && dt != HHG_F32) THROW(HHG_ERR_ARG, "dtype");
    const int n = L.n;
    const int M = (int)c->tets.size();
    std::map<std::array<int64_t, 3>, int> fcount;
    auto face_key = [&](int t, int f) {
      std::array<int64_t, 3> key;
      int r = 0;
      for (int q = 0; q < 4; ++q)
        if (q != f) key[r++] = c->tets[t][q];
      std::sort(key.begin(), key.end());
      return key;
    };
    for (int t = 0; t < M; ++t)
      for (int f = 0; f < 4; ++f) fcount[face_key(t, f)]++;
    // flagged faces: their area per refined triangle and the entries of their lattice points
    const int npf = (n + 1) * (n + 2) / 2;
    std::vector<double> area;
    std::vector<int64_t> pent;
    for (int t = 0; t < M; ++t)
      for (int f = 0; f < 4; ++f) {
        if (!face_flags[4 * t + f]) continue;
        if (fcount[face_key(t, f)] != 1) THROW(HHG_ERR_ARG, "face %d of tetrahedron %d is not on the boundary", f, t);
        int v[3], r = 0;
        for (int q = 0; q < 4; ++q)
          if (q != f) v[r++] = (int)c->tets[t][q];
        const Vec3d& A = c->xyz[v[0]];
        const Vec3d& B = c->xyz[v[1]];
        const Vec3d& C = c->xyz[v[2]];
        const double ux = B.x - A.x, uy = B.y - A.y, uz = B.z - A.z;
        const double wx = C.x - A.x, wy = C.y - A.y, wz = C.z - A.z;
        const double cx = uy * wz - uz * wy, cy = uz * wx - ux * wz, cz = ux * wy - uy * wx;
        area.push_back(0.5 * std::sqrt(cx * cx + cy * cy + cz * cz) / ((double)n * n));
        // face point (a, b) -> lattice point (i, j, k) of macro t on face f (f = 0: i + j + k = n,
        // 1: i = 0, 2: j = 0, 3: k = 0)
        for (int b = 0; b <= n; ++b)
          for (int a = 0; a + b <= n; ++a) {
            int i, j, k;
            if (f == 0) {
              j = a; k = b; i = n - a - b;
            } else if (f == 1) {
              i = 0; j = a; k = b;
            } else if (f == 2) {
              j = 0; i = a; k = b;
            } else {
              k = 0; i = a; j = b;
            }
            pent.push_back((int64_t)t * L.nt + lattice_index(n, i, j, k));
          }
      }
    const int nslots = (int)area.size();
    if (nslots == 0) return;
    // per free boundary node: its contributions (slot-major order) and all its copies
    std::map<int64_t, std::vector<int64_t>> contrib_of;
    for (int64_t g = 0; g < (int64_t)pent.size(); ++g) {
      const int64_t u = L.entry_to_unique[pent[g]];
      if (!L.unique_dir[u]) contrib_of[u].push_back(g);
    }
    std::map<int64_t, std::vector<int64_t>> copies;
    for (const auto& kv : contrib_of) copies[kv.first];
    for (int64_t e = 0; e < L.entries; ++e) {
      auto it = copies.find(L.entry_to_unique[e]);
      if (it != copies.end()) it->second.push_back(e);
    }
    std::vector<int64_t> cptr{0}, cidx, eptr{0}, eidx;
    for (const auto& kv : contrib_of) {
      cidx.insert(cidx.end(), kv.second.begin(), kv.second.end());
      cptr.push_back((int64_t)cidx.size());
      const auto& cp = copies[kv.first];
      eidx.insert(eidx.end(), cp.begin(), cp.end());
      eptr.push_back((int64_t)eidx.size());
    }
    DevMem d_area, d_pent, d_contrib, d_cptr, d_cidx, d_eptr, d_eidx;
    upload(d_area, area);
    upload(d_pent, pent);
    upload(d_cptr, cptr);
    upload(d_cidx, cidx);
    upload(d_eptr, eptr);
    upload(d_eidx, eidx);
    CK(d_contrib.alloc(3 * pent.size() * sizeof(double)));
    const int64_t nn = (int64_t)contrib_of.size();
    if (dt == HHG_F64)
      CK(launch_traction_load<double>(n, nslots, d_area.as<double>(), d_pent.as<int64_t>(), L.entries,
                                      (const double*)t_dev, d_contrib.as<double>(), nn, d_cptr.as<int64_t>(),
                                      d_cidx.as<int64_t>(), d_eptr.as<int64_t>(), d_eidx.as<int64_t>(),
                                      (double*)f_dev, c->stream));
    else
      CK(launch_traction_load<float>(n, nslots, d_area.as<double>(), d_pent.as<int64_t>(), L.entries,
                                     (const float*)t_dev, d_contrib.as<double>(), nn, d_cptr.as<int64_t>(),
                                     d_cidx.as<int64_t>(), d_eptr.as<int64_t>(), d_eidx.as<int64_t>(),
                                     (float*)f_dev, c->stream));
    wait_stream(c);  // the temporaries are freed on return
  });
}

hhg_status hhg_apply_2d(hhg_ctx* c, const double* tri_host, int level, double nu, int variant, hhg_dtype dt,
                        const void* k_dev, const void* x_dev, void* y_dev) {
  return guard(c, [&] {
    if (!tri_host || !k_dev || !x_dev || !y_dev) THROW(HHG_ERR_ARG, "null argument");
    if (x_dev == y_dev) THROW(HHG_ERR_ARG, "x and y must be distinct buffers");
    if (level < 1 || level > 14) THROW(HHG_ERR_ARG, "level must be in [1, 14]");
    if (!(nu > -1.0 && nu < 0.5)) THROW(HHG_ERR_ARG, "Poisson ratio out of range");
    if (variant != HHG_PHYSICAL && variant != HHG_UNPHYSICAL && variant != HHG_NODAL)
      THROW(HHG_ERR_UNSUPPORTED, "the 2D variant is built for the physical and unphysical scalings and nodal "
                                 "integration");
    const double ce = 1.0 / (1.0 + nu), cd = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    Stencil2D<double> st64{};
    const int n = 1 << level;
    if (stencil_2d(tri_host, n, ce, cd, variant == HHG_PHYSICAL ? 1 : variant == HHG_NODAL ? 2 : 0, &st64) != 0)
      THROW(HHG_ERR_ARG, "degenerate macro triangle");
    if (dt == HHG_F64) {
      CK(launch_apply_2d<double>(n, st64, (const double*)k_dev, (const double*)x_dev, (double*)y_dev, c->stream));
    } else if (dt == HHG_F32) {
      Stencil2D<float> st32{};
      for (int d = 0; d < 6; ++d) {
        for (int q = 0; q < 4; ++q) st32.S[d][q] = (float)st64.S[d][q];
        st32.w[d] = (float)st64.w[d];
        st32.p[d] = st64.p[d];
        st32.pm[d] = st64.pm[d];
        for (int q = 0; q < 4; ++q) {
          st32.Kt[d][q] = (float)st64.Kt[d][q];
          st32.Ktm[d][q] = (float)st64.Ktm[d][q];
        }
      }
      st32.nodal = st64.nodal;
      CK(launch_apply_2d<float>(n, st32, (const float*)k_dev, (const float*)x_dev, (float*)y_dev, c->stream));
    } else {
      THROW(HHG_ERR_ARG, "dtype");
    }
  });
}

hhg_status hhg_set_strain_fit(hhg_ctx* c, int degree) {
  return guard(c, [&] {
    if (degree != 1 && degree != 2) THROW(HHG_ERR_ARG, "strain-rate fit degree must be 1 or 2");
    c->strain_degree = degree;
  });
}

hhg_status hhg_set_coarsest_level(hhg_ctx* c, int level) {
  return guard(c, [&] {
    if (level < 0 || level > 9) THROW(HHG_ERR_ARG, "coarsest level must be in [0, 9]");
    if (c->level_max >= 0) THROW(HHG_ERR_STATE, "set the coarsest level before hhg_refine");
    c->level_min = level;
  });
}

hhg_status hhg_refine(hhg_ctx* c, int level_max) {
  return guard(c, [&] {
    if (!c->have_mesh) THROW(HHG_ERR_STATE, "mesh not set");
    if (level_max < c->level_min || level_max > 9)
      THROW(HHG_ERR_ARG, "level_max must be in [%d, 9] (the coarsest level to 9)", c->level_min);
    c->levels.clear();
    c->levels.resize(level_max + 1);
    c->level_max = level_max;
    for (int l = c->level_min; l <= level_max; ++l) build_level(c, l);
    for (int l = c->level_min; l < level_max; ++l) build_restriction(c, l);
    for (int l = c->level_min; l <= level_max; ++l) upload_level(c, *c->levels[l]);
    CK(c->scratch.alloc(max_partials(c) * sizeof(double)));
    c->have_problem = false;
    c->have_coeff = false;
  });
}

hhg_status hhg_set_problem(hhg_ctx* c, const hhg_problem* p) {
  return guard(c, [&] {
    c->drop_graphs();
    if (!p) THROW(HHG_ERR_ARG, "null problem");
    if (!c->have_mesh || c->level_max < 0) THROW(HHG_ERR_STATE, "refine first");
    double ce, cd;
    if (p->kind == HHG_ELASTICITY) {
      if (!(p->nu > -1.0 && p->nu < 0.5)) THROW(HHG_ERR_ARG, "Poisson ratio out of range");
      ce = 1.0 / (1.0 + p->nu);
      cd = p->nu / ((1.0 + p->nu) * (1.0 - 2.0 * p->nu));
    } else if (p->kind == HHG_STOKES) {
      ce = 2.0;
      cd = 0.0;
    } else {
      THROW(HHG_ERR_ARG, "unknown problem kind");
    }
    if (p->variant != HHG_PHYSICAL && p->variant != HHG_UNPHYSICAL && p->variant != HHG_NODAL &&
        p->variant != HHG_STORED)
      THROW(HHG_ERR_ARG, "bad variant");
    if ((p->variant == HHG_NODAL || p->variant == HHG_STORED) && p->kind != HHG_ELASTICITY)
      THROW(HHG_ERR_UNSUPPORTED, "the nodal-integration and stored-stencil variants are built for elasticity");
    if (p->khat != HHG_KHAT_PATCH && p->khat != HHG_KHAT_EDGE) THROW(HHG_ERR_ARG, "bad khat");
    if (p->iface != HHG_IFACE_SYMMETRIC && p->iface != HHG_IFACE_PRACTICAL) THROW(HHG_ERR_ARG, "bad iface");
    for (int l = c->level_min; l <= c->level_max; ++l) {
      LevelHost& L = *c->levels[l];
      const int M = (int)c->tets.size();
      std::vector<MacroConsts<double>> mc64(M);
      std::vector<MacroConsts<float>> mc32(M);
      L.st64.resize(M);
      L.st32.resize(M);
      L.nc64.resize(M);
      L.nc32.resize(M);
      for (int m = 0; m < M; ++m) {
        MacroGeom G;
        for (int q = 0; q < 4; ++q) G.v[q] = c->xyz[c->tets[m][q]];
        macro_constants(G, L.n, ce, cd, mc64[m]);
        check_stokes_row_sums(mc64[m]);
        mc32[m] = cast_consts<float>(mc64[m]);
        L.st64[m] = mc64[m].st;
        L.st32[m] = mc32[m].st;
        std::memcpy(L.nc64[m].ke, mc64[m].ke, sizeof(L.nc64[m].ke));
        std::memcpy(L.nc32[m].ke, mc32[m].ke, sizeof(L.nc32[m].ke));
      }
      upload(L.d_mc64, mc64);
      upload(L.d_mc32, mc32);
      if (p->kind == HHG_STOKES) {
        // diagonal of -C (pressure stabilisation) at every node: sum over the elements
        // around it, in every incident macro, of the element matrix's diagonal entry
        const int n = L.n;
        auto inside = [&](int i, int j, int k, int pp, int av) {
          const int X = i + j + k, Y = j + k, Z = k;
          int P[4][3];
          kuhn_vertices(pp, P);
          for (int v = 0; v < 4; ++v) {
            const int VX = X - P[av][0] + P[v][0], VY = Y - P[av][1] + P[v][1], VZ = Z - P[av][2] + P[v][2];
            if (!(0 <= VZ && VZ <= VY && VY <= VX && VX <= n)) return false;
          }
          return true;
        };
        std::vector<double> du(L.nunique, 0.0);
        const int64_t nint = L.nunique - (int64_t)L.skel_dir.size();
        std::vector<double> dint(M, 0.0);
        for (int m = 0; m < M; ++m)
          for (int pp = 0; pp < 6; ++pp)
            for (int av = 0; av < 4; ++av) dint[m] -= mc64[m].lc[pp][av][av];
        for (int m = 0; m < M; ++m)
          for (int64_t q = 0; q < L.nt; ++q) {
            const int64_t u = L.entry_to_unique[(int64_t)m * L.nt + q];
            if (u < nint) du[u] = dint[m];
          }
        for (int64_t sk = 0; sk < (int64_t)L.skel_dir.size(); ++sk)
          for (int q = L.skel_ptr[sk]; q < L.skel_ptr[sk + 1]; ++q) {
            const SkelInc& I = L.skel_inc[q];
            for (int pp = 0; pp < 6; ++pp)
              for (int av = 0; av < 4; ++av)
                if (inside(I.i, I.j, I.k, pp, av)) du[nint + sk] -= mc64[I.macro].lc[pp][av][av];
          }
        std::vector<double> d64(L.entries);
        for (int64_t e = 0; e < L.entries; ++e) d64[e] = du[L.entry_to_unique[e]];
        std::vector<float> d32(d64.begin(), d64.end());
        upload(L.d_sdiag64, d64);
        upload(L.d_sdiag32, d32);
      }
    }
    c->prob = *p;
    c->flags.physical = (p->variant == HHG_PHYSICAL || p->variant == HHG_STORED) ? 1 : 0;
    c->flags.stored = p->variant == HHG_STORED ? 1 : 0;
    ++c->problem_version;
    c->flags.khat_edge = p->khat == HHG_KHAT_EDGE ? 1 : 0;
    // the nodal variant is a_h on every row: skeleton rows by the a_h (practical) rule
    c->flags.practical = (p->iface == HHG_IFACE_PRACTICAL || p->variant == HHG_NODAL) ? 1 : 0;
    c->flags.nodal = p->variant == HHG_NODAL ? 1 : 0;
    c->have_problem = true;
  });
}

hhg_status hhg_num_nodes(hhg_ctx* c, int level, int64_t* entries, int64_t* unique_nodes, int64_t* free_nodes) {
  return guard(c, [&] {
    LevelHost& L = c->lv(level);
    if (entries) *entries = L.entries;
    if (unique_nodes) *unique_nodes = L.nunique;
    if (free_nodes) *free_nodes = L.nfree;
  });
}

hhg_status hhg_entry_coords(hhg_ctx* c, int level, double* xyz) {
  return guard(c, [&] {
    LevelHost& L = c->lv(level);
    if (!xyz) THROW(HHG_ERR_ARG, "null output");
    const int n = L.n;
    for (size_t m = 0; m < c->tets.size(); ++m) {
      Vec3d v[4];
      for (int q = 0; q < 4; ++q) v[q] = c->xyz[c->tets[m][q]];
      for (int k = 0; k <= n; ++k)
        for (int j = 0; j <= n - k; ++j)
          for (int i = 0; i <= n - k - j; ++i) {
            const int64_t e = (int64_t)m * L.nt + lattice_index(n, i, j, k);
            const double a = (double)i / n, b = (double)j / n, g = (double)k / n;
            xyz[3 * e] = v[0].x + a * (v[1].x - v[0].x) + b * (v[2].x - v[0].x) + g * (v[3].x - v[0].x);
            xyz[3 * e + 1] = v[0].y + a * (v[1].y - v[0].y) + b * (v[2].y - v[0].y) + g * (v[3].y - v[0].y);
            xyz[3 * e + 2] = v[0].z + a * (v[1].z - v[0].z) + b * (v[2].z - v[0].z) + g * (v[3].z - v[0].z);
          }
    }
  });
}

hhg_status hhg_entry_to_unique(hhg_ctx* c, int level, int64_t* map, int8_t* dir) {
  return guard(c, [&] {
    LevelHost& L = c->lv(level);
    if (!map) THROW(HHG_ERR_ARG, "null output");
    std::memcpy(map, L.entry_to_unique.data(), L.entries * sizeof(int64_t));
    if (dir) std::memcpy(dir, L.unique_dir.data(), L.nunique);
  });
}

hhg_status hhg_gather_unique(hhg_ctx* c, int level, hhg_dtype dt, int comps, const void* src, void* dst) {
  return guard(c, [&] {
    LevelHost& L = c->lv(level);
    if (!src || !dst || comps < 1 || comps > 4) THROW(HHG_ERR_ARG, "bad arguments");
    if (dt == HHG_F64)
      CK(launch_gather<double>(L.nunique, comps, L.entries, L.nunique, L.d_first.as<int64_t>(), (const double*)src,
                               (double*)dst, c->stream));
    else if (dt == HHG_F32)
      CK(launch_gather<float>(L.nunique, comps, L.entries, L.nunique, L.d_first.as<int64_t>(), (const float*)src,
                              (float*)dst, c->stream));
    else
      THROW(HHG_ERR_ARG, "dtype");
  });
}

hhg_status hhg_scatter_unique(hhg_ctx* c, int level, hhg_dtype dt, int comps, const void* src, void* dst) {
  return guard(c, [&] {
    LevelHost& L = c->lv(level);
    if (!src || !dst || comps < 1 || comps > 4) THROW(HHG_ERR_ARG, "bad arguments");
    if (dt == HHG_F64)
      CK(launch_gather<double>(L.entries, comps, L.nunique, L.entries, L.d_e2u.as<int64_t>(), (const double*)src,
                               (double*)dst, c->stream));
    else if (dt == HHG_F32)
      CK(launch_gather<float>(L.entries, comps, L.nunique, L.entries, L.d_e2u.as<int64_t>(), (const float*)src,
                              (float*)dst, c->stream));
    else
      THROW(HHG_ERR_ARG, "dtype");
  });
}

hhg_status hhg_set_coefficient(hhg_ctx* c, const void* k, hhg_dtype dt) {
  return guard(c, [&] {
    c->drop_graphs();
    if (!c->have_mesh || c->level_max < 0) THROW(HHG_ERR_STATE, "refine first");
    if (!k) THROW(HHG_ERR_ARG, "null coefficient");
    LevelHost& F = *c->levels[c->level_max];
    if (dt == HHG_F64) {
      CK(cudaMemcpyAsync(F.d_k64.p, k, F.entries * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    } else if (dt == HHG_F32) {
      CK(launch_convert<float, double>(F.entries, (const float*)k, F.d_k64.as<double>(), c->stream));
    } else if (dt == HHG_BF16) {
      CK(launch_bf16_to_f64(F.entries, (const uint16_t*)k, F.d_k64.as<double>(), c->stream));
    } else {
      THROW(HHG_ERR_ARG, "coefficient dtype");
    }
    c->coeff_bf16 = dt == HHG_BF16;
    for (int l = c->level_max; l > c->level_min; --l) {
      LevelHost& Lf = *c->levels[l];
      LevelHost& Lc = *c->levels[l - 1];
      CK(launch_inject<double>(Lf.dev, Lc.dev, Lf.d_k64.as<double>(), Lc.d_k64.as<double>(), c->stream));
    }
    for (int l = c->level_min; l <= c->level_max; ++l) {
      LevelHost& L = *c->levels[l];
      if (c->coeff_bf16) {  // values are BF16 already: the rounding below is exact
        if (!L.d_k16.p) CK(L.d_k16.alloc(L.entries * sizeof(uint16_t)));
        CK(launch_round_bf16(L.entries, L.d_k64.as<double>(), L.d_k32.as<float>(), L.d_k16.as<uint16_t>(),
                             c->stream));
      } else {
        CK(launch_convert<double, float>(L.entries, L.d_k64.as<double>(), L.d_k32.as<float>(), c->stream));
      }
    }
    c->have_coeff = true;
    ++c->coeff_version;
    // the multigrid data (diagonals, lambda_max, coarse inverse) depend on the coefficient
    c->mg_ready = false;
    for (int l = c->level_min; l <= c->level_max; ++l) c->levels[l]->lambda_set = false;
  });
}

hhg_status hhg_apply(hhg_ctx* c, int level, hhg_dtype dt, const void* x, void* y) {
  return guard(c, [&] {
    need_ready(c, true);
    if (!x || !y || x == y) THROW(HHG_ERR_ARG, "x and y must be distinct device buffers");
    if (dt == HHG_F64) {
      SweepArgs<double> a{};
      a.x = (const double*)x;
      a.out = (double*)y;
      sweep<double>(c, level, OP_APPLY, a, nullptr);
    } else if (dt == HHG_F32) {
      SweepArgs<float> a{};
      a.x = (const float*)x;
      a.out = (float*)y;
      sweep<float>(c, level, OP_APPLY, a, nullptr);
    } else {
      THROW(HHG_ERR_ARG, "dtype");
    }
  });
}

hhg_status hhg_residual(hhg_ctx* c, int level, hhg_dtype dt, const void* f, const void* x, void* r, double* norm2) {
  return guard(c, [&] {
    need_ready(c, true);
    if (!x || !r || !f || x == r || f == r) THROW(HHG_ERR_ARG, "bad buffers");
    if (dt == HHG_F64) {
      SweepArgs<double> a{};
      a.x = (const double*)x;
      a.f = (const double*)f;
      a.out = (double*)r;
      sweep<double>(c, level, OP_RESID, a, norm2);
    } else if (dt == HHG_F32) {
      SweepArgs<float> a{};
      a.x = (const float*)x;
      a.f = (const float*)f;
      a.out = (float*)r;
      sweep<float>(c, level, OP_RESID, a, norm2);
    } else {
      THROW(HHG_ERR_ARG, "dtype");
    }
  });
}

hhg_status hhg_apply_host(hhg_ctx* c, int level, hhg_dtype dt, const void* x_host, void* y_host) {
  return guard(c, [&] {
    need_ready(c, true);
    if (!x_host || !y_host) THROW(HHG_ERR_ARG, "null host buffer");
    LevelHost& L = c->lv(level);
    const size_t es = dt == HHG_F64 ? sizeof(double) : dt == HHG_F32 ? sizeof(float) : 0;
    if (!es) THROW(HHG_ERR_ARG, "dtype");
    const size_t bytes = 3 * (size_t)L.entries * es;
    if (c->hx.bytes < bytes) {
      CK(c->hx.alloc(bytes));
      CK(c->hy.alloc(bytes));
    }
    CK(cudaMemcpyAsync(c->hx.p, x_host, bytes, cudaMemcpyHostToDevice, c->stream));
    if (dt == HHG_F64) {
      SweepArgs<double> a{};
      a.x = c->hx.as<double>();
      a.out = c->hy.as<double>();
      sweep<double>(c, level, OP_APPLY, a, nullptr);
    } else {
      SweepArgs<float> a{};
      a.x = c->hx.as<float>();
      a.out = c->hy.as<float>();
      sweep<float>(c, level, OP_APPLY, a, nullptr);
    }
    CK(cudaMemcpyAsync(y_host, c->hy.p, bytes, cudaMemcpyDeviceToHost, c->stream));
    wait_stream(c);
  });
}

// Allocation-free residual with norm: same result as hhg_residual(..., norm2_host), with
// the scratch in a static device array instead of context-owned memory (see hhg.h).
hhg_status hhg_residual_noalloc(hhg_ctx* c, int level, hhg_dtype dt, const void* f, const void* x, void* r,
                                double* norm2_host) {
  return guard(c, [&] {
    need_ready(c, true);
    if (!x || !r || !f || !norm2_host || x == r || f == r) THROW(HHG_ERR_ARG, "bad buffers");
    LevelHost& L = c->lv(level);
    if (c->flags.nodal) THROW(HHG_ERR_UNSUPPORTED, "the no-alloc residual is built for the scaled-stencil variants");
    const int64_t need = noalloc_partials_needed(L.dev);
    if (need > NOALLOC_SLOTS)
      THROW(HHG_ERR_ARG, "level %d needs %lld partial sums; the no-alloc scratch holds %lld (use hhg_residual)", level,
            (long long)need, (long long)NOALLOC_SLOTS);
    double* scratch = nullptr;
    CK(noalloc_scratch_address(c->device, &scratch));
    if (dt == HHG_F64) {
      SweepArgs<double> a{};
      a.x = (const double*)x;
      a.f = (const double*)f;
      a.out = (double*)r;
      a.k = L.d_k64.as<double>();
      CK(launch_residual_noalloc<double>(L.dev, L.st64.data(), L.d_mc64.as<MacroConsts<double>>(), c->flags, a,
                                         scratch, c->stream));
    } else if (dt == HHG_F32) {
      SweepArgs<float> a{};
      a.x = (const float*)x;
      a.f = (const float*)f;
      a.out = (float*)r;
      a.k = L.d_k32.as<float>();
      CK(launch_residual_noalloc<float>(L.dev, L.st32.data(), L.d_mc32.as<MacroConsts<float>>(), c->flags, a, scratch,
                                        c->stream));
    } else {
      THROW(HHG_ERR_ARG, "dtype");
    }
    CK(cudaMemcpyAsync(c->pinned, scratch + NOALLOC_SLOTS, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    wait_stream_noalloc(c);
    *norm2_host = c->pinned[0];
  });
}

hhg_status hhg_profile(hhg_ctx* c, int enable, double* ms_host, int64_t* launches_host) {
  return guard(c, [&] {
    if (ms_host || launches_host) {
      wait_stream(c);
      for (int part = 0; part < 2; ++part) {
        double tot = 0.0;
        for (auto& pr : c->prof_ev[part]) {
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, pr[0], pr[1]));
          tot += ms;
        }
        if (ms_host) ms_host[part] = tot;
        if (launches_host) launches_host[part] = c->prof_launches[part];
      }
    }
    for (int part = 0; part < 2; ++part) {
      for (auto& pr : c->prof_ev[part]) {
        c->ev_pool.push_back(pr[0]);
        c->ev_pool.push_back(pr[1]);
      }
      c->prof_ev[part].clear();
      c->prof_launches[part] = 0;
    }
    c->prof = enable != 0;
  });
}

hhg_status hhg_set_interior_kernel(hhg_ctx* c, int kernel) {
  return guard(c, [&] {
    if (kernel < 0 || kernel > 3) THROW(HHG_ERR_ARG, "interior kernel must be 0, 1, 2 or 3");
    c->drop_graphs();
    c->interior_kernel = kernel;
    c->flags.tile = kernel == 1;
  });
}

hhg_status hhg_fp32_fma_probe(hhg_ctx* c, int packed, int64_t iterations, float* out_dev, double* flops_host,
                              int* sm_count_host) {
  return guard(c, [&] {
    if (!out_dev || !flops_host || iterations < 1 || (packed != 0 && packed != 1)) THROW(HHG_ERR_ARG, "probe arguments");
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    if (sm_count_host) *sm_count_host = sms;
    CK(launch_fma_probe(packed, iterations, sms, out_dev, flops_host, c->stream));
  });
}

}  // extern "C"
