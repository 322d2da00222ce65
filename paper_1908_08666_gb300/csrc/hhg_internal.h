// Internal structures shared by the host setup (hhg_host.cpp) and the CUDA
// kernels (hhg_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define HHG_HD __host__ __device__ __forceinline__
#else
#define HHG_HD inline
#endif

namespace hhg {

// ---------------------------------------------------------------------------
// Lattice of one refined macro.  Corner coordinates (i, j, k) with i+j+k <= n
// address the point v0 + (i (v1-v0) + j (v2-v0) + k (v3-v0)) / n.  In the
// coordinates X = i+j+k, Y = j+k, Z = k the macro is {0 <= Z <= Y <= X <= n}
// and Bey's refinement is the Freudenthal (Kuhn) lattice: its edges are the
// seven 0/1 vectors and their negatives, its elements the Kuhn simplices
// c, c+e_p0, c+e_p0+e_p1, c+(1,1,1) for the 6 permutations p (Sec. 2.4).
// ---------------------------------------------------------------------------

// The 14 stencil directions in corner coordinates.  d < 7 are the Kuhn 0/1
// vectors (1,0,0) (0,1,0) (0,0,1) (1,1,0) (0,1,1) (1,0,1) (1,1,1); d+7 = -d.
// Directions 0,1,2,6 (and negatives) lie in six elements ("red" edges),
// directions 3,4,5 (and negatives) in four.
constexpr int NDIR = 14;
HHG_HD int dir_di(int d) {
  const int t[7] = {1, -1, 0, 0, -1, 1, 0};
  return d < 7 ? t[d] : -t[d - 7];
}
HHG_HD int dir_dj(int d) {
  const int t[7] = {0, 1, -1, 1, 0, -1, 0};
  return d < 7 ? t[d] : -t[d - 7];
}
HHG_HD int dir_dk(int d) {
  const int t[7] = {0, 0, 1, 0, 1, 1, 1};
  return d < 7 ? t[d] : -t[d - 7];
}
HHG_HD int dir_neg(int d) { return d < 7 ? d + 7 : d - 7; }
HHG_HD bool dir_red(int d) {
  int e = d < 7 ? d : d - 7;
  return e == 0 || e == 1 || e == 2 || e == 6;
}
// Ring pairs of the edge (0, d): for every c the nodes r_c and its point
// reflection r_c^m = d - r_c through the edge midpoint, both neighbours of 0
// (stencil direction indices).  Red edges have three pairs, the others two.
HHG_HD int ring_count(int d) { return dir_red(d) ? 3 : 2; }
HHG_HD int ring_a(int d, int c) {
  const int t[7][3] = {{3, 5, 6}, {3, 4, 6}, {5, 4, 6}, {0, 6, -1}, {1, 6, -1}, {0, 6, -1}, {0, 1, 2}};
  return d < 7 ? t[d][c] : dir_neg(t[d - 7][c]);
}
HHG_HD int ring_b(int d, int c) {
  const int t[7][3] = {{8, 9, 11}, {7, 9, 12}, {7, 8, 10}, {1, 9, -1}, {2, 7, -1}, {2, 8, -1}, {4, 5, 3}};
  return d < 7 ? t[d][c] : dir_neg(t[d - 7][c]);
}

// direction index of the corner offset (di, dj, dk), -1 if it is not a stencil direction
HHG_HD int dir_of_offset(int di, int dj, int dk) {
  int r = -1;
#pragma unroll
  for (int d = 0; d < NDIR; ++d)
    if (dir_di(d) == di && dir_dj(d) == dj && dir_dk(d) == dk) r = d;
  return r;
}

HHG_HD int64_t tetnum(int64_t a) { return a * (a + 1) * (a + 2) / 6; }
HHG_HD int64_t lattice_size(int n) { return tetnum(n + 1); }
// compact index of (i, j, k) inside one macro
HHG_HD int64_t lattice_index(int n, int i, int j, int k) {
  const int64_t m = n - k;
  return tetnum(n + 1) - tetnum(n + 1 - k) + (int64_t)j * (2 * m + 3 - j) / 2 + i;
}
// 32-bit version for kernels (valid for n <= 1000)
HHG_HD int lattice_index32(int n, int i, int j, int k) {
  const int m = n - k;
  const int a = n + 1, b = n + 1 - k;
  return a * (a + 1) * (a + 2) / 6 - b * (b + 1) * (b + 2) / 6 + ((j * (2 * m + 3 - j)) >> 1) + i;
}
// compact indices of the 14 neighbours of (i, j, k) (32-bit, n <= 1000), from the
// starts of the seven lattice rows they lie in; an entry is meaningful only where that
// neighbour is a lattice point
HHG_HD void lattice_neighbours(int n, int i, int j, int k, int nb[NDIR]) {
  const int m = n - k;
  const int r00 = lattice_index32(n, i, j, k);
  const int r10 = r00 + (m + 1 - j);
  const int rm0 = r00 - (m + 2 - j);
  const int sz = (m + 1) * (m + 2) / 2;
  const int szm = (m + 2) * (m + 3) / 2;
  const int r01 = r00 + sz - j;
  const int r0m = r00 - szm + j;
  const int rm1 = rm0 + sz - j + 1;
  const int r1m = r10 - szm + j + 1;
  nb[0] = r00 + 1;
  nb[7] = r00 - 1;
  nb[1] = r10 - 1;
  nb[3] = r10;
  nb[2] = rm1;
  nb[5] = rm1 + 1;
  nb[4] = r01 - 1;
  nb[6] = r01;
  nb[8] = rm0 + 1;
  nb[10] = rm0;
  nb[9] = r1m;
  nb[12] = r1m - 1;
  nb[11] = r0m + 1;
  nb[13] = r0m;
}
HHG_HD bool lattice_inside(int n, int i, int j, int k) { return i >= 0 && j >= 0 && k >= 0 && i + j + k <= n; }
HHG_HD bool lattice_interior(int n, int i, int j, int k) {
  return i >= 1 && j >= 1 && k >= 1 && i + j + k <= n - 1;
}

// Kuhn element of permutation p: vertex a = c + P_a(p) (Kuhn coordinates).
HHG_HD void kuhn_perm(int p, int& a0, int& a1, int& a2) {
  const int t[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  a0 = t[p][0];
  a1 = t[p][1];
  a2 = t[p][2];
}

// ---------------------------------------------------------------------------
// per-macro constants
// ---------------------------------------------------------------------------

// Interior stencil of one macro (kernel parameter).  Shat for the 7 positive
// directions (Shat_{-d} = Shat_d), symmetric 3x3 stored xx yy zz xy xz yz; axial
// vectors of the correction matrices (eq. correctionterm3D): the antisymmetric
// matrix of ring pair c of direction d is [s[d][c]]_x, acting as s x v.
//
// Stokes blocks (Sec. 5.2, stabilised P1-P1; coefficient-free): divergence B,
// gradient B^T and stabilisation C = -(h^2/12)(grad p, grad q) in difference form
// over the 14 directions (their row sums vanish at macro-interior nodes):
//   (B u)_i = sum_d B[d] . (u_{i+d} - u_i),  (B^T p)_i = sum_d G[d] (p_{i+d} - p_i),
//   (C p)_i = sum_d C[d] (p_{i+d} - p_i).
template <typename T>
struct MacroStencil {
  T S[7][6];
  T s[NDIR][3][3];
  T B[NDIR][3];
  T G[NDIR][3];
  T C[NDIR];
};

// Constants of one macro for the skeleton kernel (global memory): the interior
// stencil plus the 6 element stiffness matrices K[type][a][b][m][l] (test
// vertex a, trial vertex b) of the Kuhn element types.
// Element matrices for the Stokes blocks: bd[type][a][b][l] = -int phi_a d_l phi_b
// (pressure test vertex a, velocity trial vertex b), lc[type][a][b] = -(h^2/12) int
// grad phi_a . grad phi_b.
// Element stiffness of one macro's 6 Kuhn element types for the nodal-integration
// interior kernel (kernel parameter, 864 values): ke[type][a][b][3 m + l].
template <typename T>
struct NodalConsts {
  T ke[6][4][4][9];
};

template <typename T>
struct MacroConsts {
  MacroStencil<T> st;
  T ke[6][4][4][9];
  T bd[6][4][4][3];
  T lc[6][4][4];
};

// one incidence of a skeleton node in a macro
struct SkelInc {
  int32_t macro;
  int16_t i, j, k;
  int16_t pad;
};

// one incidence of a node on a macro face (face-interior node) in a macro;
// f = which barycentric coordinate vanishes (0: i+j+k = n, 1: i = 0, 2: j = 0, 3: k = 0)
struct FaceItem {
  int32_t macro;
  int32_t node;  // index into the face-node list
  int16_t i, j, k;
  int16_t f;
};

// device view of one level
struct LevelDev {
  int n;
  int nmacro;
  int64_t nt;          // entries per macro
  int64_t entries;     // nmacro * nt
  int32_t ntiles_int;  // interior tiles
  int32_t ntiles_all;  // tiles over all lattice points
  int32_t ntiles_lin;  // 128-node chunks of the interior points of each slice: (k << 20) | start
  const int32_t* tiles_lin;
  int32_t ntiles_pair;  // 128-pair chunks of the point pairs of each slice (FP32 sweeps): (k << 20) | start
  const int32_t* tiles_pair;
  int32_t ntiles3;      // boxes of the shared-memory tile kernel: (k0 << 20) | (j0 << 10) | i0
  const int32_t* tiles3;
  // hybrid Gauss-Seidel: chunks of up to 32 macro-interior points of one colour along a row,
  // (k << 20) | (j << 10) | i0 (points i0, i0 + 2, ...), colour c's at [gs_ptr[c], gs_ptr[c+1]);
  // colour = 4 (i % 2) + 2 (j % 2) + (k % 2) of the point's lattice coordinates
  int32_t gs_ptr[9];
  const int32_t* gs_chunks;
  int64_t nskel_entries;           // entries of skeleton nodes (every copy)
  const int64_t* skel_entries;
  const int32_t* tiles_int;  // packed (k << 20) | (j0 << 10) | i0
  const int32_t* tiles_all;
  int32_t nskel;
  const int32_t* skel_ptr;   // [nskel+1]
  const SkelInc* skel_inc;   // incidences
  const int8_t* skel_dir;    // Dirichlet flag per skeleton node
  const uint8_t* mask;       // [entries] 1 = owned copy of a free node (dot products)
  // skeleton split: free face-interior nodes (per-incidence items + accumulator),
  // free edge/vertex nodes (warp kernel), Dirichlet nodes
  int32_t nface_items, nface_nodes, nev, ndir;
  const FaceItem* face_items;
  const int32_t* face_nodes;  // skeleton id of each face node
  const int32_t* ev_nodes;    // skeleton ids
  const int32_t* dir_nodes;   // skeleton ids
  uint32_t face_mask[4];      // candidate elements (bit 4p+av) inside the macro, per face type
  float* acc32;               // [nface_nodes_all * 8] accumulators, zero between sweeps
  double* acc64;
  // the same split including Dirichlet skeleton nodes (the Stokes pressure rows of
  // velocity-Dirichlet nodes are free)
  int32_t nface_items_all, nface_nodes_all, nev_all;
  const FaceItem* face_items_all;
  const int32_t* face_nodes_all;
  const int32_t* ev_all;
};

constexpr int INTERIOR_BLOCK = 128;
// boxes of the shared-memory tile kernel (k_interior_tile): 30 x 4 x 4 lattice points, so that a
// box row plus its halo is 32 points, one warp
constexpr int TILE3_I = 30, TILE3_J = 4, TILE3_K = 4;
constexpr int TILE_I = 32;
constexpr int TILE_J = 4;

}  // namespace hhg
