// Kernel launchers (C++ linkage, internal).  Each returns a cudaError_t as int.
#pragma once
#include <cstdint>

#include "hhg_internal.h"

namespace hhg {

enum OpKind { OP_APPLY = 0, OP_RESID = 1, OP_JACOBI = 2, OP_CHEBY = 3, OP_DIAG = 4 };

// Flags of the operator variant, uniform per launch.
struct OpFlags {
  int physical;   // 1: add the correction R (physical scaling); 0: unphysical
  int khat_edge;  // 1: khat = (k_i + k_j)/2; 0: patch mean
  int practical;  // 1: skeleton rows are the a_h rows; 0: symmetric interface rows
  int nodal = 0;  // 1: macro-interior rows by nodal integration a_h (the NODAL variant)
  int stored = 0; // 1: macro-interior rows from the stored stencil blocks (the STORED variant)
  int tile = 0;   // 1: macro-interior sweeps by the shared-memory tile kernel (k_interior_tile)
  int batch = 0;  // 1: the macro-interior sweeps of all macros in one launch (stencils staged in shared memory)
};

// Arguments of one stencil sweep.  Vectors are component-major over the level
// (component stride = entries).  Scalars for the smoothers:
//   JACOBI: x_out = x + omega * D^{-1} (f - A x)
//   CHEBY:  d_out = rho1 * d + rho2 * D^{-1} (f - A x);  x_out = x + d_out  (d may be null: 0)
//   DIAG:   out = point diagonal of A (1 on Dirichlet rows)
template <typename T>
struct SweepArgs {
  const T* x;
  const T* f;
  const T* k;
  const T* d;
  T* out;   // y (APPLY), r (RESID), x_out (JACOBI, CHEBY)
  T* dout;  // CHEBY only
  double* partial;  // RESID: per-block partial sums of |r|^2 (nullable)
  double omega, rho1, rho2;
  // BF16 bits of the coefficient (FP32 sweeps only; nullable): the macro-interior kernels
  // read k from here (2 B per node); k holds the same values widened, for the others
  const uint16_t* k16 = nullptr;
  // stored stencil blocks of the macro-interior rows (STORED variant): value r (row-major 3x3
  // entry) of block q (direction q < 14, q = 14 the centre) of entry e at [(9 q + r) * entries + e]
  const T* stencil = nullptr;
};

// The stored stencil blocks (layout of SweepArgs::stencil) of macro m's interior rows, computed in
// FP64 from the FP64 coefficient and rounded to T: for each direction d the scaled block
// khat_d Shat_d + [w_d]_x of Lemma 2.1, and the centre block minus their sum.
template <typename T>
int launch_store_stencil(const LevelDev& L, const MacroStencil<double>* st_host, const OpFlags& fl, const double* k64,
                         T* out, void* stream);

// parts: 1 = macro-interior kernels (one launch per macro), 2 = skeleton kernel, 3 = both.
// partial_offset: first partial slot used (the interior launches take ntiles_lin slots per
// macro, then the skeleton kernel one per block); *partial_count returns the slots used.
// stream_ev / stream_dir (nullable: `stream`): streams of the edge/vertex and Dirichlet
// skeleton kernels, which write disjoint entries and may run concurrently.
template <typename T>
int launch_sweep(const LevelDev& L, const MacroStencil<T>* st_host, const MacroConsts<T>* mc_dev, OpKind op,
                 const OpFlags& fl, const SweepArgs<T>& a, void* stream, int parts, int64_t partial_offset,
                 int64_t* partial_count, void* stream_ev = nullptr, void* stream_dir = nullptr);

// The macro-interior sweeps of all macros of the level in one launch (k_interior_pair_batched for
// FP32, k_interior_batched for FP64; each block stages its macro's stencil from mc_dev in shared
// memory), partial slots from partial_offset in the order of the per-macro launches.
template <typename T>
int launch_sweep_batched(const LevelDev& L, const MacroConsts<T>* mc_dev, OpKind op, const OpFlags& fl,
                         const SweepArgs<T>& a, void* stream, int64_t partial_offset, int64_t* partial_count);

// The macro-interior launch of macro m alone (partial slots from partial_offset; *partial_count
// returns the slots used).
// nc_host: per-macro element stiffness, used when fl.nodal is set.
template <typename T>
int launch_sweep_macro(const LevelDev& L, const MacroStencil<T>* st_host, const NodalConsts<T>* nc_host, int m,
                       OpKind op, const OpFlags& fl, const SweepArgs<T>& a, void* stream, int64_t partial_offset,
                       int64_t* partial_count);

// No-alloc residual (see hhg_residual_noalloc): static device scratch of
// NOALLOC_SLOTS partial sums plus the result slot at index NOALLOC_SLOTS.
constexpr int64_t NOALLOC_SLOTS = 262144;
constexpr int NOALLOC_MAX_DEVICES = 64;
int noalloc_scratch_address(int device, double** ptr);
int64_t noalloc_partials_needed(const LevelDev& L);
template <typename T>
int launch_residual_noalloc(const LevelDev& L, const MacroStencil<T>* st_host, const MacroConsts<T>* mc_dev,
                            const OpFlags& fl, SweepArgs<T> a, double* scratch, void* stream);

// One colour pass of the hybrid Gauss-Seidel smoother on the macro interiors: every
// macro-interior point of the colour, x_i += D_ii^-1 (f - A x)_i in place (a.x == a.out, a.omega
// = 1); points of one colour are never neighbours.  mc_dev non-null: one launch for all macros
// (stencils staged in shared memory); null: one launch per macro with st_host[m].
template <typename T>
int launch_gs_colour(const LevelDev& L, const MacroStencil<T>* st_host, const MacroConsts<T>* mc_dev, const OpFlags& fl,
                     const SweepArgs<T>& a, int colour, void* stream);
// dst[c * E + idx[u]] = src[c * E + idx[u]] for u < count, c < comps
template <typename T>
int launch_copy_entries(int64_t count, const int64_t* idx, int comps, int64_t E, const T* src, T* dst, void* stream);

// constant-memory direction tables of the skeleton kernels (once per device)
int upload_direction_tables();

// Stokes saddle operator on (u, v, w, p) vectors (4 components): apply or residual
// side (nullable): three side streams for the face-node chain, every second macro's
// interior launch and the edge/vertex nodes (they write disjoint entries).
template <typename T>
int launch_stokes_sweep(const LevelDev& L, const MacroStencil<T>* st_host, const MacroConsts<T>* mc_dev, OpKind op,
                        const OpFlags& fl, const SweepArgs<T>& a, void* stream, int64_t* partial_count,
                        void* const* side = nullptr);

// Carreau viscosity from the nodal least-squares strain rate (Sec. 3, eq. carreau):
// interior nodes with the per-macro slope operator Q (grad u_c = sum_d Q[d] (u_c(i+d) - u_c(i))),
// skeleton nodes from their precomputed patch lists (general affine least squares).
struct CarreauParams {
  double eta0, eta_inf, kappa, r;
};
struct SlopeOp {
  double Q[NDIR][3];
};
struct PatchLists {
  int32_t nnodes;
  const int32_t* node;   // skeleton id
  const int32_t* ptr;    // [nnodes+1]
  const int64_t* ent;    // entry of each patch point (the node itself included)
  const double* dx;      // 3 per patch point: x_point - x_node
};
// degree 2: quadratic least squares on the skeleton where the patch determines it (affine
// elsewhere); the interior slope operator serves both degrees (the fits agree there, Sec. 3)
int launch_carreau(const LevelDev& L, const SlopeOp* q_host, const PatchLists& P, const CarreauParams& cp,
                   const double* u, double* mu, void* stream, int degree = 1);

// Boundary traction load: nslots flagged macro faces, each a lattice of (n+1)(n+2)/2 points whose
// entries are pent[s * npf + p] and whose n^2 triangles have area area[s]; t: nodal traction (3
// components of stride E); contrib: scratch of 3 doubles per face point; then for each of nnodes
// boundary nodes the contributions cidx[cptr[u] .. cptr[u+1]) are summed and added to f at its
// entries eidx[eptr[u] .. eptr[u+1]).
template <typename T>
int launch_traction_load(int n, int nslots, const double* area, const int64_t* pent, int64_t E, const T* t,
                         double* contrib, int64_t nnodes, const int64_t* cptr, const int64_t* cidx,
                         const int64_t* eptr, const int64_t* eidx, T* f, void* stream);

// out[0] = max over masked entries of |a - b|_2 over comps components (b nullable)
int launch_node_maxnorm(const uint8_t* mask, int64_t E, int comps, const double* a, const double* b,
                        double* partials, double* out, void* stream);

// sum of partials[0..count) into out[0] (single block), deterministic
int launch_reduce(const double* partials, int64_t count, double* out, void* stream);

// dot over unique free nodes: sum_e mask[e] * sum_c a[c][e] b[c][e]
template <typename T>
int launch_dot(const LevelDev& L, int comps, const T* a, const T* b, double* partials, int64_t* partial_count,
               void* stream);

// dot over entries with mask[e] != 0 (comps components of stride E)
template <typename T>
int launch_dot_masked(const uint8_t* mask, int64_t E, int comps, const T* a, const T* b, double* partials,
                      int64_t* partial_count, void* stream);
template <typename T>
int launch_mul3(int64_t n, const T* a, const T* b, const T* c, T* out, void* stream);  // out = a * b * c
template <typename T>
int launch_add_const(int64_t n, T v, T* dst, void* stream);                           // dst += v
// out = r / (m / mu + s): the pressure Schur-complement diagonal of the Stokes solvers
template <typename T>
int launch_schur_diag(int64_t n, const T* r, const T* mu, const T* m, const T* s, T* out, void* stream);

// multigrid transfers and coefficient injection (all on the fine level's lattice)
// comps: components of the fields (3 velocity, 1 pressure); use_dir = 0: the coarse skeleton
// rows of Dirichlet nodes are restricted too (pressure, with lists over all fine nodes)
template <typename T>
int launch_prolong_add(const LevelDev& Lf, const LevelDev& Lc, const T* ec, T* ef, void* stream, int comps = 3);
template <typename T>
int launch_restrict(const LevelDev& Lf, const LevelDev& Lc, const int32_t* rptr, const int64_t* rent, const T* rw,
                    const T* rf, T* rc, void* stream, int comps = 3, int use_dir = 1);
template <typename T>
int launch_inject(const LevelDev& Lf, const LevelDev& Lc, const T* kf, T* kc, void* stream);
// coefficient copies: k64[e] <- FP64 widening of BF16 bits (bf16_to_f64); or round k64 to the
// nearest BF16 and write the value to k64, k32 and its bits to k16 (round_bf16)
int launch_bf16_to_f64(int64_t n, const uint16_t* src, double* dst, void* stream);
int launch_round_bf16(int64_t n, double* k64, float* k32, uint16_t* k16, void* stream);
// coarse macro-interior nodes: kc = weighted mean (harmonic = 1: of 1/k, inverted) of kf over the
// coincident fine node (weight 1) and its 14 fine neighbours (weight 1/2); other nodes untouched
int launch_average_coeff(const LevelDev& Lf, const LevelDev& Lc, const double* kf, double* kc, int harmonic,
                         void* stream);

// vector kernels over n elements
template <typename T>
int launch_axpby(int64_t n, T a, const T* x, T b, T* y, void* stream);  // y = a x + b y
template <typename T, typename U>
int launch_convert(int64_t n, const T* src, U* dst, void* stream);
template <typename T>
int launch_gather(int64_t count, int comps, int64_t src_stride, int64_t dst_stride, const int64_t* idx, const T* src,
                  T* dst, void* stream);  // dst[c*dst_stride + u] = src[c*src_stride + idx[u]]
template <typename T>
int launch_fill(int64_t n, T v, T* dst, void* stream);
template <typename T>
int launch_mul(int64_t n, const T* a, const T* b, T* out, void* stream);  // out = a * b
template <typename T>
int launch_recip(int64_t n, const T* a, T* out, void* stream);             // out = 1 / a
int launch_add_f32_to_f64(int64_t n, const float* e, double* x, void* stream);  // x += e
// unique-node vector of hashed values in [-1, 1), 0 on Dirichlet nodes
template <typename T>
int launch_hash_unique(int64_t U, int comps, const int8_t* udir, T* u, void* stream);
// dst_u[idx[i]] = sum_j A[i*N + j] src_u[idx[j]]  (dense coarse solve)
template <typename T>
int launch_dense_matvec(int N, const T* A, const int64_t* idx, const T* src_u, T* dst_u, void* stream);

// 2D variant (Sec. 2.3) on one refined macro triangle: per direction d of the 7-point stencil
// the constant-coefficient 2x2 block S[d] (row-major), the weight w[d] of the correction
// (k_p - k_pm) [[0, -w], [w, 0]], and the directions p[d], pm[d] of the third vertices of the
// edge's two elements
template <typename T>
struct Stencil2D {
  T S[6][4];
  T w[6];
  int p[6], pm[6];
  // nodal integration (nodal = 1): the two element blocks of each direction's edge, of the
  // element with third vertex p[d] (Kt) and of the one with third vertex pm[d] (Ktm), each
  // scaled by its own vertex mean
  int nodal;
  T Kt[6][4], Ktm[6][4];
};
// constants in FP64 for tri[6] at n intervals per edge; 0 on success
int stencil_2d(const double* tri, int n, double c_eps, double c_div, int physical, Stencil2D<double>* out);
// variant: 0 unphysical, 1 physical, 2 nodal integration
// y = A x on the lattice (2 components of stride (n+1)(n+2)/2; k one value per point)
template <typename T>
int launch_apply_2d(int n, const Stencil2D<T>& st, const T* k, const T* x, T* y, void* stream);

// FP32 FMA issue-rate probe on sm_count * 8 blocks of 256 threads; *flops = flops of the launch
int launch_fma_probe(int packed, int64_t iters, int sm_count, float* out, double* flops, void* stream);

}  // namespace hhg
