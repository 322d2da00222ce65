// Scaled-stencil sweeps on one level: operator apply, residual, Jacobi and
// Chebyshev smoothing steps (Sec. 2 and Sec. 4.1 of arXiv 1908.08666).
//
// Macro-interior rows (k_interior): for the interior node i and each of the 14
// stencil directions d (edge (i, i+d) lies in 6 or 4 elements, Sec. 2.4)
//     khat_d = (k_i + k_{i+d})/4 + w_d * sum_{ring nodes r of the edge} k_r
// with w_d = 1/12 for six-element edges and 1/8 for four-element edges (this is
// the patch mean of the element means, eq. patchmean), and
//     S_d = khat_d * Shat_d + sum_c (k_{r_c} - k_{r_c^m}) [s_{d,c}]_x
// (Lemma 2.1 with the correction of eq. correctionterm3D written as the cross
// product with an axial vector).  The centre block is -sum_d S_d, so
//     (A x)_i = sum_d S_d (x_{i+d} - x_i).
// Shat_{-d} = Shat_d, so the symmetric part is applied once per direction pair:
// Shat_d (khat_d dx_d + khat_{-d} dx_{-d}).
//
// Skeleton rows (k_skeleton, nodes on macro faces/edges/vertices, Sec. 2.2):
// pairs of skeleton nodes use nodal integration a_h, summed over the incident
// elements of every incident macro; pairs with a macro-interior neighbour use
// that macro's scaled block; the centre block is minus the off-diagonal row
// sum.  With the practical interface rule the whole row is the a_h row.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "hhg_internal.h"
#include "hhg_launch.h"

namespace hhg {

namespace {

template <typename T>
__device__ __forceinline__ void block_sum_store(double v, double* out) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nw = (blockDim.x * blockDim.y + 31) / 32;
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    double s = tid < nw ? red[tid] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (tid == 0) *out = s;
  }
}

template <typename T, int OP>
__device__ __forceinline__ void epilogue(const SweepArgs<T>& a, int64_t e, int64_t E, T ax, T ay, T az, T dgx, T dgy,
                                         T dgz, T x0, T y0, T z0, double& r2) {
  if (OP == OP_APPLY) {
    a.out[e] = ax;
    a.out[e + E] = ay;
    a.out[e + 2 * E] = az;
  } else if (OP == OP_DIAG) {
    a.out[e] = dgx;
    a.out[e + E] = dgy;
    a.out[e + 2 * E] = dgz;
  } else {
    const T rx = a.f[e] - ax, ry = a.f[e + E] - ay, rz = a.f[e + 2 * E] - az;
    if (OP == OP_RESID) {
      a.out[e] = rx;
      a.out[e + E] = ry;
      a.out[e + 2 * E] = rz;
      r2 += (double)rx * rx + (double)ry * ry + (double)rz * rz;
    } else if (OP == OP_JACOBI) {
      const T om = (T)a.omega;
      a.out[e] = x0 + om * rx / dgx;
      a.out[e + E] = y0 + om * ry / dgy;
      a.out[e + 2 * E] = z0 + om * rz / dgz;
    } else if (OP == OP_CHEBY) {
      const T r1 = (T)a.rho1, r2c = (T)a.rho2;
      const T ux = (a.d ? r1 * a.d[e] : (T)0) + r2c * rx / dgx;
      const T uy = (a.d ? r1 * a.d[e + E] : (T)0) + r2c * ry / dgy;
      const T uz = (a.d ? r1 * a.d[e + 2 * E] : (T)0) + r2c * rz / dgz;
      a.dout[e] = ux;
      a.dout[e + E] = uy;
      a.dout[e + 2 * E] = uz;
      a.out[e] = x0 + ux;
      a.out[e + E] = y0 + uy;
      a.out[e + 2 * E] = z0 + uz;
    }
  }
}

// (j, i) of the t-th interior point of a slice with M = n-1-k: rows j = 1..M-1 hold
// M-j points; C(j) = (j-1)(2M-j)/2 points precede row j.
__device__ __forceinline__ void slice_decode(int M, int t, int& j, int& i) {
  const float b = (float)(2 * M - 1);
  int u = (int)floorf(0.5f * (b - sqrtf(fmaxf(b * b - 8.0f * (float)t, 0.0f))));
  u = max(0, min(u, M - 2));
  // exact correction: C(u+1) <= t < C(u+2)
  if (((u + 1) * (2 * M - u - 2)) / 2 <= t) ++u;
  if ((u * (2 * M - u - 1)) / 2 > t) --u;
  j = u + 1;
  i = t - (u * (2 * M - u - 1)) / 2 + 1;
}

// The scaled-stencil row of one macro-interior node (Lemma 2.1, eq. correctionterm3D) from
// the coefficients kk[d] = k_{i+d}, k0 = k_i and the neighbour differences
// dx/dy/dz[d] = x_{i+d} - x_i of its 14 stencil directions: (A x)_i = (ax, ay, az) and, with
// DIAG, the point diagonal (dgx, dgy, dgz) = -sum_d khat_d diag(Shat_d).
// GEN = 0: physical scaling with the patch mean (flags folded at compile time); GEN = 1:
// variant and khat rule from the run-time flags.
// The neighbour values come through an accessor nb: nb.k(d) = k_{i+d}, nb.dx(d) = x_{i+d} - x_i
// (likewise dy, dz); the accessor decides where they are read from (registers or shared
// memory) and the compiler when.
template <typename T>
struct Diff3 {
  T x, y, z;
};

template <typename T>
struct RegNeighbours {
  const T (&kk)[NDIR];
  const T (&x)[NDIR];
  const T (&y)[NDIR];
  const T (&z)[NDIR];
  __device__ __forceinline__ T k(int d) const { return kk[d]; }
  __device__ __forceinline__ Diff3<T> diff(int d) const { return {x[d], y[d], z[d]}; }
  __device__ __forceinline__ void next_pair() {}
};

// Packed FP32 arithmetic (the two-point kernel below) has no negated operands: differences and
// negations go through a packed subtraction.  For scalar types both are the plain forms (the
// negation folds into the FMA).
struct P2;
template <typename T>
struct Packed {
  static constexpr bool value = false;
};
template <>
struct Packed<P2> {
  static constexpr bool value = true;
};
template <typename T>
__device__ __forceinline__ T sub(T a, T b) {
  return a - b;
}
template <typename T>
__device__ __forceinline__ T neg(T a) {
  if constexpr (Packed<T>::value)
    return sub(T(0.0), a);
  else
    return -a;
}

template <typename T, bool DIAG, int GEN, typename NB, typename C>
__device__ __forceinline__ void interior_row(const MacroStencil<C>& st, const OpFlags& fl, NB& nb, T k0,
                                             T& ax, T& ay, T& az, T& dgx, T& dgy, T& dgz) {
  const bool physical = GEN ? fl.physical != 0 : true;
  const bool khat_edge = GEN ? fl.khat_edge != 0 : false;
  ax = 0;
  ay = 0;
  az = 0;
  dgx = 0;
  dgy = 0;
  dgz = 0;
  const T k0q = (T)0.25 * k0;
  // the vector differences of a direction pair are read one pair ahead of their use
  Diff3<T> pn = nb.diff(0), mn = nb.diff(7);
#pragma unroll
  for (int d = 0; d < 7; ++d) {
    const Diff3<T> p = pn, m = mn;
    nb.next_pair();
    if (d < 6) {
      pn = nb.diff(d + 1);
      mn = nb.diff(d + 8);
    }
    const int e = d + 7;
    const T wr = dir_red(d) ? (T)(1.0 / 12.0) : (T)0.125;
    T rsp = 0, rsm = 0;
    T wpx = 0, wpy = 0, wpz = 0, wmx = 0, wmy = 0, wmz = 0;
    // the correction stencils of d and -d are equal, s[d + 7] = s[d] (checked on the host
    // when they are built), so one set of constants serves the pair
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (c < ring_count(d)) {
        const T ka = nb.k(ring_a(d, c)), kb = nb.k(ring_b(d, c));
        const T la = nb.k(ring_a(e, c)), lb = nb.k(ring_b(e, c));
        rsp += ka + kb;
        rsm += la + lb;
        if (physical) {
          const T dp = sub(ka, kb), dm = sub(la, lb);
          wpx = fma(dp, st.s[d][c][0], wpx);
          wpy = fma(dp, st.s[d][c][1], wpy);
          wpz = fma(dp, st.s[d][c][2], wpz);
          wmx = fma(dm, st.s[d][c][0], wmx);
          wmy = fma(dm, st.s[d][c][1], wmy);
          wmz = fma(dm, st.s[d][c][2], wmz);
        }
      }
    }
    T khp, khm;
    if (khat_edge) {
      khp = (T)0.5 * (k0 + nb.k(d));
      khm = (T)0.5 * (k0 + nb.k(e));
    } else {
      khp = fma(wr, rsp, fma((T)0.25, nb.k(d), k0q));
      khm = fma(wr, rsm, fma((T)0.25, nb.k(e), k0q));
    }
    const T vx = fma(khp, p.x, khm * m.x);
    const T vy = fma(khp, p.y, khm * m.y);
    const T vz = fma(khp, p.z, khm * m.z);
    const C* S = st.S[d];
    ax = fma(S[0], vx, ax);
    ax = fma(S[3], vy, ax);
    ax = fma(S[4], vz, ax);
    ay = fma(S[3], vx, ay);
    ay = fma(S[1], vy, ay);
    ay = fma(S[5], vz, ay);
    az = fma(S[4], vx, az);
    az = fma(S[5], vy, az);
    az = fma(S[2], vz, az);
    if (physical) {
      // w x delta for both directions
      const Diff3<T> np{neg(p.x), neg(p.y), neg(p.z)}, nm{neg(m.x), neg(m.y), neg(m.z)};
      ax = fma(wpy, p.z, ax);
      ax = fma(wpz, np.y, ax);
      ax = fma(wmy, m.z, ax);
      ax = fma(wmz, nm.y, ax);
      ay = fma(wpz, p.x, ay);
      ay = fma(wpx, np.z, ay);
      ay = fma(wmz, m.x, ay);
      ay = fma(wmx, nm.z, ay);
      az = fma(wpx, p.y, az);
      az = fma(wpy, np.x, az);
      az = fma(wmx, m.y, az);
      az = fma(wmy, nm.x, az);
    }
    if (DIAG) {
      const T nks = neg(khp + khm);
      dgx = fma(nks, S[0], dgx);
      dgy = fma(nks, S[1], dgy);
      dgz = fma(nks, S[2], dgz);
    }
  }
}

// Stokes epilogue (apply / residual) for one copy: velocity rows (identity on
// velocity-Dirichlet nodes) and the pressure row.
template <typename T, int OP>
__device__ __forceinline__ void stokes_epilogue(const SweepArgs<T>& a, int64_t e, int64_t E, T ax, T ay, T az, T yp,
                                                T x0, T y0, T z0, bool vdir, double& r2) {
  if (OP == OP_APPLY) {
    a.out[e] = vdir ? x0 : ax;
    a.out[e + E] = vdir ? y0 : ay;
    a.out[e + 2 * E] = vdir ? z0 : az;
    a.out[e + 3 * E] = yp;
  } else {
    const T rx = vdir ? (T)0 : a.f[e] - ax, ry = vdir ? (T)0 : a.f[e + E] - ay, rz = vdir ? (T)0 : a.f[e + 2 * E] - az;
    const T rp = a.f[e + 3 * E] - yp;
    a.out[e] = rx;
    a.out[e + E] = ry;
    a.out[e + 2 * E] = rz;
    a.out[e + 3 * E] = rp;
    r2 += (double)rx * rx + (double)ry * ry + (double)rz * rz + (double)rp * rp;
  }
}

// STK = 1: the Stokes saddle operator [[A(mu), B^T], [B, C]] on (u, v, w, p) (Sec. 5.2),
// the velocity block being the scaled-stencil operator of the 2 mu eps(u) form.
// KB = 1 (FP32, default operator only): the coefficient is read as BF16 bits from a.k16.
// GS = 1 (a colour pass of the hybrid Gauss-Seidel smoother): the block takes four chunks of
// colour `colour`'s list (a warp each; lane l the point i0 + 2 l of the chunk's row) instead
// of a slice chunk.
// The body takes its block's index among the macro's blocks (`block`) and the slot of its
// partial sum (`partial`, nullable) from the kernel around it.
template <typename T, int OP, int GEN, int STK, int KB, int GS>
__device__ __forceinline__ void interior_point_body(const LevelDev& L, const MacroStencil<T>& st, const int macro,
                                                    const int block, double* partial, const OpFlags& fl,
                                                    const SweepArgs<T>& a, const int colour) {
  const int n = L.n;
  int i = 0, j = 0, k = 0;
  bool valid;
  if constexpr (GS) {
    const int q = block * (INTERIOR_BLOCK / 32) + (threadIdx.x >> 5);
    valid = q < L.gs_ptr[colour + 1] - L.gs_ptr[colour];
    if (valid) {
      const int32_t ch = L.gs_chunks[L.gs_ptr[colour] + q];
      k = ch >> 20;
      j = (ch >> 10) & 0x3FF;
      i = (ch & 0x3FF) + 2 * (threadIdx.x & 31);
      valid = i + j + k <= n - 1;
    }
  } else {
    const int32_t tile = L.tiles_lin[block];
    k = tile >> 20;
    const int M = n - 1 - k;
    const int t = (tile & 0xFFFFF) + threadIdx.x;
    valid = t < (M - 1) * M / 2;
    if (valid) slice_decode(M, t, j, i);
  }
  double r2 = 0.0;
  if (valid) {
    const int64_t E = L.entries;
    const int64_t base = (int64_t)macro * L.nt;
    // starts of the seven lattice rows the stencil touches (plus i)
    const int m = n - k;
    const int r00 = (int)(tetnum(n + 1) - tetnum(n + 1 - k)) + j * (2 * m + 3 - j) / 2 + i;
    const int r10 = r00 + (m + 1 - j);
    const int rm0 = r00 - (m + 2 - j);
    const int sz = (m + 1) * (m + 2) / 2;
    const int szm = (m + 2) * (m + 3) / 2;
    const int r01 = r00 + sz - j;
    const int r0m = r00 - szm + j;
    const int rm1 = rm0 + sz - j + 1;
    const int r1m = r10 - szm + j + 1;
    // neighbour d lies in row rowof[d] at column offset -1, 0 or +1: load through one
    // pointer per (row, array) with immediate offsets
    T kk[NDIR], dx[NDIR], dy[NDIR], dz[NDIR];
    T x0, y0, z0, k0;
    T dp[STK ? NDIR : 1];
    T p0 = 0;
    if constexpr (STK) {
      const T* __restrict__ P = a.x + base + 3 * E;
      p0 = P[r00];
      dp[0] = P[r00 + 1] - p0;
      dp[7] = P[r00 - 1] - p0;
      dp[1] = P[r10 - 1] - p0;
      dp[3] = P[r10] - p0;
      dp[2] = P[rm1] - p0;
      dp[5] = P[rm1 + 1] - p0;
      dp[4] = P[r01 - 1] - p0;
      dp[6] = P[r01] - p0;
      dp[8] = P[rm0 + 1] - p0;
      dp[10] = P[rm0] - p0;
      dp[9] = P[r1m] - p0;
      dp[12] = P[r1m - 1] - p0;
      dp[11] = P[r0m + 1] - p0;
      dp[13] = P[r0m] - p0;
    }
    {
      const T* __restrict__ X = a.x + base;
      const T* __restrict__ K = a.k + base;
      const uint16_t* __restrict__ K16 = KB ? a.k16 + base : nullptr;
#define HHG_ROW(R, ...)                                                                                   \
  {                                                                                                      \
    const T* px_ = X + (R);                                                                              \
    const T* py_ = px_ + E;                                                                              \
    const T* pz_ = py_ + E;                                                                              \
    const T* pk_ = K + (R);                                                                              \
    const uint16_t* pk16_ = KB ? K16 + (R) : nullptr;                                                    \
    __VA_ARGS__                                                                                          \
  }
#define HHG_K(OFF) (KB ? (T)__uint_as_float((uint32_t)pk16_[OFF] << 16) : pk_[OFF])
#define HHG_NB(D, OFF)                                                                                    \
  kk[D] = HHG_K(OFF);                                                                                    \
  dx[D] = px_[OFF];                                                                                      \
      dy[D] = py_[OFF];                                                                                  \
      dz[D] = pz_[OFF];
      HHG_ROW(r00, x0 = px_[0]; y0 = py_[0]; z0 = pz_[0]; k0 = HHG_K(0); HHG_NB(0, 1) HHG_NB(7, -1))
      HHG_ROW(r10, HHG_NB(1, -1) HHG_NB(3, 0))
      HHG_ROW(rm1, HHG_NB(2, 0) HHG_NB(5, 1))
      HHG_ROW(r01, HHG_NB(4, -1) HHG_NB(6, 0))
      HHG_ROW(rm0, HHG_NB(8, 1) HHG_NB(10, 0))
      HHG_ROW(r1m, HHG_NB(9, 0) HHG_NB(12, -1))
      HHG_ROW(r0m, HHG_NB(11, 1) HHG_NB(13, 0))
#undef HHG_NB
#undef HHG_K
#undef HHG_ROW
    }
#pragma unroll
    for (int d = 0; d < NDIR; ++d) {
      dx[d] -= x0;
      dy[d] -= y0;
      dz[d] -= z0;
    }
    T ax, ay, az, dgx, dgy, dgz;
    RegNeighbours<T> nb{kk, dx, dy, dz};
    interior_row<T, OP == OP_JACOBI || OP == OP_CHEBY || OP == OP_DIAG, GEN>(st, fl, nb, k0, ax, ay, az, dgx, dgy,
                                                                             dgz);
    if constexpr (STK) {
      T yp = 0;
#pragma unroll
      for (int d = 0; d < NDIR; ++d) {
        ax = fma(st.G[d][0], dp[d], ax);
        ay = fma(st.G[d][1], dp[d], ay);
        az = fma(st.G[d][2], dp[d], az);
        yp = fma(st.B[d][0], dx[d], yp);
        yp = fma(st.B[d][1], dy[d], yp);
        yp = fma(st.B[d][2], dz[d], yp);
        yp = fma(st.C[d], dp[d], yp);
      }
      stokes_epilogue<T, OP>(a, base + r00, E, ax, ay, az, yp, x0, y0, z0, false, r2);
    } else {
      epilogue<T, OP>(a, base + r00, E, ax, ay, az, dgx, dgy, dgz, x0, y0, z0, r2);
    }
  }
  if (OP == OP_RESID && partial != nullptr) block_sum_store<T>(r2, partial);
}

// one launch per macro: the stencil is a kernel parameter
template <typename T, int OP, int GEN, int STK = 0, int KB = 0, int GS = 0>
__global__ void __launch_bounds__(INTERIOR_BLOCK) k_interior(const LevelDev L, const MacroStencil<T> st,
                                                              const int macro, const OpFlags fl,
                                                              const SweepArgs<T> a, const int colour) {
  interior_point_body<T, OP, GEN, STK, KB, GS>(L, st, macro, blockIdx.x, a.partial ? a.partial + blockIdx.x : nullptr,
                                               fl, a, colour);
}

// The interior stencil of one macro copied into shared memory by the whole block, each value
// as stored (C = T) or as the lane pair (v, v) of the packed FP32 arithmetic (C = float2).
__device__ __forceinline__ float2 stencil_value(float v, float2) { return make_float2(v, v); }
__device__ __forceinline__ float stencil_value(float v, float) { return v; }
__device__ __forceinline__ double stencil_value(double v, double) { return v; }
template <typename C, typename T>
__device__ __forceinline__ void stage_stencil(MacroStencil<C>& dst, const MacroStencil<T>* __restrict__ src) {
  const T* s = &src->S[0][0];
  C* d = &dst.S[0][0];
  for (int q = threadIdx.x; q < (int)(sizeof(MacroStencil<T>) / sizeof(T)); q += blockDim.x)
    d[q] = stencil_value(__ldg(s + q), C());
  __syncthreads();
}

// All macros of a level in one launch (grid: the macro's blocks x macros macro0 ..): each block
// stages its macro's stencil in shared memory.  Partial-sum slots macro-major, as the per-macro
// launches place them.
template <typename T, int OP, int GEN, int STK = 0, int KB = 0>
__global__ void __launch_bounds__(INTERIOR_BLOCK) k_interior_batched(const LevelDev L,
                                                                      const MacroConsts<T>* __restrict__ mc,
                                                                      const int macro0, const OpFlags fl,
                                                                      const SweepArgs<T> a) {
  __shared__ MacroStencil<T> sst;
  const int m = macro0 + blockIdx.y;
  stage_stencil(sst, &mc[m].st);
  double* partial = a.partial ? a.partial + (int64_t)blockIdx.y * gridDim.x + blockIdx.x : nullptr;
  interior_point_body<T, OP, GEN, STK, KB, 0>(L, sst, m, blockIdx.x, partial, fl, a, 0);
}

// ---------------------------------------------------------------------------
// FP32 macro-interior sweep on pairs of points (k_interior_pair).  A thread takes the
// neighbouring points A = (i, j, k) and B = (i + 1, j, k) of one lattice row and evaluates
// both in the two lanes of packed FP32 arithmetic (fma.rn.f32x2 and friends): every
// instruction of interior_row serves both points.  The two points share their seven row
// addresses, and their neighbours overlap (the points of a row at column offsets -1..2).
// A row of odd length pairs its last point with the face point after it, a lattice point
// whose neighbours are lattice points or the next row's: its lane is computed and dropped.
// Pairs are numbered densely per slice: slice k (M = n - 1 - k) has floor(M^2 / 4) pairs,
// rows j = 1 .. M - 1 holding ceil((M - j) / 2) of them.
// ---------------------------------------------------------------------------
// the float/double fma stays visible next to the packed overloads below
using ::fma;

struct P2 {
  float2 v;
  __device__ __forceinline__ P2() {}
  __device__ __forceinline__ P2(float2 a) : v(a) {}
  __device__ __forceinline__ P2(double a) : v(make_float2((float)a, (float)a)) {}
  __device__ __forceinline__ P2(float a, float b) : v(make_float2(a, b)) {}
};
__device__ __forceinline__ P2 operator+(P2 a, P2 b) { return P2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ P2 operator-(P2 a) { return P2(make_float2(-a.v.x, -a.v.y)); }
__device__ __forceinline__ P2 operator-(P2 a, P2 b) { return P2(__fadd2_rn(a.v, (-b).v)); }
__device__ __forceinline__ P2 operator*(P2 a, P2 b) { return P2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ P2& operator+=(P2& a, P2 b) { return a = a + b; }
__device__ __forceinline__ P2 fma(P2 a, P2 b, P2 c) { return P2(__ffma2_rn(a.v, b.v, c.v)); }
// packed subtraction (sub.rn.f32x2)
template <>
__device__ __forceinline__ P2 sub<P2>(P2 a, P2 b) {
  unsigned long long r;
  const unsigned long long x = *reinterpret_cast<const unsigned long long*>(&a.v);
  const unsigned long long y = *reinterpret_cast<const unsigned long long*>(&b.v);
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
  return P2(*reinterpret_cast<const float2*>(&r));
}
__device__ __forceinline__ P2 fma(float a, P2 b, P2 c) { return fma(P2(a, a), b, c); }
__device__ __forceinline__ P2 fma(P2 a, float b, P2 c) { return fma(a, P2(b, b), c); }
// stencil constants stored as lane pairs (c, c)
__device__ __forceinline__ P2 fma(float2 a, P2 b, P2 c) { return P2(__ffma2_rn(a, b.v, c.v)); }
__device__ __forceinline__ P2 fma(P2 a, float2 b, P2 c) { return P2(__ffma2_rn(a.v, b, c.v)); }

// the lane pair (p[0], p[1]) read from global memory (read-only path); one load per lane and
// pair, so the two values land in the pair's own registers
__device__ __forceinline__ P2 ldg2(const float* p) {
  float a, b;
  asm volatile("ld.global.nc.f32 %0, [%2];\n\tld.global.nc.f32 %1, [%2+4];" : "=f"(a), "=f"(b) : "l"(p));
  return P2(a, b);
}

// pair number t of a slice with M = n - 1 - k -> row j and pair p (points i = 2p + 1, 2p + 2)
__device__ __forceinline__ void pair_decode(int M, int t, int& j, int& p) {
  const int R = (M * M) / 4 - t;  // pairs from the one of t to the end of the slice
  int s = (int)ceilf(sqrtf(4.0f * (float)R));
  if (s * s < 4 * R) ++s;
  if ((s - 1) * (s - 1) >= 4 * R) --s;
  j = M - s + 1;  // rows before j hold floor(M^2/4) - floor(s^2/4) pairs
  p = t - ((M * M) / 4 - (s * s) / 4);
}

// neighbour values of a pair of points: coefficients held in registers, vector values read
// from global memory per direction (next_pair() keeps the reads of later direction pairs
// below it)
struct PairNeighbours {
  const float* __restrict__ X;
  const float* __restrict__ Y;
  const float* __restrict__ Z;
  int row[7];   // entry (in the macro) of column 0 of the seven rows, relative to point A
  P2 kk[NDIR];
  P2 x0, y0, z0;
  // row index and column offset (relative to point A) of direction d
  __device__ __forceinline__ static int rowof(int d) {
    const int t[NDIR] = {0, 1, 2, 1, 3, 2, 3, 0, 4, 5, 4, 6, 5, 6};
    return t[d];
  }
  __device__ __forceinline__ static int colof(int d) {
    const int t[NDIR] = {1, -1, 0, 0, -1, 1, 0, -1, 1, 0, 0, 1, -1, 0};
    return t[d];
  }
  __device__ __forceinline__ P2 k(int d) const { return kk[d]; }
  __device__ __forceinline__ Diff3<P2> diff(int d) const {
    const int q = row[rowof(d)] + colof(d);
    return {sub(ldg2(X + q), x0), sub(ldg2(Y + q), y0), sub(ldg2(Z + q), z0)};
  }
  __device__ __forceinline__ void next_pair() {
    asm volatile("" : "+r"(row[0]), "+r"(row[1]), "+r"(row[2]), "+r"(row[3]), "+r"(row[4]), "+r"(row[5]),
                 "+r"(row[6]));
  }
};

template <typename T>
__device__ __forceinline__ float lane_x(T v) { return v.v.x; }

template <int OP, int GEN, int KB>
__device__ __forceinline__ void interior_pair_body(const LevelDev& L, const MacroStencil<float2>& st, const int macro,
                                                   const int block, double* partial, const OpFlags& fl,
                                                   const SweepArgs<float>& a) {
  const int32_t tile = L.tiles_pair[block];
  const int n = L.n;
  const int k = tile >> 20;
  const int M = n - 1 - k;
  const int t = (tile & 0xFFFFF) + threadIdx.x;
  double r2 = 0.0;
  if (t < (M * M) / 4) {
    int j, pp;
    pair_decode(M, t, j, pp);
    const int i = 2 * pp + 1;
    const bool second = i + 1 <= M - j;  // point B is macro-interior
    const int64_t E = L.entries;
    const int64_t base = (int64_t)macro * L.nt;
    const int m = n - k;
    const int r00 = (int)(tetnum(n + 1) - tetnum(n + 1 - k)) + j * (2 * m + 3 - j) / 2 + i;
    const int r10 = r00 + (m + 1 - j);
    const int rm0 = r00 - (m + 2 - j);
    const int sz = (m + 1) * (m + 2) / 2;
    const int szm = (m + 2) * (m + 3) / 2;
    PairNeighbours nb;
    nb.X = a.x + base;
    nb.Y = nb.X + E;
    nb.Z = nb.Y + E;
    nb.row[0] = r00;
    nb.row[1] = r10;
    nb.row[2] = rm0 + sz - j + 1;  // rm1
    nb.row[3] = r00 + sz - j;      // r01
    nb.row[4] = rm0;
    nb.row[5] = r10 - szm + j + 1; // r1m
    nb.row[6] = r00 - szm + j;     // r0m
    P2 k0;
    {
      const float* __restrict__ K = a.k + base;
      const uint16_t* __restrict__ K16 = a.k16 + base;
      auto kload = [&](int q) -> float {
        if constexpr (KB)
          return __uint_as_float((uint32_t)__ldg(K16 + q) << 16);
        else
          return __ldg(K + q);
      };
      auto kload2 = [&](int q) -> P2 {
        if constexpr (KB)
          return P2(kload(q), kload(q + 1));
        else
          return ldg2(K + q);
      };
      k0 = kload2(r00);
#pragma unroll
      for (int d = 0; d < NDIR; ++d) nb.kk[d] = kload2(nb.row[PairNeighbours::rowof(d)] + PairNeighbours::colof(d));
    }
    nb.x0 = ldg2(nb.X + r00);
    nb.y0 = ldg2(nb.Y + r00);
    nb.z0 = ldg2(nb.Z + r00);
    P2 ax, ay, az, dgx, dgy, dgz;
    interior_row<P2, OP == OP_JACOBI || OP == OP_CHEBY || OP == OP_DIAG, GEN>(st, fl, nb, k0, ax, ay, az, dgx, dgy,
                                                                              dgz);
    const int64_t e = base + r00;
    epilogue<float, OP>(a, e, E, ax.v.x, ay.v.x, az.v.x, dgx.v.x, dgy.v.x, dgz.v.x, nb.x0.v.x, nb.y0.v.x, nb.z0.v.x,
                        r2);
    if (second)
      epilogue<float, OP>(a, e + 1, E, ax.v.y, ay.v.y, az.v.y, dgx.v.y, dgy.v.y, dgz.v.y, nb.x0.v.y, nb.y0.v.y,
                          nb.z0.v.y, r2);
  }
  if (OP == OP_RESID && partial != nullptr) block_sum_store<float>(r2, partial);
}

// one launch per macro: the stencil (as lane pairs) is a kernel parameter
template <int OP, int GEN, int KB>
__global__ void __launch_bounds__(INTERIOR_BLOCK, 4) k_interior_pair(const LevelDev L, const MacroStencil<float2> st,
                                                                   const int macro, const OpFlags fl,
                                                                   const SweepArgs<float> a) {
  interior_pair_body<OP, GEN, KB>(L, st, macro, blockIdx.x, a.partial ? a.partial + blockIdx.x : nullptr, fl, a);
}

// a colour pass of the hybrid Gauss-Seidel smoother over all macros (grid.y), each block staging
// its macro's stencil in shared memory
template <typename T, int GEN>
__global__ void __launch_bounds__(INTERIOR_BLOCK) k_gs_colour_batched(const LevelDev L,
                                                                       const MacroConsts<T>* __restrict__ mc,
                                                                       const int macro0, const OpFlags fl,
                                                                       const SweepArgs<T> a, const int colour) {
  __shared__ MacroStencil<T> sst;
  const int m = macro0 + blockIdx.y;
  stage_stencil(sst, &mc[m].st);
  interior_point_body<T, OP_JACOBI, GEN, 0, 0, 1>(L, sst, m, blockIdx.x, nullptr, fl, a, colour);
}

// all macros in one launch, as k_interior_batched: the block stages its macro's stencil as lane
// pairs in shared memory
template <int OP, int GEN, int KB>
__global__ void __launch_bounds__(INTERIOR_BLOCK, 4) k_interior_pair_batched(const LevelDev L,
                                                                           const MacroConsts<float>* __restrict__ mc,
                                                                           const int macro0, const OpFlags fl,
                                                                           const SweepArgs<float> a) {
  __shared__ MacroStencil<float2> sst;
  const int m = macro0 + blockIdx.y;
  stage_stencil(sst, &mc[m].st);
  double* partial = a.partial ? a.partial + (int64_t)blockIdx.y * gridDim.x + blockIdx.x : nullptr;
  interior_pair_body<OP, GEN, KB>(L, sst, m, blockIdx.x, partial, fl, a);
}

// Macro-interior sweep from a shared-memory tile.  Each block takes one box of
// T3_I x T3_J x T3_K lattice points (i, j, k) of one macro and stages the box plus a
// one-point halo in shared memory as (x, y, z, k) quadruples: one coalesced global read per
// array and point (a warp per 32-point region row), then one 16-byte shared-memory read per
// stencil neighbour (two in FP64), at offsets fixed at compile time.  The macro interior
// i, j, k >= 1, i + j + k <= n - 1 is a tetrahedron, so boxes along its slanted face are
// partly empty; the threads take the box's interior points densely (through a table of
// (row, i) built with the staging), so no lane idles on an empty point.  The arithmetic per
// point is interior_row, as in k_interior.
constexpr int T3_I = TILE3_I, T3_J = TILE3_J, T3_K = TILE3_K;
constexpr int R3_I = T3_I + 2, R3_J = T3_J + 2, R3_K = T3_K + 2;
constexpr int T3_ROWS = T3_J * T3_K;
constexpr int T3_THREADS = 256;
static_assert(R3_I == 32, "a region row is one warp");

template <typename T>
struct alignas(4 * sizeof(T)) Quad {
  T x, y, z, k;
};

// shared-memory offset of stencil direction d in the staged region
__device__ __forceinline__ int region_offset(int d) {
  return (dir_dk(d) * R3_J + dir_dj(d)) * R3_I + dir_di(d);
}

// shared-memory reads at a 32-bit shared-window address
__device__ __forceinline__ float lds(uint32_t a, float) {
  float v;
  asm("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ double lds(uint32_t a, double) {
  double v;
  asm("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ Diff3<float> lds3(uint32_t a, float) {
  float x, y, z, w;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(x), "=f"(y), "=f"(z), "=f"(w) : "r"(a));
  return {x, y, z};
}
__device__ __forceinline__ Diff3<double> lds3(uint32_t a, double) {
  double x, y, z;
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%3];\n\tld.shared.f64 %2, [%4];" : "=d"(x), "=d"(y), "=d"(z) : "r"(a), "r"(a + 16));
  return {x, y, z};
}

// Neighbour values of a point of the staged region (a: shared address of the point's own
// quadruple): the 14 coefficients are held in registers, the vector values are read from
// shared memory per direction pair; next_pair() redefines the address for the compiler, so
// the reads of later pairs cannot move above it (which would hold all 42 values in registers
// at once).
template <typename T>
struct SmemNeighbours {
  uint32_t a;
  T x0, y0, z0;
  T kk[NDIR];
  __device__ __forceinline__ T k(int d) const { return kk[d]; }
  __device__ __forceinline__ Diff3<T> diff(int d) const {
    const Diff3<T> v = lds3(a + region_offset(d) * (int)sizeof(Quad<T>), T());
    return {v.x - x0, v.y - y0, v.z - z0};
  }
  __device__ __forceinline__ void next_pair() { asm volatile("" : "+r"(a)); }
};

// asynchronous copy of one FP32 / FP64 element from global to shared memory (zero-filled when
// !valid: nothing is read then)
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src), "n"(sizeof(T)),
               "r"(valid ? (int)sizeof(T) : 0));
}

template <typename T, int OP, int GEN, int KB>
__global__ void __launch_bounds__(T3_THREADS, sizeof(T) == 4 ? 3 : 1) k_interior_tile(const LevelDev L,
                                                                                          const MacroStencil<T> st,
                                                                                          const int macro,
                                                                                          const OpFlags fl,
                                                                                          const SweepArgs<T> a) {
  __shared__ Quad<T> q[R3_K * R3_J * R3_I];
  __shared__ int row_start[R3_K * R3_J];  // entry (in the macro) of point i = 0 of each region row
  __shared__ int row_first[T3_ROWS + 1];  // dense numbering of the box's interior points, per row
  __shared__ uint16_t point[T3_ROWS * T3_I];  // dense number -> (box row << 8) | i - i0
  const int32_t tile = L.tiles3[blockIdx.x];
  const int n = L.n;
  const int i0 = tile & 0x3FF, j0 = (tile >> 10) & 0x3FF, k0 = tile >> 20;
  const int64_t E = L.entries;
  const int64_t base = (int64_t)macro * L.nt;
  const int tid = threadIdx.x;
  if (tid < R3_K * R3_J) {
    const int j = j0 - 1 + tid % R3_J, k = k0 - 1 + tid / R3_J;
    row_start[tid] = (j >= 0 && k >= 0 && j + k <= n) ? lattice_index32(n, 0, j, k) : -1;
  }
  if (tid == 0) {
    // interior points of box row (tj, tk): i0 .. min(i0 + T3_I - 1, n - 1 - j - k)
    int acc = 0;
    for (int r = 0; r < T3_ROWS; ++r) {
      row_first[r] = acc;
      const int j = j0 + r % T3_J, k = k0 + r / T3_J;
      acc += max(0, min(T3_I, n - j - k - i0));
    }
    row_first[T3_ROWS] = acc;
  }
  __syncthreads();
  for (int s = tid; s < T3_ROWS * T3_I; s += T3_THREADS) {
    const int r = s / T3_I, ti = s - r * T3_I;
    if (row_first[r] + ti < row_first[r + 1]) point[row_first[r] + ti] = (uint16_t)((r << 8) | ti);
  }
  // stage the region: warp w takes region rows w, w + 8, ...; lane l the point i0 - 1 + l,
  // copied asynchronously (cp.async) into the fields of its quadruple; points outside the
  // macro's lattice are zero-filled (no interior point reads them)
  {
    const int lane = tid & 31;
    const int i = i0 - 1 + lane;
    const T* __restrict__ X = a.x + base;
    for (int r = tid >> 5; r < R3_K * R3_J; r += T3_THREADS / 32) {
      const int start = row_start[r];
      const int imax = n - (j0 - 1 + r % R3_J) - (k0 - 1 + r / R3_J);
      const bool valid = start >= 0 && i <= imax;
      const int64_t off = valid ? (int64_t)start + i : 0;
      Quad<T>* dst = q + r * R3_I + lane;
      cp_async_elem(&dst->x, X + off, valid);
      cp_async_elem(&dst->y, X + E + off, valid);
      cp_async_elem(&dst->z, X + 2 * E + off, valid);
      if constexpr (KB) {
        dst->k = valid ? (T)__uint_as_float((uint32_t)a.k16[base + off] << 16) : (T)0;
      } else {
        cp_async_elem(&dst->k, a.k + base + off, valid);
      }
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
  }
  __syncthreads();
  double r2 = 0.0;
  const int count = row_first[T3_ROWS];
#pragma unroll 1
  for (int t = tid; t < count; t += T3_THREADS) {
    const int pr = point[t];
    const int r = pr >> 8, ti = pr & 0xFF;
    const int tj = r % T3_J, tk = r / T3_J;
    const Quad<T>* c = q + ((tk + 1) * R3_J + (tj + 1)) * R3_I + (ti + 1);
    const Quad<T> c0 = c[0];
    SmemNeighbours<T> nb{(uint32_t)__cvta_generic_to_shared(c), c0.x, c0.y, c0.z, {}};
#pragma unroll
    for (int d = 0; d < NDIR; ++d) nb.kk[d] = lds(nb.a + region_offset(d) * (int)sizeof(Quad<T>) + 3 * (int)sizeof(T), T());
    T ax, ay, az, dgx, dgy, dgz;
    interior_row<T, OP == OP_JACOBI || OP == OP_CHEBY || OP == OP_DIAG, GEN>(st, fl, nb, c0.k, ax, ay, az, dgx, dgy,
                                                                             dgz);
    const int64_t e = base + row_start[(tk + 1) * R3_J + (tj + 1)] + i0 + ti;
    epilogue<T, OP>(a, e, E, ax, ay, az, dgx, dgy, dgz, c0.x, c0.y, c0.z, r2);
  }
  if (OP == OP_RESID && a.partial != nullptr) block_sum_store<T>(r2, a.partial + blockIdx.x);
}

// Macro-interior rows by nodal integration (the NODAL variant, eq. nodalintegration):
// (A x)_i = sum over the 24 elements t around i of kbar^t sum_{b != a} K^t_ab (x_b - x_i),
// kbar^t the mean of the element's 4 nodal coefficients, K^t the element stiffness of the
// element's Kuhn type (kernel parameter).  Each element vertex b is a stencil neighbour of
// i; the unrolled loops make all element/vertex/direction indices compile-time constants.
template <typename T, int OP>
__global__ void __launch_bounds__(INTERIOR_BLOCK) k_interior_nodal(const LevelDev L, const NodalConsts<T> nc,
                                                                    const int macro, const SweepArgs<T> a) {
  const int32_t tile = L.tiles_lin[blockIdx.x];
  const int n = L.n;
  const int k = tile >> 20;
  const int M = n - 1 - k;
  const int t = (tile & 0xFFFFF) + threadIdx.x;
  double r2 = 0.0;
  if (t < (M - 1) * M / 2) {
    int j, i;
    slice_decode(M, t, j, i);
    const int64_t E = L.entries;
    const int64_t base = (int64_t)macro * L.nt;
    int nb[NDIR];
    lattice_neighbours(n, i, j, k, nb);
    const int c0 = lattice_index32(n, i, j, k);
    const T* __restrict__ X = a.x + base;
    const T* __restrict__ K = a.k + base;
    const T x0 = X[c0], y0 = X[c0 + E], z0 = X[c0 + 2 * E], k0 = K[c0];
    T kk[NDIR], dx[NDIR], dy[NDIR], dz[NDIR];
#pragma unroll
    for (int d = 0; d < NDIR; ++d) {
      kk[d] = K[nb[d]];
      dx[d] = X[nb[d]] - x0;
      dy[d] = X[nb[d] + E] - y0;
      dz[d] = X[nb[d] + 2 * E] - z0;
    }
    T ax = 0, ay = 0, az = 0, dgx = 0, dgy = 0, dgz = 0;
#pragma unroll
    for (int bit = 0; bit < 24; ++bit) {
      const int p = bit >> 2, av = bit & 3;
      int a0, a1, a2;
      kuhn_perm(p, a0, a1, a2);
      int PX[4], PY[4], PZ[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        PX[v] = (v >= 1 && a0 == 0) + (v >= 2 && a1 == 0) + (v >= 3 && a2 == 0);
        PY[v] = (v >= 1 && a0 == 1) + (v >= 2 && a1 == 1) + (v >= 3 && a2 == 1);
        PZ[v] = (v >= 1 && a0 == 2) + (v >= 2 && a1 == 2) + (v >= 3 && a2 == 2);
      }
      int dv[4];
      T ks = k0;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int oX = PX[v] - PX[av], oY = PY[v] - PY[av], oZ = PZ[v] - PZ[av];
        dv[v] = v == av ? -1 : dir_of_offset(oX - oY, oY - oZ, oZ);
        if (v != av) ks += kk[dv[v]];
      }
      const T kb = (T)0.25 * ks;
      T ex = 0, ey = 0, ez = 0;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        if (v == av) continue;
        const T* Kt = nc.ke[p][av][v];
        const int d = dv[v];
        ex = fma(Kt[0], dx[d], fma(Kt[1], dy[d], fma(Kt[2], dz[d], ex)));
        ey = fma(Kt[3], dx[d], fma(Kt[4], dy[d], fma(Kt[5], dz[d], ey)));
        ez = fma(Kt[6], dx[d], fma(Kt[7], dy[d], fma(Kt[8], dz[d], ez)));
        if (OP == OP_JACOBI || OP == OP_CHEBY || OP == OP_DIAG) {
          dgx = fma(-kb, Kt[0], dgx);
          dgy = fma(-kb, Kt[4], dgy);
          dgz = fma(-kb, Kt[8], dgz);
        }
      }
      ax = fma(kb, ex, ax);
      ay = fma(kb, ey, ay);
      az = fma(kb, ez, az);
    }
    epilogue<T, OP>(a, base + c0, E, ax, ay, az, dgx, dgy, dgz, x0, y0, z0, r2);
  }
  if (OP == OP_RESID && a.partial != nullptr) block_sum_store<T>(r2, a.partial + blockIdx.x);
}

// ---------------------------------------------------------------------------
// Stored stencils (Sec. 4, the paper's third method): the 15 blocks of every macro-interior
// row (135 values, Table memorytotal) are computed once per coefficient by k_store_stencil and
// streamed by k_interior_stored, which evaluates the row as the plain product
// sum_q B_q x_{i+q} over the centre and the 14 neighbours.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(INTERIOR_BLOCK) k_store_stencil(const LevelDev L, const MacroStencil<double> st,
                                                                   const int macro, const OpFlags fl,
                                                                   const double* __restrict__ k64,
                                                                   T* __restrict__ out) {
  const int32_t tile = L.tiles_lin[blockIdx.x];
  const int n = L.n;
  const int k = tile >> 20;
  const int M = n - 1 - k;
  const int t = (tile & 0xFFFFF) + threadIdx.x;
  if (t >= (M - 1) * M / 2) return;
  int j, i;
  slice_decode(M, t, j, i);
  const int64_t E = L.entries;
  const int64_t base = (int64_t)macro * L.nt;
  int nb[NDIR];
  lattice_neighbours(n, i, j, k, nb);
  const int c0 = lattice_index32(n, i, j, k);
  const int64_t e = base + c0;
  const double k0 = k64[e];
  double kk[NDIR];
#pragma unroll
  for (int d = 0; d < NDIR; ++d) kk[d] = k64[base + nb[d]];
  double cen[9];
#pragma unroll
  for (int r = 0; r < 9; ++r) cen[r] = 0.0;
#pragma unroll
  for (int d = 0; d < NDIR; ++d) {
    const int dd = d < 7 ? d : d - 7;  // Shat_{-d} = Shat_d, s[-d] = s[d]
    double rs = 0.0, wx = 0.0, wy = 0.0, wz = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (c >= ring_count(d)) continue;
      const double ka = kk[ring_a(d, c)], kb = kk[ring_b(d, c)];
      rs += ka + kb;
      wx = fma(ka - kb, st.s[dd][c][0], wx);
      wy = fma(ka - kb, st.s[dd][c][1], wy);
      wz = fma(ka - kb, st.s[dd][c][2], wz);
    }
    if (!fl.physical) wx = wy = wz = 0.0;
    const double kh = fl.khat_edge ? 0.5 * (k0 + kk[d]) : 0.25 * (k0 + kk[d]) + (dir_red(d) ? 1.0 / 12.0 : 0.125) * rs;
    const double* S = st.S[dd];
    const double blk[9] = {kh * S[0], kh * S[3] - wz, kh * S[4] + wy,
                           kh * S[3] + wz, kh * S[1], kh * S[5] - wx,
                           kh * S[4] - wy, kh * S[5] + wx, kh * S[2]};
#pragma unroll
    for (int r = 0; r < 9; ++r) {
      out[(int64_t)(9 * d + r) * E + e] = (T)blk[r];
      cen[r] -= blk[r];
    }
  }
#pragma unroll
  for (int r = 0; r < 9; ++r) out[(int64_t)(9 * NDIR + r) * E + e] = (T)cen[r];
}

template <typename T, int OP>
__global__ void __launch_bounds__(INTERIOR_BLOCK) k_interior_stored(const LevelDev L, const int macro,
                                                                     const SweepArgs<T> a) {
  const int32_t tile = L.tiles_lin[blockIdx.x];
  const int n = L.n;
  const int k = tile >> 20;
  const int M = n - 1 - k;
  const int t = (tile & 0xFFFFF) + threadIdx.x;
  double r2 = 0.0;
  if (t < (M - 1) * M / 2) {
    int j, i;
    slice_decode(M, t, j, i);
    const int64_t E = L.entries;
    const int64_t base = (int64_t)macro * L.nt;
    int nb[NDIR];
    lattice_neighbours(n, i, j, k, nb);
    const int64_t e = base + lattice_index32(n, i, j, k);
    const T* __restrict__ X = a.x + base;
    const T* __restrict__ B = a.stencil + e;
    const T x0 = a.x[e], y0 = a.x[e + E], z0 = a.x[e + 2 * E];
    T ax = B[(int64_t)(9 * NDIR + 0) * E] * x0, ay = B[(int64_t)(9 * NDIR + 3) * E] * x0,
      az = B[(int64_t)(9 * NDIR + 6) * E] * x0;
    ax = fma(B[(int64_t)(9 * NDIR + 1) * E], y0, fma(B[(int64_t)(9 * NDIR + 2) * E], z0, ax));
    ay = fma(B[(int64_t)(9 * NDIR + 4) * E], y0, fma(B[(int64_t)(9 * NDIR + 5) * E], z0, ay));
    az = fma(B[(int64_t)(9 * NDIR + 7) * E], y0, fma(B[(int64_t)(9 * NDIR + 8) * E], z0, az));
#pragma unroll
    for (int d = 0; d < NDIR; ++d) {
      const int q = nb[d];
      const T vx = X[q], vy = X[q + E], vz = X[q + 2 * E];
      const T* b = B + (int64_t)(9 * d) * E;
      ax = fma(b[0], vx, fma(b[E], vy, fma(b[2 * E], vz, ax)));
      ay = fma(b[3 * E], vx, fma(b[4 * E], vy, fma(b[5 * E], vz, ay)));
      az = fma(b[6 * E], vx, fma(b[7 * E], vy, fma(b[8 * E], vz, az)));
    }
    T dgx = 0, dgy = 0, dgz = 0;
    if (OP == OP_JACOBI || OP == OP_CHEBY || OP == OP_DIAG) {
      dgx = B[(int64_t)(9 * NDIR + 0) * E];
      dgy = B[(int64_t)(9 * NDIR + 4) * E];
      dgz = B[(int64_t)(9 * NDIR + 8) * E];
    }
    epilogue<T, OP>(a, e, E, ax, ay, az, dgx, dgy, dgz, x0, y0, z0, r2);
  }
  if (OP == OP_RESID && a.partial != nullptr) block_sum_store<T>(r2, a.partial + blockIdx.x);
}

// Kuhn coordinates of corner (i, j, k): X = i+j+k, Y = j+k, Z = k.
__device__ __forceinline__ bool kuhn_inside(int n, int X, int Y, int Z) {
  return 0 <= Z && Z <= Y && Y <= X && X <= n;
}
__device__ __forceinline__ bool kuhn_interior(int n, int X, int Y, int Z) {
  return 1 <= Z && Z < Y && Y < X && X <= n - 1;
}

// Contribution of one incident macro to the row of a skeleton node at corner
// (i, j, k) of that macro: a_h terms over the candidate elements `cand` (bit
// 4p+av: Kuhn permutation p, node at vertex av) for partner vertices on the
// skeleton (every partner with the practical rule), and the scaled blocks of
// the directions that end at a macro-interior node (symmetric rule).
// Candidates bit in [B0, B1) and directions in [D0, D1) only (a part of the row).
template <typename T, int B0 = 0, int B1 = 24, int D0 = 0, int D1 = NDIR>
__device__ __forceinline__ void incidence_row(const MacroConsts<T>& C, const T* __restrict__ px,
                                              const T* __restrict__ pk, int64_t E, int n, int i, int j, int k,
                                              uint32_t cand, uint32_t dirs, T x0, T y0, T z0, const OpFlags& fl,
                                              T& ax, T& ay, T& az, T& dgx, T& dgy, T& dgz) {
  const int X = i + j + k, Y = j + k, Z = k;
  int nb[NDIR];
  lattice_neighbours(n, i, j, k, nb);
  const int c0 = lattice_index32(n, i, j, k);
  // fully unrolled over the 24 candidates so that permutation, vertex offsets, the
  // neighbour direction of every vertex and stiffness offsets are compile-time constants
#pragma unroll
  for (int bit = B0; bit < B1; ++bit) {
    if (!((cand >> bit) & 1u)) continue;
    const int p = bit >> 2, av = bit & 3;
    int a0, a1, a2;
    kuhn_perm(p, a0, a1, a2);
    int PX[4], PY[4], PZ[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      PX[v] = (v >= 1 && a0 == 0) + (v >= 2 && a1 == 0) + (v >= 3 && a2 == 0);
      PY[v] = (v >= 1 && a0 == 1) + (v >= 2 && a1 == 1) + (v >= 3 && a2 == 1);
      PZ[v] = (v >= 1 && a0 == 2) + (v >= 2 && a1 == 2) + (v >= 3 && a2 == 2);
    }
    const int cX = X - PX[av], cY = Y - PY[av], cZ = Z - PZ[av];
    bool ok = true;
    int idx[4];
    bool inner[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int VX = cX + PX[v], VY = cY + PY[v], VZ = cZ + PZ[v];
      ok = ok && kuhn_inside(n, VX, VY, VZ);
      // Kuhn offset of vertex v from the node, as a corner offset -> stencil direction
      const int oX = PX[v] - PX[av], oY = PY[v] - PY[av], oZ = PZ[v] - PZ[av];
      idx[v] = v == av ? c0 : nb[dir_of_offset(oX - oY, oY - oZ, oZ)];
      inner[v] = kuhn_interior(n, VX, VY, VZ);
    }
    if (!ok) continue;
    const T kb = (T)0.25 * (pk[idx[0]] + pk[idx[1]] + pk[idx[2]] + pk[idx[3]]);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      if (v == av) continue;
      if (!fl.practical && inner[v]) continue;
      const T* K = C.ke[p][av][v];
      const T ddx = px[idx[v]] - x0, ddy = px[idx[v] + E] - y0, ddz = px[idx[v] + 2 * E] - z0;
      ax += kb * (K[0] * ddx + K[1] * ddy + K[2] * ddz);
      ay += kb * (K[3] * ddx + K[4] * ddy + K[5] * ddz);
      az += kb * (K[6] * ddx + K[7] * ddy + K[8] * ddz);
      dgx -= kb * K[0];
      dgy -= kb * K[4];
      dgz -= kb * K[8];
    }
  }
  if (fl.practical || !dirs) return;
  const T k0 = pk[c0];
#pragma unroll
  for (int d = D0; d < D1; ++d) {
    if (!((dirs >> d) & 1u)) continue;
    const int qi = i + dir_di(d), qj = j + dir_dj(d), qk = k + dir_dk(d);
    if (!lattice_interior(n, qi, qj, qk)) continue;
    const int qe = nb[d];
    T rs = 0, wx = 0, wy = 0, wz = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (c >= ring_count(d)) continue;
      const T ka = pk[nb[ring_a(d, c)]];
      const T kb = pk[nb[ring_b(d, c)]];
      rs += ka + kb;
      const T dk = ka - kb;
      wx += dk * C.st.s[d][c][0];
      wy += dk * C.st.s[d][c][1];
      wz += dk * C.st.s[d][c][2];
    }
    const T kq = pk[qe];
    const T kh = fl.khat_edge ? (T)0.5 * (k0 + kq)
                              : (T)0.25 * (k0 + kq) + (dir_red(d) ? (T)(1.0 / 12.0) : (T)0.125) * rs;
    const T* S = C.st.S[d < 7 ? d : d - 7];
    const T ddx = px[qe] - x0, ddy = px[qe + E] - y0, ddz = px[qe + 2 * E] - z0;
    ax += kh * (S[0] * ddx + S[3] * ddy + S[4] * ddz);
    ay += kh * (S[3] * ddx + S[1] * ddy + S[5] * ddz);
    az += kh * (S[4] * ddx + S[5] * ddy + S[2] * ddz);
    if (fl.physical) {
      ax += wy * ddz - wz * ddy;
      ay += wz * ddx - wx * ddz;
      az += wx * ddy - wy * ddx;
    }
    dgx -= kh * S[0];
    dgy -= kh * S[1];
    dgz -= kh * S[2];
  }
}

__constant__ int c_dir[NDIR][3];
__constant__ int c_ring[NDIR][3][2];
__constant__ int c_ring_n[NDIR];

// Lane version of incidence_row for the block kernels: lane l evaluates candidate
// element l (l < 24) and stencil direction l (l < 14) with run-time indices, so
// the lanes of a warp run the same element/direction body concurrently.
template <typename T>
__device__ __forceinline__ void incidence_lane(const MacroConsts<T>& C, const T* __restrict__ px,
                                               const T* __restrict__ pk, int64_t E, int n, int i, int j, int k,
                                               int lane, T x0, T y0, T z0, const OpFlags& fl, T& ax, T& ay, T& az,
                                               T& dgx, T& dgy, T& dgz) {
  if (lane < 24) {
    const int X = i + j + k, Y = j + k, Z = k;
    const int p = lane >> 2, av = lane & 3;
    // Kuhn permutation p (lexicographic order 012 021 102 120 201 210)
    const int a0 = p >> 1;
    const int lo = a0 == 0 ? 1 : 0, hi = a0 == 2 ? 1 : 2;
    const int a1 = (p & 1) ? hi : lo, a2 = (p & 1) ? lo : hi;
    const int oX = (av >= 1 && a0 == 0) + (av >= 2 && a1 == 0) + (av >= 3 && a2 == 0);
    const int oY = (av >= 1 && a0 == 1) + (av >= 2 && a1 == 1) + (av >= 3 && a2 == 1);
    const int oZ = (av >= 1 && a0 == 2) + (av >= 2 && a1 == 2) + (av >= 3 && a2 == 2);
    bool ok = true;
    int idx[4];
    bool inner[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int VX = X - oX + (v >= 1 && a0 == 0) + (v >= 2 && a1 == 0) + (v >= 3 && a2 == 0);
      const int VY = Y - oY + (v >= 1 && a0 == 1) + (v >= 2 && a1 == 1) + (v >= 3 && a2 == 1);
      const int VZ = Z - oZ + (v >= 1 && a0 == 2) + (v >= 2 && a1 == 2) + (v >= 3 && a2 == 2);
      ok = ok && kuhn_inside(n, VX, VY, VZ);
      idx[v] = ok ? lattice_index32(n, VX - VY, VY - VZ, VZ) : 0;
      inner[v] = kuhn_interior(n, VX, VY, VZ);
    }
    if (ok) {
      const T kb = (T)0.25 * (pk[idx[0]] + pk[idx[1]] + pk[idx[2]] + pk[idx[3]]);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        if (v == av) continue;
        if (!fl.practical && inner[v]) continue;
        const T* K = C.ke[p][av][v];
        const T ddx = px[idx[v]] - x0, ddy = px[idx[v] + E] - y0, ddz = px[idx[v] + 2 * E] - z0;
        ax += kb * (K[0] * ddx + K[1] * ddy + K[2] * ddz);
        ay += kb * (K[3] * ddx + K[4] * ddy + K[5] * ddz);
        az += kb * (K[6] * ddx + K[7] * ddy + K[8] * ddz);
        dgx -= kb * K[0];
        dgy -= kb * K[4];
        dgz -= kb * K[8];
      }
    }
  }
  if (fl.practical || lane >= NDIR) return;
  const int d = lane;
  const int qi = i + c_dir[d][0], qj = j + c_dir[d][1], qk = k + c_dir[d][2];
  if (!lattice_interior(n, qi, qj, qk)) return;
  const T k0 = pk[lattice_index32(n, i, j, k)];
  const int qe = lattice_index32(n, qi, qj, qk);
  T rs = 0, wx = 0, wy = 0, wz = 0;
  for (int c = 0; c < c_ring_n[d]; ++c) {
    const int ra = c_ring[d][c][0], rb = c_ring[d][c][1];
    const T ka = pk[lattice_index32(n, i + c_dir[ra][0], j + c_dir[ra][1], k + c_dir[ra][2])];
    const T kb = pk[lattice_index32(n, i + c_dir[rb][0], j + c_dir[rb][1], k + c_dir[rb][2])];
    rs += ka + kb;
    const T dk = ka - kb;
    wx += dk * C.st.s[d][c][0];
    wy += dk * C.st.s[d][c][1];
    wz += dk * C.st.s[d][c][2];
  }
  const T kq = pk[qe];
  const T kh = fl.khat_edge ? (T)0.5 * (k0 + kq)
                            : (T)0.25 * (k0 + kq) + (c_ring_n[d] == 3 ? (T)(1.0 / 12.0) : (T)0.125) * rs;
  const T* S = C.st.S[d < 7 ? d : d - 7];
  const T ddx = px[qe] - x0, ddy = px[qe + E] - y0, ddz = px[qe + 2 * E] - z0;
  ax += kh * (S[0] * ddx + S[3] * ddy + S[4] * ddz);
  ay += kh * (S[3] * ddx + S[1] * ddy + S[5] * ddz);
  az += kh * (S[4] * ddx + S[5] * ddy + S[2] * ddz);
  if (fl.physical) {
    ax += wy * ddz - wz * ddy;
    ay += wz * ddx - wx * ddz;
    az += wx * ddy - wy * ddx;
  }
  dgx -= kh * S[0];
  dgy -= kh * S[1];
  dgz -= kh * S[2];
}

template <typename T>
__device__ __forceinline__ T* acc_of(const LevelDev& L);
template <>
__device__ __forceinline__ float* acc_of<float>(const LevelDev& L) {
  return L.acc32;
}
template <>
__device__ __forceinline__ double* acc_of<double>(const LevelDev& L) {
  return L.acc64;
}

// ---------------------------------------------------------------------------
// Free face-interior skeleton nodes, one thread per node (k_face_rows).  A node on a macro
// face has one incidence per macro sharing the face (two on an interior face); in macro T
// the node sits on face F of T's lattice (F = 0: i + j + k = n, 1: i = 0, 2: j = 0,
// 3: k = 0), so the elements of T around it, the stencil directions that stay in T and
// those that can end at a macro-interior node are fixed by F.  face_incidence<F> evaluates
// T's part of the row with those sets fixed at compile time (the representative
// face-interior point of each face type, on a lattice with 16 intervals, decides them);
// only whether a neighbour is macro-interior (next to the face's edges it is not) is
// decided at run time.  The symmetric interface rule of Sec. 2.2: pairs of skeleton nodes
// by nodal integration a_h over T's elements, pairs with a macro-interior neighbour by T's
// scaled block; the practical rule: a_h for every pair.  Rows are in difference form, so
// the centre block is minus the sum of the off-diagonal blocks.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void face_rep(int F, int& i, int& j, int& k) {
  i = F == 1 ? 0 : 5;
  j = F == 2 ? 0 : 5;
  k = F == 3 ? 0 : (F == 0 ? 6 : 5);
}
// direction d stays in the macro's closed lattice from a face-interior point of face F
__device__ __forceinline__ bool face_dir_valid(int F, int d) {
  int i, j, k;
  face_rep(F, i, j, k);
  return lattice_inside(16, i + dir_di(d), j + dir_dj(d), k + dir_dk(d));
}
// direction d can end at a macro-interior point
__device__ __forceinline__ bool face_dir_inward(int F, int d) {
  int i, j, k;
  face_rep(F, i, j, k);
  return lattice_interior(16, i + dir_di(d), j + dir_dj(d), k + dir_dk(d));
}
// candidate element (bit 4 p + av: Kuhn permutation p, the point at vertex av) lies in the macro
__device__ __forceinline__ bool face_cand_inside(int F, int bit) {
  int i, j, k;
  face_rep(F, i, j, k);
  const int p = bit >> 2, av = bit & 3;
  int a0, a1, a2;
  kuhn_perm(p, a0, a1, a2);
  const int X = i + j + k, Y = j + k, Z = k;
  bool ok = true;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int VX = X + ((v >= 1 && a0 == 0) + (v >= 2 && a1 == 0) + (v >= 3 && a2 == 0)) -
                   ((av >= 1 && a0 == 0) + (av >= 2 && a1 == 0) + (av >= 3 && a2 == 0));
    const int VY = Y + ((v >= 1 && a0 == 1) + (v >= 2 && a1 == 1) + (v >= 3 && a2 == 1)) -
                   ((av >= 1 && a0 == 1) + (av >= 2 && a1 == 1) + (av >= 3 && a2 == 1));
    const int VZ = Z + ((v >= 1 && a0 == 2) + (v >= 2 && a1 == 2) + (v >= 3 && a2 == 2)) -
                   ((av >= 1 && a0 == 2) + (av >= 2 && a1 == 2) + (av >= 3 && a2 == 2));
    ok = ok && kuhn_inside(16, VX, VY, VZ);
  }
  return ok;
}

template <typename T, int F, bool DIAG>
__device__ __forceinline__ void face_incidence(const MacroConsts<T>& C, const T* __restrict__ px,
                                               const T* __restrict__ pk, int64_t E, int n, int i, int j, int k,
                                               const OpFlags& fl, T x0, T y0, T z0, T& ax, T& ay, T& az, T& dgx,
                                               T& dgy, T& dgz) {
  int nb[NDIR];
  lattice_neighbours(n, i, j, k, nb);
  const T k0 = pk[lattice_index32(n, i, j, k)];
  T kv[NDIR], dx[NDIR], dy[NDIR], dz[NDIR];
  bool in[NDIR];
#pragma unroll
  for (int d = 0; d < NDIR; ++d) {
    kv[d] = dx[d] = dy[d] = dz[d] = (T)0;
    in[d] = false;
    if (face_dir_valid(F, d)) {
      const int q = nb[d];
      kv[d] = pk[q];
      dx[d] = px[q] - x0;
      dy[d] = px[q + E] - y0;
      dz[d] = px[q + 2 * E] - z0;
      in[d] = face_dir_inward(F, d) && lattice_interior(n, i + dir_di(d), j + dir_dj(d), k + dir_dk(d));
    }
  }
  // nodal-integration terms over the macro's elements around the point
#pragma unroll
  for (int bit = 0; bit < 24; ++bit) {
    if (!face_cand_inside(F, bit)) continue;
    const int p = bit >> 2, av = bit & 3;
    int a0, a1, a2;
    kuhn_perm(p, a0, a1, a2);
    int dv[4];
    T ks = k0;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int oX = ((v >= 1 && a0 == 0) + (v >= 2 && a1 == 0) + (v >= 3 && a2 == 0)) -
                     ((av >= 1 && a0 == 0) + (av >= 2 && a1 == 0) + (av >= 3 && a2 == 0));
      const int oY = ((v >= 1 && a0 == 1) + (v >= 2 && a1 == 1) + (v >= 3 && a2 == 1)) -
                     ((av >= 1 && a0 == 1) + (av >= 2 && a1 == 1) + (av >= 3 && a2 == 1));
      const int oZ = ((v >= 1 && a0 == 2) + (v >= 2 && a1 == 2) + (v >= 3 && a2 == 2)) -
                     ((av >= 1 && a0 == 2) + (av >= 2 && a1 == 2) + (av >= 3 && a2 == 2));
      dv[v] = v == av ? -1 : dir_of_offset(oX - oY, oY - oZ, oZ);
      if (v != av) ks += kv[dv[v]];
    }
    const T kb = (T)0.25 * ks;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      if (v == av) continue;
      const int d = dv[v];
      if (!fl.practical && in[d]) continue;
      const T* K = C.ke[p][av][v];
      ax = fma(kb, fma(K[0], dx[d], fma(K[1], dy[d], K[2] * dz[d])), ax);
      ay = fma(kb, fma(K[3], dx[d], fma(K[4], dy[d], K[5] * dz[d])), ay);
      az = fma(kb, fma(K[6], dx[d], fma(K[7], dy[d], K[8] * dz[d])), az);
      if (DIAG) {
        dgx = fma(-kb, K[0], dgx);
        dgy = fma(-kb, K[4], dgy);
        dgz = fma(-kb, K[8], dgz);
      }
    }
  }
  if (fl.practical) return;
  // scaled blocks of the directions that end at a macro-interior point (their ring nodes
  // are neighbours of that point, so they lie in the macro)
#pragma unroll
  for (int d = 0; d < NDIR; ++d) {
    if (!face_dir_inward(F, d)) continue;
    if (!in[d]) continue;
    T rs = 0, wx = 0, wy = 0, wz = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (c >= ring_count(d)) continue;
      const T ka = kv[ring_a(d, c)], kb = kv[ring_b(d, c)];
      rs += ka + kb;
      const T dk = ka - kb;
      wx = fma(dk, C.st.s[d][c][0], wx);
      wy = fma(dk, C.st.s[d][c][1], wy);
      wz = fma(dk, C.st.s[d][c][2], wz);
    }
    const T kh = fl.khat_edge ? (T)0.5 * (k0 + kv[d])
                              : fma((dir_red(d) ? (T)(1.0 / 12.0) : (T)0.125), rs, (T)0.25 * (k0 + kv[d]));
    const T* S = C.st.S[d < 7 ? d : d - 7];
    const T vx = kh * dx[d], vy = kh * dy[d], vz = kh * dz[d];
    ax = fma(S[0], vx, fma(S[3], vy, fma(S[4], vz, ax)));
    ay = fma(S[3], vx, fma(S[1], vy, fma(S[5], vz, ay)));
    az = fma(S[4], vx, fma(S[5], vy, fma(S[2], vz, az)));
    if (fl.physical) {
      ax = fma(wy, dz[d], fma(-wz, dy[d], ax));
      ay = fma(wz, dx[d], fma(-wx, dz[d], ay));
      az = fma(wx, dy[d], fma(-wy, dx[d], az));
    }
    if (DIAG) {
      dgx = fma(-kh, S[0], dgx);
      dgy = fma(-kh, S[1], dgy);
      dgz = fma(-kh, S[2], dgz);
    }
  }
}

template <typename T, int OP>
__global__ void __launch_bounds__(128) k_face_rows(const LevelDev L, const MacroConsts<T>* __restrict__ mc,
                                                    const OpFlags fl, const SweepArgs<T> a) {
  constexpr bool DIAG = OP == OP_JACOBI || OP == OP_CHEBY || OP == OP_DIAG;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double r2 = 0.0;
  if (t < L.nface_nodes) {
    const int n = L.n;
    const int64_t E = L.entries;
    const int s = L.face_nodes[t];
    const int b0 = L.skel_ptr[s], b1 = L.skel_ptr[s + 1];
    const SkelInc I0 = L.skel_inc[b0];
    const int64_t e0 = (int64_t)I0.macro * L.nt + lattice_index32(n, I0.i, I0.j, I0.k);
    const T x0 = a.x[e0], y0 = a.x[e0 + E], z0 = a.x[e0 + 2 * E];
    T ax = 0, ay = 0, az = 0, dgx = 0, dgy = 0, dgz = 0;
    for (int q = b0; q < b1; ++q) {
      const SkelInc I = L.skel_inc[q];
      const int64_t base = (int64_t)I.macro * L.nt;
      const T* px = a.x + base;
      const T* pk = a.k + base;
      const MacroConsts<T>& C = mc[I.macro];
      const int f = (I.i + I.j + I.k == n) ? 0 : (I.i == 0) ? 1 : (I.j == 0) ? 2 : 3;
      switch (f) {
        case 0: face_incidence<T, 0, DIAG>(C, px, pk, E, n, I.i, I.j, I.k, fl, x0, y0, z0, ax, ay, az, dgx, dgy, dgz); break;
        case 1: face_incidence<T, 1, DIAG>(C, px, pk, E, n, I.i, I.j, I.k, fl, x0, y0, z0, ax, ay, az, dgx, dgy, dgz); break;
        case 2: face_incidence<T, 2, DIAG>(C, px, pk, E, n, I.i, I.j, I.k, fl, x0, y0, z0, ax, ay, az, dgx, dgy, dgz); break;
        default: face_incidence<T, 3, DIAG>(C, px, pk, E, n, I.i, I.j, I.k, fl, x0, y0, z0, ax, ay, az, dgx, dgy, dgz); break;
      }
    }
    for (int q = b0; q < b1; ++q) {
      const SkelInc I = L.skel_inc[q];
      const int64_t e = (int64_t)I.macro * L.nt + lattice_index32(n, I.i, I.j, I.k);
      double tmp = 0.0;
      epilogue<T, OP>(a, e, E, ax, ay, az, dgx, dgy, dgz, x0, y0, z0, tmp);
      if (q == b0) r2 = tmp;
    }
  }
  if (OP == OP_RESID && a.partial != nullptr) block_sum_store<T>(r2, a.partial + blockIdx.x);
}

// Dirichlet skeleton nodes: identity rows (residual 0), every copy.
template <typename T, int OP>
__global__ void __launch_bounds__(128) k_dirichlet(const LevelDev L, const SweepArgs<T> a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L.ndir) return;
  const int n = L.n;
  const int64_t E = L.entries;
  const int s = L.dir_nodes[t];
  const int b0 = L.skel_ptr[s], b1 = L.skel_ptr[s + 1];
  const SkelInc I0 = L.skel_inc[b0];
  const int64_t e0 = (int64_t)I0.macro * L.nt + lattice_index32(n, I0.i, I0.j, I0.k);
  const T x0 = a.x[e0], y0 = a.x[e0 + E], z0 = a.x[e0 + 2 * E];
  for (int q = b0; q < b1; ++q) {
    const SkelInc I = L.skel_inc[q];
    const int64_t e = (int64_t)I.macro * L.nt + lattice_index32(n, I.i, I.j, I.k);
    if (OP == OP_RESID) {
      a.out[e] = 0;
      a.out[e + E] = 0;
      a.out[e + 2 * E] = 0;
    } else if (OP == OP_DIAG) {
      a.out[e] = 1;
      a.out[e + E] = 1;
      a.out[e + 2 * E] = 1;
    } else {
      a.out[e] = x0;
      a.out[e + E] = y0;
      a.out[e + 2 * E] = z0;
      if (OP == OP_CHEBY) {
        a.dout[e] = 0;
        a.dout[e + E] = 0;
        a.dout[e + 2 * E] = 0;
      }
    }
  }
}

// Free nodes on macro edges and vertices: one 128-thread block per node; warp w
// takes incidences w, w+4, ...; lanes take candidate elements and directions
// (incidence_lane).  Warp sums are combined in a fixed order, so the row is
// deterministic, and it is written to every copy of the node.
template <typename T, int OP>
__global__ void __launch_bounds__(128) k_skeleton_ev(const LevelDev L, const MacroConsts<T>* __restrict__ mc,
                                                      const OpFlags fl, const SweepArgs<T> a) {
  __shared__ T part[4][6];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double r2 = 0.0;
  const int s = L.ev_nodes[blockIdx.x];
  const int n = L.n;
  const int64_t E = L.entries;
  const int b0 = L.skel_ptr[s], b1 = L.skel_ptr[s + 1];
  const SkelInc I0 = L.skel_inc[b0];
  const int64_t e0 = (int64_t)I0.macro * L.nt + lattice_index32(n, I0.i, I0.j, I0.k);
  const T x0 = a.x[e0], y0 = a.x[e0 + E], z0 = a.x[e0 + 2 * E];
  T ax = 0, ay = 0, az = 0, dgx = 0, dgy = 0, dgz = 0;
  for (int q = b0 + warp; q < b1; q += 4) {
    const SkelInc I = L.skel_inc[q];
    const int64_t base = (int64_t)I.macro * L.nt;
    incidence_lane<T>(mc[I.macro], a.x + base, a.k + base, E, n, I.i, I.j, I.k, lane, x0, y0, z0, fl, ax, ay, az,
                      dgx, dgy, dgz);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ax += __shfl_xor_sync(0xffffffffu, ax, o);
    ay += __shfl_xor_sync(0xffffffffu, ay, o);
    az += __shfl_xor_sync(0xffffffffu, az, o);
    dgx += __shfl_xor_sync(0xffffffffu, dgx, o);
    dgy += __shfl_xor_sync(0xffffffffu, dgy, o);
    dgz += __shfl_xor_sync(0xffffffffu, dgz, o);
  }
  if (lane == 0) {
    part[warp][0] = ax;
    part[warp][1] = ay;
    part[warp][2] = az;
    part[warp][3] = dgx;
    part[warp][4] = dgy;
    part[warp][5] = dgz;
  }
  __syncthreads();
  ax = (part[0][0] + part[1][0]) + (part[2][0] + part[3][0]);
  ay = (part[0][1] + part[1][1]) + (part[2][1] + part[3][1]);
  az = (part[0][2] + part[1][2]) + (part[2][2] + part[3][2]);
  dgx = (part[0][3] + part[1][3]) + (part[2][3] + part[3][3]);
  dgy = (part[0][4] + part[1][4]) + (part[2][4] + part[3][4]);
  dgz = (part[0][5] + part[1][5]) + (part[2][5] + part[3][5]);
  for (int q = b0 + threadIdx.x; q < b1; q += blockDim.x) {
    const SkelInc I = L.skel_inc[q];
    const int64_t e = (int64_t)I.macro * L.nt + lattice_index32(n, I.i, I.j, I.k);
    double tmp = 0.0;
    epilogue<T, OP>(a, e, E, ax, ay, az, dgx, dgy, dgz, x0, y0, z0, tmp);
    if (q == b0) r2 = tmp;
  }
  if (OP == OP_RESID && a.partial != nullptr) block_sum_store<T>(r2, a.partial + blockIdx.x);
}

// Stokes element terms of one candidate element (permutation p, node at vertex av)
// of one incident macro for the skeleton node at Kuhn coordinates (X, Y, Z): full
// element sums of B u, C p (pressure row) and B^T p (velocity rows) -- no interface
// rule applies to these coefficient-free blocks.
template <typename T>
__device__ __forceinline__ void stokes_candidate(const MacroConsts<T>& C, const T* __restrict__ px, int64_t E, int n,
                                                 int X, int Y, int Z, int p, int av, T& ax, T& ay, T& az, T& yp) {
  const int a0 = p >> 1;
  const int lo = a0 == 0 ? 1 : 0, hi = a0 == 2 ? 1 : 2;
  const int a1 = (p & 1) ? hi : lo, a2 = (p & 1) ? lo : hi;
  const int oX = (av >= 1 && a0 == 0) + (av >= 2 && a1 == 0) + (av >= 3 && a2 == 0);
  const int oY = (av >= 1 && a0 == 1) + (av >= 2 && a1 == 1) + (av >= 3 && a2 == 1);
  const int oZ = (av >= 1 && a0 == 2) + (av >= 2 && a1 == 2) + (av >= 3 && a2 == 2);
  bool ok = true;
  int idx[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int VX = X - oX + (v >= 1 && a0 == 0) + (v >= 2 && a1 == 0) + (v >= 3 && a2 == 0);
    const int VY = Y - oY + (v >= 1 && a0 == 1) + (v >= 2 && a1 == 1) + (v >= 3 && a2 == 1);
    const int VZ = Z - oZ + (v >= 1 && a0 == 2) + (v >= 2 && a1 == 2) + (v >= 3 && a2 == 2);
    ok = ok && kuhn_inside(n, VX, VY, VZ);
    idx[v] = ok ? lattice_index32(n, VX - VY, VY - VZ, VZ) : 0;
  }
  if (!ok) return;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const T ux = px[idx[v]], uy = px[idx[v] + E], uz = px[idx[v] + 2 * E], pv = px[idx[v] + 3 * E];
    const T* b = C.bd[p][av][v];
    yp = fma(b[0], ux, yp);
    yp = fma(b[1], uy, yp);
    yp = fma(b[2], uz, yp);
    yp = fma(C.lc[p][av][v], pv, yp);
    const T* g = C.bd[p][v][av];
    ax = fma(g[0], pv, ax);
    ay = fma(g[1], pv, ay);
    az = fma(g[2], pv, az);
  }
}

// Stokes: face-interior skeleton nodes (Dirichlet ones included), one thread per
// (node, incident macro); velocity part as in k_face_items unless the node is
// velocity-Dirichlet, plus the element terms of B, B^T and C.
template <typename T>
__global__ void __launch_bounds__(128) k_face_items_stk(const LevelDev L, const MacroConsts<T>* __restrict__ mc,
                                                         const OpFlags fl, const T* __restrict__ x,
                                                         const T* __restrict__ kc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L.nface_items_all) return;
  const FaceItem it = L.face_items_all[t];
  const int n = L.n;
  const int64_t E = L.entries;
  const int64_t base = (int64_t)it.macro * L.nt;
  const T* px = x + base;
  const T* pk = kc + base;
  const int c0 = lattice_index32(n, it.i, it.j, it.k);
  const T x0 = px[c0], y0 = px[c0 + E], z0 = px[c0 + 2 * E];
  T ax = 0, ay = 0, az = 0, dgx = 0, dgy = 0, dgz = 0, yp = 0;
  const bool vdir = L.skel_dir[L.face_nodes_all[it.node]] != 0;
  const MacroConsts<T>& C = mc[it.macro];
  if (!vdir)
    incidence_row<T>(C, px, pk, E, n, it.i, it.j, it.k, L.face_mask[it.f], (1u << NDIR) - 1u, x0, y0, z0, fl, ax, ay,
                     az, dgx, dgy, dgz);
  const uint32_t cand = L.face_mask[it.f];
  const int X = it.i + it.j + it.k, Y = it.j + it.k, Z = it.k;
#pragma unroll
  for (int bit = 0; bit < 24; ++bit)
    if ((cand >> bit) & 1u) stokes_candidate<T>(C, px, E, n, X, Y, Z, bit >> 2, bit & 3, ax, ay, az, yp);
  T* acc = acc_of<T>(L) + 8 * (int64_t)it.node;
  atomicAdd(acc + 0, ax);
  atomicAdd(acc + 1, ay);
  atomicAdd(acc + 2, az);
  atomicAdd(acc + 6, yp);
}

template <typename T, int OP>
__global__ void __launch_bounds__(128) k_face_finalize_stk(const LevelDev L, const SweepArgs<T> a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double r2 = 0.0;
  if (t < L.nface_nodes_all) {
    const int n = L.n;
    const int64_t E = L.entries;
    T* acc = acc_of<T>(L) + 8 * (int64_t)t;
    const T ax = acc[0], ay = acc[1], az = acc[2], yp = acc[6];
    acc[0] = 0;
    acc[1] = 0;
    acc[2] = 0;
    acc[6] = 0;
    const int s = L.face_nodes_all[t];
    const bool vdir = L.skel_dir[s] != 0;
    const int b0 = L.skel_ptr[s], b1 = L.skel_ptr[s + 1];
    const SkelInc I0 = L.skel_inc[b0];
    const int64_t e0 = (int64_t)I0.macro * L.nt + lattice_index32(n, I0.i, I0.j, I0.k);
    const T x0 = a.x[e0], y0 = a.x[e0 + E], z0 = a.x[e0 + 2 * E];
    for (int q = b0; q < b1; ++q) {
      const SkelInc I = L.skel_inc[q];
      const int64_t e = (int64_t)I.macro * L.nt + lattice_index32(n, I.i, I.j, I.k);
      double tmp = 0.0;
      stokes_epilogue<T, OP>(a, e, E, ax, ay, az, yp, x0, y0, z0, vdir, tmp);
      if (q == b0) r2 = tmp;
    }
  }
  if (OP == OP_RESID && a.partial != nullptr) block_sum_store<T>(r2, a.partial + blockIdx.x);
}

// Stokes: macro edge/vertex skeleton nodes (Dirichlet ones included), one block per node.
template <typename T, int OP>
__global__ void __launch_bounds__(128) k_skeleton_ev_stk(const LevelDev L, const MacroConsts<T>* __restrict__ mc,
                                                          const OpFlags fl, const SweepArgs<T> a) {
  __shared__ T part[4][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double r2 = 0.0;
  const int s = L.ev_all[blockIdx.x];
  const bool vdir = L.skel_dir[s] != 0;
  const int n = L.n;
  const int64_t E = L.entries;
  const int b0 = L.skel_ptr[s], b1 = L.skel_ptr[s + 1];
  const SkelInc I0 = L.skel_inc[b0];
  const int64_t e0 = (int64_t)I0.macro * L.nt + lattice_index32(n, I0.i, I0.j, I0.k);
  const T x0 = a.x[e0], y0 = a.x[e0 + E], z0 = a.x[e0 + 2 * E];
  T ax = 0, ay = 0, az = 0, dgx = 0, dgy = 0, dgz = 0, yp = 0;
  for (int q = b0 + warp; q < b1; q += 4) {
    const SkelInc I = L.skel_inc[q];
    const int64_t base = (int64_t)I.macro * L.nt;
    if (!vdir)
      incidence_lane<T>(mc[I.macro], a.x + base, a.k + base, E, n, I.i, I.j, I.k, lane, x0, y0, z0, fl, ax, ay, az,
                        dgx, dgy, dgz);
    if (lane < 24)
      stokes_candidate<T>(mc[I.macro], a.x + base, E, n, I.i + I.j + I.k, I.j + I.k, I.k, lane >> 2, lane & 3, ax, ay,
                          az, yp);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ax += __shfl_xor_sync(0xffffffffu, ax, o);
    ay += __shfl_xor_sync(0xffffffffu, ay, o);
    az += __shfl_xor_sync(0xffffffffu, az, o);
    yp += __shfl_xor_sync(0xffffffffu, yp, o);
  }
  if (lane == 0) {
    part[warp][0] = ax;
    part[warp][1] = ay;
    part[warp][2] = az;
    part[warp][3] = yp;
  }
  __syncthreads();
  ax = (part[0][0] + part[1][0]) + (part[2][0] + part[3][0]);
  ay = (part[0][1] + part[1][1]) + (part[2][1] + part[3][1]);
  az = (part[0][2] + part[1][2]) + (part[2][2] + part[3][2]);
  yp = (part[0][3] + part[1][3]) + (part[2][3] + part[3][3]);
  for (int q = b0 + threadIdx.x; q < b1; q += blockDim.x) {
    const SkelInc I = L.skel_inc[q];
    const int64_t e = (int64_t)I.macro * L.nt + lattice_index32(n, I.i, I.j, I.k);
    double tmp = 0.0;
    stokes_epilogue<T, OP>(a, e, E, ax, ay, az, yp, x0, y0, z0, vdir, tmp);
    if (q == b0) r2 = tmp;
  }
  if (OP == OP_RESID && a.partial != nullptr) block_sum_store<T>(r2, a.partial + blockIdx.x);
}

}  // namespace

// one macro's interior launch: the BF16-coefficient kernel for FP32 sweeps of the default
// operator when a.k16 is set, else the FP32/FP64 coefficient kernel
// one macro's interior launch: FP32 sweeps on point pairs (the BF16-coefficient kernel for the
// default operator when a.k16 is set), FP64 sweeps one point per thread; returns the number
// of blocks (partial-sum slots)
// the interior stencil with every value as a lane pair (c, c), the operand form of the packed
// FP32 arithmetic
inline MacroStencil<float2> lane_pairs(const MacroStencil<float>& st) {
  MacroStencil<float2> p;
  const float* a = &st.S[0][0];
  float2* b = &p.S[0][0];
  for (size_t q = 0; q < sizeof(st) / sizeof(float); ++q) b[q] = make_float2(a[q], a[q]);
  return p;
}

template <typename T, int OP>
int launch_interior(bool gen, const LevelDev& L, const MacroStencil<T>& st, int m, const OpFlags& fl,
                    const SweepArgs<T>& am, cudaStream_t s) {
  if (fl.tile) {
    if (L.ntiles3 == 0) return 0;
    if (am.k16 && !gen)
      k_interior_tile<T, OP, 0, 1><<<L.ntiles3, T3_THREADS, 0, s>>>(L, st, m, fl, am);
    else if (gen)
      k_interior_tile<T, OP, 1, 0><<<L.ntiles3, T3_THREADS, 0, s>>>(L, st, m, fl, am);
    else
      k_interior_tile<T, OP, 0, 0><<<L.ntiles3, T3_THREADS, 0, s>>>(L, st, m, fl, am);
    return L.ntiles3;
  }
  if constexpr (std::is_same<T, float>::value) {
    if (L.ntiles_pair == 0) return 0;
    const MacroStencil<float2> st2 = lane_pairs(st);
    if (am.k16 && !gen)
      k_interior_pair<OP, 0, 1><<<L.ntiles_pair, INTERIOR_BLOCK, 0, s>>>(L, st2, m, fl, am);
    else if (gen)
      k_interior_pair<OP, 1, 0><<<L.ntiles_pair, INTERIOR_BLOCK, 0, s>>>(L, st2, m, fl, am);
    else
      k_interior_pair<OP, 0, 0><<<L.ntiles_pair, INTERIOR_BLOCK, 0, s>>>(L, st2, m, fl, am);
    return L.ntiles_pair;
  } else {
    if (L.ntiles_lin == 0) return 0;
    if (gen)
      k_interior<T, OP, 1><<<L.ntiles_lin, INTERIOR_BLOCK, 0, s>>>(L, st, m, fl, am, 0);
    else
      k_interior<T, OP, 0><<<L.ntiles_lin, INTERIOR_BLOCK, 0, s>>>(L, st, m, fl, am, 0);
    return L.ntiles_lin;
  }
}

// All macros' interior sweeps in launches of up to 65535 macros (grid.y); returns the number of
// blocks (partial-sum slots, macro-major).
constexpr int BATCH_MAX_MACROS = 65535;
template <typename T, int OP>
int64_t launch_interior_batched(bool gen, const LevelDev& L, const MacroConsts<T>* mc, const OpFlags& fl,
                                const SweepArgs<T>& a, cudaStream_t s) {
  const int nb = std::is_same<T, float>::value ? L.ntiles_pair : L.ntiles_lin;
  if (nb == 0) return 0;
  int64_t used = 0;
  for (int m0 = 0; m0 < L.nmacro; m0 += BATCH_MAX_MACROS) {
    const dim3 g(nb, std::min(BATCH_MAX_MACROS, L.nmacro - m0));
    SweepArgs<T> am = a;
    if (a.partial) am.partial = a.partial + used;
    if constexpr (std::is_same<T, float>::value) {
      if (am.k16 && !gen)
        k_interior_pair_batched<OP, 0, 1><<<g, INTERIOR_BLOCK, 0, s>>>(L, mc, m0, fl, am);
      else if (gen)
        k_interior_pair_batched<OP, 1, 0><<<g, INTERIOR_BLOCK, 0, s>>>(L, mc, m0, fl, am);
      else
        k_interior_pair_batched<OP, 0, 0><<<g, INTERIOR_BLOCK, 0, s>>>(L, mc, m0, fl, am);
    } else {
      if (gen)
        k_interior_batched<T, OP, 1><<<g, INTERIOR_BLOCK, 0, s>>>(L, mc, m0, fl, am);
      else
        k_interior_batched<T, OP, 0><<<g, INTERIOR_BLOCK, 0, s>>>(L, mc, m0, fl, am);
    }
    used += (int64_t)g.x * g.y;
  }
  return used;
}

template <typename T>
int launch_sweep_batched(const LevelDev& L, const MacroConsts<T>* mc_dev, OpKind op, const OpFlags& fl,
                         const SweepArgs<T>& a, void* stream, int64_t partial_offset, int64_t* partial_count) {
  cudaStream_t s = (cudaStream_t)stream;
  const bool gen = !(fl.physical == 1 && fl.khat_edge == 0);
  SweepArgs<T> am = a;
  if (a.partial) am.partial = a.partial + partial_offset;
  int64_t nb = 0;
  switch (op) {
    case OP_APPLY: nb = launch_interior_batched<T, OP_APPLY>(gen, L, mc_dev, fl, am, s); break;
    case OP_RESID: nb = launch_interior_batched<T, OP_RESID>(gen, L, mc_dev, fl, am, s); break;
    case OP_JACOBI: nb = launch_interior_batched<T, OP_JACOBI>(gen, L, mc_dev, fl, am, s); break;
    case OP_CHEBY: nb = launch_interior_batched<T, OP_CHEBY>(gen, L, mc_dev, fl, am, s); break;
    case OP_DIAG: nb = launch_interior_batched<T, OP_DIAG>(gen, L, mc_dev, fl, am, s); break;
  }
  if (partial_count) *partial_count = nb;
  return (int)cudaGetLastError();
}
template int launch_sweep_batched<float>(const LevelDev&, const MacroConsts<float>*, OpKind, const OpFlags&,
                                         const SweepArgs<float>&, void*, int64_t, int64_t*);
template int launch_sweep_batched<double>(const LevelDev&, const MacroConsts<double>*, OpKind, const OpFlags&,
                                          const SweepArgs<double>&, void*, int64_t, int64_t*);

template <typename T>
int launch_sweep_macro(const LevelDev& L, const MacroStencil<T>* st_host, const NodalConsts<T>* nc_host, int m,
                       OpKind op, const OpFlags& fl, const SweepArgs<T>& a, void* stream, int64_t partial_offset,
                       int64_t* partial_count) {
  if (partial_count) *partial_count = 0;
  if (L.ntiles_lin == 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  const bool gen = !(fl.physical == 1 && fl.khat_edge == 0);
  SweepArgs<T> am = a;
  if (a.partial) am.partial = a.partial + partial_offset;
  if (fl.stored) {
    const dim3 g(L.ntiles_lin);
    switch (op) {
      case OP_APPLY: k_interior_stored<T, OP_APPLY><<<g, INTERIOR_BLOCK, 0, s>>>(L, m, am); break;
      case OP_RESID: k_interior_stored<T, OP_RESID><<<g, INTERIOR_BLOCK, 0, s>>>(L, m, am); break;
      case OP_JACOBI: k_interior_stored<T, OP_JACOBI><<<g, INTERIOR_BLOCK, 0, s>>>(L, m, am); break;
      case OP_CHEBY: k_interior_stored<T, OP_CHEBY><<<g, INTERIOR_BLOCK, 0, s>>>(L, m, am); break;
      case OP_DIAG: k_interior_stored<T, OP_DIAG><<<g, INTERIOR_BLOCK, 0, s>>>(L, m, am); break;
    }
    if (partial_count) *partial_count = L.ntiles_lin;
    return (int)cudaGetLastError();
  }
  if (fl.nodal) {
    const dim3 g(L.ntiles_lin);
    switch (op) {
      case OP_APPLY: k_interior_nodal<T, OP_APPLY><<<g, INTERIOR_BLOCK, 0, s>>>(L, nc_host[m], m, am); break;
      case OP_RESID: k_interior_nodal<T, OP_RESID><<<g, INTERIOR_BLOCK, 0, s>>>(L, nc_host[m], m, am); break;
      case OP_JACOBI: k_interior_nodal<T, OP_JACOBI><<<g, INTERIOR_BLOCK, 0, s>>>(L, nc_host[m], m, am); break;
      case OP_CHEBY: k_interior_nodal<T, OP_CHEBY><<<g, INTERIOR_BLOCK, 0, s>>>(L, nc_host[m], m, am); break;
      case OP_DIAG: k_interior_nodal<T, OP_DIAG><<<g, INTERIOR_BLOCK, 0, s>>>(L, nc_host[m], m, am); break;
    }
    if (partial_count) *partial_count = L.ntiles_lin;
    return (int)cudaGetLastError();
  }
  int nb = 0;
  switch (op) {
    case OP_APPLY: nb = launch_interior<T, OP_APPLY>(gen, L, st_host[m], m, fl, am, s); break;
    case OP_RESID: nb = launch_interior<T, OP_RESID>(gen, L, st_host[m], m, fl, am, s); break;
    case OP_JACOBI: nb = launch_interior<T, OP_JACOBI>(gen, L, st_host[m], m, fl, am, s); break;
    case OP_CHEBY: nb = launch_interior<T, OP_CHEBY>(gen, L, st_host[m], m, fl, am, s); break;
    case OP_DIAG: nb = launch_interior<T, OP_DIAG>(gen, L, st_host[m], m, fl, am, s); break;
  }
  if (partial_count) *partial_count = nb;
  return (int)cudaGetLastError();
}

template <typename T>
int launch_sweep(const LevelDev& L, const MacroStencil<T>* st_host, const MacroConsts<T>* mc_dev, OpKind op,
                 const OpFlags& fl, const SweepArgs<T>& a, void* stream, int parts, int64_t partial_offset,
                 int64_t* partial_count, void* stream_ev, void* stream_dir) {
  cudaStream_t s = (cudaStream_t)stream;
  cudaStream_t s_ev = stream_ev ? (cudaStream_t)stream_ev : s;
  cudaStream_t s_dir = stream_dir ? (cudaStream_t)stream_dir : s;
  const dim3 blk(TILE_I, TILE_J);
  int64_t used = partial_offset;
  const bool gen = !(fl.physical == 1 && fl.khat_edge == 0);
  if ((parts & 1) && fl.batch && !fl.tile) {
    int64_t nb = 0;
    const int e = launch_sweep_batched<T>(L, mc_dev, op, fl, a, stream, used, &nb);
    if (e != 0) return e;
    used += nb;
    parts &= ~1;
  }
  for (int m = 0; m < L.nmacro && (parts & 1); ++m) {
    SweepArgs<T> am = a;
    if (a.partial) am.partial = a.partial + used;
    int nb = 0;
    switch (op) {
      case OP_APPLY: nb = launch_interior<T, OP_APPLY>(gen, L, st_host[m], m, fl, am, s); break;
      case OP_RESID: nb = launch_interior<T, OP_RESID>(gen, L, st_host[m], m, fl, am, s); break;
      case OP_JACOBI: nb = launch_interior<T, OP_JACOBI>(gen, L, st_host[m], m, fl, am, s); break;
      case OP_CHEBY: nb = launch_interior<T, OP_CHEBY>(gen, L, st_host[m], m, fl, am, s); break;
      case OP_DIAG: nb = launch_interior<T, OP_DIAG>(gen, L, st_host[m], m, fl, am, s); break;
    }
    used += nb;
  }
  if (parts & 2) {
    if (L.nface_nodes > 0) {
      const int nb = (L.nface_nodes + 127) / 128;
      SweepArgs<T> am = a;
      if (a.partial) am.partial = a.partial + used;
      switch (op) {
        case OP_APPLY: k_face_rows<T, OP_APPLY><<<nb, 128, 0, s>>>(L, mc_dev, fl, am); break;
        case OP_RESID: k_face_rows<T, OP_RESID><<<nb, 128, 0, s>>>(L, mc_dev, fl, am); break;
        case OP_JACOBI: k_face_rows<T, OP_JACOBI><<<nb, 128, 0, s>>>(L, mc_dev, fl, am); break;
        case OP_CHEBY: k_face_rows<T, OP_CHEBY><<<nb, 128, 0, s>>>(L, mc_dev, fl, am); break;
        case OP_DIAG: k_face_rows<T, OP_DIAG><<<nb, 128, 0, s>>>(L, mc_dev, fl, am); break;
      }
      used += nb;
    }
    if (L.nev > 0) {
      const int nb = L.nev;
      SweepArgs<T> am = a;
      if (a.partial) am.partial = a.partial + used;
      switch (op) {
        case OP_APPLY: k_skeleton_ev<T, OP_APPLY><<<nb, 128, 0, s_ev>>>(L, mc_dev, fl, am); break;
        case OP_RESID: k_skeleton_ev<T, OP_RESID><<<nb, 128, 0, s_ev>>>(L, mc_dev, fl, am); break;
        case OP_JACOBI: k_skeleton_ev<T, OP_JACOBI><<<nb, 128, 0, s_ev>>>(L, mc_dev, fl, am); break;
        case OP_CHEBY: k_skeleton_ev<T, OP_CHEBY><<<nb, 128, 0, s_ev>>>(L, mc_dev, fl, am); break;
        case OP_DIAG: k_skeleton_ev<T, OP_DIAG><<<nb, 128, 0, s_ev>>>(L, mc_dev, fl, am); break;
      }
      used += nb;
    }
    if (L.ndir > 0) {
      const int nb = (L.ndir + 127) / 128;
      switch (op) {
        case OP_APPLY: k_dirichlet<T, OP_APPLY><<<nb, 128, 0, s_dir>>>(L, a); break;
        case OP_RESID: k_dirichlet<T, OP_RESID><<<nb, 128, 0, s_dir>>>(L, a); break;
        case OP_JACOBI: k_dirichlet<T, OP_JACOBI><<<nb, 128, 0, s_dir>>>(L, a); break;
        case OP_CHEBY: k_dirichlet<T, OP_CHEBY><<<nb, 128, 0, s_dir>>>(L, a); break;
        case OP_DIAG: k_dirichlet<T, OP_DIAG><<<nb, 128, 0, s_dir>>>(L, a); break;
      }
    }
  }
  if (partial_count) *partial_count = used - partial_offset;
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Residual with norm that allocates nothing.  Its scratch (per-block partial
// sums of |r|^2 and the reduced result) lives in this file-scope device array,
// which every GPU that loads the library holds until the process exits.  Host
// code never uses the array's name as an address: the device address is looked
// up once per device with cudaGetSymbolAddress.  Face-interior skeleton nodes
// go through the warp-per-node kernel here, so no accumulator is needed.
// Calls that overlap on the GPU share the array and race.
// ---------------------------------------------------------------------------
__device__ __align__(256) static double g_noalloc_scratch[NOALLOC_SLOTS + 32];

namespace {
std::mutex g_noalloc_mutex;
double* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};
}  // namespace

int noalloc_scratch_address(int device, double** ptr) {
  if (device < 0 || device >= NOALLOC_MAX_DEVICES) return (int)cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return (int)e;
    g_noalloc_addr[device] = (double*)p;
  }
  *ptr = g_noalloc_addr[device];
  return 0;
}

int64_t noalloc_partials_needed(const LevelDev& L) {
  return (int64_t)L.nmacro * L.ntiles_lin + L.nface_nodes + L.nev;
}

template <typename T>
int launch_residual_noalloc(const LevelDev& L, const MacroStencil<T>* st_host, const MacroConsts<T>* mc_dev,
                            const OpFlags& fl, SweepArgs<T> a, double* scratch, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  int64_t used = 0;
  const bool gen = !(fl.physical == 1 && fl.khat_edge == 0);
  for (int m = 0; m < L.nmacro && L.ntiles_lin > 0; ++m) {
    SweepArgs<T> am = a;
    am.partial = scratch + used;
    (gen ? k_interior<T, OP_RESID, 1> : k_interior<T, OP_RESID, 0>)<<<L.ntiles_lin, INTERIOR_BLOCK, 0, s>>>(L, st_host[m], m, fl, am, 0);
    used += L.ntiles_lin;
  }
  if (L.nface_nodes > 0) {
    LevelDev Lf = L;  // face-interior nodes through the warp-per-node path
    Lf.ev_nodes = L.face_nodes;
    Lf.nev = L.nface_nodes;
    const int nb = L.nface_nodes;
    SweepArgs<T> am = a;
    am.partial = scratch + used;
    k_skeleton_ev<T, OP_RESID><<<nb, 128, 0, s>>>(Lf, mc_dev, fl, am);
    used += nb;
  }
  if (L.nev > 0) {
    const int nb = L.nev;
    SweepArgs<T> am = a;
    am.partial = scratch + used;
    k_skeleton_ev<T, OP_RESID><<<nb, 128, 0, s>>>(L, mc_dev, fl, am);
    used += nb;
  }
  if (L.ndir > 0) k_dirichlet<T, OP_RESID><<<(L.ndir + 127) / 128, 128, 0, s>>>(L, a);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return (int)e;
  return launch_reduce(scratch, used, scratch + NOALLOC_SLOTS, stream);
}

template int launch_residual_noalloc<float>(const LevelDev&, const MacroStencil<float>*, const MacroConsts<float>*,
                                            const OpFlags&, SweepArgs<float>, double*, void*);
template int launch_residual_noalloc<double>(const LevelDev&, const MacroStencil<double>*,
                                             const MacroConsts<double>*, const OpFlags&, SweepArgs<double>, double*,
                                             void*);

template <typename T>
int launch_stokes_sweep(const LevelDev& L, const MacroStencil<T>* st_host, const MacroConsts<T>* mc_dev, OpKind op,
                        const OpFlags& fl, const SweepArgs<T>& a, void* stream, int64_t* partial_count,
                        void* const* side) {
  if (op != OP_APPLY && op != OP_RESID) return (int)cudaErrorInvalidValue;
  cudaStream_t s = (cudaStream_t)stream;
  // side streams (nullable): [0] face chain, [1] every second macro, [2] edge/vertex nodes
  cudaStream_t s_face = side ? (cudaStream_t)side[0] : s;
  cudaStream_t s_odd = side ? (cudaStream_t)side[1] : s;
  cudaStream_t s_ev = side ? (cudaStream_t)side[2] : s;
  int64_t used = 0;
  const bool gen = !(fl.physical == 1 && fl.khat_edge == 0);
  if (fl.batch && L.ntiles_lin > 0) {
    for (int m0 = 0; m0 < L.nmacro; m0 += BATCH_MAX_MACROS) {
      const dim3 g(L.ntiles_lin, std::min(BATCH_MAX_MACROS, L.nmacro - m0));
      SweepArgs<T> am = a;
      if (a.partial) am.partial = a.partial + used;
      if (op == OP_APPLY)
        (gen ? k_interior_batched<T, OP_APPLY, 1, 1> : k_interior_batched<T, OP_APPLY, 0, 1>)<<<g, INTERIOR_BLOCK, 0,
                                                                                                s>>>(L, mc_dev, m0, fl,
                                                                                                     am);
      else
        (gen ? k_interior_batched<T, OP_RESID, 1, 1> : k_interior_batched<T, OP_RESID, 0, 1>)<<<g, INTERIOR_BLOCK, 0,
                                                                                                s>>>(L, mc_dev, m0, fl,
                                                                                                     am);
      used += (int64_t)g.x * g.y;
    }
  }
  for (int m = 0; m < L.nmacro && L.ntiles_lin > 0 && !fl.batch; ++m) {
    SweepArgs<T> am = a;
    if (a.partial) am.partial = a.partial + used;
    cudaStream_t sm = m % 2 ? s_odd : s;
    if (op == OP_APPLY)
      (gen ? k_interior<T, OP_APPLY, 1, 1> : k_interior<T, OP_APPLY, 0, 1>)<<<L.ntiles_lin, INTERIOR_BLOCK, 0, sm>>>(
          L, st_host[m], m, fl, am, 0);
    else
      (gen ? k_interior<T, OP_RESID, 1, 1> : k_interior<T, OP_RESID, 0, 1>)<<<L.ntiles_lin, INTERIOR_BLOCK, 0, sm>>>(
          L, st_host[m], m, fl, am, 0);
    used += L.ntiles_lin;
  }
  if (L.nface_items_all > 0)
    k_face_items_stk<T><<<(L.nface_items_all + 127) / 128, 128, 0, s_face>>>(L, mc_dev, fl, a.x, a.k);
  if (L.nface_nodes_all > 0) {
    const int nb = (L.nface_nodes_all + 127) / 128;
    SweepArgs<T> am = a;
    if (a.partial) am.partial = a.partial + used;
    if (op == OP_APPLY)
      k_face_finalize_stk<T, OP_APPLY><<<nb, 128, 0, s_face>>>(L, am);
    else
      k_face_finalize_stk<T, OP_RESID><<<nb, 128, 0, s_face>>>(L, am);
    used += nb;
  }
  if (L.nev_all > 0) {
    SweepArgs<T> am = a;
    if (a.partial) am.partial = a.partial + used;
    if (op == OP_APPLY)
      k_skeleton_ev_stk<T, OP_APPLY><<<L.nev_all, 128, 0, s_ev>>>(L, mc_dev, fl, am);
    else
      k_skeleton_ev_stk<T, OP_RESID><<<L.nev_all, 128, 0, s_ev>>>(L, mc_dev, fl, am);
    used += L.nev_all;
  }
  if (partial_count) *partial_count = used;
  return (int)cudaGetLastError();
}

template int launch_stokes_sweep<float>(const LevelDev&, const MacroStencil<float>*, const MacroConsts<float>*, OpKind,
                                        const OpFlags&, const SweepArgs<float>&, void*, int64_t*, void* const*);
template int launch_stokes_sweep<double>(const LevelDev&, const MacroStencil<double>*, const MacroConsts<double>*,
                                         OpKind, const OpFlags&, const SweepArgs<double>&, void*, int64_t*,
                                         void* const*);

// fills the direction / ring tables used with run-time indices
int upload_direction_tables() {
  int dir[NDIR][3], ring[NDIR][3][2], rn[NDIR];
  for (int d = 0; d < NDIR; ++d) {
    dir[d][0] = dir_di(d);
    dir[d][1] = dir_dj(d);
    dir[d][2] = dir_dk(d);
    rn[d] = ring_count(d);
    for (int c = 0; c < 3; ++c) {
      ring[d][c][0] = c < rn[d] ? ring_a(d, c) : 0;
      ring[d][c][1] = c < rn[d] ? ring_b(d, c) : 0;
    }
  }
  cudaError_t e = cudaMemcpyToSymbol(c_dir, dir, sizeof(dir));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_ring, ring, sizeof(ring));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_ring_n, rn, sizeof(rn));
  // the copies may still be landing on the legacy stream, which library streams do not wait for
  if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
  return (int)e;
}

template <typename T>
int launch_gs_colour(const LevelDev& L, const MacroStencil<T>* st_host, const MacroConsts<T>* mc_dev, const OpFlags& fl,
                     const SweepArgs<T>& a, int colour, void* stream) {
  const int count = L.gs_ptr[colour + 1] - L.gs_ptr[colour];
  if (count == 0) return 0;
  const int per = INTERIOR_BLOCK / 32;
  const bool gen = !(fl.physical == 1 && fl.khat_edge == 0);
  // all macros of the level in one launch per colour (grid.y: macros), or one launch per macro
  // when only the stencil-parameter kernel applies (mc_dev null)
  if (mc_dev) {
    for (int m0 = 0; m0 < L.nmacro; m0 += BATCH_MAX_MACROS) {
      const dim3 g((count + per - 1) / per, std::min(BATCH_MAX_MACROS, L.nmacro - m0));
      if (gen)
        k_gs_colour_batched<T, 1><<<g, INTERIOR_BLOCK, 0, (cudaStream_t)stream>>>(L, mc_dev, m0, fl, a, colour);
      else
        k_gs_colour_batched<T, 0><<<g, INTERIOR_BLOCK, 0, (cudaStream_t)stream>>>(L, mc_dev, m0, fl, a, colour);
    }
    return (int)cudaGetLastError();
  }
  const dim3 g((count + per - 1) / per);
  for (int m = 0; m < L.nmacro; ++m) {
    if (gen)
      k_interior<T, OP_JACOBI, 1, 0, 0, 1><<<g, INTERIOR_BLOCK, 0, (cudaStream_t)stream>>>(L, st_host[m], m, fl, a,
                                                                                            colour);
    else
      k_interior<T, OP_JACOBI, 0, 0, 0, 1><<<g, INTERIOR_BLOCK, 0, (cudaStream_t)stream>>>(L, st_host[m], m, fl, a,
                                                                                            colour);
  }
  return (int)cudaGetLastError();
}
template int launch_gs_colour<float>(const LevelDev&, const MacroStencil<float>*, const MacroConsts<float>*,
                                     const OpFlags&, const SweepArgs<float>&, int, void*);
template int launch_gs_colour<double>(const LevelDev&, const MacroStencil<double>*, const MacroConsts<double>*,
                                      const OpFlags&, const SweepArgs<double>&, int, void*);

template <typename T>
int launch_store_stencil(const LevelDev& L, const MacroStencil<double>* st_host, const OpFlags& fl, const double* k64,
                         T* out, void* stream) {
  if (L.ntiles_lin == 0) return 0;
  for (int m = 0; m < L.nmacro; ++m)
    k_store_stencil<T><<<L.ntiles_lin, INTERIOR_BLOCK, 0, (cudaStream_t)stream>>>(L, st_host[m], m, fl, k64, out);
  return (int)cudaGetLastError();
}
template int launch_store_stencil<float>(const LevelDev&, const MacroStencil<double>*, const OpFlags&, const double*,
                                         float*, void*);
template int launch_store_stencil<double>(const LevelDev&, const MacroStencil<double>*, const OpFlags&, const double*,
                                          double*, void*);

template int launch_sweep_macro<float>(const LevelDev&, const MacroStencil<float>*, const NodalConsts<float>*, int,
                                       OpKind, const OpFlags&, const SweepArgs<float>&, void*, int64_t, int64_t*);
template int launch_sweep_macro<double>(const LevelDev&, const MacroStencil<double>*, const NodalConsts<double>*,
                                        int, OpKind, const OpFlags&, const SweepArgs<double>&, void*, int64_t,
                                        int64_t*);
template int launch_sweep<float>(const LevelDev&, const MacroStencil<float>*, const MacroConsts<float>*, OpKind,
                                 const OpFlags&, const SweepArgs<float>&, void*, int, int64_t, int64_t*, void*, void*);
template int launch_sweep<double>(const LevelDev&, const MacroStencil<double>*, const MacroConsts<double>*, OpKind,
                                  const OpFlags&, const SweepArgs<double>&, void*, int, int64_t, int64_t*, void*, void*);

}  // namespace hhg
