// Reductions, multigrid transfers and vector kernels on the HHG lattice layout.
//
// Transfers (Sec. 5: matrix-free linear interpolation and its transpose):
// a fine lattice point q either coincides with the coarse point q/2 or is the
// midpoint of the coarse edge (q - d, q + d)/2, where d is the stencil
// direction whose Kuhn coordinates are the parities (X mod 2, Y mod 2, Z mod 2)
// of q.  Prolongation takes 1 resp. 1/2 of the parents; restriction is the
// exact transpose: coarse point p collects r(2p) + 1/2 sum_d r(2p + d).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "hhg_internal.h"
#include "hhg_launch.h"

namespace hhg {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void block_store(double v, double* out) {
  __shared__ double red[32];
  v = warp_sum(v);
  const int tid = threadIdx.x;
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    double s = tid < (int)((blockDim.x + 31) / 32) ? red[tid] : 0.0;
    s = warp_sum(s);
    if (tid == 0) *out = s;
  }
}

__global__ void k_reduce(const double* __restrict__ p, int64_t count, double* out) {
  double v = 0.0;
  for (int64_t q = threadIdx.x; q < count; q += blockDim.x) v += p[q];
  block_store(v, out);
}

template <typename T>
__global__ void k_dot(const uint8_t* __restrict__ mask, int64_t E, int comps, const T* __restrict__ a,
                      const T* __restrict__ b, double* partials) {
  double v = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    if (mask[e]) {
      for (int c = 0; c < comps; ++c) v += (double)a[e + c * E] * (double)b[e + c * E];
    }
  }
  block_store(v, partials + blockIdx.x);
}

// fine point (i, j, k) of macro `m` of the fine level; adds P e_c
template <typename T>
__global__ void k_prolong_add(const LevelDev Lf, const LevelDev Lc, const T* __restrict__ ec, T* __restrict__ ef,
                              int comps) {
  const int m = blockIdx.y;
  const int32_t tile = Lf.tiles_all[blockIdx.x];
  const int k = tile >> 20;
  const int j = ((tile >> 10) & 1023) + threadIdx.y;
  const int i = (tile & 1023) + threadIdx.x;
  const int n = Lf.n, nc = Lc.n;
  if (i + j + k > n) return;
  const int X = i + j + k, Y = j + k, Z = k;
  const int pX = X & 1, pY = Y & 1, pZ = Z & 1;
  const int64_t ef0 = (int64_t)m * Lf.nt + lattice_index(n, i, j, k);
  const int64_t cb = (int64_t)m * Lc.nt;
  if (!(pX | pY | pZ)) {
    const int64_t c = cb + lattice_index(nc, i >> 1, j >> 1, k >> 1);
    for (int q = 0; q < comps; ++q) ef[ef0 + q * Lf.entries] += ec[c + q * Lc.entries];
  } else {
    const int di = pX - pY, dj = pY - pZ, dk = pZ;
    const int64_t ca = cb + lattice_index(nc, (i - di) >> 1, (j - dj) >> 1, (k - dk) >> 1);
    const int64_t cc = cb + lattice_index(nc, (i + di) >> 1, (j + dj) >> 1, (k + dk) >> 1);
    for (int q = 0; q < comps; ++q)
      ef[ef0 + q * Lf.entries] += (T)0.5 * (ec[ca + q * Lc.entries] + ec[cc + q * Lc.entries]);
  }
}

// coarse macro-interior points: rc(p) = rf(2p) + 1/2 sum_d rf(2p + d)
template <typename T>
__global__ void k_restrict_interior(const LevelDev Lf, const LevelDev Lc, const T* __restrict__ rf,
                                    T* __restrict__ rc, int comps) {
  const int m = blockIdx.y;
  const int32_t tile = Lc.tiles_int[blockIdx.x];
  const int k = tile >> 20;
  const int j = ((tile >> 10) & 1023) + threadIdx.y;
  const int i = (tile & 1023) + threadIdx.x;
  const int n = Lf.n, nc = Lc.n;
  if (i + j + k > nc - 1) return;
  const int64_t fb = (int64_t)m * Lf.nt;
  const int64_t c = (int64_t)m * Lc.nt + lattice_index(nc, i, j, k);
  const int64_t f0 = fb + lattice_index(n, 2 * i, 2 * j, 2 * k);
  for (int q = 0; q < comps; ++q) {
    const T* r = rf + q * Lf.entries;
    T s = 0;
#pragma unroll
    for (int d = 0; d < NDIR; ++d) s += r[fb + lattice_index(n, 2 * i + dir_di(d), 2 * j + dir_dj(d), 2 * k + dir_dk(d))];
    rc[c + q * Lc.entries] = r[f0] + (T)0.5 * s;
  }
}

// coarse skeleton points: precomputed list of unique fine points and weights
template <typename T>
__global__ void k_restrict_skeleton(const LevelDev Lc, const int32_t* __restrict__ rptr,
                                    const int64_t* __restrict__ rent, const T* __restrict__ rw, int64_t Ef,
                                    const T* __restrict__ rf, T* __restrict__ rc, int comps, int use_dir) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Lc.nskel) return;
  T acc[3] = {0, 0, 0};
  if (!(use_dir && Lc.skel_dir[s])) {
    for (int q = rptr[s]; q < rptr[s + 1]; ++q) {
      const int64_t e = rent[q];
      const T w = rw[q];
      for (int c = 0; c < comps; ++c) acc[c] += w * rf[e + c * Ef];
    }
  }
  for (int q = Lc.skel_ptr[s]; q < Lc.skel_ptr[s + 1]; ++q) {
    const SkelInc I = Lc.skel_inc[q];
    const int64_t e = (int64_t)I.macro * Lc.nt + lattice_index(Lc.n, I.i, I.j, I.k);
    for (int c = 0; c < comps; ++c) rc[e + c * Lc.entries] = acc[c];
  }
}

__global__ void k_bf16_to_f64(int64_t n, const uint16_t* __restrict__ src, double* __restrict__ dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (double)__uint_as_float((uint32_t)src[e] << 16);
}

__global__ void k_round_bf16(int64_t n, double* __restrict__ k64, float* __restrict__ k32, uint16_t* __restrict__ k16) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const __nv_bfloat16 b = __double2bfloat16(k64[e]);
    const float f = __bfloat162float(b);
    k16[e] = __bfloat16_as_ushort(b);
    k32[e] = f;
    k64[e] = (double)f;
  }
}

// coarse macro-interior nodes: local weighted mean of the fine coefficient (or of its inverse)
__global__ void k_average_coeff(const LevelDev Lf, const LevelDev Lc, const double* __restrict__ kf,
                                double* __restrict__ kc, int harmonic) {
  const int m = blockIdx.y;
  const int32_t tile = Lc.tiles_int[blockIdx.x];
  const int k = tile >> 20;
  const int j = ((tile >> 10) & 1023) + threadIdx.y;
  const int i = (tile & 1023) + threadIdx.x;
  const int n = Lf.n, nc = Lc.n;
  if (i + j + k > nc - 1) return;
  const int64_t fb = (int64_t)m * Lf.nt;
  auto val = [&](int64_t e) { return harmonic ? 1.0 / kf[e] : kf[e]; };
  double s = val(fb + lattice_index(n, 2 * i, 2 * j, 2 * k));
#pragma unroll
  for (int d = 0; d < NDIR; ++d)
    s += 0.5 * val(fb + lattice_index(n, 2 * i + dir_di(d), 2 * j + dir_dj(d), 2 * k + dir_dk(d)));
  s /= 1.0 + 0.5 * NDIR;
  kc[(int64_t)m * Lc.nt + lattice_index(nc, i, j, k)] = harmonic ? 1.0 / s : s;
}

// coefficient injection: coarse points are fine points
template <typename T>
__global__ void k_inject(const LevelDev Lf, const LevelDev Lc, const T* __restrict__ kf, T* __restrict__ kc) {
  const int m = blockIdx.y;
  const int32_t tile = Lc.tiles_all[blockIdx.x];
  const int k = tile >> 20;
  const int j = ((tile >> 10) & 1023) + threadIdx.y;
  const int i = (tile & 1023) + threadIdx.x;
  if (i + j + k > Lc.n) return;
  kc[(int64_t)m * Lc.nt + lattice_index(Lc.n, i, j, k)] =
      kf[(int64_t)m * Lf.nt + lattice_index(Lf.n, 2 * i, 2 * j, 2 * k)];
}

template <typename T>
__global__ void k_schur_diag(int64_t n, const T* __restrict__ r, const T* __restrict__ mu, const T* __restrict__ m,
                             const T* __restrict__ sd, T* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = r[e] / (m[e] / mu[e] + sd[e]);
}

template <typename T>
__global__ void k_axpby(int64_t n, T a, const T* __restrict__ x, T b, T* __restrict__ y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = a * x[e] + b * y[e];
}

template <typename T, typename U>
__global__ void k_convert(int64_t n, const T* __restrict__ s, U* __restrict__ d) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    d[e] = (U)s[e];
}

template <typename T>
__global__ void k_gather(int64_t count, int comps, int64_t ss, int64_t ds, const int64_t* __restrict__ idx,
                         const T* __restrict__ src, T* __restrict__ dst) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < count; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = idx[u];
    for (int c = 0; c < comps; ++c) dst[c * ds + u] = src[c * ss + e];
  }
}

template <typename T>
__global__ void k_fill(int64_t n, T v, T* __restrict__ d) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    d[e] = v;
}

template <typename T>
__global__ void k_mul(int64_t n, const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = a[e] * b[e];
}

template <typename T>
__global__ void k_recip(int64_t n, const T* __restrict__ a, T* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (T)1 / a[e];
}

__global__ void k_add_f32_to_f64(int64_t n, const float* __restrict__ e32, double* __restrict__ x) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    x[e] += (double)e32[e];
}

// splitmix64 of (node, component): a deterministic start vector that depends on the
// unique node only, so every copy of a skeleton node gets the same value
template <typename T>
__global__ void k_hash_unique(int64_t U, int comps, const int8_t* __restrict__ udir, T* __restrict__ u) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < U; q += (int64_t)gridDim.x * blockDim.x) {
    for (int c = 0; c < comps; ++c) {
      uint64_t z = (uint64_t)(q * comps + c) + 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z = z ^ (z >> 31);
      const double v = (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
      u[c * U + q] = udir[q] ? (T)0 : (T)v;
    }
  }
}

template <typename T>
__global__ void k_dense_matvec(int N, const T* __restrict__ A, const int64_t* __restrict__ idx,
                               const T* __restrict__ src, T* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  T acc = 0;
  for (int j = 0; j < N; ++j) acc += A[(int64_t)i * N + j] * src[idx[j]];
  dst[idx[i]] = acc;
}

template <typename T>
__global__ void k_mul3(int64_t n, const T* __restrict__ a, const T* __restrict__ b, const T* __restrict__ c,
                       T* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = a[e] * b[e] * c[e];
}

template <typename T>
__global__ void k_add_const(int64_t n, T v, T* __restrict__ d) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    d[e] += v;
}

__device__ __forceinline__ double carreau_mu(const CarreauParams& cp, const double g[3][3]) {
  // |eps(u)|^2 = eps : eps with eps = (grad u + grad u^T) / 2
  double e2 = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double e = 0.5 * (g[c][j] + g[j][c]);
      e2 += e * e;
    }
  return cp.eta_inf + (cp.eta0 - cp.eta_inf) * pow(1.0 + cp.kappa * e2, cp.r);
}

// macro-interior nodes: the patch is point-symmetric, so the affine least-squares slope is
// G^{-1} sum_d dx_d (u(i+d) - u(i)) with G = sum_d dx_d dx_d^T (precomputed as Q)
__global__ void k_carreau_interior(const LevelDev L, const SlopeOp q, int macro, CarreauParams cp,
                                   const double* __restrict__ u, double* __restrict__ mu) {
  const int32_t tile = L.tiles_lin[blockIdx.x];
  const int n = L.n;
  const int k = tile >> 20;
  const int M = n - 1 - k;
  const int t = (tile & 0xFFFFF) + threadIdx.x;
  if (t >= (M - 1) * M / 2) return;
  // (j, i) of the t-th interior point of the slice
  const float b = (float)(2 * M - 1);
  int uu = (int)floorf(0.5f * (b - sqrtf(fmaxf(b * b - 8.0f * (float)t, 0.0f))));
  uu = max(0, min(uu, M - 2));
  if (((uu + 1) * (2 * M - uu - 2)) / 2 <= t) ++uu;
  if ((uu * (2 * M - uu - 1)) / 2 > t) --uu;
  const int j = uu + 1;
  const int i = t - (uu * (2 * M - uu - 1)) / 2 + 1;
  const int64_t E = L.entries;
  const int64_t base = (int64_t)macro * L.nt;
  const int64_t c0 = base + lattice_index(n, i, j, k);
  double g[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
  for (int d = 0; d < NDIR; ++d) {
    const int64_t e = base + lattice_index(n, i + dir_di(d), j + dir_dj(d), k + dir_dk(d));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double du = u[e + c * E] - u[c0 + c * E];
#pragma unroll
      for (int a = 0; a < 3; ++a) g[c][a] = fma(q.Q[d][a], du, g[c][a]);
    }
  }
  mu[c0] = carreau_mu(cp, g);
}

// Quadratic least squares (eq. minimization_problem, m = 2) over the patch of skeleton node t,
// in the coordinates y = dx / rho (rho = the patch's largest |dx| component): Cholesky of the
// 10 x 10 normal equations in the monomials 1, y_a, y_a y_b (a <= b).  Returns false, leaving
// g untouched, when the patch does not determine the quadratic (fewer than 10 points or a
// pivot at most QUAD_PIVOT_TOL times the largest diagonal entry: one-sided patches, on which
// y_a and y_a^2 agree); else g[c][a] = d u_c / d x_a of the fit at the node.
constexpr double QUAD_PIVOT_TOL = 1e-10;
__device__ bool quadratic_gradient(const PatchLists& P, int t, int64_t E, const double* __restrict__ u,
                                   double g[3][3]) {
  const int q0 = P.ptr[t], q1 = P.ptr[t + 1];
  if (q1 - q0 < 10) return false;
  double rho = 0.0;
  for (int q = q0; q < q1; ++q)
    for (int a = 0; a < 3; ++a) rho = fmax(rho, fabs(P.dx[3 * q + a]));
  if (!(rho > 0.0)) return false;
  const double ir = 1.0 / rho;
  double N[10][10], R[10][3];
  for (int a = 0; a < 10; ++a) {
    for (int b = 0; b < 10; ++b) N[a][b] = 0.0;
    for (int c = 0; c < 3; ++c) R[a][c] = 0.0;
  }
  for (int q = q0; q < q1; ++q) {
    const double y0 = P.dx[3 * q] * ir, y1 = P.dx[3 * q + 1] * ir, y2 = P.dx[3 * q + 2] * ir;
    const double w[10] = {1.0, y0, y1, y2, y0 * y0, y0 * y1, y0 * y2, y1 * y1, y1 * y2, y2 * y2};
    const int64_t e = P.ent[q];
    const double uv[3] = {u[e], u[e + E], u[e + 2 * E]};
    for (int a = 0; a < 10; ++a) {
      for (int b = 0; b <= a; ++b) N[a][b] += w[a] * w[b];
      for (int c = 0; c < 3; ++c) R[a][c] += w[a] * uv[c];
    }
  }
  double dmax = 0.0;
  for (int a = 0; a < 10; ++a) dmax = fmax(dmax, N[a][a]);
  // Cholesky N = L L^T in place (lower triangle)
  for (int k = 0; k < 10; ++k) {
    double s = N[k][k];
    for (int j = 0; j < k; ++j) s -= N[k][j] * N[k][j];
    if (!(s > QUAD_PIVOT_TOL * dmax)) return false;
    const double l = sqrt(s);
    N[k][k] = l;
    for (int r = k + 1; r < 10; ++r) {
      double v = N[r][k];
      for (int j = 0; j < k; ++j) v -= N[r][j] * N[k][j];
      N[r][k] = v / l;
    }
  }
  // forward (L z = R) and backward (L^T c = z) substitution, three right-hand sides
  for (int k = 0; k < 10; ++k)
    for (int c = 0; c < 3; ++c) {
      double v = R[k][c];
      for (int j = 0; j < k; ++j) v -= N[k][j] * R[j][c];
      R[k][c] = v / N[k][k];
    }
  for (int k = 9; k >= 0; --k)
    for (int c = 0; c < 3; ++c) {
      double v = R[k][c];
      for (int j = k + 1; j < 10; ++j) v -= N[j][k] * R[j][c];
      R[k][c] = v / N[k][k];
    }
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) g[c][a] = R[a + 1][c] * ir;
  return true;
}

// skeleton nodes: general affine least squares min sum (c + b.dx - u)^2 over the patch
// (normal equations, 4x4, Gaussian elimination with partial pivoting), or with QUAD the
// quadratic fit where the patch determines it (affine elsewhere); every copy written
template <int QUAD>
__global__ void k_carreau_skeleton(const LevelDev L, const PatchLists P, CarreauParams cp,
                                   const double* __restrict__ u, double* __restrict__ mu) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P.nnodes) return;
  const int64_t E = L.entries;
  double g[3][3];
  if (QUAD && quadratic_gradient(P, t, E, u, g)) {
    const double m = carreau_mu(cp, g);
    const int s = P.node[t];
    for (int q = L.skel_ptr[s]; q < L.skel_ptr[s + 1]; ++q) {
      const SkelInc I = L.skel_inc[q];
      mu[(int64_t)I.macro * L.nt + lattice_index(L.n, I.i, I.j, I.k)] = m;
    }
    return;
  }
  double A[4][4] = {{0}}, R[4][3] = {{0}};
  for (int q = P.ptr[t]; q < P.ptr[t + 1]; ++q) {
    const double w[4] = {1.0, P.dx[3 * q], P.dx[3 * q + 1], P.dx[3 * q + 2]};
    const int64_t e = P.ent[q];
    const double uv[3] = {u[e], u[e + E], u[e + 2 * E]};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
      for (int b = 0; b < 4; ++b) A[a][b] += w[a] * w[b];
#pragma unroll
      for (int c = 0; c < 3; ++c) R[a][c] += w[a] * uv[c];
    }
  }
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int r = col + 1; r < 4; ++r)
      if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
    if (piv != col) {
      for (int q = 0; q < 4; ++q) {
        const double tmp = A[piv][q];
        A[piv][q] = A[col][q];
        A[col][q] = tmp;
      }
      for (int c = 0; c < 3; ++c) {
        const double tmp = R[piv][c];
        R[piv][c] = R[col][c];
        R[col][c] = tmp;
      }
    }
    const double inv = 1.0 / A[col][col];
    for (int r = 0; r < 4; ++r) {
      if (r == col) continue;
      const double f = A[r][col] * inv;
      for (int q = col; q < 4; ++q) A[r][q] -= f * A[col][q];
      for (int c = 0; c < 3; ++c) R[r][c] -= f * R[col][c];
    }
  }
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) g[c][a] = R[a + 1][c] / A[a + 1][a + 1];
  const double m = carreau_mu(cp, g);
  const int s = P.node[t];
  for (int q = L.skel_ptr[s]; q < L.skel_ptr[s + 1]; ++q) {
    const SkelInc I = L.skel_inc[q];
    mu[(int64_t)I.macro * L.nt + lattice_index(L.n, I.i, I.j, I.k)] = m;
  }
}

// ---------------------------------------------------------------------------
// Boundary traction load (the Neumann term of the weak form, Sec. 5.1.3): on each flagged
// macro face (slot s) the refined face is a triangular lattice of (n+1)(n+2)/2 points
// (a, b), a + b <= n, point index b (n + 1) - b (b - 1) / 2 + a, split into n^2 congruent
// triangles of area A_s: "up" (a, b), (a+1, b), (a, b+1) and "down" (a+1, b), (a, b+1),
// (a+1, b+1).  With the P1 interpolant of the nodal traction t, each triangle adds
// (A / 12) (2 t_p + t_q + t_r) to the load of its point p (exact P1 face mass matrix).
// k_traction_face: one thread per face point, the sum over its (up to six) triangles of
// its face, into contrib[3 (s npf + p) + c]; k_traction_gather: one thread per boundary
// node, the sum of its contributions (fixed order) added to every copy of the node.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int face_point(int n, int a, int b) { return b * (n + 1) - b * (b - 1) / 2 + a; }

template <typename T>
__global__ void k_traction_face(int n, int nslots, const double* __restrict__ area, const int64_t* __restrict__ pent,
                                int64_t E, const T* __restrict__ t, double* __restrict__ contrib) {
  const int npf = (n + 1) * (n + 2) / 2;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= (int64_t)nslots * npf) return;
  const int s = (int)(g / npf);
  const int p = (int)(g % npf);
  int b = 0;
  while (face_point(n, 0, b + 1) <= p && b < n) ++b;
  const int a = p - face_point(n, 0, b);
  const int64_t* pe = pent + (int64_t)s * npf;
  double acc[3] = {0.0, 0.0, 0.0};
  auto add = [&](int a1, int b1, int a2, int b2) {  // triangle (a, b), (a1, b1), (a2, b2)
    const int64_t e0 = pe[p], e1 = pe[face_point(n, a1, b1)], e2 = pe[face_point(n, a2, b2)];
    for (int c = 0; c < 3; ++c)
      acc[c] += 2.0 * (double)t[e0 + c * E] + (double)t[e1 + c * E] + (double)t[e2 + c * E];
  };
  // up triangles with (a, b) as their first, second or third vertex
  if (a + b + 1 <= n) add(a + 1, b, a, b + 1);
  if (a >= 1) add(a - 1, b, a - 1, b + 1);
  if (b >= 1) add(a, b - 1, a + 1, b - 1);
  // down triangles with (a, b) as their first, second or third vertex
  if (a >= 1 && b >= 1) add(a - 1, b, a, b - 1);          // down(a-1, b-1): (a, b-1), (a-1, b), (a, b)
  if (a >= 1 && a + b + 1 <= n) add(a - 1, b + 1, a, b + 1);  // down(a-1, b): (a, b), (a-1, b+1), (a, b+1)
  if (b >= 1 && a + b + 1 <= n) add(a + 1, b - 1, a + 1, b);  // down(a, b-1): (a+1, b-1), (a, b), (a+1, b)
  const double w = area[s] / 12.0;
  for (int c = 0; c < 3; ++c) contrib[3 * g + c] = w * acc[c];
}

template <typename T>
__global__ void k_traction_gather(int64_t nnodes, const int64_t* __restrict__ cptr, const int64_t* __restrict__ cidx,
                                  const int64_t* __restrict__ eptr, const int64_t* __restrict__ eidx, int64_t E,
                                  const double* __restrict__ contrib, T* __restrict__ f) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= nnodes) return;
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t q = cptr[u]; q < cptr[u + 1]; ++q)
    for (int c = 0; c < 3; ++c) v[c] += contrib[3 * cidx[q] + c];
  for (int64_t q = eptr[u]; q < eptr[u + 1]; ++q)
    for (int c = 0; c < 3; ++c) f[eidx[q] + c * E] += (T)v[c];
}

// max over masked entries of the 2-norm of (a - b) over `comps` components (b nullable)
__global__ void k_node_maxnorm(const uint8_t* __restrict__ mask, int64_t E, int comps, const double* __restrict__ a,
                               const double* __restrict__ b, double* partials) {
  double v = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    if (!mask[e]) continue;
    double s = 0.0;
    for (int c = 0; c < comps; ++c) {
      const double d = a[e + c * E] - (b ? b[e + c * E] : 0.0);
      s += d * d;
    }
    v = fmax(v, sqrt(s));
  }
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double m = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) partials[blockIdx.x] = m;
  }
}

__global__ void k_reduce_max(const double* __restrict__ p, int64_t count, double* out) {
  double v = 0.0;
  for (int64_t q = threadIdx.x; q < count; q += blockDim.x) v = fmax(v, p[q]);
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double m = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) *out = m;
  }
}

inline int grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

template <typename T>
int launch_traction_load(int n, int nslots, const double* area, const int64_t* pent, int64_t E, const T* t,
                         double* contrib, int64_t nnodes, const int64_t* cptr, const int64_t* cidx,
                         const int64_t* eptr, const int64_t* eidx, T* f, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t pts = (int64_t)nslots * (n + 1) * (n + 2) / 2;
  if (pts > 0) k_traction_face<T><<<(unsigned)((pts + 127) / 128), 128, 0, s>>>(n, nslots, area, pent, E, t, contrib);
  if (nnodes > 0)
    k_traction_gather<T><<<(unsigned)((nnodes + 127) / 128), 128, 0, s>>>(nnodes, cptr, cidx, eptr, eidx, E, contrib,
                                                                          f);
  return (int)cudaGetLastError();
}
template int launch_traction_load<float>(int, int, const double*, const int64_t*, int64_t, const float*, double*,
                                         int64_t, const int64_t*, const int64_t*, const int64_t*, const int64_t*,
                                         float*, void*);
template int launch_traction_load<double>(int, int, const double*, const int64_t*, int64_t, const double*, double*,
                                          int64_t, const int64_t*, const int64_t*, const int64_t*, const int64_t*,
                                          double*, void*);


int launch_reduce(const double* partials, int64_t count, double* out, void* stream) {
  k_reduce<<<1, 1024, 0, (cudaStream_t)stream>>>(partials, count, out);
  return (int)cudaGetLastError();
}

constexpr int DOT_BLOCKS = 1024;

template <typename T>
int launch_dot(const LevelDev& L, int comps, const T* a, const T* b, double* partials, int64_t* partial_count,
               void* stream) {
  k_dot<T><<<DOT_BLOCKS, 256, 0, (cudaStream_t)stream>>>(L.mask, L.entries, comps, a, b, partials);
  *partial_count = DOT_BLOCKS;
  return (int)cudaGetLastError();
}

template <typename T>
int launch_dot_masked(const uint8_t* mask, int64_t E, int comps, const T* a, const T* b, double* partials,
                      int64_t* partial_count, void* stream) {
  k_dot<T><<<DOT_BLOCKS, 256, 0, (cudaStream_t)stream>>>(mask, E, comps, a, b, partials);
  *partial_count = DOT_BLOCKS;
  return (int)cudaGetLastError();
}

int launch_node_maxnorm(const uint8_t* mask, int64_t E, int comps, const double* a, const double* b,
                        double* partials, double* out, void* stream) {
  k_node_maxnorm<<<DOT_BLOCKS, 256, 0, (cudaStream_t)stream>>>(mask, E, comps, a, b, partials);
  k_reduce_max<<<1, 1024, 0, (cudaStream_t)stream>>>(partials, DOT_BLOCKS, out);
  return (int)cudaGetLastError();
}

int launch_carreau(const LevelDev& L, const SlopeOp* q_host, const PatchLists& P, const CarreauParams& cp,
                   const double* u, double* mu, void* stream, int degree) {
  cudaStream_t s = (cudaStream_t)stream;
  for (int m = 0; m < L.nmacro && L.ntiles_lin > 0; ++m)
    k_carreau_interior<<<L.ntiles_lin, INTERIOR_BLOCK, 0, s>>>(L, q_host[m], m, cp, u, mu);
  if (P.nnodes > 0) {
    if (degree == 2)
      k_carreau_skeleton<1><<<(P.nnodes + 127) / 128, 128, 0, s>>>(L, P, cp, u, mu);
    else
      k_carreau_skeleton<0><<<(P.nnodes + 127) / 128, 128, 0, s>>>(L, P, cp, u, mu);
  }
  return (int)cudaGetLastError();
}

template <typename T>
int launch_mul3(int64_t n, const T* a, const T* b, const T* c, T* out, void* stream) {
  k_mul3<T><<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(n, a, b, c, out);
  return (int)cudaGetLastError();
}

template <typename T>
int launch_add_const(int64_t n, T v, T* dst, void* stream) {
  k_add_const<T><<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(n, v, dst);
  return (int)cudaGetLastError();
}

template <typename T>
int launch_prolong_add(const LevelDev& Lf, const LevelDev& Lc, const T* ec, T* ef, void* stream, int comps) {
  dim3 grid(Lf.ntiles_all, Lf.nmacro);
  k_prolong_add<T><<<grid, dim3(TILE_I, TILE_J), 0, (cudaStream_t)stream>>>(Lf, Lc, ec, ef, comps);
  return (int)cudaGetLastError();
}

template <typename T>
int launch_restrict(const LevelDev& Lf, const LevelDev& Lc, const int32_t* rptr, const int64_t* rent, const T* rw,
                    const T* rf, T* rc, void* stream, int comps, int use_dir) {
  cudaStream_t s = (cudaStream_t)stream;
  if (Lc.ntiles_int > 0) {
    dim3 grid(Lc.ntiles_int, Lc.nmacro);
    k_restrict_interior<T><<<grid, dim3(TILE_I, TILE_J), 0, s>>>(Lf, Lc, rf, rc, comps);
  }
  if (Lc.nskel > 0)
    k_restrict_skeleton<T><<<(Lc.nskel + 127) / 128, 128, 0, s>>>(Lc, rptr, rent, rw, Lf.entries, rf, rc, comps,
                                                                  use_dir);
  return (int)cudaGetLastError();
}

template <typename T>
int launch_schur_diag(int64_t n, const T* r, const T* mu, const T* m, const T* sd, T* out, void* stream) {
  k_schur_diag<T><<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, (cudaStream_t)stream>>>(n, r, mu, m,
                                                                                                        sd, out);
  return (int)cudaGetLastError();
}
template int launch_schur_diag<float>(int64_t, const float*, const float*, const float*, const float*, float*, void*);
template int launch_schur_diag<double>(int64_t, const double*, const double*, const double*, const double*, double*,
                                       void*);

int launch_bf16_to_f64(int64_t n, const uint16_t* src, double* dst, void* stream) {
  k_bf16_to_f64<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, (cudaStream_t)stream>>>(n, src, dst);
  return (int)cudaGetLastError();
}

int launch_round_bf16(int64_t n, double* k64, float* k32, uint16_t* k16, void* stream) {
  k_round_bf16<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, (cudaStream_t)stream>>>(n, k64, k32,
                                                                                                     k16);
  return (int)cudaGetLastError();
}

int launch_average_coeff(const LevelDev& Lf, const LevelDev& Lc, const double* kf, double* kc, int harmonic,
                         void* stream) {
  if (Lc.ntiles_int == 0) return 0;
  dim3 grid(Lc.ntiles_int, Lc.nmacro);
  k_average_coeff<<<grid, dim3(TILE_I, TILE_J), 0, (cudaStream_t)stream>>>(Lf, Lc, kf, kc, harmonic);
  return (int)cudaGetLastError();
}

template <typename T>
int launch_inject(const LevelDev& Lf, const LevelDev& Lc, const T* kf, T* kc, void* stream) {
  dim3 grid(Lc.ntiles_all, Lc.nmacro);
  k_inject<T><<<grid, dim3(TILE_I, TILE_J), 0, (cudaStream_t)stream>>>(Lf, Lc, kf, kc);
  return (int)cudaGetLastError();
}

template <typename T>
int launch_axpby(int64_t n, T a, const T* x, T b, T* y, void* stream) {
  k_axpby<T><<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(n, a, x, b, y);
  return (int)cudaGetLastError();
}

template <typename T, typename U>
int launch_convert(int64_t n, const T* src, U* dst, void* stream) {
  k_convert<T, U><<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(n, src, dst);
  return (int)cudaGetLastError();
}

template <typename T>
int launch_gather(int64_t count, int comps, int64_t ss, int64_t ds, const int64_t* idx, const T* src, T* dst,
                  void* stream) {
  k_gather<T><<<grid_for(count, 256), 256, 0, (cudaStream_t)stream>>>(count, comps, ss, ds, idx, src, dst);
  return (int)cudaGetLastError();
}

template <typename T>
int launch_fill(int64_t n, T v, T* dst, void* stream) {
  k_fill<T><<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(n, v, dst);
  return (int)cudaGetLastError();
}

template <typename T>
int launch_mul(int64_t n, const T* a, const T* b, T* out, void* stream) {
  k_mul<T><<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(n, a, b, out);
  return (int)cudaGetLastError();
}

template <typename T>
int launch_recip(int64_t n, const T* a, T* out, void* stream) {
  k_recip<T><<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(n, a, out);
  return (int)cudaGetLastError();
}

int launch_add_f32_to_f64(int64_t n, const float* e, double* x, void* stream) {
  k_add_f32_to_f64<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(n, e, x);
  return (int)cudaGetLastError();
}

template <typename T>
int launch_hash_unique(int64_t U, int comps, const int8_t* udir, T* u, void* stream) {
  k_hash_unique<T><<<grid_for(U, 256), 256, 0, (cudaStream_t)stream>>>(U, comps, udir, u);
  return (int)cudaGetLastError();
}

template <typename T>
int launch_dense_matvec(int N, const T* A, const int64_t* idx, const T* src_u, T* dst_u, void* stream) {
  k_dense_matvec<T><<<(N + 127) / 128, 128, 0, (cudaStream_t)stream>>>(N, A, idx, src_u, dst_u);
  return (int)cudaGetLastError();
}

#define HHG_INST(T)                                                                                              \
  template int launch_dot<T>(const LevelDev&, int, const T*, const T*, double*, int64_t*, void*);               \
  template int launch_prolong_add<T>(const LevelDev&, const LevelDev&, const T*, T*, void*, int);                     \
  template int launch_restrict<T>(const LevelDev&, const LevelDev&, const int32_t*, const int64_t*, const T*,   \
                                  const T*, T*, void*, int, int);                                                \
  template int launch_inject<T>(const LevelDev&, const LevelDev&, const T*, T*, void*);                          \
  template int launch_axpby<T>(int64_t, T, const T*, T, T*, void*);                                              \
  template int launch_gather<T>(int64_t, int, int64_t, int64_t, const int64_t*, const T*, T*, void*);            \
  template int launch_fill<T>(int64_t, T, T*, void*);                                                           \
  template int launch_dot_masked<T>(const uint8_t*, int64_t, int, const T*, const T*, double*, int64_t*, void*);  \
  template int launch_mul3<T>(int64_t, const T*, const T*, const T*, T*, void*);                                  \
  template int launch_add_const<T>(int64_t, T, T*, void*);                                                        \
  template int launch_mul<T>(int64_t, const T*, const T*, T*, void*);                                           \
  template int launch_recip<T>(int64_t, const T*, T*, void*);                                                    \
  template int launch_hash_unique<T>(int64_t, int, const int8_t*, T*, void*);                                    \
  template int launch_dense_matvec<T>(int, const T*, const int64_t*, const T*, T*, void*);
HHG_INST(float)
HHG_INST(double)
template int launch_convert<double, float>(int64_t, const double*, float*, void*);
template int launch_convert<float, double>(int64_t, const float*, double*, void*);

template <typename T>
__global__ void k_copy_entries(int64_t count, const int64_t* __restrict__ idx, int comps, int64_t E,
                               const T* __restrict__ src, T* __restrict__ dst) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= count) return;
  const int64_t e = idx[u];
  for (int c = 0; c < comps; ++c) dst[c * E + e] = src[c * E + e];
}

template <typename T>
int launch_copy_entries(int64_t count, const int64_t* idx, int comps, int64_t E, const T* src, T* dst, void* stream) {
  if (count == 0) return 0;
  k_copy_entries<T><<<(unsigned)((count + 255) / 256), 256, 0, (cudaStream_t)stream>>>(count, idx, comps, E, src, dst);
  return (int)cudaGetLastError();
}
template int launch_copy_entries<float>(int64_t, const int64_t*, int, int64_t, const float*, float*, void*);
template int launch_copy_entries<double>(int64_t, const int64_t*, int, int64_t, const double*, double*, void*);

// ---------------------------------------------------------------------------
// FP32 FMA issue-rate probe (a measurement aid: the denominator of the ALU roofline
// of the stencil kernels).  Every thread runs 8 independent FMA chains a <- a * b + c
// (PACKED: 8 chains of packed two-lane FMAs, fma.rn.f32x2, 16 FMAs per step); the
// result is stored only under a condition that never holds, so nothing is removed.
// ---------------------------------------------------------------------------
constexpr int PROBE_THREADS = 256;
constexpr int PROBE_BLOCKS_PER_SM = 8;

template <int PACKED>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(int64_t iters, float* out) {
  const float b = 0.9999999f, c = 1.0e-7f;
  const float s0 = 1.0f + 1.0e-6f * (float)(threadIdx.x & 63);
  if constexpr (PACKED) {
    float2 a[8];
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = make_float2(s0 + q, s0 - q);
#pragma unroll 4
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = __ffma2_rn(a[q], b2, c2);
    }
    float sum = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) sum += a[q].x + a[q].y;
    if (sum == -1.0f) out[0] = sum;
  } else {
    float a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = s0 + q;
#pragma unroll 8
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = fmaf(a[q], b, c);
    }
    float sum = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) sum += a[q];
    if (sum == -1.0f) out[0] = sum;
  }
}

int launch_fma_probe(int packed, int64_t iters, int sm_count, float* out, double* flops, void* stream) {
  const int64_t blocks = (int64_t)sm_count * PROBE_BLOCKS_PER_SM;
  if (packed)
    k_fma_probe<1><<<(unsigned)blocks, PROBE_THREADS, 0, (cudaStream_t)stream>>>(iters, out);
  else
    k_fma_probe<0><<<(unsigned)blocks, PROBE_THREADS, 0, (cudaStream_t)stream>>>(iters, out);
  *flops = 2.0 * (packed ? 16.0 : 8.0) * (double)iters * (double)(blocks * PROBE_THREADS);
  return (int)cudaGetLastError();
}

}  // namespace hhg
