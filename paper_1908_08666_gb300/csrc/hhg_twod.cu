// 2D variant of the stencil scaling (Sec. 2.1 and Sec. 2.3): the vector P1 operator of
// c_eps (eps(u), eps(v)) + c_div (div u, div v) with a scalar nodal coefficient on one macro
// triangle refined uniformly, applied with the scaled 7-point stencil of 2x2 blocks.
//
// Lattice: points (i, j), i + j <= n, at v0 + (i (v1 - v0) + j (v2 - v0)) / n, index
// j (n + 1) - j (j - 1) / 2 + i; "up" elements (i, j), (i+1, j), (i, j+1), "down" elements
// (i+1, j), (i, j+1), (i+1, j+1).  Every interior edge lies in one up and one down element, t
// and t^m, with third vertices p and p^m.  Per direction d the block is
//   S_d = khat_d Shat_d + (k_p - k_{p^m}) [[0, -w_d], [w_d, 0]],
// khat_d = (kbar^t + kbar^{t^m}) / 2 (vertex means), Shat_d the constant-coefficient block and
// w_d from the antisymmetric parts of the two element blocks (eq. corrtermgeneral; in 2D the
// value does not depend on the triangle's shape, eq. correction2d).  Interior rows are
// y_i = sum_d S_d (x_{i+d} - x_i); the boundary of the triangle is Dirichlet (y = x).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "hhg_launch.h"

namespace hhg {

namespace {

// directions (1,0), (0,1), (-1,1), (-1,0), (0,-1), (1,-1); d + 3 is the opposite of d
__host__ __device__ __forceinline__ int d2_di(int d) {
  const int t[6] = {1, 0, -1, -1, 0, 1};
  return t[d];
}
__host__ __device__ __forceinline__ int d2_dj(int d) {
  const int t[6] = {0, 1, 1, 0, -1, -1};
  return t[d];
}
__host__ __device__ __forceinline__ int64_t idx2(int n, int i, int j) {
  return (int64_t)j * (n + 1) - (int64_t)j * (j - 1) / 2 + i;
}

// v[q] for a run-time q in 0..5 by selects (keeps v in registers)
template <typename T>
__device__ __forceinline__ T pick6(const T v[6], int q) {
  T r = v[0];
#pragma unroll
  for (int s = 1; s < 6; ++s) r = q == s ? v[s] : r;
  return r;
}

template <typename T>
__global__ void __launch_bounds__(128) k_apply_2d(int n, const Stencil2D<T> st, const T* __restrict__ k,
                                                  const T* __restrict__ x, T* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i + j > n) return;
  const int64_t N = (int64_t)(n + 1) * (n + 2) / 2;
  const int64_t e = idx2(n, i, j);
  const T x0 = x[e], y0 = x[e + N];
  if (i == 0 || j == 0 || i + j == n) {
    y[e] = x0;
    y[e + N] = y0;
    return;
  }
  // neighbour indices from the point's own: row j + 1 starts n + 1 - j entries after row j,
  // row j starts n + 2 - j entries after row j - 1
  const int up = n + 1 - j, dn = n + 2 - j;
  const int off[6] = {1, up, up - 1, -1, -dn, -dn + 1};  // (1,0) (0,1) (-1,1) (-1,0) (0,-1) (1,-1)
  T kk[6], dx[6], dy[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const int64_t q = e + off[d];
    kk[d] = k[q];
    dx[d] = x[q] - x0;
    dy[d] = x[q + N] - y0;
  }
  const T k0 = k[e];
  T ax = 0, ay = 0;
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const T kp = pick6(kk, st.p[d]), kpm = pick6(kk, st.pm[d]);
    if (st.nodal) {
      // a_h: each element block scaled by its own vertex mean
      const T kt = (k0 + kk[d] + kp) * (T)(1.0 / 3.0), ktm = (k0 + kk[d] + kpm) * (T)(1.0 / 3.0);
      const T* A = st.Kt[d];
      const T* C = st.Ktm[d];
      ax += kt * (A[0] * dx[d] + A[1] * dy[d]) + ktm * (C[0] * dx[d] + C[1] * dy[d]);
      ay += kt * (A[2] * dx[d] + A[3] * dy[d]) + ktm * (C[2] * dx[d] + C[3] * dy[d]);
      continue;
    }
    const T khat = ((T)2 * (k0 + kk[d]) + kp + kpm) * (T)(1.0 / 6.0);
    const T dk = kp - kpm;
    const T* S = st.S[d];  // row-major 2x2
    const T w = dk * st.w[d];
    ax += khat * (S[0] * dx[d] + S[1] * dy[d]) - w * dy[d];
    ay += khat * (S[2] * dx[d] + S[3] * dy[d]) + w * dx[d];
  }
  y[e] = ax;
  y[e + N] = ay;
}

}  // namespace

template <typename T>
int launch_apply_2d(int n, const Stencil2D<T>& st, const T* k, const T* x, T* y, void* stream) {
  const dim3 g((n + 1 + 127) / 128, n + 1);
  k_apply_2d<T><<<g, 128, 0, (cudaStream_t)stream>>>(n, st, k, x, y);
  return (int)cudaGetLastError();
}
template int launch_apply_2d<float>(int, const Stencil2D<float>&, const float*, const float*, float*, void*);
template int launch_apply_2d<double>(int, const Stencil2D<double>&, const double*, const double*, double*, void*);

// The constants of Stencil2D for the macro triangle tri[6] = (x0, y0, x1, y1, x2, y2) at n
// intervals per edge, in FP64: the element blocks of the up and down element types, then per
// direction the sum of the two blocks of its edge and the antisymmetric weight w_d.
// physical = 0 leaves w_d = 0 (the unphysical scaling); physical = 2 selects nodal integration
// (the two element blocks are kept apart).
int stencil_2d(const double* tri, int n, double c_eps, double c_div, int physical, Stencil2D<double>* out) {
  const double e1x = (tri[2] - tri[0]) / n, e1y = (tri[3] - tri[1]) / n;
  const double e2x = (tri[4] - tri[0]) / n, e2y = (tri[5] - tri[1]) / n;
  const double det = e1x * e2y - e1y * e2x;
  if (!(std::fabs(det) > 0.0)) return 1;
  // barycentric gradients of the up element (0,0), (1,0), (0,1): rows of [-1 -1; 1 0; 0 1] J^-1
  // with J = [e1 e2]; the down element (1,0), (0,1), (1,1) is its point reflection, so its
  // gradients are the negated ones of the opposite vertices
  const double inv[2][2] = {{e2y / det, -e2x / det}, {-e1y / det, e1x / det}};
  double gu[3][2];
  const double ref[3][2] = {{-1.0, -1.0}, {1.0, 0.0}, {0.0, 1.0}};
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 2; ++c) gu[a][c] = ref[a][0] * inv[0][c] + ref[a][1] * inv[1][c];
  // down element local order: (1,0), (0,1), (1,1); (1,1) = -(0,0) reflected, (1,0) <-> (0,1) swap
  double gd[3][2];
  for (int c = 0; c < 2; ++c) {
    gd[0][c] = -gu[2][c];  // (1,0) is the reflection image of (0,1)
    gd[1][c] = -gu[1][c];  // (0,1) is the reflection image of (1,0)
    gd[2][c] = -gu[0][c];  // (1,1) is the reflection image of (0,0)
  }
  const double area = 0.5 * std::fabs(det);
  // element block K[a][b][m][l] = a(phi_b e_l, phi_a e_m)
  auto block = [&](const double g[3][2], int a, int b, double K[2][2]) {
    for (int m = 0; m < 2; ++m)
      for (int l = 0; l < 2; ++l) {
        const double dot = g[a][0] * g[b][0] + g[a][1] * g[b][1];
        const double eps = 0.5 * ((m == l ? dot : 0.0) + g[a][l] * g[b][m]);
        const double dv = g[b][l] * g[a][m];
        K[m][l] = area * (c_eps * eps + c_div * dv);
      }
  };
  // local vertex offsets of the two element types
  const int up[3][2] = {{0, 0}, {1, 0}, {0, 1}};
  const int dn[3][2] = {{1, 0}, {0, 1}, {1, 1}};
  for (int d = 0; d < 6; ++d) {
    const int di = d2_di(d), dj = d2_dj(d);
    double S[2][2] = {{0, 0}, {0, 0}}, A[2] = {0, 0};
    int third[2][2], found = 0;
    // elements containing the edge from the point (0,0) to (di, dj): bases within +-1
    for (int type = 0; type < 2; ++type)
      for (int bi = -1; bi <= 0; ++bi)
        for (int bj = -1; bj <= 0; ++bj) {
          const int(*v)[2] = type == 0 ? up : dn;
          int la = -1, lb = -1, lt = -1;
          for (int q = 0; q < 3; ++q) {
            const int oi = bi + v[q][0], oj = bj + v[q][1];
            if (oi == 0 && oj == 0)
              la = q;
            else if (oi == di && oj == dj)
              lb = q;
            else
              lt = q;
          }
          if (la < 0 || lb < 0) continue;
          double K[2][2];
          block(type == 0 ? gu : gd, la, lb, K);
          for (int m = 0; m < 2; ++m)
            for (int l = 0; l < 2; ++l) S[m][l] += K[m][l];
          if (found < 2)
            for (int m = 0; m < 2; ++m)
              for (int l = 0; l < 2; ++l) (found == 0 ? out->Kt : out->Ktm)[d][2 * m + l] = K[m][l];
          if (found < 2) {
            third[found][0] = bi + v[lt][0];
            third[found][1] = bj + v[lt][1];
            A[found] = 0.5 * (K[1][0] - K[0][1]);  // the (2,1) entry of the antisymmetric part
          }
          ++found;
        }
    if (found != 2) return 2;
    for (int m = 0; m < 2; ++m)
      for (int l = 0; l < 2; ++l) out->S[d][2 * m + l] = S[m][l];
    // R = 1/2 [(kbar^t - kbar^{t^m}) a^{a;t} + (kbar^{t^m} - kbar^t) a^{a;t^m}],
    // kbar^t - kbar^{t^m} = (k_p - k_{p^m}) / 3 with p the third vertex of t = the first element
    int pdir = -1, pmdir = -1;
    for (int q = 0; q < 6; ++q) {
      if (d2_di(q) == third[0][0] && d2_dj(q) == third[0][1]) pdir = q;
      if (d2_di(q) == third[1][0] && d2_dj(q) == third[1][1]) pmdir = q;
    }
    if (pdir < 0 || pmdir < 0) return 3;
    out->p[d] = pdir;
    out->pm[d] = pmdir;
    out->w[d] = physical == 1 ? 0.5 * (A[0] - A[1]) / 3.0 : 0.0;
  }
  out->nodal = physical == 2;
  return 0;
}

}  // namespace hhg
