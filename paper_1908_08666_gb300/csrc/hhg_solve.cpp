// libhhgs solvers: point-Jacobi / Chebyshev smoothing, geometric multigrid
// V-cycles, (preconditioned) conjugate gradients and FP64 iterative refinement
// around an FP32 multigrid-preconditioned CG.
//
// Sec. 5 of the paper solves with geometric multigrid V-cycles: matrix-free
// linear interpolation between levels and its transpose as restriction, a
// smoother on every level, and a coarse-grid solve on the mesh with one
// interior node per macro.  Coarse operators are rediscretisations with the
// injected nodal coefficient.  Here the smoother is point Jacobi or Chebyshev
// (on D^-1 A, interval [lo, hi] * lambda_max with lambda_max from power
// iterations), and the coarsest level (level 2) is solved exactly with a dense
// inverse of its matrix restricted to the free degrees of freedom.
#include "hhg_ctx.h"
#include "hhg_solver.h"

namespace {

template <typename T>
DevMem* work(LevelHost& L);
template <>
DevMem* work<double>(LevelHost& L) {
  return L.w64;
}
template <>
DevMem* work<float>(LevelHost& L) {
  return L.w32;
}
template <typename T>
DevMem& uvec(LevelHost& L);
template <>
DevMem& uvec<double>(LevelHost& L) {
  return L.u64;
}
template <>
DevMem& uvec<float>(LevelHost& L) {
  return L.u32;
}
template <typename T>
DevMem& dinv(LevelHost& L);
template <>
DevMem& dinv<double>(LevelHost& L) {
  return L.dinv64;
}
template <>
DevMem& dinv<float>(LevelHost& L) {
  return L.dinv32;
}
template <typename T>
DevMem& cinv(LevelHost& L);
template <>
DevMem& cinv<double>(LevelHost& L) {
  return L.d_cinv64;
}
template <>
DevMem& cinv<float>(LevelHost& L) {
  return L.d_cinv32;
}

constexpr int NWORK = 12;

template <typename T>
void ensure_work(hhg_ctx* c, int l) {
  LevelHost& L = c->lv(l);
  DevMem* W = work<T>(L);
  if (W[0].p) return;
  for (int q = 0; q < NWORK; ++q) {
    CK(W[q].alloc(3 * (size_t)L.entries * sizeof(T)));
    CK(cudaMemsetAsync(W[q].p, 0, W[q].bytes, c->stream));
  }
  CK(uvec<T>(L).alloc(2 * 3 * (size_t)L.nunique * sizeof(T)));
  CK(cudaMemsetAsync(uvec<T>(L).p, 0, uvec<T>(L).bytes, c->stream));
  if (!L.d_udir.p) upload(L.d_udir, L.unique_dir);
}

template <typename T>
double dot(hhg_ctx* c, int l, const T* a, const T* b) {
  LevelHost& L = c->lv(l);
  int64_t np = 0;
  CK(launch_dot<T>(L.dev, 3, a, b, c->scratch.as<double>(), &np, c->stream));
  CK(launch_reduce(c->scratch.as<double>(), np, c->scalar.as<double>(), c->stream));
  CK(cudaMemcpyAsync(c->pinned, c->scalar.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  wait_stream(c);
  return c->pinned[0];
}

template <typename T>
void apply_op(hhg_ctx* c, int l, const T* x, T* y) {
  SweepArgs<T> a{};
  a.x = x;
  a.out = y;
  sweep<T>(c, l, OP_APPLY, a, nullptr);
}

template <typename T>
double residual_op(hhg_ctx* c, int l, const T* f, const T* x, T* r, bool norm) {
  SweepArgs<T> a{};
  a.x = x;
  a.f = f;
  a.out = r;
  double n2 = 0.0;
  sweep<T>(c, l, OP_RESID, a, norm ? &n2 : nullptr);
  return n2;
}

template <typename T>
void compute_diag(hhg_ctx* c, int l) {
  ensure_work<T>(c, l);
  LevelHost& L = c->lv(l);
  DevMem* W = work<T>(L);
  SweepArgs<T> a{};
  a.x = W[1].as<T>();  // read by the interface kernels, value irrelevant
  a.out = W[0].as<T>();
  sweep<T>(c, l, OP_DIAG, a, nullptr);
  if (!dinv<T>(L).p) CK(dinv<T>(L).alloc(3 * (size_t)L.entries * sizeof(T)));
  CK(launch_recip<T>(3 * L.entries, W[0].as<T>(), dinv<T>(L).template as<T>(), c->stream));
}

// lambda_max of D^{-1} A by power iterations from a hashed start vector (zero on
// Dirichlet nodes), in FP64
double power_lambda(hhg_ctx* c, int l, int iters) {
  ensure_work<double>(c, l);
  LevelHost& L = c->lv(l);
  DevMem* W = work<double>(L);
  double* v = W[0].as<double>();
  double* y = W[1].as<double>();
  double* u = uvec<double>(L).as<double>();
  CK(launch_hash_unique<double>(L.nunique, 3, L.d_udir.as<int8_t>(), u, c->stream));
  CK(launch_gather<double>(L.entries, 3, L.nunique, L.entries, L.d_e2u.as<int64_t>(), u, v, c->stream));
  double lam = 0.0;
  for (int it = 0; it < iters; ++it) {
    apply_op<double>(c, l, v, y);
    CK(launch_mul<double>(3 * L.entries, y, L.dinv64.as<double>(), y, c->stream));
    const double nv = dot<double>(c, l, v, v);
    const double ny = dot<double>(c, l, y, y);
    if (!(ny > 0.0) || !std::isfinite(ny)) THROW(HHG_ERR_NUMERIC, "power iteration failed on level %d", l);
    lam = std::sqrt(ny / nv);
    CK(launch_axpby<double>(3 * L.entries, 1.0 / std::sqrt(ny), y, 0.0, v, c->stream));
  }
  // leave the work vectors zero (the interface kernels read W[1] as a dummy input)
  CK(cudaMemsetAsync(W[1].p, 0, W[1].bytes, c->stream));
  return lam;
}

// dense inverse (Gauss-Jordan with partial pivoting), row-major N x N, FP64
void invert_dense(std::vector<double>& A, int N) {
  std::vector<double> I((size_t)N * N, 0.0);
  for (int i = 0; i < N; ++i) I[(size_t)i * N + i] = 1.0;
  for (int col = 0; col < N; ++col) {
    int piv = col;
    double best = std::fabs(A[(size_t)col * N + col]);
    for (int r = col + 1; r < N; ++r)
      if (std::fabs(A[(size_t)r * N + col]) > best) {
        best = std::fabs(A[(size_t)r * N + col]);
        piv = r;
      }
    if (!(best > 0.0)) THROW(HHG_ERR_NUMERIC, "singular coarse matrix");
    if (piv != col)
      for (int q = 0; q < N; ++q) {
        std::swap(A[(size_t)piv * N + q], A[(size_t)col * N + q]);
        std::swap(I[(size_t)piv * N + q], I[(size_t)col * N + q]);
      }
    const double inv = 1.0 / A[(size_t)col * N + col];
    for (int q = 0; q < N; ++q) {
      A[(size_t)col * N + q] *= inv;
      I[(size_t)col * N + q] *= inv;
    }
    for (int r = 0; r < N; ++r) {
      if (r == col) continue;
      const double f = A[(size_t)r * N + col];
      if (f == 0.0) continue;
      for (int q = 0; q < N; ++q) {
        A[(size_t)r * N + q] -= f * A[(size_t)col * N + q];
        I[(size_t)r * N + q] -= f * I[(size_t)col * N + q];
      }
    }
  }
  A.swap(I);
}

constexpr int MAX_COARSE_DOFS = 3000;

// coarse matrix by applying the operator to unit vectors of the free DoFs
void coarse_setup(hhg_ctx* c) {
  const int l = c->level_min;
  ensure_work<double>(c, l);
  ensure_work<float>(c, l);
  LevelHost& L = c->lv(l);
  std::vector<int64_t> cdof;
  for (int64_t u = 0; u < L.nunique; ++u)
    if (!L.unique_dir[u])
      for (int q = 0; q < 3; ++q) cdof.push_back(q * L.nunique + u);
  const int N = (int)cdof.size();
  L.ncdof = N;
  if (N == 0) return;
  if (N > MAX_COARSE_DOFS) {
    L.ncdof = -N;  // too large for the dense coarse solve
    return;
  }
  DevMem* W = work<double>(L);
  double* u = uvec<double>(L).as<double>();
  std::vector<double> A((size_t)N * N), col(3 * L.nunique);
  const double one = 1.0;
  for (int j = 0; j < N; ++j) {
    CK(cudaMemsetAsync(u, 0, 3 * L.nunique * sizeof(double), c->stream));
    CK(cudaMemcpyAsync(u + cdof[j], &one, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(launch_gather<double>(L.entries, 3, L.nunique, L.entries, L.d_e2u.as<int64_t>(), u, W[0].as<double>(),
                             c->stream));
    apply_op<double>(c, l, W[0].as<double>(), W[1].as<double>());
    CK(launch_gather<double>(L.nunique, 3, L.entries, L.nunique, L.d_first.as<int64_t>(), W[1].as<double>(), u,
                             c->stream));
    CK(cudaMemcpyAsync(col.data(), u, col.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    wait_stream(c);
    for (int i = 0; i < N; ++i) A[(size_t)i * N + j] = col[cdof[i]];
  }
  CK(cudaMemsetAsync(W[0].p, 0, W[0].bytes, c->stream));
  CK(cudaMemsetAsync(W[1].p, 0, W[1].bytes, c->stream));
  invert_dense(A, N);
  std::vector<float> A32(A.begin(), A.end());
  upload(L.d_cdof, cdof);
  upload(L.d_cinv64, A);
  upload(L.d_cinv32, A32);
}

template <typename T>
void coarse_solve(hhg_ctx* c, int l, const T* f, T* x) {
  LevelHost& L = c->lv(l);
  if (L.ncdof < 0) THROW(HHG_ERR_UNSUPPORTED, "coarse level has %d DoFs (dense solve limit %d)", -L.ncdof,
                         MAX_COARSE_DOFS);
  T* us = uvec<T>(L).template as<T>();
  T* ud = us + 3 * L.nunique;
  CK(launch_gather<T>(L.nunique, 3, L.entries, L.nunique, L.d_first.as<int64_t>(), f, us, c->stream));
  CK(cudaMemsetAsync(ud, 0, 3 * L.nunique * sizeof(T), c->stream));
  if (L.ncdof > 0)
    CK(launch_dense_matvec<T>(L.ncdof, cinv<T>(L).template as<T>(), L.d_cdof.as<int64_t>(), us, ud, c->stream));
  CK(launch_gather<T>(L.entries, 3, L.nunique, L.entries, L.d_e2u.as<int64_t>(), ud, x, c->stream));
}

template <typename T>
void smooth(hhg_ctx* c, int l, int steps, const T* f, T* x) {
  if (steps <= 0) return;
  ensure_work<T>(c, l);
  LevelHost& L = c->lv(l);
  DevMem* W = work<T>(L);
  T* cur = x;
  T* oth = W[3].as<T>();
  if (c->mg.smoother == HHG_SMOOTH_CHEBYSHEV) {
    if (!L.lambda_set) THROW(HHG_ERR_STATE, "lambda_max of level %d unknown (call hhg_mg_setup)", l);
    const double a = c->mg.cheby_lo * L.lambda_max, b = c->mg.cheby_hi * L.lambda_max;
    const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
    double rho = 1.0 / sigma;
    const T* dprev = nullptr;
    T* dnext = W[4].as<T>();
    for (int s = 0; s < steps; ++s) {
      SweepArgs<T> a{};
      if (s == 0) {
        a.rho1 = 0.0;
        a.rho2 = 1.0 / theta;
      } else {
        const double rn = 1.0 / (2.0 * sigma - rho);
        a.rho1 = rn * rho;
        a.rho2 = 2.0 * rn / delta;
        rho = rn;
      }
      a.x = cur;
      a.f = f;
      a.d = dprev;
      a.out = oth;
      a.dout = dnext;
      sweep<T>(c, l, OP_CHEBY, a, nullptr);
      std::swap(cur, oth);
      dprev = dnext;
      dnext = dnext == W[4].as<T>() ? W[5].as<T>() : W[4].as<T>();
    }
  } else if (c->mg.smoother == HHG_SMOOTH_HYBRID_GS) {
    // hybrid Gauss-Seidel (Sec. 5): per step a damped Jacobi step on the macro skeleton (out of
    // place, copied back to every copy), then Gauss-Seidel over the macro interiors in eight
    // colour passes, each in place with the newest values
    for (int s = 0; s < steps; ++s) {
      SweepArgs<T> a{};
      a.x = x;
      a.f = f;
      a.k = kptr<T>(L);
      a.out = oth;
      a.omega = c->mg.omega;
      CK(launch_sweep<T>(L.dev, stencils<T>(L), consts_dev<T>(L), OP_JACOBI, c->flags, a, c->stream, 2, 0, nullptr));
      CK(launch_copy_entries<T>(L.dev.nskel_entries, L.dev.skel_entries, 3, L.entries, oth, x, c->stream));
      SweepArgs<T> g{};
      g.x = x;
      g.f = f;
      g.k = kptr<T>(L);
      g.out = x;
      g.omega = 1.0;
      for (int col = 0; col < 8; ++col)
        CK(launch_gs_colour<T>(L.dev, stencils<T>(L), consts_dev<T>(L), c->flags, g, col, c->stream));
    }
  } else {
    for (int s = 0; s < steps; ++s) {
      SweepArgs<T> a{};
      a.x = cur;
      a.f = f;
      a.out = oth;
      a.omega = c->mg.omega;
      sweep<T>(c, l, OP_JACOBI, a, nullptr);
      std::swap(cur, oth);
    }
  }
  if (cur != x) CK(cudaMemcpyAsync(x, cur, 3 * L.entries * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
}

template <typename T>
void restrict_op(hhg_ctx* c, int lf, const T* rf, T* rc);
template <>
void restrict_op<double>(hhg_ctx* c, int lf, const double* rf, double* rc) {
  LevelHost& F = c->lv(lf);
  LevelHost& C = c->lv(lf - 1);
  CK(launch_restrict<double>(F.dev, C.dev, C.d_rptr.as<int32_t>(), C.d_rent.as<int64_t>(), C.d_rw64.as<double>(), rf,
                             rc, c->stream));
}
template <>
void restrict_op<float>(hhg_ctx* c, int lf, const float* rf, float* rc) {
  LevelHost& F = c->lv(lf);
  LevelHost& C = c->lv(lf - 1);
  CK(launch_restrict<float>(F.dev, C.dev, C.d_rptr.as<int32_t>(), C.d_rent.as<int64_t>(), C.d_rw32.as<float>(), rf,
                            rc, c->stream));
}

template <typename T>
void vcycle(hhg_ctx* c, int l, const T* f, T* x) {
  if (l == c->level_min) {
    coarse_solve<T>(c, l, f, x);
    return;
  }
  ensure_work<T>(c, l);
  ensure_work<T>(c, l - 1);
  LevelHost& L = c->lv(l);
  LevelHost& C = c->lv(l - 1);
  DevMem* W = work<T>(L);
  DevMem* Wc = work<T>(C);
  smooth<T>(c, l, c->mg.pre, f, x);
  residual_op<T>(c, l, f, x, W[0].as<T>(), false);
  restrict_op<T>(c, l, W[0].as<T>(), Wc[1].as<T>());
  CK(cudaMemsetAsync(Wc[2].p, 0, 3 * C.entries * sizeof(T), c->stream));
  vcycle<T>(c, l - 1, Wc[1].as<T>(), Wc[2].as<T>());
  CK(launch_prolong_add<T>(L.dev, C.dev, Wc[2].as<T>(), x, c->stream));
  smooth<T>(c, l, c->mg.post, f, x);
}

// x = 0 followed by one V-cycle for f on level l.  The first call for a (precision,
// level, f, x) runs the cycle directly (allocating its work vectors), the second captures
// it as a CUDA graph on the context's capture stream, later calls replay the graph on the
// context stream.  A failed capture disables graphs for the context (direct launches).
template <typename T>
void vcycle_zero(hhg_ctx* c, int l, const T* f, T* x) {
  LevelHost& L = c->lv(l);
  auto direct = [&] {
    CK(cudaMemsetAsync(x, 0, 3 * L.entries * sizeof(T), c->stream));
    vcycle<T>(c, l, f, x);
  };
  if (!c->graphs_ok || c->prof) {
    direct();
    return;
  }
  const auto key = std::make_tuple((int)sizeof(T), l, (const void*)f, (void*)x);
  auto it = c->vc_graphs.find(key);
  if (it != c->vc_graphs.end() && it->second) {
    CK(cudaGraphLaunch(it->second, c->stream));
    return;
  }
  if (it == c->vc_graphs.end()) {  // first use: run directly, so every work vector exists
    c->vc_graphs[key] = nullptr;
    direct();
    return;
  }
  if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  // the capture stream starts after everything issued so far on the context stream
  cudaEvent_t ev = c->take_event();
  CK(cudaEventRecord(ev, c->stream));
  CK(cudaStreamWaitEvent(c->cap_stream, ev, 0));
  c->ev_pool.push_back(ev);
  cudaStream_t user = c->stream;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    c->stream = c->cap_stream;
    try {
      CK(cudaMemsetAsync(x, 0, 3 * L.entries * sizeof(T), c->stream));
      vcycle<T>(c, l, f, x);
    } catch (...) {
      c->stream = user;
      cudaStreamEndCapture(c->cap_stream, &g);
      if (g) cudaGraphDestroy(g);
      c->graphs_ok = false;
      cudaGetLastError();
      direct();
      return;
    }
    c->stream = user;
    e = cudaStreamEndCapture(c->cap_stream, &g);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->graphs_ok = false;
    direct();
    return;
  }
  c->vc_graphs[key] = ge;
  CK(cudaGraphLaunch(ge, c->stream));
}

template <typename T>
void precondition(hhg_ctx* c, int l, bool mg, const T* r, T* z) {
  LevelHost& L = c->lv(l);
  if (mg) {
    vcycle_zero<T>(c, l, r, z);
  } else {
    CK(launch_mul<T>(3 * L.entries, dinv<T>(L).template as<T>(), r, z, c->stream));
  }
}

struct CgResult {
  int iterations = 0;
  double r0 = 0.0, rel = 0.0;
  bool converged = false;
};

// (preconditioned) CG on A x = f, x updated in place; uses work vectors 6..9
template <typename T>
CgResult pcg(hhg_ctx* c, int l, bool mg, const T* f, T* x, double rtol, int max_iter) {
  ensure_work<T>(c, l);
  LevelHost& L = c->lv(l);
  DevMem* W = work<T>(L);
  T* r = W[6].as<T>();
  T* z = W[7].as<T>();
  T* p = W[8].as<T>();
  T* q = W[9].as<T>();
  const int64_t n = 3 * L.entries;
  CgResult res;
  const double r0 = residual_op<T>(c, l, f, x, r, true);
  res.r0 = std::sqrt(r0);
  if (!std::isfinite(r0)) THROW(HHG_ERR_NUMERIC, "non-finite initial residual");
  if (r0 == 0.0) {
    res.converged = true;
    return res;
  }
  precondition<T>(c, l, mg, r, z);
  CK(cudaMemcpyAsync(p, z, n * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
  double rz = dot<T>(c, l, r, z);
  double rr = r0;
  for (int it = 1; it <= max_iter; ++it) {
    apply_op<T>(c, l, p, q);
    const double pq = dot<T>(c, l, p, q);
    if (!(pq > 0.0) || !std::isfinite(pq)) THROW(HHG_ERR_NUMERIC, "CG breakdown (p.Ap = %g)", pq);
    const double alpha = rz / pq;
    CK(launch_axpby<T>(n, (T)alpha, p, (T)1, x, c->stream));
    CK(launch_axpby<T>(n, (T)(-alpha), q, (T)1, r, c->stream));
    rr = dot<T>(c, l, r, r);
    res.iterations = it;
    if (!std::isfinite(rr)) THROW(HHG_ERR_NUMERIC, "non-finite residual");
    if (std::sqrt(rr / r0) <= rtol) {
      res.converged = true;
      break;
    }
    precondition<T>(c, l, mg, r, z);
    const double rzn = dot<T>(c, l, r, z);
    const double beta = rzn / rz;
    rz = rzn;
    CK(launch_axpby<T>(n, (T)1, z, (T)beta, p, c->stream));
  }
  res.rel = std::sqrt(rr / r0);
  return res;
}

// ------------------------------------------------------------------- Stokes (Sec. 5.2)

template <typename T>
DevMem* swork(LevelHost& L);
template <>
DevMem* swork<double>(LevelHost& L) {
  return L.sw64;
}
template <>
DevMem* swork<float>(LevelHost& L) {
  return L.sw32;
}
template <typename T>
const T* mass(LevelHost& L);
template <>
const double* mass<double>(LevelHost& L) {
  return L.d_mass64.as<double>();
}
template <>
const float* mass<float>(LevelHost& L) {
  return L.d_mass32.as<float>();
}

constexpr int NSWORK = 10;

template <typename T>
void ensure_swork(hhg_ctx* c, int l) {
  LevelHost& L = c->lv(l);
  DevMem* W = swork<T>(L);
  if (W[0].p) return;
  for (int q = 0; q < NSWORK; ++q) {
    CK(W[q].alloc(4 * (size_t)L.entries * sizeof(T)));
    CK(cudaMemsetAsync(W[q].p, 0, W[q].bytes, c->stream));
  }
}

void need_stokes(hhg_ctx* c) {
  need_ready(c, true);
  if (c->prob.kind != HHG_STOKES) THROW(HHG_ERR_STATE, "problem kind is not Stokes");
}

template <typename T>
double stokes_sweep(hhg_ctx* c, int l, OpKind op, const T* f, const T* x, T* out, bool norm) {
  LevelHost& L = c->lv(l);
  SweepArgs<T> a{};
  a.x = x;
  a.f = f;
  a.out = out;
  a.k = kptr<T>(L);
  if (norm) a.partial = c->scratch.as<double>();
  int64_t np = 0;
  fork_side_streams(c);
  void* side[3] = {c->aux[0], c->aux[1], c->aux[2]};
  CK(launch_stokes_sweep<T>(L.dev, stencils<T>(L), consts_dev<T>(L), op, sweep_flags(c, L, false), a, c->stream, &np,
                            side));
  join_side_streams(c);
  if (!norm) return 0.0;
  CK(launch_reduce(c->scratch.as<double>(), np, c->scalar.as<double>(), c->stream));
  CK(cudaMemcpyAsync(c->pinned, c->scalar.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  wait_stream(c);
  return c->pinned[0];
}

// Euclidean inner product over the unique DoFs: free velocity components and all pressures
template <typename T>
double sdot(hhg_ctx* c, int l, const T* a, const T* b) {
  LevelHost& L = c->lv(l);
  int64_t n1 = 0, n2 = 0;
  double* part = c->scratch.as<double>();
  CK(launch_dot_masked<T>(L.d_mask.as<uint8_t>(), L.entries, 3, a, b, part, &n1, c->stream));
  if ((n1 + 1024) * (int64_t)sizeof(double) > (int64_t)c->scratch.bytes)
    THROW(HHG_ERR_STATE, "partial-sum scratch too small for the Stokes inner product");
  CK(launch_dot_masked<T>(L.d_mask_own.as<uint8_t>(), L.entries, 1, a + 3 * L.entries, b + 3 * L.entries, part + n1,
                          &n2, c->stream));
  CK(launch_reduce(part, n1 + n2, c->scalar.as<double>(), c->stream));
  CK(cudaMemcpyAsync(c->pinned, c->scalar.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  wait_stream(c);
  return c->pinned[0];
}

template <typename T>
const T* sdiag(LevelHost& L);
template <>
const double* sdiag<double>(LevelHost& L) {
  return L.d_sdiag64.as<double>();
}
template <>
const float* sdiag<float>(LevelHost& L) {
  return L.d_sdiag32.as<float>();
}

// Pressure Schur-complement surrogate: S = C - B A^-1 B^T is approximated by
// -diag(m_i / mu_i + (-C)_ii) (lumped mass over the viscosity, plus the stabilisation,
// which carries no 1/mu and dominates where mu is large); out = r / (m / mu + (-C)_ii).
template <typename T>
void schur_apply(hhg_ctx* c, int l, const T* r, T* out) {
  LevelHost& L = c->lv(l);
  CK(launch_schur_diag<T>(L.entries, r, kptr<T>(L), mass<T>(L), sdiag<T>(L), out, c->stream));
}

// z = blockdiag(V-cycle of A(mu), Schur surrogate^-1) r
template <typename T>
void stokes_precond(hhg_ctx* c, int l, const T* r, T* z) {
  LevelHost& L = c->lv(l);
  vcycle_zero<T>(c, l, r, z);
  schur_apply<T>(c, l, r + 3 * L.entries, z + 3 * L.entries);
}

// shift the pressure to zero mean: sum_i m_i p_i = 0 over unique nodes
template <typename T>
void project_pressure(hhg_ctx* c, int l, T* x) {
  LevelHost& L = c->lv(l);
  int64_t n1 = 0;
  double* part = c->scratch.as<double>();
  T* p = x + 3 * L.entries;
  CK(launch_dot_masked<T>(L.d_mask_own.as<uint8_t>(), L.entries, 1, mass<T>(L), p, part, &n1, c->stream));
  CK(launch_reduce(part, n1, c->scalar.as<double>(), c->stream));
  CK(cudaMemcpyAsync(c->pinned, c->scalar.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  wait_stream(c);
  double msum = 0.0;
  for (int64_t u = 0; u < L.nunique; ++u) msum += L.lumped[L.unique_first[u]];
  CK(launch_add_const<T>(L.entries, (T)(-c->pinned[0] / msum), p, c->stream));
}

struct MinresResult {
  int iterations = 0;
  double r0 = 0.0, rel = 0.0;
  bool converged = false;
};

// Preconditioned MINRES (Lanczos with Givens rotations; Elman, Silvester and Wathen,
// Finite Elements and Fast Iterative Solvers, Alg. 4.1) on K x = f; stops when the
// preconditioned residual estimate |eta| <= rtol |eta_0|; returns the true relative residual.
template <typename T>
MinresResult minres(hhg_ctx* c, int l, const T* f, T* x, double rtol, int max_iter) {
  ensure_swork<T>(c, l);
  ensure_work<T>(c, l);
  LevelHost& L = c->lv(l);
  DevMem* W = swork<T>(L);
  const int64_t n = 4 * L.entries;
  T* v_prev = W[0].as<T>();
  T* v = W[1].as<T>();
  T* q = W[2].as<T>();
  T* z = W[3].as<T>();
  T* w_prev = W[4].as<T>();
  T* w = W[5].as<T>();
  MinresResult R;
  const double r0 = stokes_sweep<T>(c, l, OP_RESID, f, x, v, true);
  R.r0 = std::sqrt(r0);
  if (!std::isfinite(r0)) THROW(HHG_ERR_NUMERIC, "non-finite initial residual");
  if (r0 == 0.0) {
    R.converged = true;
    return R;
  }
  CK(cudaMemsetAsync(v_prev, 0, n * sizeof(T), c->stream));
  CK(cudaMemsetAsync(w_prev, 0, n * sizeof(T), c->stream));
  CK(cudaMemsetAsync(w, 0, n * sizeof(T), c->stream));
  stokes_precond<T>(c, l, v, z);
  double gamma = std::sqrt(sdot<T>(c, l, z, v));
  if (!(gamma > 0.0) || !std::isfinite(gamma)) THROW(HHG_ERR_NUMERIC, "preconditioner is not positive definite");
  const double eta0 = gamma;
  double eta = gamma, gamma_prev = 1.0;
  double c_prev = 1.0, c_cur = 1.0, s_prev = 0.0, s_cur = 0.0;
  for (int it = 1; it <= max_iter; ++it) {
    CK(launch_axpby<T>(n, (T)0, z, (T)(1.0 / gamma), z, c->stream));  // z /= gamma
    stokes_sweep<T>(c, l, OP_APPLY, nullptr, z, q, false);
    const double delta = sdot<T>(c, l, q, z);
    CK(launch_axpby<T>(n, (T)(-delta / gamma), v, (T)1, q, c->stream));
    CK(launch_axpby<T>(n, (T)(-gamma / gamma_prev), v_prev, (T)1, q, c->stream));  // q = v_next
    std::swap(v_prev, v);
    std::swap(v, q);  // v = v_next, q = old v_prev (free)
    // z_next into q (z is still needed for w)
    stokes_precond<T>(c, l, v, q);
    const double gn2 = sdot<T>(c, l, q, v);
    if (!(gn2 >= 0.0) || !std::isfinite(gn2)) THROW(HHG_ERR_NUMERIC, "MINRES breakdown");
    const double gamma_next = std::sqrt(gn2);
    const double a0 = c_cur * delta - c_prev * s_cur * gamma;
    const double a1 = std::sqrt(a0 * a0 + gamma_next * gamma_next);
    const double a2 = s_cur * delta + c_prev * c_cur * gamma;
    const double a3 = s_prev * gamma;
    const double c_next = a0 / a1, s_next = gamma_next / a1;
    // w_next = (z - a3 w_prev - a2 w) / a1, stored in w_prev
    CK(launch_axpby<T>(n, (T)(1.0 / a1), z, (T)(-a3 / a1), w_prev, c->stream));
    CK(launch_axpby<T>(n, (T)(-a2 / a1), w, (T)1, w_prev, c->stream));
    std::swap(w_prev, w);  // w = w_next, w_prev = old w
    CK(launch_axpby<T>(n, (T)(c_next * eta), w, (T)1, x, c->stream));
    eta = -s_next * eta;
    std::swap(z, q);  // z = z_next
    gamma_prev = gamma;
    gamma = gamma_next;
    c_prev = c_cur;
    c_cur = c_next;
    s_prev = s_cur;
    s_cur = s_next;
    R.iterations = it;
    if (std::fabs(eta) <= rtol * eta0 || gamma == 0.0) {
      R.converged = true;
      break;
    }
  }
  T* r = W[6].as<T>();
  const double rr = stokes_sweep<T>(c, l, OP_RESID, f, x, r, true);
  R.rel = std::sqrt(rr / r0);
  return R;
}

// ------------------------------------------------ Stokes inexact Uzawa multigrid (Sec. 5.2)

template <typename T>
DevMem* uzwork(LevelHost& L);
template <>
DevMem* uzwork<double>(LevelHost& L) {
  return L.uz64;
}
template <>
DevMem* uzwork<float>(LevelHost& L) {
  return L.uz32;
}

template <typename T>
void ensure_uzwork(hhg_ctx* c, int l) {
  LevelHost& L = c->lv(l);
  DevMem* W = uzwork<T>(L);
  if (W[0].p) return;
  for (int q = 0; q < 4; ++q) {
    CK(W[q].alloc(4 * (size_t)L.entries * sizeof(T)));
    CK(cudaMemsetAsync(W[q].p, 0, W[q].bytes, c->stream));
  }
}

// restriction lists of the pressure: the coarse skeleton node lc gathers every unique fine
// node of its restriction stencil (weights 1 and 1/2), Dirichlet or not
void build_pressure_restriction(hhg_ctx* c, int lc) {
  LevelHost& C = c->lv(lc);
  if (C.rlist_p) return;
  LevelHost& F = c->lv(lc + 1);
  const int nf = F.n;
  const int64_t nskel = (int64_t)C.skel_dir.size();
  std::vector<int32_t> ptr(nskel + 1, 0);
  std::vector<int64_t> ent;
  std::vector<double> w;
  for (int64_t s = 0; s < nskel; ++s) {
    std::map<int64_t, std::pair<int64_t, double>> fine;
    for (int q = C.skel_ptr[s]; q < C.skel_ptr[s + 1]; ++q) {
      const SkelInc& I = C.skel_inc[q];
      const int fi = 2 * I.i, fj = 2 * I.j, fk = 2 * I.k;
      for (int d = -1; d < NDIR; ++d) {
        const int qi = fi + (d < 0 ? 0 : dir_di(d)), qj = fj + (d < 0 ? 0 : dir_dj(d)), qk = fk + (d < 0 ? 0 : dir_dk(d));
        if (!lattice_inside(nf, qi, qj, qk)) continue;
        const int64_t e = (int64_t)I.macro * F.nt + lattice_index(nf, qi, qj, qk);
        fine.emplace(F.entry_to_unique[e], std::make_pair(e, d < 0 ? 1.0 : 0.5));
      }
    }
    for (auto& kv : fine) {
      ent.push_back(kv.second.first);
      w.push_back(kv.second.second);
    }
    ptr[s + 1] = (int32_t)ent.size();
  }
  std::vector<float> w32(w.begin(), w.end());
  upload(C.d_rptr_p, ptr);
  upload(C.d_rent_p, ent);
  upload(C.d_rw64_p, w);
  upload(C.d_rw32_p, w32);
  C.rlist_p = true;
}

template <typename T>
const T* rw_p(LevelHost& L);
template <>
const double* rw_p<double>(LevelHost& L) {
  return L.d_rw64_p.as<double>();
}
template <>
const float* rw_p<float>(LevelHost& L) {
  return L.d_rw32_p.as<float>();
}

// (velocity, pressure) restriction of a saddle residual from level lf to lf - 1
template <typename T>
void stokes_restrict(hhg_ctx* c, int lf, const T* rf, T* rc) {
  LevelHost& F = c->lv(lf);
  LevelHost& C = c->lv(lf - 1);
  restrict_op<T>(c, lf, rf, rc);
  CK(launch_restrict<T>(F.dev, C.dev, C.d_rptr_p.as<int32_t>(), C.d_rent_p.as<int64_t>(), rw_p<T>(C),
                        rf + 3 * F.entries, rc + 3 * C.entries, c->stream, 1, 0));
}

template <typename T>
DevMem& scinv(LevelHost& L);
template <>
DevMem& scinv<double>(LevelHost& L) {
  return L.d_scinv64;
}
template <>
DevMem& scinv<float>(LevelHost& L) {
  return L.d_scinv32;
}
template <typename T>
DevMem& suvec(LevelHost& L);
template <>
DevMem& suvec<double>(LevelHost& L) {
  return L.su64;
}
template <>
DevMem& suvec<float>(LevelHost& L) {
  return L.su32;
}

// Dense inverse of the coarsest saddle matrix on its free velocity DoFs and all pressure
// DoFs, with beta u u^T added to the pressure block (u = normalised constant pressure,
// the kernel of the matrix): for a right-hand side orthogonal to that kernel the
// shifted system has the zero-mean solution of the singular one.
void stokes_coarse_setup(hhg_ctx* c) {
  const int l = c->level_min;
  LevelHost& L = c->lv(l);
  ensure_swork<double>(c, l);
  const int64_t U = L.nunique;
  std::vector<int64_t> dof;
  for (int64_t u = 0; u < U; ++u)
    if (!L.unique_dir[u])
      for (int q = 0; q < 3; ++q) dof.push_back(q * U + u);
  const int nvel = (int)dof.size();
  for (int64_t u = 0; u < U; ++u) dof.push_back(3 * U + u);
  const int N = (int)dof.size();
  if (N > MAX_COARSE_DOFS) THROW(HHG_ERR_UNSUPPORTED, "coarse saddle system too large (%d DoFs)", N);
  for (DevMem* d : {&L.su64, &L.su32})
    if (!d->p) CK(d->alloc(2 * 4 * (size_t)U * (d == &L.su64 ? sizeof(double) : sizeof(float))));
  double* u = L.su64.as<double>();
  DevMem* W = swork<double>(L);
  std::vector<double> A((size_t)N * N), col(4 * U);
  const double one = 1.0;
  for (int j = 0; j < N; ++j) {
    CK(cudaMemsetAsync(u, 0, 4 * U * sizeof(double), c->stream));
    CK(cudaMemcpyAsync(u + dof[j], &one, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(launch_gather<double>(L.entries, 4, U, L.entries, L.d_e2u.as<int64_t>(), u, W[0].as<double>(), c->stream));
    stokes_sweep<double>(c, l, OP_APPLY, nullptr, W[0].as<double>(), W[1].as<double>(), false);
    CK(launch_gather<double>(U, 4, L.entries, U, L.d_first.as<int64_t>(), W[1].as<double>(), u, c->stream));
    CK(cudaMemcpyAsync(col.data(), u, col.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    wait_stream(c);
    for (int i = 0; i < N; ++i) A[(size_t)i * N + j] = col[dof[i]];
  }
  double beta = 0.0;
  for (double v : A) beta = std::max(beta, std::fabs(v));
  const int np = N - nvel;
  for (int i = nvel; i < N; ++i)
    for (int j = nvel; j < N; ++j) A[(size_t)i * N + j] += beta / np;
  invert_dense(A, N);
  std::vector<float> A32(A.begin(), A.end());
  upload(L.d_scdof, dof);
  upload(L.d_scinv64, A);
  upload(L.d_scinv32, A32);
  L.nscdof = N;
  CK(cudaMemsetAsync(W[0].p, 0, W[0].bytes, c->stream));
  CK(cudaMemsetAsync(W[1].p, 0, W[1].bytes, c->stream));
}

template <typename T>
void stokes_coarse_solve(hhg_ctx* c, int l, const T* f, T* x) {
  LevelHost& L = c->lv(l);
  if (L.nscdof <= 0) THROW(HHG_ERR_STATE, "coarse saddle inverse missing (call hhg_mg_setup)");
  const int64_t U = L.nunique;
  T* us = suvec<T>(L).template as<T>();
  T* ud = us + 4 * U;
  CK(launch_gather<T>(U, 4, L.entries, U, L.d_first.as<int64_t>(), f, us, c->stream));
  CK(cudaMemsetAsync(ud, 0, 4 * U * sizeof(T), c->stream));
  CK(launch_dense_matvec<T>(L.nscdof, scinv<T>(L).template as<T>(), L.d_scdof.as<int64_t>(), us, ud, c->stream));
  CK(launch_gather<T>(L.entries, 4, U, L.entries, L.d_e2u.as<int64_t>(), ud, x, c->stream));
}

// One inexact Uzawa step on K (u, p) = (f, g): velocity smoothing of A du = f - A u - B^T p
// (pressure fixed), u += du, then p -= omega S^-1 (g - B u - C p) with the diagonal Schur
// surrogate S = m / mu + (-C)_ii.
template <typename T>
void uzawa_step(hhg_ctx* c, int l, const T* f, T* x) {
  LevelHost& L = c->lv(l);
  const int64_t E = L.entries;
  DevMem* Z = uzwork<T>(L);
  T* r = Z[0].as<T>();
  T* du = Z[1].as<T>();
  stokes_sweep<T>(c, l, OP_RESID, f, x, r, false);
  CK(cudaMemsetAsync(du, 0, 3 * E * sizeof(T), c->stream));
  smooth<T>(c, l, c->mg.uzawa_vsteps, r, du);
  CK(launch_axpby<T>(3 * E, (T)1, du, (T)1, x, c->stream));
  stokes_sweep<T>(c, l, OP_RESID, f, x, r, false);
  T* dp = du + 3 * E;
  schur_apply<T>(c, l, r + 3 * E, dp);
  CK(launch_axpby<T>(E, (T)(-c->mg.uzawa_omega), dp, (T)1, x + 3 * E, c->stream));
}

// Variable V-cycle: uzawa_pre / uzawa_post steps on the finest level, uzawa_extra more on
// every coarser one; exact solve on the coarsest.  Work vectors of a level: [0], [1]
// scratch of its Uzawa steps, [2] and [3] its right-hand side and iterate when it is the
// coarse level of the cycle.
template <typename T>
void uzawa_vcycle(hhg_ctx* c, int l, const T* f, T* x) {
  if (l == c->level_min) {
    stokes_coarse_solve<T>(c, l, f, x);
    return;
  }
  ensure_uzwork<T>(c, l);
  ensure_uzwork<T>(c, l - 1);
  ensure_work<T>(c, l);
  build_pressure_restriction(c, l - 1);
  LevelHost& L = c->lv(l);
  LevelHost& C = c->lv(l - 1);
  DevMem* Z = uzwork<T>(L);
  DevMem* Zc = uzwork<T>(C);
  const int extra = c->mg.uzawa_extra * (c->level_max - l);
  for (int s = 0; s < c->mg.uzawa_pre + extra; ++s) uzawa_step<T>(c, l, f, x);
  T* r = Z[0].as<T>();
  T* fc = Zc[2].as<T>();
  T* xc = Zc[3].as<T>();
  stokes_sweep<T>(c, l, OP_RESID, f, x, r, false);
  stokes_restrict<T>(c, l, r, fc);
  CK(cudaMemsetAsync(xc, 0, 4 * C.entries * sizeof(T), c->stream));
  uzawa_vcycle<T>(c, l - 1, fc, xc);
  CK(launch_prolong_add<T>(L.dev, C.dev, xc, x, c->stream, 3));
  CK(launch_prolong_add<T>(L.dev, C.dev, xc + 3 * C.entries, x + 3 * L.entries, c->stream, 1));
  for (int s = 0; s < c->mg.uzawa_post + extra; ++s) uzawa_step<T>(c, l, f, x);
}

// Stationary Uzawa V-cycles on K x = f until |f - K x| <= rtol |f - K x0|.
template <typename T>
MinresResult uzawa_solve(hhg_ctx* c, int l, const T* f, T* x, double rtol, int max_iter) {
  ensure_uzwork<T>(c, l);
  T* r = uzwork<T>(c->lv(l))[0].template as<T>();  // free between cycles
  MinresResult res;
  const double r0 = stokes_sweep<T>(c, l, OP_RESID, f, x, r, true);
  res.r0 = std::sqrt(r0);
  if (!std::isfinite(r0)) THROW(HHG_ERR_NUMERIC, "non-finite initial residual");
  double rr = r0;
  for (int it = 1; it <= max_iter && r0 > 0.0; ++it) {
    uzawa_vcycle<T>(c, l, f, x);
    rr = stokes_sweep<T>(c, l, OP_RESID, f, x, r, true);
    res.iterations = it;
    if (!std::isfinite(rr)) THROW(HHG_ERR_NUMERIC, "non-finite residual");
    if (std::sqrt(rr / r0) <= rtol) break;
  }
  res.rel = r0 > 0.0 ? std::sqrt(rr / r0) : 0.0;
  res.converged = res.rel <= rtol;
  return res;
}

// ------------------------------------------------------------------- Carreau (Sec. 3, 5.2.2)

// per-macro slope operators and skeleton patch lists of the level (host, once)
void carreau_setup(hhg_ctx* c, int l) {
  LevelHost& L = c->lv(l);
  if (L.carreau_ready) return;
  const int n = L.n;
  const int M = (int)c->tets.size();
  auto phys = [&](int m, double i, double j, double k, double out[3]) {
    const Vec3d& v0 = c->xyz[c->tets[m][0]];
    const Vec3d& v1 = c->xyz[c->tets[m][1]];
    const Vec3d& v2 = c->xyz[c->tets[m][2]];
    const Vec3d& v3 = c->xyz[c->tets[m][3]];
    out[0] = v0.x + (i * (v1.x - v0.x) + j * (v2.x - v0.x) + k * (v3.x - v0.x)) / n;
    out[1] = v0.y + (i * (v1.y - v0.y) + j * (v2.y - v0.y) + k * (v3.y - v0.y)) / n;
    out[2] = v0.z + (i * (v1.z - v0.z) + j * (v2.z - v0.z) + k * (v3.z - v0.z)) / n;
  };
  L.slope.resize(M);
  for (int m = 0; m < M; ++m) {
    double dx[NDIR][3], G[3][3] = {{0}};
    double o[3];
    phys(m, 0, 0, 0, o);
    for (int d = 0; d < NDIR; ++d) {
      double q[3];
      phys(m, dir_di(d), dir_dj(d), dir_dk(d), q);
      for (int a = 0; a < 3; ++a) dx[d][a] = q[a] - o[a];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) G[a][b] += dx[d][a] * dx[d][b];
    }
    // G^{-1} by cofactors
    const double det = G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) -
                       G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) +
                       G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]);
    double Gi[3][3];
    Gi[0][0] = (G[1][1] * G[2][2] - G[1][2] * G[2][1]) / det;
    Gi[0][1] = (G[0][2] * G[2][1] - G[0][1] * G[2][2]) / det;
    Gi[0][2] = (G[0][1] * G[1][2] - G[0][2] * G[1][1]) / det;
    Gi[1][0] = (G[1][2] * G[2][0] - G[1][0] * G[2][2]) / det;
    Gi[1][1] = (G[0][0] * G[2][2] - G[0][2] * G[2][0]) / det;
    Gi[1][2] = (G[0][2] * G[1][0] - G[0][0] * G[1][2]) / det;
    Gi[2][0] = (G[1][0] * G[2][1] - G[1][1] * G[2][0]) / det;
    Gi[2][1] = (G[0][1] * G[2][0] - G[0][0] * G[2][1]) / det;
    Gi[2][2] = (G[0][0] * G[1][1] - G[0][1] * G[1][0]) / det;
    for (int d = 0; d < NDIR; ++d)
      for (int a = 0; a < 3; ++a)
        L.slope[m].Q[d][a] = Gi[a][0] * dx[d][0] + Gi[a][1] * dx[d][1] + Gi[a][2] * dx[d][2];
  }
  // skeleton patches: the node and its lattice neighbours in every incident macro (unique)
  std::vector<int32_t> node, ptr(1, 0);
  std::vector<int64_t> ent;
  std::vector<double> dxs;
  const int64_t nskel = (int64_t)L.skel_dir.size();
  for (int64_t s = 0; s < nskel; ++s) {
    node.push_back((int32_t)s);
    std::map<int64_t, std::array<double, 4>> pts;  // unique node -> (entry, dx)
    for (int q = L.skel_ptr[s]; q < L.skel_ptr[s + 1]; ++q) {
      const SkelInc& I = L.skel_inc[q];
      double o[3];
      phys(I.macro, I.i, I.j, I.k, o);
      for (int d = -1; d < NDIR; ++d) {
        const int qi = I.i + (d < 0 ? 0 : dir_di(d)), qj = I.j + (d < 0 ? 0 : dir_dj(d)),
                  qk = I.k + (d < 0 ? 0 : dir_dk(d));
        if (!lattice_inside(n, qi, qj, qk)) continue;
        const int64_t e = (int64_t)I.macro * L.nt + lattice_index(n, qi, qj, qk);
        const int64_t u = L.entry_to_unique[e];
        if (pts.count(u)) continue;
        double x[3];
        phys(I.macro, qi, qj, qk, x);
        pts[u] = {(double)e, x[0] - o[0], x[1] - o[1], x[2] - o[2]};
      }
    }
    for (auto& kv : pts) {
      ent.push_back((int64_t)kv.second[0]);
      dxs.push_back(kv.second[1]);
      dxs.push_back(kv.second[2]);
      dxs.push_back(kv.second[3]);
    }
    ptr.push_back((int32_t)ent.size());
  }
  upload(L.d_pnode, node);
  upload(L.d_pptr, ptr);
  upload(L.d_pent, ent);
  upload(L.d_pdx, dxs);
  L.plist.nnodes = (int32_t)node.size();
  L.plist.node = L.d_pnode.as<int32_t>();
  L.plist.ptr = L.d_pptr.as<int32_t>();
  L.plist.ent = L.d_pent.as<int64_t>();
  L.plist.dx = L.d_pdx.as<double>();
  L.carreau_ready = true;
}

void carreau_viscosity(hhg_ctx* c, int l, const hhg_carreau& p, const double* u, double* mu) {
  carreau_setup(c, l);
  LevelHost& L = c->lv(l);
  CarreauParams cp{p.eta0, p.eta_inf, p.kappa, p.r};
  CK(launch_carreau(L.dev, L.slope.data(), L.plist, cp, u, mu, c->stream, c->strain_degree));
}

void mg_check(hhg_ctx* c) {
  need_ready(c, true);
  if (!c->mg_ready) THROW(HHG_ERR_STATE, "call hhg_mg_setup after setting the coefficient");
}

template <typename F>
hhg_status dispatch(hhg_ctx* c, hhg_dtype dt, F&& f) {
  return guard(c, [&] {
    if (dt == HHG_F64)
      f((double*)nullptr);
    else if (dt == HHG_F32)
      f((float*)nullptr);
    else
      THROW(HHG_ERR_ARG, "dtype");
  });
}

}  // namespace

namespace hhg {
namespace host {

void mg_ready_check(hhg_ctx* c) { mg_check(c); }
void apply32(hhg_ctx* c, int l, const float* x, float* y) { apply_op<float>(c, l, x, y); }
double dot32(hhg_ctx* c, int l, const float* a, const float* b) { return dot<float>(c, l, a, b); }
void vcycle32(hhg_ctx* c, int l, const float* f, float* x) {
  ensure_work<float>(c, l);
  vcycle<float>(c, l, f, x);
}
void vcycle_zero32(hhg_ctx* c, int l, const float* f, float* x) {
  ensure_work<float>(c, l);
  vcycle_zero<float>(c, l, f, x);
}
const float* dinv32(hhg_ctx* c, int l) {
  LevelHost& L = c->lv(l);
  if (!L.dinv32.p) compute_diag<float>(c, l);
  return L.dinv32.as<float>();
}
double residual32(hhg_ctx* c, int l, const float* f, const float* x, float* r) {
  return residual_op<float>(c, l, f, x, r, true);
}
double residual64(hhg_ctx* c, int l, const double* f, const double* x, double* r) {
  return residual_op<double>(c, l, f, x, r, true);
}
void ensure_work64(hhg_ctx* c, int l) {
  ensure_work<double>(c, l);
  ensure_work<float>(c, l);
}
double* work64(hhg_ctx* c, int l, int q) { return work<double>(c->lv(l))[q].as<double>(); }
float* work32(hhg_ctx* c, int l, int q) { return work<float>(c->lv(l))[q].as<float>(); }

void restrict32(hhg_ctx* c, int lf, const float* rf, float* rc) { restrict_op<float>(c, lf, rf, rc); }
void prolong_add32(hhg_ctx* c, int lf, const float* xc, float* xf) {
  CK(launch_prolong_add<float>(c->lv(lf).dev, c->lv(lf - 1).dev, xc, xf, c->stream));
}
void inject32(hhg_ctx* c, int lf, const float* xf, float* xc) {
  LevelHost& F = c->lv(lf);
  LevelHost& C = c->lv(lf - 1);
  for (int q = 0; q < 3; ++q)
    CK(launch_inject<float>(F.dev, C.dev, xf + q * F.entries, xc + q * C.entries, c->stream));
}

void need_stokes_problem(hhg_ctx* c) { need_stokes(c); }
void stokes_apply32(hhg_ctx* c, int l, const float* x, float* y) {
  stokes_sweep<float>(c, l, OP_APPLY, nullptr, x, y, false);
}
double stokes_dot32(hhg_ctx* c, int l, const float* a, const float* b) { return sdot<float>(c, l, a, b); }
double stokes_residual32(hhg_ctx* c, int l, const float* f, const float* x, float* r) {
  return stokes_sweep<float>(c, l, OP_RESID, f, x, r, true);
}
double stokes_residual64(hhg_ctx* c, int l, const double* f, const double* x, double* r) {
  return stokes_sweep<double>(c, l, OP_RESID, f, x, r, true);
}
void uzawa_zero32(hhg_ctx* c, int l, const float* f, float* x) {
  CK(cudaMemsetAsync(x, 0, 4 * (size_t)c->lv(l).entries * sizeof(float), c->stream));
  uzawa_vcycle<float>(c, l, f, x);
}
void schur_inv32(hhg_ctx* c, int l, const float* r, float* out) { schur_apply<float>(c, l, r, out); }
void project_pressure32(hhg_ctx* c, int l, float* x) { project_pressure<float>(c, l, x); }
void project_pressure64(hhg_ctx* c, int l, double* x) { project_pressure<double>(c, l, x); }
void ensure_stokes_work(hhg_ctx* c, int l) {
  ensure_swork<double>(c, l);
  ensure_swork<float>(c, l);
}
double* stokes_work64(hhg_ctx* c, int l, int q) { return swork<double>(c->lv(l))[q].as<double>(); }
float* stokes_work32(hhg_ctx* c, int l, int q) { return swork<float>(c->lv(l))[q].as<float>(); }

}  // namespace host
}  // namespace hhg

extern "C" {

hhg_status hhg_set_mg_params(hhg_ctx* c, const hhg_mg_params* p) {
  return guard(c, [&] {
    c->drop_graphs();
    if (!p) THROW(HHG_ERR_ARG, "null params");
    if (p->smoother != HHG_SMOOTH_JACOBI && p->smoother != HHG_SMOOTH_CHEBYSHEV && p->smoother != HHG_SMOOTH_HYBRID_GS)
      THROW(HHG_ERR_ARG, "smoother");
    if (p->pre < 0 || p->post < 0 || p->pre + p->post == 0) THROW(HHG_ERR_ARG, "smoothing steps");
    if (!(p->omega > 0.0 && p->omega < 2.0)) THROW(HHG_ERR_ARG, "omega");
    if (!(p->cheby_lo > 0.0 && p->cheby_hi > p->cheby_lo)) THROW(HHG_ERR_ARG, "Chebyshev interval");
    if (p->power_iters < 1) THROW(HHG_ERR_ARG, "power_iters");
    if (p->coarse_coeff < HHG_COARSE_INJECT || p->coarse_coeff > HHG_COARSE_HARMONIC) THROW(HHG_ERR_ARG, "coarse_coeff");
    if (p->uzawa_pre < 0 || p->uzawa_post < 0 || p->uzawa_pre + p->uzawa_post == 0 || p->uzawa_extra < 0 ||
        p->uzawa_vsteps < 1 || !(p->uzawa_omega > 0.0 && p->uzawa_omega < 2.0))
      THROW(HHG_ERR_ARG, "Uzawa parameters");
    c->mg = *p;
  });
}

hhg_status hhg_mg_setup(hhg_ctx* c) {
  return guard(c, [&] {
    c->drop_graphs();
    need_ready(c, true);
    if (c->mg.coarse_coeff != HHG_COARSE_INJECT) {
      for (int l = c->level_max; l > c->level_min; --l) {
        LevelHost& Lf = c->lv(l);
        LevelHost& Lc = c->lv(l - 1);
        CK(launch_inject<double>(Lf.dev, Lc.dev, Lf.d_k64.as<double>(), Lc.d_k64.as<double>(), c->stream));
        CK(launch_average_coeff(Lf.dev, Lc.dev, Lf.d_k64.as<double>(), Lc.d_k64.as<double>(),
                                c->mg.coarse_coeff == HHG_COARSE_HARMONIC, c->stream));
        if (c->coeff_bf16)  // keep every copy of the coarse coefficient a BF16 value
          CK(launch_round_bf16(Lc.entries, Lc.d_k64.as<double>(), Lc.d_k32.as<float>(), Lc.d_k16.as<uint16_t>(),
                               c->stream));
        else
          CK(launch_convert<double, float>(Lc.entries, Lc.d_k64.as<double>(), Lc.d_k32.as<float>(), c->stream));
        Lc.lambda_set = false;
        Lc.stencil_version[0][0] = Lc.stencil_version[1][0] = -1;  // stored stencils of the old coefficient
      }
    }
    // (with the STORED variant the diagonal sweeps below also compute every level's stored
    // stencils, so that no V-cycle captured in a graph later has to)
    for (int l = c->level_min; l <= c->level_max; ++l) {
      compute_diag<double>(c, l);
      compute_diag<float>(c, l);
      LevelHost& L = c->lv(l);
      if (!L.lambda_set) {
        L.lambda_max = power_lambda(c, l, c->mg.power_iters);
        L.lambda_set = true;
      }
    }
    coarse_setup(c);
    if (c->prob.kind == HHG_STOKES) stokes_coarse_setup(c);
    wait_stream(c);
    c->mg_ready = true;
  });
}

hhg_status hhg_get_lambda_max(hhg_ctx* c, int level, double* lambda) {
  return guard(c, [&] {
    LevelHost& L = c->lv(level);
    if (!lambda) THROW(HHG_ERR_ARG, "null output");
    if (!L.lambda_set) THROW(HHG_ERR_STATE, "lambda_max not computed");
    *lambda = L.lambda_max;
  });
}

hhg_status hhg_set_lambda_max(hhg_ctx* c, int level, double lambda) {
  return guard(c, [&] {
    c->drop_graphs();
    LevelHost& L = c->lv(level);
    if (!(lambda > 0.0)) THROW(HHG_ERR_ARG, "lambda must be positive");
    L.lambda_max = lambda;
    L.lambda_set = true;
  });
}

hhg_status hhg_diagonal(hhg_ctx* c, int level, hhg_dtype dt, void* d) {
  return dispatch(c, dt, [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    need_ready(c, true);
    if (!d) THROW(HHG_ERR_ARG, "null output");
    ensure_work<T>(c, level);
    LevelHost& L = c->lv(level);
    SweepArgs<T> a{};
    a.x = work<T>(L)[1].template as<T>();
    a.out = (T*)d;
    sweep<T>(c, level, OP_DIAG, a, nullptr);
  });
}

hhg_status hhg_smooth(hhg_ctx* c, int level, hhg_dtype dt, int steps, const void* f, void* x) {
  return dispatch(c, dt, [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    mg_check(c);
    if (!f || !x || steps < 0) THROW(HHG_ERR_ARG, "bad arguments");
    smooth<T>(c, level, steps, (const T*)f, (T*)x);
  });
}

hhg_status hhg_prolongate_add(hhg_ctx* c, int fine, hhg_dtype dt, const void* xc, void* xf) {
  return dispatch(c, dt, [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    need_ready(c, false);
    if (fine <= c->level_min) THROW(HHG_ERR_ARG, "fine level must be above the coarsest level");
    if (!xc || !xf) THROW(HHG_ERR_ARG, "null buffer");
    CK(launch_prolong_add<T>(c->lv(fine).dev, c->lv(fine - 1).dev, (const T*)xc, (T*)xf, c->stream));
  });
}

hhg_status hhg_restrict(hhg_ctx* c, int fine, hhg_dtype dt, const void* rf, void* rc) {
  return dispatch(c, dt, [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    need_ready(c, false);
    if (fine <= c->level_min) THROW(HHG_ERR_ARG, "fine level must be above the coarsest level");
    if (!rf || !rc) THROW(HHG_ERR_ARG, "null buffer");
    restrict_op<T>(c, fine, (const T*)rf, (T*)rc);
  });
}

hhg_status hhg_vcycle(hhg_ctx* c, int level, hhg_dtype dt, const void* f, void* x) {
  return dispatch(c, dt, [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    mg_check(c);
    if (!f || !x) THROW(HHG_ERR_ARG, "null buffer");
    c->lv(level);
    vcycle<T>(c, level, (const T*)f, (T*)x);
  });
}

hhg_status hhg_stokes_apply(hhg_ctx* c, int level, hhg_dtype dt, const void* x, void* y) {
  return dispatch(c, dt, [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    need_stokes(c);
    if (!x || !y || x == y) THROW(HHG_ERR_ARG, "x and y must be distinct device buffers");
    c->lv(level);
    stokes_sweep<T>(c, level, OP_APPLY, nullptr, (const T*)x, (T*)y, false);
  });
}

hhg_status hhg_stokes_residual(hhg_ctx* c, int level, hhg_dtype dt, const void* f, const void* x, void* r,
                               double* norm2) {
  return dispatch(c, dt, [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    need_stokes(c);
    if (!f || !x || !r || x == r || f == r) THROW(HHG_ERR_ARG, "bad buffers");
    c->lv(level);
    const double n2 = stokes_sweep<T>(c, level, OP_RESID, (const T*)f, (const T*)x, (T*)r, norm2 != nullptr);
    if (norm2) *norm2 = n2;
  });
}

hhg_status hhg_carreau_viscosity(hhg_ctx* c, int level, const hhg_carreau* p, const void* u, void* mu) {
  return guard(c, [&] {
    need_ready(c, false);
    if (!p || !u || !mu) THROW(HHG_ERR_ARG, "null argument");
    if (!(p->eta0 > 0.0 && p->eta_inf >= 0.0 && p->kappa >= 0.0)) THROW(HHG_ERR_ARG, "Carreau parameters");
    carreau_viscosity(c, level, *p, (const double*)u, (double*)mu);
  });
}

double node_maxnorm(hhg_ctx* c, int l, int comps, const double* a, const double* b) {
  LevelHost& L = c->lv(l);
  CK(launch_node_maxnorm(L.d_mask_own.as<uint8_t>(), L.entries, comps, a, b, c->scratch.as<double>(),
                         c->scalar.as<double>(), c->stream));
  CK(cudaMemcpyAsync(c->pinned, c->scalar.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  wait_stream(c);
  return c->pinned[0];
}

hhg_status hhg_picard(hhg_ctx* c, const hhg_picard_opts* o, const void* f, void* x, hhg_picard_report* rep) {
  bool not_converged = false;
  hhg_status st = guard(c, [&] {
    if (!o || !f || !x) THROW(HHG_ERR_ARG, "null argument");
    need_stokes(c);
    const int l = o->level;
    if (l != c->level_max) THROW(HHG_ERR_ARG, "the Picard iteration runs on the finest level");
    LevelHost& L = c->lv(l);
    if (o->max_picard < 1 || !(o->picard_tol > 0.0) || !(o->final_rtol > 0.0) || !(o->step_rtol > 0.0) ||
        o->step_max_iter < 1)
      THROW(HHG_ERR_ARG, "Picard options");
    const auto t0 = std::chrono::steady_clock::now();
    if (!L.d_mu64.p || L.d_mu64.bytes < L.entries * sizeof(double)) CK(L.d_mu64.alloc(L.entries * sizeof(double)));
    ensure_swork<double>(c, l);
    double* mu = L.d_mu64.as<double>();
    double* xprev = swork<double>(L)[7].as<double>();
    const int64_t n4 = 4 * L.entries;
    auto check = [&](hhg_status s) {
      if (s != HHG_OK && s != HHG_ERR_NOT_CONVERGED) THROW(s, "%s", c->err.c_str());
    };
    auto update_mu = [&]() {
      carreau_viscosity(c, l, o->carreau, (const double*)x, mu);
      check(hhg_set_coefficient(c, mu, HHG_F64));
      check(hhg_mg_setup(c));
    };
    hhg_picard_report R{};
    update_mu();  // mu^0 = mu(u^0)
    hhg_solve_opts so{};
    so.method = HHG_SOLVE_STOKES_IR_MINRES;
    so.level = l;
    so.dt = HHG_F64;
    so.rtol = o->step_rtol;
    // one refinement step when the FP32 inner solve reaches step_rtol by itself; below what
    // FP32 reaches, refinement steps with inner solves to 1e-3 (at most 50)
    const bool exact_steps = o->step_rtol < 1e-6;
    so.max_iter = exact_steps ? 50 : 1;
    so.inner_rtol = exact_steps ? 1e-3 : o->step_rtol;
    so.inner_max_iter = o->step_max_iter;
    double change = 1.0;
    for (int it = 1; it <= o->max_picard; ++it) {
      CK(cudaMemcpyAsync(xprev, x, n4 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      hhg_solve_report sr{};
      check(hhg_solve(c, &so, f, x, &sr));
      R.minres_iterations += sr.inner_iterations;
      const double du = node_maxnorm(c, l, 3, (const double*)x, xprev);
      const double um = node_maxnorm(c, l, 3, (const double*)x, nullptr);
      change = um > 0.0 ? du / um : 0.0;
      R.picard_iterations = it;
      update_mu();  // mu^{n+1} = mu(u^{n+1})
      if (!std::isfinite(change)) THROW(HHG_ERR_NUMERIC, "non-finite velocity");
      if (change < o->picard_tol) break;
    }
    R.last_change = change;
    // final solve to final_rtol and the last viscosity update (Alg. 1)
    hhg_solve_opts fo = so;
    fo.rtol = o->final_rtol;
    fo.max_iter = 50;
    fo.inner_rtol = o->final_rtol < 1e-6 ? 1e-3 : std::min(1e-2, o->final_rtol);
    hhg_solve_report fr{};
    check(hhg_solve(c, &fo, f, x, &fr));
    R.minres_iterations += fr.inner_iterations;
    R.final_rel_residual = fr.rel_residual;
    carreau_viscosity(c, l, o->carreau, (const double*)x, mu);
    check(hhg_set_coefficient(c, mu, HHG_F64));
    R.mu_max = node_maxnorm(c, l, 1, mu, nullptr);
    {
      std::vector<double> h(L.entries);
      CK(cudaMemcpyAsync(h.data(), mu, L.entries * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      wait_stream(c);
      R.mu_min = *std::min_element(h.begin(), h.end());
    }
    R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    R.converged = change < o->picard_tol && fr.converged;
    if (rep) *rep = R;
    not_converged = !R.converged;
  });
  if (st == HHG_OK && not_converged) {
    c->err = "Picard iteration did not converge";
    return HHG_ERR_NOT_CONVERGED;
  }
  return st;
}

hhg_status hhg_solve(hhg_ctx* c, const hhg_solve_opts* o, const void* f, void* x, hhg_solve_report* rep) {
  bool not_converged = false;
  hhg_status st = guard(c, [&] {
    if (!o || !f || !x) THROW(HHG_ERR_ARG, "null argument");
    need_ready(c, true);
    const int l = o->level;
    c->lv(l);
    if (!(o->rtol > 0.0) || o->max_iter < 1) THROW(HHG_ERR_ARG, "rtol / max_iter");
    if (o->method != HHG_SOLVE_PCG_JACOBI) mg_check(c);
    const auto t0 = std::chrono::steady_clock::now();
    hhg_solve_report R{};
    if (o->method == HHG_SOLVE_PCG_JACOBI || o->method == HHG_SOLVE_MG_CG) {
      const bool mg = o->method == HHG_SOLVE_MG_CG;
      if (o->dt == HHG_F64) {
        if (!mg && !c->lv(l).dinv64.p) compute_diag<double>(c, l);
        CgResult cr = pcg<double>(c, l, mg, (const double*)f, (double*)x, o->rtol, o->max_iter);
        R.iterations = cr.iterations;
        R.residual0 = cr.r0;
        R.rel_residual = cr.rel;
        R.converged = cr.converged;
      } else if (o->dt == HHG_F32) {
        if (!mg && !c->lv(l).dinv32.p) compute_diag<float>(c, l);
        CgResult cr = pcg<float>(c, l, mg, (const float*)f, (float*)x, o->rtol, o->max_iter);
        R.iterations = cr.iterations;
        R.residual0 = cr.r0;
        R.rel_residual = cr.rel;
        R.converged = cr.converged;
      } else {
        THROW(HHG_ERR_ARG, "dtype");
      }
    } else if (o->method == HHG_SOLVE_MG) {
      auto run = [&](auto* tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        ensure_work<T>(c, l);
        T* r = work<T>(c->lv(l))[6].template as<T>();
        const double r0 = residual_op<T>(c, l, (const T*)f, (const T*)x, r, true);
        R.residual0 = std::sqrt(r0);
        double rr = r0;
        for (int it = 1; it <= o->max_iter && r0 > 0.0; ++it) {
          vcycle<T>(c, l, (const T*)f, (T*)x);
          rr = residual_op<T>(c, l, (const T*)f, (const T*)x, r, true);
          R.iterations = it;
          if (!std::isfinite(rr)) THROW(HHG_ERR_NUMERIC, "non-finite residual");
          if (std::sqrt(rr / r0) <= o->rtol) break;
        }
        R.rel_residual = r0 > 0.0 ? std::sqrt(rr / r0) : 0.0;
        R.converged = R.rel_residual <= o->rtol;
      };
      if (o->dt == HHG_F64)
        run((double*)nullptr);
      else if (o->dt == HHG_F32)
        run((float*)nullptr);
      else
        THROW(HHG_ERR_ARG, "dtype");
    } else if (o->method == HHG_SOLVE_IR_MG_CG) {
      if (o->dt != HHG_F64) THROW(HHG_ERR_ARG, "iterative refinement needs FP64 f and x");
      if (!(o->inner_rtol > 0.0 && o->inner_rtol < 1.0) || o->inner_max_iter < 1) THROW(HHG_ERR_ARG, "inner tol");
      ensure_work<double>(c, l);
      ensure_work<float>(c, l);
      LevelHost& L = c->lv(l);
      const int64_t n = 3 * L.entries;
      double* r64 = work<double>(L)[10].as<double>();
      float* r32 = work<float>(L)[10].as<float>();
      float* e32 = work<float>(L)[11].as<float>();
      const double r0 = residual_op<double>(c, l, (const double*)f, (const double*)x, r64, true);
      R.residual0 = std::sqrt(r0);
      double rr = r0;
      for (int it = 1; it <= o->max_iter && r0 > 0.0 && std::sqrt(rr / r0) > o->rtol; ++it) {
        CK(launch_convert<double, float>(n, r64, r32, c->stream));
        CK(cudaMemsetAsync(e32, 0, n * sizeof(float), c->stream));
        CgResult cr = pcg<float>(c, l, true, r32, e32, o->inner_rtol, o->inner_max_iter);
        R.inner_iterations += cr.iterations;
        CK(launch_add_f32_to_f64(n, e32, (double*)x, c->stream));
        rr = residual_op<double>(c, l, (const double*)f, (const double*)x, r64, true);
        R.iterations = it;
        if (!std::isfinite(rr)) THROW(HHG_ERR_NUMERIC, "non-finite residual");
      }
      R.rel_residual = r0 > 0.0 ? std::sqrt(rr / r0) : 0.0;
      R.converged = R.rel_residual <= o->rtol;
    } else if (o->method == HHG_SOLVE_STOKES_MINRES) {
      need_stokes(c);
      auto run = [&](auto* tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        MinresResult mr = minres<T>(c, l, (const T*)f, (T*)x, o->rtol, o->max_iter);
        project_pressure<T>(c, l, (T*)x);
        R.iterations = mr.iterations;
        R.residual0 = mr.r0;
        R.rel_residual = mr.rel;
        R.converged = mr.converged && mr.rel <= 10.0 * o->rtol;
      };
      if (o->dt == HHG_F64)
        run((double*)nullptr);
      else if (o->dt == HHG_F32)
        run((float*)nullptr);
      else
        THROW(HHG_ERR_ARG, "dtype");
    } else if (o->method == HHG_SOLVE_STOKES_IR_MINRES) {
      need_stokes(c);
      if (o->dt != HHG_F64) THROW(HHG_ERR_ARG, "iterative refinement needs FP64 f and x");
      if (!(o->inner_rtol > 0.0 && o->inner_rtol < 1.0) || o->inner_max_iter < 1) THROW(HHG_ERR_ARG, "inner tol");
      ensure_swork<double>(c, l);
      ensure_swork<float>(c, l);
      LevelHost& L = c->lv(l);
      const int64_t n = 4 * L.entries;
      double* r64 = swork<double>(L)[8].as<double>();
      float* r32 = swork<float>(L)[8].as<float>();
      float* e32 = swork<float>(L)[9].as<float>();
      const double r0 = stokes_sweep<double>(c, l, OP_RESID, (const double*)f, (const double*)x, r64, true);
      R.residual0 = std::sqrt(r0);
      double rr = r0;
      for (int it = 1; it <= o->max_iter && r0 > 0.0 && std::sqrt(rr / r0) > o->rtol; ++it) {
        CK(launch_convert<double, float>(n, r64, r32, c->stream));
        CK(cudaMemsetAsync(e32, 0, n * sizeof(float), c->stream));
        MinresResult mr = minres<float>(c, l, r32, e32, o->inner_rtol, o->inner_max_iter);
        R.inner_iterations += mr.iterations;
        CK(launch_add_f32_to_f64(n, e32, (double*)x, c->stream));
        rr = stokes_sweep<double>(c, l, OP_RESID, (const double*)f, (const double*)x, r64, true);
        R.iterations = it;
        if (!std::isfinite(rr)) THROW(HHG_ERR_NUMERIC, "non-finite residual");
      }
      project_pressure<double>(c, l, (double*)x);
      R.rel_residual = r0 > 0.0 ? std::sqrt(rr / r0) : 0.0;
      R.converged = R.rel_residual <= o->rtol;
    } else if (o->method == HHG_SOLVE_STOKES_UZAWA) {
      need_stokes(c);
      auto run = [&](auto* tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        MinresResult mr = uzawa_solve<T>(c, l, (const T*)f, (T*)x, o->rtol, o->max_iter);
        project_pressure<T>(c, l, (T*)x);
        R.iterations = mr.iterations;
        R.residual0 = mr.r0;
        R.rel_residual = mr.rel;
        R.converged = mr.converged;
      };
      if (o->dt == HHG_F64)
        run((double*)nullptr);
      else if (o->dt == HHG_F32)
        run((float*)nullptr);
      else
        THROW(HHG_ERR_ARG, "dtype");
    } else if (o->method == HHG_SOLVE_STOKES_IR_UZAWA) {
      need_stokes(c);
      if (o->dt != HHG_F64) THROW(HHG_ERR_ARG, "iterative refinement needs FP64 f and x");
      if (!(o->inner_rtol > 0.0 && o->inner_rtol < 1.0) || o->inner_max_iter < 1) THROW(HHG_ERR_ARG, "inner tol");
      ensure_swork<double>(c, l);
      ensure_swork<float>(c, l);
      LevelHost& L = c->lv(l);
      const int64_t n = 4 * L.entries;
      double* r64 = swork<double>(L)[8].as<double>();
      float* r32 = swork<float>(L)[8].as<float>();
      float* e32 = swork<float>(L)[9].as<float>();
      const double r0 = stokes_sweep<double>(c, l, OP_RESID, (const double*)f, (const double*)x, r64, true);
      R.residual0 = std::sqrt(r0);
      double rr = r0;
      for (int it = 1; it <= o->max_iter && r0 > 0.0 && std::sqrt(rr / r0) > o->rtol; ++it) {
        CK(launch_convert<double, float>(n, r64, r32, c->stream));
        CK(cudaMemsetAsync(e32, 0, n * sizeof(float), c->stream));
        MinresResult mr = uzawa_solve<float>(c, l, r32, e32, o->inner_rtol, o->inner_max_iter);
        R.inner_iterations += mr.iterations;
        CK(launch_add_f32_to_f64(n, e32, (double*)x, c->stream));
        rr = stokes_sweep<double>(c, l, OP_RESID, (const double*)f, (const double*)x, r64, true);
        R.iterations = it;
        if (!std::isfinite(rr)) THROW(HHG_ERR_NUMERIC, "non-finite residual");
      }
      project_pressure<double>(c, l, (double*)x);
      R.rel_residual = r0 > 0.0 ? std::sqrt(rr / r0) : 0.0;
      R.converged = R.rel_residual <= o->rtol;
    } else if (o->method == HHG_SOLVE_IR_FCG_LEARNED || o->method == HHG_SOLVE_IR_FCG ||
               o->method == HHG_SOLVE_STOKES_IR_FGCR_LEARNED || o->method == HHG_SOLVE_STOKES_IR_FGCR) {
      if (o->dt != HHG_F64) THROW(HHG_ERR_ARG, "iterative refinement needs FP64 f and x");
      const bool st = o->method == HHG_SOLVE_STOKES_IR_FGCR_LEARNED || o->method == HHG_SOLVE_STOKES_IR_FGCR;
      if (st) need_stokes(c);
      learned_ir(c, o, (const double*)f, (double*)x,
                 o->method == HHG_SOLVE_IR_FCG_LEARNED || o->method == HHG_SOLVE_STOKES_IR_FGCR_LEARNED, R);
    } else {
      THROW(HHG_ERR_ARG, "method");
    }
    wait_stream(c);
    R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (rep) *rep = R;
    not_converged = !R.converged;
  });
  if (st == HHG_OK && not_converged) {
    c->err = "maximum number of iterations reached";
    return HHG_ERR_NOT_CONVERGED;
  }
  return st;
}

}  // extern "C"
