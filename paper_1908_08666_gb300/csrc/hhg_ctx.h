// Host-side context of libhhgs, shared by hhg_host.cpp (mesh, levels, operator)
// and hhg_solve.cpp (smoothers, multigrid, solvers).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <set>
#include <string>
#include <thread>
#include <tuple>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "../../include/hhg.h"
#include "hhg_internal.h"
#include "hhg_launch.h"

namespace hhg {
namespace host {


struct DevMem {
  void* p = nullptr;
  size_t bytes = 0;
  DevMem() = default;
  DevMem(const DevMem&) = delete;
  DevMem& operator=(const DevMem&) = delete;
  ~DevMem() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t b) {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = b;
    if (b == 0) return cudaSuccess;
    return cudaMalloc(&p, b);
  }
  template <typename T>
  T* as() const {
    return (T*)p;
  }
};

struct HhgError {
  hhg_status st;
  std::string msg;
};

#define THROW(st, ...)                                      \
  do {                                                      \
    char _b[512];                                           \
    snprintf(_b, sizeof(_b), __VA_ARGS__);                  \
    throw HhgError{st, std::string(_b)};                    \
  } while (0)

#define CK(...)                                                                                      \
  do {                                                                                               \
    cudaError_t _e = (cudaError_t)(__VA_ARGS__);                                                         \
    if (_e != cudaSuccess) {                                                                         \
      hhg_status _s = (_e == cudaErrorMemoryAllocation) ? HHG_ERR_OOM : HHG_ERR_CUDA;                \
      THROW(_s, "%s failed: %s (%s:%d)", #__VA_ARGS__, cudaGetErrorString(_e), __FILE__, __LINE__);        \
    }                                                                                                \
  } while (0)

// Host -> device copy that has landed when it returns.  cudaMemcpy from pageable memory returns
// once the data is staged, with the DMA into device memory possibly still running on the legacy
// stream, which the library's non-blocking streams do not wait for; the synchronisation keeps a
// kernel queued next on a library stream from reading the old contents.
inline void copy_h2d(void* dst, const void* src, size_t bytes) {
  CK(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice));
  CK(cudaStreamSynchronize(cudaStreamLegacy));
}

template <typename T>
void upload(DevMem& d, const std::vector<T>& h) {
  CK(d.alloc(h.size() * sizeof(T)));
  if (!h.empty()) copy_h2d(d.p, h.data(), h.size() * sizeof(T));
}

struct Vec3d {
  double x, y, z;
};


struct KeyHash {
  size_t operator()(const std::array<int64_t, 3>& k) const {
    size_t h = 1469598103934665603ull;
    for (int q = 0; q < 3; ++q) h = (h ^ (size_t)k[q]) * 1099511628211ull;
    return h;
  }
};

struct LevelHost {
  int level = 0, n = 0;
  int64_t nt = 0, entries = 0;
  std::vector<int32_t> tiles_int, tiles_all, tiles_lin, tiles_pair, tiles3, gs_chunks;
  int32_t gs_ptr[9] = {0};
  std::vector<int64_t> skel_entries;
  std::vector<int32_t> skel_ptr;
  std::vector<SkelInc> skel_inc;
  std::vector<int8_t> skel_dir;
  std::vector<int8_t> skel_support;  // number of macro vertices spanning the node's primitive
  std::vector<std::array<int64_t, 3>> skel_key;
  std::vector<FaceItem> face_items;
  std::vector<int32_t> face_nodes, ev_nodes, dir_nodes;
  std::vector<FaceItem> face_items_all;
  std::vector<int32_t> face_nodes_all, ev_all;
  uint32_t face_mask[4] = {0, 0, 0, 0};
  std::vector<uint8_t> mask, mask_own;  // owned copy of a free node / of any node
  std::vector<double> lumped;           // lumped P1 mass of every entry's node
  std::vector<int64_t> entry_to_unique, unique_first;
  std::vector<int8_t> unique_dir;
  int64_t nunique = 0, nfree = 0;
  // restriction lists for the skeleton nodes of this level as the coarse level
  std::vector<int32_t> rptr;
  std::vector<int64_t> rent;
  std::vector<double> rw;
  // device
  DevMem d_tiles_pair, d_tiles3, d_gs_chunks, d_skel_entries;
  DevMem d_tiles_int, d_tiles_all, d_tiles_lin, d_skel_ptr, d_skel_inc, d_skel_dir, d_mask, d_first, d_e2u;
  DevMem d_face_items, d_face_nodes, d_ev_nodes, d_dir_nodes, d_acc32, d_acc64;
  DevMem d_face_items_all, d_face_nodes_all, d_ev_all;
  DevMem d_mask_own, d_invm64, d_invm32;  // owned-node mask; inverse lumped mass
  DevMem d_mass64, d_mass32;              // lumped mass
  DevMem d_sdiag64, d_sdiag32;            // Stokes: diagonal of -C (pressure stabilisation)
  DevMem sw64[10], sw32[10];               // Stokes work vectors (4*E)
  // Stokes all-at-once multigrid: pressure restriction lists over all fine nodes (this
  // level as the coarse one), Uzawa work vectors (4*E), dense coarse saddle inverse
  bool rlist_p = false;
  DevMem d_rptr_p, d_rent_p, d_rw64_p, d_rw32_p;
  DevMem uz64[4], uz32[4];
  int nscdof = 0;
  DevMem d_scdof, d_scinv64, d_scinv32, su64, su32;
  // Carreau viscosity: per-macro slope operators and skeleton patch lists (built on first use)
  std::vector<SlopeOp> slope;
  DevMem d_pnode, d_pptr, d_pent, d_pdx;
  PatchLists plist{};
  bool carreau_ready = false;
  DevMem d_mu64;  // viscosity of the Picard iteration
  DevMem d_rptr, d_rent, d_rw64, d_rw32;
  DevMem d_mc64, d_mc32;
  DevMem d_k64, d_k32;
  DevMem d_k16;  // BF16 bits of the coefficient (BF16 coefficient mode)
  // stored stencil blocks of the macro-interior rows (STORED variant), per precision, and the
  // (coefficient, problem) versions they were computed for
  DevMem stencil32, stencil64;
  int64_t stencil_version[2][2] = {{-1, -1}, {-1, -1}};
  std::vector<MacroStencil<double>> st64;
  std::vector<MacroStencil<float>> st32;
  std::vector<NodalConsts<double>> nc64;  // element stiffness per macro (NODAL variant)
  std::vector<NodalConsts<float>> nc32;
  LevelDev dev{};
  // multigrid / solver state (hhg_mg_setup and the solvers)
  DevMem d_udir;                    // int8 Dirichlet flag per unique node
  DevMem dinv64, dinv32;            // inverse point diagonal, 3*E
  double lambda_max = 0.0;          // of D^{-1} A, power iteration
  bool lambda_set = false;
  DevMem w64[12], w32[12];          // work vectors, 3*E each
  DevMem u64, u32;                  // two unique-node vectors, 2 * 3*U
  int ncdof = 0;                    // dense coarse solve: free DoFs, their index in the unique vector,
  DevMem d_cdof, d_cinv64, d_cinv32;  // and the inverse of the coarse matrix restricted to them
};

// Node grid of a level whose nodes lie on an axis-aligned uniform lattice (learned
// preconditioner): voxel g = (z * H + y) * W + x.
struct LearnGrid {
  int D = 0, H = 0, W = 0;
  int64_t V = 0, nfree = 0, nnode = 0;  // voxels; with a free node; with a node
  int64_t coeff_version = -1;  // of the log-coefficient feature
  DevMem gent, gfree, e2g, efree, logk;
  DevMem lw[16];  // FP32 work vectors (4*E) of the learned preconditioner and its Krylov solvers
  DevMem lw64[2]; // FP64 work vectors (4*E) of the pair collection
  // Stokes: inverse diagonal of the features (velocity point diagonal, pressure Schur
  // surrogate; 4*E) and the coefficient version it was computed for
  DevMem dinv4;
  int64_t dinv4_version = -1;
  // flexible GCR search directions p_j and K p_j (4*E each; the solver restarts after
  // GCR_DIRS directions)
  static constexpr int GCR_DIRS = 30;
  DevMem gcr_p[GCR_DIRS], gcr_q[GCR_DIRS];
};

// Learned preconditioner: network parameters, optimiser state, training pairs, buffers.
struct LearnState {
  bool have_params = false;
  int adam_step = 0;
  DevMem params, grad, m, v, fwd, bwd;  // LN_NPARAM floats; packed fragments LN_LAYERS * LN_PACK words
  DevMem fwd_u, bwd_u;                   // tcgen05 operands, LN_LAYERS * LN_UMMA bytes
  int conv_kernel = 0;                   // 0 warp MMA, 1 tcgen05 per tile, 2 TMA + tcgen05 pipeline
  int64_t conv_wait_polls = -1;          // bound of kernel 1's wait for its MMAs (-1: the default)
  std::map<int, std::unique_ptr<LearnGrid>> grids;
  // training pairs of one level: inputs (ln_pair_in(pair_nc) BF16 per voxel) and targets
  // (pair_nc FP32), pair_nc = components of the problem they came from
  int pair_level = -1, pair_nc = 3;
  int pair_coarsen = 0;  // the coarsening the pairs were stored with (their grid: pair_level - it)
  int coarsen = 0;       // the network runs on the node grid this many levels below the solve's
  // per-pair factor of the targets in training (Stokes: 1 / RMS of the pair's target, so
  // that every pair weighs the same; elasticity: 1)
  std::vector<float> pair_tscale;
  int64_t pair_cap = 0, pair_count = 0;
  DevMem pin, ptg;
  // activation buffers (16-channel BF16), outputs, gradients, partial sums
  int64_t act_voxels = 0;
  DevMem act[4], gb[2], out, tgt;
  DevMem wpart, bpart, dpart, dscal;
  // statistics of the preconditioner applications
  int64_t applications = 0, fallbacks = 0;
  double alpha_sum = 0.0, alpha_min = 0.0, alpha_max = 0.0, gain_sum = 0.0;
};


}  // namespace host
}  // namespace hhg

using namespace hhg;
using namespace hhg::host;

struct hhg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int64_t timeout_ms = 120000;
  std::string err;
  // macro mesh
  std::vector<Vec3d> xyz;
  std::vector<std::array<int64_t, 4>> tets;
  std::set<std::array<int64_t, 3>> dir_faces;
  std::set<std::array<int64_t, 2>> dir_edges;
  std::set<int64_t> dir_verts;
  bool have_mesh = false;
  int level_min = 2, level_max = -1;
  std::vector<std::unique_ptr<LevelHost>> levels;  // index = level
  hhg_problem prob{};
  bool have_problem = false;
  bool have_coeff = false;
  int64_t coeff_version = 0;  // incremented by hhg_set_coefficient
  int64_t problem_version = 0;  // incremented by hhg_set_problem
  bool coeff_bf16 = false;     // the coefficient was given in BF16 (k16 holds it on every level)
  std::unique_ptr<LearnState> learn;
  OpFlags flags{1, 0, 0};
  // macro-interior kernel choice (hhg_set_interior_kernel): 0 automatic, 1 shared-memory tile,
  // 2 one launch per macro, 3 all macros in one launch
  int interior_kernel = 0;
  int sm_count = 0;  // SMs of the device (read on first use)
  int strain_degree = 1;  // least-squares strain-rate fit on the skeleton (hhg_set_strain_fit)
  DevMem scratch;   // reduction partials
  DevMem scalar;    // device scalars
  double* pinned = nullptr;
  // host-buffer apply (hhg_apply_host)
  DevMem hx, hy;
  // kernel timing (hhg_profile): event pairs per part (0 interior, 1 skeleton)
  hhg_mg_params mg{HHG_SMOOTH_CHEBYSHEV, 2, 2, 2.0 / 3.0, 1.0 / 8.0, 1.1, 15, HHG_COARSE_INJECT, 3, 3, 2, 2, 0.5};
  bool mg_ready = false;
  bool prof = false;
  // side streams of a sweep: aux[0] runs the face-node skeleton kernels, aux[1] every
  // second macro's interior launch, aux[2] the edge/vertex kernel, aux[3] the Dirichlet
  // rows; all forked from and joined back into `stream` by events
  cudaStream_t aux[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[4] = {nullptr, nullptr, nullptr, nullptr};
  // CUDA graphs of "x = 0; one V-cycle for f" per (precision, level, f, x), replayed by
  // the solvers; dropped whenever the multigrid data change (hhg_mg_setup and friends)
  std::map<std::tuple<int, int, const void*, void*>, cudaGraphExec_t> vc_graphs;
  cudaStream_t cap_stream = nullptr;  // capture stream (the caller's may be the legacy one)
  bool graphs_ok = true;              // false after a failed capture: launch directly
  void drop_graphs() {
    for (auto& kv : vc_graphs)
      if (kv.second) cudaGraphExecDestroy(kv.second);  // null: the first-use marker
    vc_graphs.clear();
  }
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::array<cudaEvent_t, 2>> prof_ev[2];
  int64_t prof_launches[2] = {0, 0};
  ~hhg_ctx() {
    drop_graphs();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (pinned) cudaFreeHost(pinned);
    for (auto st : aux)
      if (st) cudaStreamDestroy(st);
    if (ev_fork) cudaEventDestroy(ev_fork);
    for (auto e : ev_join)
      if (e) cudaEventDestroy(e);
    for (auto e : ev_pool) cudaEventDestroy(e);
    for (int q = 0; q < 2; ++q)
      for (auto& pr : prof_ev[q]) {
        cudaEventDestroy(pr[0]);
        cudaEventDestroy(pr[1]);
      }
  }
  cudaEvent_t take_event() {
    if (!ev_pool.empty()) {
      cudaEvent_t e = ev_pool.back();
      ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) throw HhgError{HHG_ERR_CUDA, "cudaEventCreate failed"};
    return e;
  }
  LevelHost& lv(int l) {
    if (l < level_min || l > level_max || !levels[l]) THROW(HHG_ERR_ARG, "level %d not built", l);
    return *levels[l];
  }
};


namespace hhg {
namespace host {

// Slots of the partial-sum scratch: the largest sweep's blocks, and at least the partials of two
// dot-product launches in a row (1024 blocks each: the Stokes inner product over the velocity and
// the pressure components writes both before reducing them together).
inline int64_t max_partials(hhg_ctx* c) {
  int64_t mx = 2 * 1024;
  for (int l = c->level_min; l <= c->level_max; ++l) {
    const LevelHost& L = *c->levels[l];
    mx = std::max<int64_t>(mx, (int64_t)std::max(L.tiles_lin.size(), L.tiles3.size()) * (int64_t)c->tets.size() +
                                   (L.face_nodes_all.size() + 127) / 128 + L.ev_all.size() + 8);
  }
  return mx;
}

inline void wait_stream(hhg_ctx* c) {
  cudaEvent_t ev;
  CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t e = cudaEventRecord(ev, c->stream);
  if (e != cudaSuccess) {
    cudaEventDestroy(ev);
    CK(e);
  }
  const auto t0 = std::chrono::steady_clock::now();
  while (true) {
    e = cudaEventQuery(ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) {
      cudaEventDestroy(ev);
      CK(e);
    }
    const auto us =
        std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
    if (us > 1000 * c->timeout_ms) {
      cudaEventDestroy(ev);
      THROW(HHG_ERR_TIMEOUT, "stream did not finish within %lld ms", (long long)c->timeout_ms);
    }
    // poll without sleeping for the first 2 ms (short solver waits), then every 50 us
    if (us < 2000)
      std::this_thread::yield();
    else
      std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  cudaEventDestroy(ev);
}

// bounded wait that creates nothing: polls the stream itself
inline void wait_stream_noalloc(hhg_ctx* c) {
  const auto t0 = std::chrono::steady_clock::now();
  while (true) {
    const cudaError_t e = cudaStreamQuery(c->stream);
    if (e == cudaSuccess) return;
    if (e != cudaErrorNotReady) CK(e);
    const auto ms =
        std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
    if (ms > c->timeout_ms) THROW(HHG_ERR_TIMEOUT, "stream did not finish within %lld ms", (long long)c->timeout_ms);
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

template <typename F>
hhg_status guard(hhg_ctx* c, F&& f) {
  if (!c) return HHG_ERR_ARG;
  try {
    CK(cudaSetDevice(c->device));
    f();
    return HHG_OK;
  } catch (const HhgError& e) {
    c->err = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    c->err = "host allocation failed";
    return HHG_ERR_OOM;
  } catch (...) {
    c->err = "unknown error";
    return HHG_ERR_STATE;
  }
}

inline void need_ready(hhg_ctx* c, bool coeff) {
  if (!c->have_mesh || c->level_max < 0) THROW(HHG_ERR_STATE, "mesh/levels not set");
  if (!c->have_problem) THROW(HHG_ERR_STATE, "problem not set");
  if (coeff && !c->have_coeff) THROW(HHG_ERR_STATE, "coefficient not set");
}

template <typename T>
const T* kptr(LevelHost& L);
template <>
inline const double* kptr<double>(LevelHost& L) {
  return L.d_k64.as<double>();
}
template <>
inline const float* kptr<float>(LevelHost& L) {
  return L.d_k32.as<float>();
}
template <typename T>
const MacroStencil<T>* stencils(LevelHost& L);
template <>
inline const MacroStencil<double>* stencils<double>(LevelHost& L) {
  return L.st64.data();
}
template <>
inline const MacroStencil<float>* stencils<float>(LevelHost& L) {
  return L.st32.data();
}
template <typename T>
const NodalConsts<T>* nodal_consts(LevelHost& L);
template <>
inline const NodalConsts<double>* nodal_consts<double>(LevelHost& L) {
  return L.nc64.data();
}
template <>
inline const NodalConsts<float>* nodal_consts<float>(LevelHost& L) {
  return L.nc32.data();
}
template <typename T>
const MacroConsts<T>* consts_dev(LevelHost& L);
template <>
inline const MacroConsts<double>* consts_dev<double>(LevelHost& L) {
  return L.d_mc64.as<MacroConsts<double>>();
}
template <>
inline const MacroConsts<float>* consts_dev<float>(LevelHost& L) {
  return L.d_mc32.as<MacroConsts<float>>();
}

// Fork the side streams from `stream` (they start after everything issued so far).
inline void fork_side_streams(hhg_ctx* c) {
  if (!c->aux[0]) {
    for (auto& st : c->aux) CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    for (auto& e : c->ev_join) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  CK(cudaEventRecord(c->ev_fork, c->stream));
  for (auto st : c->aux) CK(cudaStreamWaitEvent(st, c->ev_fork, 0));
}

// Join the side streams back into `stream`.
inline void join_side_streams(hhg_ctx* c) {
  for (int q = 0; q < 4; ++q) {
    CK(cudaEventRecord(c->ev_join[q], c->aux[q]));
    CK(cudaStreamWaitEvent(c->stream, c->ev_join[q], 0));
  }
}

// One operator sweep on a level.  The macro-interior launches (one per macro) alternate
// between `stream` and aux[1] so that the tail of one overlaps the next, and the skeleton
// kernels run concurrently on aux[0] (they write disjoint entries and their own partial-sum
// slots); both side streams are joined back into `stream`.  With profiling on, the
// interior span (fork to join of the interior launches) and the skeleton span are timed.
// The stored stencil blocks of a level in precision T (STORED variant), computed on the stream
// when the coefficient or the problem changed since they were last computed.
template <typename T>
const T* stored_stencil(hhg_ctx* c, LevelHost& L) {
  const int q = std::is_same<T, float>::value ? 0 : 1;
  DevMem& S = q == 0 ? L.stencil32 : L.stencil64;
  if (!S.p) CK(S.alloc((size_t)135 * L.entries * sizeof(T)));
  if (L.stencil_version[q][0] != c->coeff_version || L.stencil_version[q][1] != c->problem_version) {
    CK(launch_store_stencil<T>(L.dev, L.st64.data(), c->flags, L.d_k64.as<double>(), S.as<T>(), c->stream));
    L.stencil_version[q][0] = c->coeff_version;
    L.stencil_version[q][1] = c->problem_version;
  }
  return S.as<T>();
}

// The operator flags of a sweep on level L, with the launch shape of its macro-interior part:
// all macros in one launch when chosen (interior kernel 3) or, automatically, when the mesh has
// several macros and one macro's launch (FP32 point pairs or one point per thread) fills
// fewer than two waves of four 128-thread blocks per SM.
inline OpFlags sweep_flags(hhg_ctx* c, const LevelHost& L, bool pairs) {
  OpFlags f = c->flags;
  f.batch = 0;
  if (f.stored || f.nodal || f.tile || c->interior_kernel == 2) return f;
  if (c->interior_kernel == 3) {
    f.batch = 1;
    return f;
  }
  if (L.dev.nmacro < 2) return f;
  if (c->sm_count == 0) CK(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device));
  const int per_macro = pairs ? L.dev.ntiles_pair : L.dev.ntiles_lin;
  f.batch = per_macro < 2 * 4 * c->sm_count;
  return f;
}

template <typename T>
void sweep(hhg_ctx* c, int level, OpKind op, SweepArgs<T> a, double* norm2) {
  LevelHost& L = c->lv(level);
  a.k = kptr<T>(L);
  if (c->flags.stored) a.stencil = stored_stencil<T>(c, L);
  if (std::is_same<T, float>::value && c->coeff_bf16) a.k16 = L.d_k16.as<uint16_t>();
  if (norm2) a.partial = c->scratch.as<double>();
  if (!c->aux[0]) {
    for (auto& st : c->aux) CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    for (auto& e : c->ev_join) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  std::array<cudaEvent_t, 2> pi{}, ps{};
  if (c->prof) {
    pi = {c->take_event(), c->take_event()};
    ps = {c->take_event(), c->take_event()};
    CK(cudaEventRecord(pi[0], c->stream));
  }
  CK(cudaEventRecord(c->ev_fork, c->stream));
  for (auto st : c->aux) CK(cudaStreamWaitEvent(st, c->ev_fork, 0));
  // interior: all macros in one launch, or macro m on stream (m even) or aux[1] (m odd); partial
  // slots in macro order
  const OpFlags fl = sweep_flags(c, L, std::is_same<T, float>::value);
  int64_t used = 0;
  if (fl.batch) {
    CK(launch_sweep_batched<T>(L.dev, consts_dev<T>(L), op, fl, a, c->stream, 0, &used));
  } else {
    for (int m = 0; m < L.dev.nmacro; ++m) {
      int64_t cnt = 0;
      CK(launch_sweep_macro<T>(L.dev, stencils<T>(L), nodal_consts<T>(L), m, op, c->flags, a,
                               m % 2 ? c->aux[1] : c->stream, used, &cnt));
      used += cnt;
    }
  }
  if (c->prof) {
    CK(cudaEventRecord(c->ev_join[1], c->aux[1]));
    CK(cudaStreamWaitEvent(c->stream, c->ev_join[1], 0));
    CK(cudaEventRecord(pi[1], c->stream));
    CK(cudaEventRecord(ps[0], c->aux[0]));
  }
  int64_t used_sk = 0;
  CK(launch_sweep<T>(L.dev, stencils<T>(L), consts_dev<T>(L), op, c->flags, a, c->aux[0], 2, used, &used_sk,
                     c->aux[2], c->aux[3]));
  if (c->prof) {
    for (int q = 2; q < 4; ++q) {  // the skeleton span ends when all three skeleton streams have
      CK(cudaEventRecord(c->ev_join[q], c->aux[q]));
      CK(cudaStreamWaitEvent(c->aux[0], c->ev_join[q], 0));
    }
    CK(cudaEventRecord(ps[1], c->aux[0]));
    c->prof_ev[0].push_back(pi);
    c->prof_ev[1].push_back(ps);
    c->prof_launches[0] += L.dev.ntiles_lin > 0 ? (fl.batch ? (L.dev.nmacro + 65534) / 65535 : L.dev.nmacro) : 0;
    c->prof_launches[1] += (L.dev.nface_nodes > 0) + (L.dev.nev > 0) + (L.dev.ndir > 0);
  }
  for (int q = 0; q < 4; ++q) {
    CK(cudaEventRecord(c->ev_join[q], c->aux[q]));
    CK(cudaStreamWaitEvent(c->stream, c->ev_join[q], 0));
  }
  const int64_t np = used + used_sk;
  if (norm2) {
    CK(launch_reduce(c->scratch.as<double>(), np, c->scalar.as<double>(), c->stream));
    CK(cudaMemcpyAsync(c->pinned, c->scalar.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    wait_stream(c);
    *norm2 = c->pinned[0];
  }
}


}  // namespace host
}  // namespace hhg
