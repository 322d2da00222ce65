// Learned preconditioner of libhhgs (not part of the paper): a 4-layer 3x3x3 conv net
// with 16 channels on the node grid, trained on the GPU on residual/error pairs that the
// multigrid solver itself produces, and used inside a flexible Krylov solver as a
// correction after the multigrid cycle: flexible CG after the V-cycle for elasticity
// (nc = 3 unknowns per node), flexible GCR after the inexact Uzawa V-cycle for Stokes
// (nc = 4: velocity and pressure).  Kernels in hhg_learn.cu; conventions in hhg_learn.h.
//
// Preconditioner application for a residual r (FP32), K the system operator, MG one cycle:
//   z0 = a0 MG(r), a0 = the energy-optimal step length (z0, r) / (z0, K z0) of the cycle's
//        output for elasticity; a0 = 1 for Stokes (the Uzawa cycle is itself a convergent
//        iteration, and K is indefinite),
//   r1 = r - K z0       (the residual the step leaves),
//   c  = s D^-1 N(features(r1, z0, log k))   (network correction),
//   z  = a z0 + b c,  (a, b) minimising over span{z0, c} the energy norm of the error
//        K^-1 r - z (elasticity) or the residual norm |r - K z|_2 (Stokes) (2x2 normal
//        equations).
// Hence an application never does worse (in that norm) than the best multiple of the
// cycle's output alone, and
// the network is not rewarded for what a rescaling of z0 would do (the Krylov solvers are
// invariant to that); when the 2x2 system is singular or not finite the application falls
// back to z = z0.
//
// Training pairs: for an error e, one multigrid step gives z0 = a0 MG(K e) (a0 as above), the
// remaining error e1 = e - z0 (Stokes: pressure shifted to zero mean, the constant being
// invisible to K) and residual r1 = K e1; the pair is (features(r1, z0), D e1 / s).  The
// errors are either random (further steps continue from e1) or the errors of the plain
// multigrid-preconditioned Krylov iterates (hhg_learn_collect_cg).
//
// Coarse-grid mode (elasticity, hhg_learn_set_coarsening(q)): the network sees r1
// restricted q levels and z0 injected there, with that level's diagonal and log k; its
// correction is prolongated back before the 2x2 combination, and pairs are stored on the
// coarse grid with the error injected.
#include <cmath>
#include <cstring>
#include <functional>

#include "hhg_ctx.h"
#include "hhg_learn.h"
#include "hhg_solver.h"

namespace {

using namespace hhg;
using namespace hhg::host;

// work vectors of LearnGrid::lw
// (CR, CZ, CE, CC: restricted residual, injected correction and error, and the network's
// correction, on the coarser levels of the coarse-grid mode)
enum { LW_Z0 = 0, LW_AZ0, LW_R1, LW_C, LW_AC, LW_R, LW_Z, LW_AZ, LW_P, LW_Q, LW_X, LW_XS, LW_E, LW_CR, LW_CZ, LW_CE };

LearnState& state(hhg_ctx* c) {
  if (!c->learn) c->learn.reset(new LearnState());
  return *c->learn;
}

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double uniform01(uint64_t& s) { return ((splitmix64(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

// standard normal by the Box-Muller transform
double normal(uint64_t& s) {
  const double u1 = uniform01(s), u2 = uniform01(s);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

// nearest BF16 value (ties to even) of a float
float round_bf16(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u = ((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16) << 16;
  float y;
  std::memcpy(&y, &u, 4);
  return y;
}

void need_elasticity(hhg_ctx* c) {
  need_ready(c, true);
  if (c->prob.kind != HHG_ELASTICITY) THROW(HHG_ERR_UNSUPPORTED, "flexible CG needs an elasticity problem");
}

bool is_stokes(hhg_ctx* c) { return c->prob.kind == HHG_STOKES; }
int ncomp(hhg_ctx* c) { return is_stokes(c) ? 4 : 3; }

// the system operator K of the problem kind, its inner product over the unique free DoFs,
// its residual (returns |r|^2) and one multigrid cycle from zero, all FP32
void sys_apply(hhg_ctx* c, int l, const float* x, float* y) {
  if (is_stokes(c))
    stokes_apply32(c, l, x, y);
  else
    apply32(c, l, x, y);
}
double sys_dot(hhg_ctx* c, int l, const float* a, const float* b) {
  return is_stokes(c) ? stokes_dot32(c, l, a, b) : dot32(c, l, a, b);
}
double sys_residual(hhg_ctx* c, int l, const float* f, const float* x, float* r) {
  return is_stokes(c) ? stokes_residual32(c, l, f, x, r) : residual32(c, l, f, x, r);
}
void sys_mg(hhg_ctx* c, int l, const float* r, float* z) {
  if (is_stokes(c))
    uzawa_zero32(c, l, r, z);
  else
    vcycle_zero32(c, l, r, z);
}

void need_params(LearnState& S) {
  if (!S.have_params) THROW(HHG_ERR_STATE, "network parameters not set (hhg_learn_init or hhg_learn_set_params)");
}

void repack(hhg_ctx* c, LearnState& S) {
  CK(launch_pack(S.params.as<float>(), S.fwd.as<uint32_t>(), S.bwd.as<uint32_t>(), c->stream));
  CK(launch_pack_umma(S.params.as<float>(), S.fwd_u.p, S.bwd_u.p, c->stream));
}

// after a wait on the stream: a tensor-core convolution whose bounded wait ran out disables
// that kernel for the context (the warp-MMA convolution takes over) and fails the call
void check_conv(LearnState& S) {
  int flag = 0;
  CK(conv_take_error(&flag));
  if (flag) {
    S.conv_kernel = 0;
    THROW(HHG_ERR_TIMEOUT, "tensor-core convolution timed out (switched to the warp-MMA kernel)");
  }
}

void alloc_params(hhg_ctx* c, LearnState& S) {
  if (S.params.p) return;
  const size_t nb = LN_NPARAM * sizeof(float);
  CK(S.params.alloc(nb));
  CK(S.grad.alloc(nb));
  CK(S.m.alloc(nb));
  CK(S.v.alloc(nb));
  CK(S.fwd.alloc(LN_LAYERS * LN_PACK * sizeof(uint32_t)));
  CK(S.bwd.alloc(LN_LAYERS * LN_PACK * sizeof(uint32_t)));
  CK(S.fwd_u.alloc((size_t)LN_LAYERS * LN_UMMA));
  CK(S.bwd_u.alloc((size_t)LN_LAYERS * LN_UMMA));
  CK(S.dscal.alloc(8 * sizeof(double)));
}

void reset_adam(hhg_ctx* c, LearnState& S) {
  CK(cudaMemsetAsync(S.m.p, 0, S.m.bytes, c->stream));
  CK(cudaMemsetAsync(S.v.p, 0, S.v.bytes, c->stream));
  S.adam_step = 0;
}

void upload_params(hhg_ctx* c, LearnState& S, const std::vector<float>& h) {
  alloc_params(c, S);
  CK(cudaMemcpyAsync(S.params.p, h.data(), LN_NPARAM * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  wait_stream(c);  // h is the caller's or a temporary buffer
  repack(c, S);
  reset_adam(c, S);
  S.have_params = true;
}

// activation buffers for V voxels (outputs and targets of up to 4 channels)
void ensure_acts(hhg_ctx* c, LearnState& S, int64_t V) {
  if (S.act_voxels >= V) return;
  const size_t b16 = (size_t)V * LN_C * 2;
  for (auto& a : S.act) CK(a.alloc(b16));
  for (auto& g : S.gb) CK(g.alloc(b16));
  CK(S.out.alloc((size_t)V * 4 * sizeof(float)));
  CK(S.tgt.alloc((size_t)V * 4 * sizeof(float)));
  CK(S.dpart.alloc((size_t)std::max<int64_t>(mse_partials(V), 1) * sizeof(double)));
  S.act_voxels = V;
}

void ensure_grad_scratch(hhg_ctx* c, LearnState& S, GridShape s) {
  const size_t wp = (size_t)wgrad_partials(s) * LN_WSIZE * sizeof(float);
  if (S.wpart.bytes < wp) CK(S.wpart.alloc(wp));
  const size_t bp = (size_t)bgrad_partials(s.voxels()) * 16 * sizeof(float);
  if (S.bpart.bytes < bp) CK(S.bpart.alloc(bp));
}

const float* layer_bias(LearnState& S, int l) { return S.params.as<float>() + (int64_t)l * LN_LSIZE + LN_WSIZE; }
const uint32_t* layer_fwd(LearnState& S, int l) { return S.fwd.as<uint32_t>() + (int64_t)l * LN_PACK; }
const uint32_t* layer_bwd(LearnState& S, int l) { return S.bwd.as<uint32_t>() + (int64_t)l * LN_PACK; }
const void* layer_fwd_u(LearnState& S, int l) { return (const char*)S.fwd_u.p + (size_t)l * LN_UMMA; }
const void* layer_bwd_u(LearnState& S, int l) { return (const char*)S.bwd_u.p + (size_t)l * LN_UMMA; }

// one convolution with the context's kernel choice (bwd: input-gradient weights)
void conv(hhg_ctx* c, LearnState& S, int l, bool bwd, const void* X, const float* bias, void* Y, float* Yf, int nf,
          const void* mask, GridShape s, int relu) {
  const uint32_t* wp = bwd ? layer_bwd(S, l) : layer_fwd(S, l);
  const void* wu = bwd ? layer_bwd_u(S, l) : layer_fwd_u(S, l);
  if (S.conv_kernel == 2)
    CK(launch_conv_tma(X, wu, bias, Y, Yf, nf, mask, s, relu, c->stream));
  else
    CK(launch_conv(X, wp, S.conv_kernel == 1 ? wu : nullptr, bias, Y, Yf, nf, mask, s, relu, c->stream,
                   S.conv_wait_polls));
}

// forward pass from act[0]: act[1..3] = hidden activations, out = the first nout FP32
// output channels
void forward(hhg_ctx* c, LearnState& S, GridShape s, float* out, int nout) {
  for (int l = 0; l < LN_LAYERS; ++l) {
    const bool last = l == LN_LAYERS - 1;
    conv(c, S, l, false, S.act[l].p, layer_bias(S, l), last ? nullptr : S.act[l + 1].p, last ? out : nullptr, nout,
         nullptr, s, last ? 0 : 1);
  }
}

// inference with two activation buffers (act[0] holds the input; act[0] and act[1] alternate)
void forward_inference(hhg_ctx* c, LearnState& S, GridShape s, float* out, int nout) {
  for (int l = 0; l < LN_LAYERS; ++l) {
    const bool last = l == LN_LAYERS - 1;
    conv(c, S, l, false, S.act[l & 1].p, layer_bias(S, l), last ? nullptr : S.act[(l + 1) & 1].p,
         last ? out : nullptr, nout, nullptr, s, last ? 0 : 1);
  }
}

// backward pass after forward(): MSE over nout channels against tgt into *loss (device),
// gradients into S.grad
void backward(hhg_ctx* c, LearnState& S, GridShape s, const float* out, const float* tgt, int nout, double* loss) {
  const int64_t V = s.voxels();
  ensure_grad_scratch(c, S, s);
  CK(launch_mse(out, tgt, V, nout, S.gb[0].p, S.dpart.as<double>(), loss, c->stream));
  int cur = 0;
  for (int l = LN_LAYERS - 1; l >= 0; --l) {
    float* gW = S.grad.as<float>() + (int64_t)l * LN_LSIZE;
    CK(launch_wgrad(S.act[l].p, S.gb[cur].p, S.wpart.as<float>(), gW, s, c->stream));
    CK(launch_bgrad(S.gb[cur].p, V, S.bpart.as<float>(), gW + LN_WSIZE, c->stream));
    if (l > 0) {
      conv(c, S, l, true, S.gb[cur].p, nullptr, S.gb[cur ^ 1].p, nullptr, 0, S.act[l].p, s, 0);
      cur ^= 1;
    }
  }
}

// Node grid of level l: every entry's lattice point must sit on an axis-aligned uniform
// lattice (spacing = the smallest nonzero coordinate step of the macros' lattice vectors).
LearnGrid& grid(hhg_ctx* c, int l) {
  LearnState& S = state(c);
  LevelHost& L = c->lv(l);
  auto it = S.grids.find(l);
  LearnGrid* G = it == S.grids.end() ? nullptr : it->second.get();
  if (!G) {
    const int n = L.n;
    const int M = (int)c->tets.size();
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300}, h[3] = {1e300, 1e300, 1e300};
    for (int m = 0; m < M; ++m)
      for (int q = 0; q < 4; ++q) {
        const Vec3d& v = c->xyz[c->tets[m][q]];
        const double p[3] = {v.x, v.y, v.z};
        for (int a = 0; a < 3; ++a) {
          lo[a] = std::min(lo[a], p[a]);
          hi[a] = std::max(hi[a], p[a]);
        }
        if (q == 0) continue;
        const Vec3d& v0 = c->xyz[c->tets[m][0]];
        const double d[3] = {(v.x - v0.x) / n, (v.y - v0.y) / n, (v.z - v0.z) / n};
        for (int a = 0; a < 3; ++a)
          if (std::fabs(d[a]) > 1e-12 * (1.0 + std::fabs(hi[a] - lo[a]))) h[a] = std::min(h[a], std::fabs(d[a]));
      }
    int dims[3];
    auto steps = [&](double x, int a) {
      const double s = x / h[a];
      const double r = std::round(s);
      if (std::fabs(s - r) > 1e-6) THROW(HHG_ERR_UNSUPPORTED, "mesh nodes do not lie on an axis-aligned uniform lattice");
      return (int64_t)r;
    };
    for (int a = 0; a < 3; ++a) {
      if (!(h[a] < 1e299)) THROW(HHG_ERR_UNSUPPORTED, "degenerate macro mesh for the node grid");
      dims[a] = (int)steps(hi[a] - lo[a], a) + 1;
    }
    const int64_t V = (int64_t)dims[0] * dims[1] * dims[2];
    if (V > 8 * L.nunique + 64) THROW(HHG_ERR_UNSUPPORTED, "node grid too sparse (%lld voxels for %lld nodes)",
                                      (long long)V, (long long)L.nunique);
    std::unique_ptr<LearnGrid> ng(new LearnGrid());
    G = ng.get();
    G->W = dims[0];
    G->H = dims[1];
    G->D = dims[2];
    G->V = V;
    std::vector<int64_t> gent(V, -1), e2g(L.entries, -1);
    std::vector<uint8_t> gfree(V, 0), efree(L.entries, 0);
    for (int m = 0; m < M; ++m) {
      int64_t o[3], s1[3], s2[3], s3[3];
      const Vec3d& v0 = c->xyz[c->tets[m][0]];
      const double p0[3] = {v0.x, v0.y, v0.z};
      const Vec3d* vv[3] = {&c->xyz[c->tets[m][1]], &c->xyz[c->tets[m][2]], &c->xyz[c->tets[m][3]]};
      int64_t* sv[3] = {s1, s2, s3};
      for (int a = 0; a < 3; ++a) o[a] = steps(p0[a] - lo[a], a);
      for (int q = 0; q < 3; ++q) {
        const double p[3] = {vv[q]->x, vv[q]->y, vv[q]->z};
        for (int a = 0; a < 3; ++a) sv[q][a] = steps((p[a] - p0[a]) / n, a);
      }
      for (int k = 0; k <= n; ++k)
        for (int j = 0; j <= n - k; ++j)
          for (int i = 0; i <= n - k - j; ++i) {
            const int64_t e = (int64_t)m * L.nt + lattice_index(n, i, j, k);
            int64_t ix[3];
            for (int a = 0; a < 3; ++a) ix[a] = o[a] + i * s1[a] + j * s2[a] + k * s3[a];
            const int64_t g = (ix[2] * dims[1] + ix[1]) * dims[0] + ix[0];
            if (g < 0 || g >= V) THROW(HHG_ERR_UNSUPPORTED, "node outside the node grid");
            const int64_t u = L.entry_to_unique[e];
            e2g[e] = g;
            efree[e] = L.unique_dir[u] ? 0 : 1;
            if (gent[g] < 0) {
              gent[g] = e;
              gfree[g] = efree[e];
            } else if (L.entry_to_unique[gent[g]] != u) {
              THROW(HHG_ERR_UNSUPPORTED, "two nodes share a grid point");
            }
          }
    }
    for (int64_t g = 0; g < V; ++g) {
      G->nfree += gfree[g];
      G->nnode += gent[g] >= 0;
    }
    upload(G->gent, gent);
    upload(G->gfree, gfree);
    upload(G->e2g, e2g);
    upload(G->efree, efree);
    CK(G->logk.alloc(V * sizeof(float)));
    S.grids[l] = std::move(ng);
  }
  if (c->have_coeff && G->coeff_version != c->coeff_version) {
    // log-coefficient feature: log k at the voxel's node minus its mean over the nodes
    std::vector<double> k(L.entries);
    CK(cudaMemcpyAsync(k.data(), L.d_k64.p, L.entries * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    wait_stream(c);
    std::vector<int64_t> gent(G->V);
    CK(cudaMemcpy(gent.data(), G->gent.p, G->V * sizeof(int64_t), cudaMemcpyDeviceToHost));
    std::vector<float> lk(G->V, 0.f);
    double sum = 0.0;
    int64_t cnt = 0;
    for (int64_t g = 0; g < G->V; ++g)
      if (gent[g] >= 0) {
        const double kv = k[gent[g]];
        if (!(kv > 0.0)) THROW(HHG_ERR_NUMERIC, "coefficient must be positive for the learned preconditioner");
        sum += std::log(kv);
        ++cnt;
      }
    const double mean = cnt ? sum / cnt : 0.0;
    for (int64_t g = 0; g < G->V; ++g)
      if (gent[g] >= 0) lk[g] = (float)(std::log(k[gent[g]]) - mean);
    copy_h2d(G->logk.p, lk.data(), G->V * sizeof(float));
    G->coeff_version = c->coeff_version;
  }
  return *G;
}

// work vector q of the grid's level (4*E floats: room for either problem kind)
float* lwork(hhg_ctx* c, LearnGrid& G, int l, int q) {
  if (!G.lw[q].p) {
    const size_t b = 4 * (size_t)c->lv(l).entries * sizeof(float);
    CK(G.lw[q].alloc(b));
    CK(cudaMemsetAsync(G.lw[q].p, 0, b, c->stream));
  }
  return G.lw[q].as<float>();
}

int64_t sys_n(hhg_ctx* c, int l) { return ncomp(c) * c->lv(l).entries; }

void copy32(hhg_ctx* c, int l, const float* src, float* dst) {
  CK(cudaMemcpyAsync(dst, src, sys_n(c, l) * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
}

// Inverse diagonal D^-1 of the features (nc*E): elasticity the point diagonal of A; Stokes
// that of the velocity block, then 1 / (m_i / mu_i + (-C)_ii) for the pressure (recomputed
// when the coefficient changes).
const float* sys_dinv(hhg_ctx* c, int l, LearnGrid& G) {
  if (!is_stokes(c)) return dinv32(c, l);
  if (!G.dinv4.p || G.dinv4_version != c->coeff_version) {
    const int64_t E = c->lv(l).entries;
    if (!G.dinv4.p) CK(G.dinv4.alloc(4 * (size_t)E * sizeof(float)));
    float* d = G.dinv4.as<float>();
    CK(cudaMemcpyAsync(d, dinv32(c, l), 3 * (size_t)E * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemsetAsync(d + 3 * E, 0, (size_t)E * sizeof(float), c->stream));
    CK(launch_add_const<float>(E, 1.f, d + 3 * E, c->stream));
    schur_inv32(c, l, d + 3 * E, d + 3 * E);
    G.dinv4_version = c->coeff_version;
  }
  return G.dinv4.as<float>();
}

// Scales of the features, as sums of squares and DoF counts: D z0 over the free
// velocity-like DoFs (S.dscal[0]) and, for Stokes, over the pressure (S.dscal[2]; its
// diagonal differs from the velocity's by orders of magnitude, so it gets its own scale)
struct FeatureScale {
  const double* su;
  double cu;
  const double* sp;
  double cp;
};

FeatureScale feature_scales(hhg_ctx* c, int l, LearnState& S, LearnGrid& G, const float* z0, const float* dinv) {
  const int nc = ncomp(c);
  const int64_t E = c->lv(l).entries;
  if (!S.dscal.p) CK(S.dscal.alloc(8 * sizeof(double)));
  if (S.dpart.bytes < (size_t)mse_partials(G.V) * sizeof(double))
    CK(S.dpart.alloc((size_t)mse_partials(G.V) * sizeof(double)));
  double* ss = S.dscal.as<double>();
  CK(launch_feature_norm(G.V, E, nc, 0, 3, G.gent.as<int64_t>(), G.gfree.as<uint8_t>(), z0, dinv,
                         S.dpart.as<double>(), ss, c->stream));
  FeatureScale f{ss, std::max(1.0, 3.0 * (double)G.nfree), nullptr, 1.0};
  if (nc == 4) {
    CK(launch_feature_norm(G.V, E, nc, 3, 4, G.gent.as<int64_t>(), G.gfree.as<uint8_t>(), z0, dinv,
                           S.dpart.as<double>(), ss + 2, c->stream));
    f.sp = ss + 2;
    f.cp = std::max(1.0, (double)G.nnode);
  }
  return f;
}

// Coarse-grid mode (elasticity, S.coarsen = q > 0): the fields the network sees at level
// l - q, r1 restricted (P^T, q times) and z0 (and e1) injected; returns the level-(l - q)
// vectors (work vectors of the intermediate levels; e1 nullable).
struct CoarseFields {
  const float *r1, *z0, *e1;
};

CoarseFields to_coarse(hhg_ctx* c, int l, int q, const float* r1, const float* z0, const float* e1) {
  CoarseFields f{r1, z0, e1};
  for (int lev = l; lev > l - q; --lev) {
    LearnGrid& Gn = grid(c, lev - 1);
    float* rn = lwork(c, Gn, lev - 1, LW_CR);
    float* zn = lwork(c, Gn, lev - 1, LW_CZ);
    restrict32(c, lev, f.r1, rn);
    inject32(c, lev, f.z0, zn);
    f.r1 = rn;
    f.z0 = zn;
    if (f.e1) {
      float* en = lwork(c, Gn, lev - 1, LW_CE);
      inject32(c, lev, f.e1, en);
      f.e1 = en;
    }
  }
  return f;
}

void need_coarse_level(hhg_ctx* c, int l, int q) {
  if (q > 0 && is_stokes(c)) THROW(HHG_ERR_UNSUPPORTED, "the coarse-grid mode is built for elasticity");
  if (l - q < c->level_min) THROW(HHG_ERR_ARG, "coarsening %d below the coarsest level from level %d", q, l);
}

// Elasticity: scale the V-cycle correction z0 (and K z0) to its energy-optimal length for
// the residual r, z0 <- a0 z0 with a0 = (z0, r) / (z0, K z0) (unchanged when that is not
// finite).  Stokes: no scaling.
void scale_mg_step(hhg_ctx* c, int l, const float* r, float* z0, float* az0) {
  if (is_stokes(c)) return;
  const int64_t n = sys_n(c, l);
  const double num = sys_dot(c, l, z0, r), den = sys_dot(c, l, z0, az0);
  const double a0 = (den > 0.0 && std::isfinite(num / den)) ? num / den : 1.0;
  CK(launch_axpby<float>(n, (float)a0, z0, 0.f, z0, c->stream));
  CK(launch_axpby<float>(n, (float)a0, az0, 0.f, az0, c->stream));
}

// z and az = K z of one preconditioner application (see the file comment); use_net =
// false: z = z0 = MG(r), unscaled.  Returns the weight b / a of the correction in z = a z0 + b c.
double precondition(hhg_ctx* c, int l, const float* r, float* z, float* az, bool use_net) {
  LearnState& S = state(c);
  LearnGrid& G = grid(c, l);
  const bool st = is_stokes(c);
  const int nc = ncomp(c);
  const int64_t E = c->lv(l).entries, n = nc * E;
  float* z0 = lwork(c, G, l, LW_Z0);
  float* az0 = lwork(c, G, l, LW_AZ0);
  sys_mg(c, l, r, z0);
  sys_apply(c, l, z0, az0);
  if (!use_net) {
    copy32(c, l, z0, z);
    copy32(c, l, az0, az);
    return 0.0;
  }
  need_params(S);
  const int q = S.coarsen;
  need_coarse_level(c, l, q);
  float* r1 = lwork(c, G, l, LW_R1);
  float* cc = lwork(c, G, l, LW_C);
  float* acc = lwork(c, G, l, LW_AC);
  scale_mg_step(c, l, r, z0, az0);
  copy32(c, l, r, r1);
  CK(launch_axpby<float>(n, -1.f, az0, 1.f, r1, c->stream));
  // the network's level (l itself unless coarse-grid mode) and its inputs there
  const int lc = l - q;
  LearnGrid& Gc = grid(c, lc);
  const int64_t Ec = c->lv(lc).entries;
  const CoarseFields cf = q ? to_coarse(c, l, q, r1, z0, nullptr) : CoarseFields{r1, z0, nullptr};
  const float* dinv = sys_dinv(c, lc, Gc);
  float* ccn = q ? lwork(c, Gc, lc, LW_C) : cc;
  ensure_acts(c, S, Gc.V);
  const FeatureScale fs = feature_scales(c, lc, S, Gc, cf.z0, dinv);
  CK(launch_features(Gc.V, Ec, nc, Gc.gent.as<int64_t>(), Gc.gfree.as<uint8_t>(), Gc.logk.as<float>(), cf.r1, cf.z0,
                     nullptr, dinv, fs.su, fs.cu, fs.sp, fs.cp, S.act[0].p, nullptr, nullptr, c->stream));
  forward_inference(c, S, GridShape{1, Gc.D, Gc.H, Gc.W}, S.out.as<float>(), nc);
  CK(launch_grid_to_lib(Ec, nc, Gc.e2g.as<int64_t>(), Gc.efree.as<uint8_t>(), S.out.as<float>(), dinv, fs.su, fs.cu,
                        fs.sp, fs.cp, ccn, c->stream));
  // coarse-grid mode: prolongate the correction back to level l
  const float* cur = ccn;
  for (int lev = lc + 1; lev <= l; ++lev) {
    float* nx = lev == l ? cc : lwork(c, grid(c, lev), lev, LW_C);
    CK(cudaMemsetAsync(nx, 0, 3 * (size_t)c->lv(lev).entries * sizeof(float), c->stream));
    prolong_add32(c, lev, cur, nx);
    cur = nx;
  }
  sys_apply(c, l, cc, acc);
  // optimal a, b: [m11 m12; m12 m22] (a, b) = (rv, rc) with the energy inner product
  // (u, K v) (elasticity) or the residual one (K u, K v) (Stokes)
  const double m11 = st ? sys_dot(c, l, az0, az0) : sys_dot(c, l, z0, az0);
  const double rv = st ? sys_dot(c, l, az0, r) : sys_dot(c, l, z0, r);
  const double m12 = st ? sys_dot(c, l, acc, az0) : sys_dot(c, l, cc, az0);
  const double m22 = st ? sys_dot(c, l, acc, acc) : sys_dot(c, l, cc, acc);
  const double rc = st ? sys_dot(c, l, acc, r) : sys_dot(c, l, cc, r);
  const double det = m11 * m22 - m12 * m12;
  // without c: the best multiple of z0, with a0 = rv / m11 (fallback a = 1 keeps z0 itself)
  const double a_only = (m11 > 0.0 && std::isfinite(rv / m11)) ? rv / m11 : 1.0;
  double a = 1.0, b = 0.0;
  if (m11 > 0.0 && m22 > 0.0 && det > 1e-6 * m11 * m22 && std::isfinite(det) && std::isfinite(rc)) {
    a = (rv * m22 - m12 * rc) / det;
    b = (m11 * rc - m12 * rv) / det;
    if (!(std::isfinite(a) && std::isfinite(b)) || a <= 0.0) {
      a = 1.0;
      b = 0.0;
    }
  }
  const double w = b / a;
  S.applications++;
  if (b == 0.0) S.fallbacks++;
  S.alpha_sum += w;
  S.alpha_min = S.applications == 1 ? w : std::min(S.alpha_min, w);
  S.alpha_max = S.applications == 1 ? w : std::max(S.alpha_max, w);
  // extra reduction of the squared norm over the best multiple of z0, relative to that
  // step's own (a_only rv)
  if (m11 > 0.0 && a_only * rv > 0.0) S.gain_sum += (a * rv + b * rc - a_only * rv) / (a_only * rv);
  copy32(c, l, z0, z);
  copy32(c, l, az0, az);
  if (b != 0.0) {
    CK(launch_axpby<float>(n, (float)b, cc, (float)a, z, c->stream));
    CK(launch_axpby<float>(n, (float)b, acc, (float)a, az, c->stream));
  }
  return w;
}

// Flexible CG (one-term A-orthogonalisation: p_k = z_k - (z_k, A p_{k-1}) / (p_{k-1}, A p_{k-1}) p_{k-1})
// on A x = f in FP32; A p follows from the preconditioner's A z by the same recurrence.
// hook (nullable) is called with the iterate before every preconditioner application.
SolverResult fcg(hhg_ctx* c, int l, const float* f, float* x, double rtol, int max_iter, bool use_net,
                 const std::function<void(const float*)>& hook = nullptr) {
  LearnGrid& G = grid(c, l);
  const int64_t n = 3 * c->lv(l).entries;
  float* r = lwork(c, G, l, LW_R);
  float* z = lwork(c, G, l, LW_Z);
  float* az = lwork(c, G, l, LW_AZ);
  float* p = lwork(c, G, l, LW_P);
  float* q = lwork(c, G, l, LW_Q);
  SolverResult res;
  const double r0 = residual32(c, l, f, x, r);
  res.r0 = std::sqrt(r0);
  if (!std::isfinite(r0)) THROW(HHG_ERR_NUMERIC, "non-finite initial residual");
  if (r0 == 0.0) {
    res.converged = true;
    return res;
  }
  if (hook) hook(x);
  precondition(c, l, r, z, az, use_net);
  copy32(c, l, z, p);
  copy32(c, l, az, q);
  double rp = dot32(c, l, r, p);
  double rr = r0;
  for (int it = 1; it <= max_iter; ++it) {
    const double pq = dot32(c, l, p, q);
    if (!(pq > 0.0) || !std::isfinite(pq)) THROW(HHG_ERR_NUMERIC, "FCG breakdown (p.Ap = %g)", pq);
    const double alpha = rp / pq;
    CK(launch_axpby<float>(n, (float)alpha, p, 1.f, x, c->stream));
    CK(launch_axpby<float>(n, (float)(-alpha), q, 1.f, r, c->stream));
    rr = dot32(c, l, r, r);
    res.iterations = it;
    if (!std::isfinite(rr)) THROW(HHG_ERR_NUMERIC, "non-finite residual");
    if (std::sqrt(rr / r0) <= rtol) {
      res.converged = true;
      break;
    }
    if (hook) hook(x);
    precondition(c, l, r, z, az, use_net);
    const double beta = -dot32(c, l, z, q) / pq;
    CK(launch_axpby<float>(n, 1.f, z, (float)beta, p, c->stream));
    CK(launch_axpby<float>(n, 1.f, az, (float)beta, q, c->stream));
    rp = dot32(c, l, r, p);
  }
  res.rel = std::sqrt(rr / r0);
  return res;
}

constexpr int GCR_RESTART = LearnGrid::GCR_DIRS;

// Flexible GCR (generalised conjugate residual with a variable preconditioner; Eisenstat,
// Elman and Schultz, SIAM J. Numer. Anal. 20 (1983), in its flexible form) on the Stokes
// system K x = f in FP32: each preconditioned direction p = z (with q = K p from the
// preconditioner) is made (q, q_j) = 0 against the stored directions by modified
// Gram-Schmidt, and the step x += alpha p, alpha = (r, q) / (q, q), minimises |r|_2 along
// it; after GCR_RESTART directions the stored ones are dropped.  hook (nullable) is
// called with the iterate before every preconditioner application.
SolverResult fgcr(hhg_ctx* c, int l, const float* f, float* x, double rtol, int max_iter, bool use_net,
                  const std::function<void(const float*)>& hook = nullptr) {
  LearnGrid& G = grid(c, l);
  const int64_t n = sys_n(c, l);
  float* r = lwork(c, G, l, LW_R);
  float* z = lwork(c, G, l, LW_Z);
  float* az = lwork(c, G, l, LW_AZ);
  std::vector<double> qq(GCR_RESTART, 0.0);
  SolverResult res;
  const double r0 = sys_residual(c, l, f, x, r);
  res.r0 = std::sqrt(r0);
  if (!std::isfinite(r0)) THROW(HHG_ERR_NUMERIC, "non-finite initial residual");
  if (r0 == 0.0) {
    res.converged = true;
    return res;
  }
  double rr = r0;
  int m = 0;
  for (int it = 1; it <= max_iter; ++it) {
    if (hook) hook(x);
    precondition(c, l, r, z, az, use_net);
    if (m == GCR_RESTART) m = 0;
    for (DevMem* d : {&G.gcr_p[m], &G.gcr_q[m]})
      if (!d->p) CK(d->alloc(4 * (size_t)c->lv(l).entries * sizeof(float)));
    float* p = G.gcr_p[m].as<float>();
    float* q = G.gcr_q[m].as<float>();
    copy32(c, l, z, p);
    copy32(c, l, az, q);
    for (int j = 0; j < m; ++j) {
      const double beta = sys_dot(c, l, q, G.gcr_q[j].as<float>()) / qq[j];
      CK(launch_axpby<float>(n, (float)(-beta), G.gcr_p[j].as<float>(), 1.f, p, c->stream));
      CK(launch_axpby<float>(n, (float)(-beta), G.gcr_q[j].as<float>(), 1.f, q, c->stream));
    }
    const double qn = sys_dot(c, l, q, q);
    if (!(qn > 0.0) || !std::isfinite(qn)) THROW(HHG_ERR_NUMERIC, "FGCR breakdown (|K p|^2 = %g)", qn);
    const double alpha = sys_dot(c, l, r, q) / qn;
    CK(launch_axpby<float>(n, (float)alpha, p, 1.f, x, c->stream));
    CK(launch_axpby<float>(n, (float)(-alpha), q, 1.f, r, c->stream));
    qq[m++] = qn;
    rr = sys_dot(c, l, r, r);
    res.iterations = it;
    if (!std::isfinite(rr)) THROW(HHG_ERR_NUMERIC, "non-finite residual");
    if (std::sqrt(rr / r0) <= rtol) {
      res.converged = true;
      break;
    }
  }
  res.rel = std::sqrt(rr / r0);
  return res;
}

// One training pair from the error e (library layout): r = K e, z0 = a0 MG(r) (elasticity:
// the energy-optimal a0; Stokes: a0 = 1), e1 = e - z0 (Stokes: pressure shifted to zero
// mean), r1 = r - K z0; stores
// (features(r1, z0), D e1 / s).  e1_out (nullable) receives e1.  Uses the work vectors
// Z0, AZ0, R1, C, AC.
void store_pair(hhg_ctx* c, int l, const float* e, float* e1_out) {
  LearnState& S = state(c);
  LearnGrid& G = grid(c, l);
  const int nc = ncomp(c);
  if (S.pair_level != l) THROW(HHG_ERR_STATE, "reserve pair storage for level %d first", l);
  if (S.pair_nc != nc) THROW(HHG_ERR_STATE, "pair storage was reserved for another problem kind");
  if (S.pair_coarsen != S.coarsen) THROW(HHG_ERR_STATE, "pair storage was reserved with another coarsening");
  if (S.pair_count >= S.pair_cap) THROW(HHG_ERR_ARG, "pair storage full (%lld)", (long long)S.pair_cap);
  const int64_t E = c->lv(l).entries, n = nc * E;
  float* z0 = lwork(c, G, l, LW_Z0);
  float* az0 = lwork(c, G, l, LW_AZ0);
  float* r1 = lwork(c, G, l, LW_R1);
  float* r = lwork(c, G, l, LW_C);
  float* e1 = lwork(c, G, l, LW_AC);
  const float* dinv = sys_dinv(c, l, G);
  sys_apply(c, l, e, r);
  sys_mg(c, l, r, z0);
  sys_apply(c, l, z0, az0);
  scale_mg_step(c, l, r, z0, az0);
  copy32(c, l, r, r1);
  CK(launch_axpby<float>(n, -1.f, az0, 1.f, r1, c->stream));
  copy32(c, l, e, e1);
  CK(launch_axpby<float>(n, -1.f, z0, 1.f, e1, c->stream));
  if (nc == 4) project_pressure32(c, l, e1);
  // the pair lives on the network's grid (level l - coarsening)
  const int q = S.pair_coarsen;
  const int lc = l - q;
  LearnGrid& Gc = grid(c, lc);
  const CoarseFields cf = q ? to_coarse(c, l, q, r1, z0, e1) : CoarseFields{r1, z0, e1};
  const float* dinv_c = q ? sys_dinv(c, lc, Gc) : dinv;
  const FeatureScale fs = feature_scales(c, lc, S, Gc, cf.z0, dinv_c);
  const int64_t p = S.pair_count++;
  float* tg = S.ptg.as<float>() + (size_t)p * Gc.V * nc;
  CK(launch_features(Gc.V, c->lv(lc).entries, nc, Gc.gent.as<int64_t>(), Gc.gfree.as<uint8_t>(), Gc.logk.as<float>(),
                     cf.r1, cf.z0, cf.e1, dinv_c, fs.su, fs.cu, fs.sp, fs.cp, nullptr,
                     (char*)S.pin.p + (size_t)p * Gc.V * ln_pair_in(nc) * 2, tg, c->stream));
  float ts = 1.f;
  if (nc == 4) {
    // the 2x2 combination fixes the size of the correction, so only its direction matters:
    // each Stokes pair's target is trained at unit RMS (the cycle's step is much smaller
    // than the error for some pairs, whose raw targets would otherwise dominate the loss)
    double* ss = S.dscal.as<double>() + 4;
    if (S.dpart.bytes < (size_t)mse_partials((int64_t)Gc.V * nc) * sizeof(double))
      CK(S.dpart.alloc((size_t)mse_partials((int64_t)Gc.V * nc) * sizeof(double)));
    CK(launch_sumsq((int64_t)Gc.V * nc, tg, S.dpart.as<double>(), ss, c->stream));
    CK(cudaMemcpyAsync(c->pinned, ss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    wait_stream(c);
    const double ms = c->pinned[0] / ((double)Gc.V * nc);
    ts = (ms > 0.0 && std::isfinite(ms)) ? (float)(1.0 / std::sqrt(ms)) : 1.f;
  }
  S.pair_tscale[p] = ts;
  if (e1_out) copy32(c, l, e1, e1_out);
}

}  // namespace

namespace hhg {
namespace host {

// FP64 iterative refinement around the FP32 flexible Krylov solver with the learned
// preconditioner (use_net = false: the same solver with the plain multigrid cycle):
// flexible CG for the elasticity methods, flexible GCR for the Stokes ones (pressure
// shifted to zero mean at the end)
void learned_ir(hhg_ctx* c, const hhg_solve_opts* o, const double* f, double* x, bool use_net, hhg_solve_report& R) {
  const bool st = o->method == HHG_SOLVE_STOKES_IR_FGCR || o->method == HHG_SOLVE_STOKES_IR_FGCR_LEARNED;
  if (st)
    need_stokes_problem(c);
  else
    need_elasticity(c);
  mg_ready_check(c);
  const int l = o->level;
  if (use_net) need_params(state(c));
  if (!(o->inner_rtol > 0.0 && o->inner_rtol < 1.0) || o->inner_max_iter < 1) THROW(HHG_ERR_ARG, "inner tol");
  const int64_t n = sys_n(c, l);
  double* r64;
  float *r32, *e32;
  if (st) {
    ensure_stokes_work(c, l);
    r64 = stokes_work64(c, l, 8);
    r32 = stokes_work32(c, l, 8);
    e32 = stokes_work32(c, l, 9);
  } else {
    ensure_work64(c, l);
    r64 = work64(c, l, 10);
    r32 = work32(c, l, 10);
    e32 = work32(c, l, 11);
  }
  auto residual = [&] { return st ? stokes_residual64(c, l, f, x, r64) : residual64(c, l, f, x, r64); };
  const double r0 = residual();
  R.residual0 = std::sqrt(r0);
  double rr = r0;
  for (int it = 1; it <= o->max_iter && r0 > 0.0 && std::sqrt(rr / r0) > o->rtol; ++it) {
    CK(launch_convert<double, float>(n, r64, r32, c->stream));
    CK(cudaMemsetAsync(e32, 0, n * sizeof(float), c->stream));
    SolverResult cr = st ? fgcr(c, l, r32, e32, o->inner_rtol, o->inner_max_iter, use_net)
                         : fcg(c, l, r32, e32, o->inner_rtol, o->inner_max_iter, use_net);
    R.inner_iterations += cr.iterations;
    CK(launch_add_f32_to_f64(n, e32, x, c->stream));
    rr = residual();
    R.iterations = it;
    if (!std::isfinite(rr)) THROW(HHG_ERR_NUMERIC, "non-finite residual");
  }
  if (st) project_pressure64(c, l, x);
  R.rel_residual = r0 > 0.0 ? std::sqrt(rr / r0) : 0.0;
  R.converged = R.rel_residual <= o->rtol;
  if (use_net) check_conv(state(c));
}

}  // namespace host
}  // namespace hhg

extern "C" {

int64_t hhg_learn_num_params(void) { return LN_NPARAM; }

hhg_status hhg_learn_init(hhg_ctx* c, uint64_t seed) {
  return guard(c, [&] {
    LearnState& S = state(c);
    std::vector<float> h(LN_NPARAM, 0.f);
    uint64_t s = seed ^ 0x6C6561726E6564ull;
    const int nc = ncomp(c);
    for (int l = 0; l < LN_LAYERS; ++l) {
      const int cin = l == 0 ? ln_cin(nc) : LN_C;
      const int cout = l == LN_LAYERS - 1 ? nc : LN_C;
      const double sd = std::sqrt(2.0 / (LN_TAPS * cin)) * (l == LN_LAYERS - 1 ? 0.1 : 1.0);
      float* W = h.data() + (int64_t)l * LN_LSIZE;
      for (int t = 0; t < LN_TAPS; ++t)
        for (int i = 0; i < cin; ++i)
          for (int o = 0; o < cout; ++o) W[(t * LN_C + i) * LN_C + o] = round_bf16((float)(sd * normal(s)));
    }
    upload_params(c, S, h);
  });
}

hhg_status hhg_learn_set_conv_kernel(hhg_ctx* c, int kernel) {
  return guard(c, [&] {
    if (kernel < 0 || kernel > 2) THROW(HHG_ERR_ARG, "conv kernel 0 (warp MMA), 1 (tcgen05) or 2 (TMA + tcgen05)");
    state(c).conv_kernel = kernel;
  });
}

hhg_status hhg_learn_set_conv_wait(hhg_ctx* c, int64_t polls) {
  return guard(c, [&] { state(c).conv_wait_polls = polls < 0 ? -1 : polls; });
}

hhg_status hhg_learn_set_coarsening(hhg_ctx* c, int levels) {
  return guard(c, [&] {
    if (levels < 0 || levels > 3) THROW(HHG_ERR_ARG, "coarsening 0..3");
    if (levels > 0 && c->prob.kind != HHG_ELASTICITY)
      THROW(HHG_ERR_UNSUPPORTED, "the coarse-grid mode is built for elasticity");
    state(c).coarsen = levels;
  });
}

hhg_status hhg_learn_get_params(hhg_ctx* c, float* params_host, int64_t n) {
  return guard(c, [&] {
    LearnState& S = state(c);
    need_params(S);
    if (!params_host || n != LN_NPARAM) THROW(HHG_ERR_ARG, "need %d parameters", LN_NPARAM);
    CK(cudaMemcpyAsync(params_host, S.params.p, LN_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    wait_stream(c);
  });
}

hhg_status hhg_learn_set_params(hhg_ctx* c, const float* params_host, int64_t n) {
  return guard(c, [&] {
    if (!params_host || n != LN_NPARAM) THROW(HHG_ERR_ARG, "need %d parameters", LN_NPARAM);
    for (int64_t q = 0; q < n; ++q)
      if (!std::isfinite(params_host[q])) THROW(HHG_ERR_ARG, "non-finite parameter %lld", (long long)q);
    std::vector<float> h(params_host, params_host + n);
    upload_params(c, state(c), h);
  });
}

hhg_status hhg_learn_grid(hhg_ctx* c, int level, int* dhw, int64_t* free_voxels) {
  return guard(c, [&] {
    need_ready(c, false);
    LearnGrid& G = grid(c, level);
    if (dhw) {
      dhw[0] = G.D;
      dhw[1] = G.H;
      dhw[2] = G.W;
    }
    if (free_voxels) *free_voxels = G.nfree;
  });
}

hhg_status hhg_learn_channels(hhg_ctx* c, int* cin, int* cout) {
  return guard(c, [&] {
    if (cin) *cin = ln_cin(ncomp(c));
    if (cout) *cout = ncomp(c);
  });
}

hhg_status hhg_learn_forward(hhg_ctx* c, const float* x, int cin, int cout, int B, int D, int H, int W, float* out) {
  return guard(c, [&] {
    LearnState& S = state(c);
    need_params(S);
    if (!x || !out || cin < 1 || cin > LN_C || (cout != 3 && cout != 4) || B < 1 || D < 1 || H < 1 || W < 1)
      THROW(HHG_ERR_ARG, "bad arguments");
    const GridShape s{B, D, H, W};
    ensure_acts(c, S, s.voxels());
    CK(launch_to_bf16(s.voxels(), cin, x, S.act[0].p, c->stream));
    forward_inference(c, S, s, out, cout);
    wait_stream(c);
    check_conv(S);
  });
}

hhg_status hhg_learn_loss_grad(hhg_ctx* c, const float* x, int cin, const float* target, int cout, int B, int D,
                               int H, int W, double* loss_host, float* grad_host) {
  return guard(c, [&] {
    LearnState& S = state(c);
    need_params(S);
    if (!x || !target || cin < 1 || cin > LN_C || (cout != 3 && cout != 4) || B < 1 || D < 1 || H < 1 || W < 1)
      THROW(HHG_ERR_ARG, "bad arguments");
    const GridShape s{B, D, H, W};
    ensure_acts(c, S, s.voxels());
    CK(launch_to_bf16(s.voxels(), cin, x, S.act[0].p, c->stream));
    forward(c, S, s, S.out.as<float>(), cout);
    double* loss = S.dscal.as<double>() + 1;
    backward(c, S, s, S.out.as<float>(), target, cout, loss);
    CK(cudaMemcpyAsync(c->pinned, loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (grad_host)
      CK(cudaMemcpyAsync(grad_host, S.grad.p, LN_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    wait_stream(c);
    check_conv(S);
    if (loss_host) *loss_host = c->pinned[0];
  });
}

hhg_status hhg_learn_reserve_pairs(hhg_ctx* c, int level, int64_t capacity) {
  return guard(c, [&] {
    need_ready(c, false);
    if (capacity < 1) THROW(HHG_ERR_ARG, "capacity");
    LearnState& S = state(c);
    need_coarse_level(c, level, S.coarsen);
    LearnGrid& G = grid(c, level - S.coarsen);
    const int nc = ncomp(c);
    CK(S.pin.alloc((size_t)capacity * G.V * ln_pair_in(nc) * 2));
    CK(S.ptg.alloc((size_t)capacity * G.V * nc * sizeof(float)));
    S.pair_nc = nc;
    S.pair_coarsen = S.coarsen;
    S.pair_tscale.assign(capacity, 1.f);
    S.pair_level = level;
    S.pair_cap = capacity;
    S.pair_count = 0;
  });
}

hhg_status hhg_learn_collect(hhg_ctx* c, int level, const float* e0_grid, int cycles, int64_t* count) {
  return guard(c, [&] {
    need_ready(c, true);
    mg_ready_check(c);
    LearnState& S = state(c);
    if (!e0_grid || cycles < 1) THROW(HHG_ERR_ARG, "bad arguments");
    if (S.pair_level != level) THROW(HHG_ERR_STATE, "reserve pair storage for level %d first", level);
    if (S.pair_count + cycles > S.pair_cap) THROW(HHG_ERR_ARG, "pair storage full (%lld)", (long long)S.pair_cap);
    LearnGrid& G = grid(c, level);
    float* e = lwork(c, G, level, LW_E);
    CK(launch_grid_to_lib(c->lv(level).entries, ncomp(c), G.e2g.as<int64_t>(), G.efree.as<uint8_t>(), e0_grid, nullptr,
                          nullptr, 1.0, nullptr, 1.0, e, c->stream));
    for (int j = 0; j < cycles; ++j) store_pair(c, level, e, e);
    wait_stream(c);
    if (count) *count = S.pair_count;
  });
}

hhg_status hhg_learn_collect_cg(hhg_ctx* c, int level, const float* f, int iters, int64_t* count) {
  return guard(c, [&] {
    need_ready(c, true);
    mg_ready_check(c);
    LearnState& S = state(c);
    if (!f || iters < 1) THROW(HHG_ERR_ARG, "bad arguments");
    if (S.pair_level != level) THROW(HHG_ERR_STATE, "reserve pair storage for level %d first", level);
    if (S.pair_count + iters > S.pair_cap) THROW(HHG_ERR_ARG, "pair storage full (%lld)", (long long)S.pair_cap);
    LearnGrid& G = grid(c, level);
    const bool st = is_stokes(c);
    const int64_t n = sys_n(c, level);
    // reference solution x* (FP64 refinement to 1e-10; Stokes: zero-mean pressure)
    for (auto& v : G.lw64)
      if (!v.p) CK(v.alloc(4 * (size_t)c->lv(level).entries * sizeof(double)));
    double* f64 = G.lw64[0].as<double>();
    double* x64 = G.lw64[1].as<double>();
    CK(launch_convert<float, double>(n, f, f64, c->stream));
    if (st) {
      // K's range is orthogonal to the constant pressure: drop that component of f (FP32
      // rounding alone leaves one of about 1e-8 relative, more than the 1e-10 asked for)
      LevelHost& L = c->lv(level);
      const int64_t E = L.entries;
      std::vector<double> hp(E);
      CK(cudaMemcpyAsync(hp.data(), f64 + 3 * E, E * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      wait_stream(c);
      double sum = 0.0;
      for (int64_t u = 0; u < L.nunique; ++u) sum += hp[L.unique_first[u]];
      CK(launch_add_const<double>(E, -sum / (double)L.nunique, f64 + 3 * E, c->stream));
    }
    CK(cudaMemsetAsync(x64, 0, n * sizeof(double), c->stream));
    hhg_solve_opts o{};
    o.method = st ? HHG_SOLVE_STOKES_IR_FGCR : HHG_SOLVE_IR_FCG;
    o.level = level;
    o.dt = HHG_F64;
    o.rtol = 1e-10;
    o.max_iter = 30;
    o.inner_rtol = 1e-3;
    o.inner_max_iter = 100;
    hhg_solve_report R{};
    learned_ir(c, &o, f64, x64, false, R);
    if (!R.converged) THROW(HHG_ERR_NOT_CONVERGED, "reference solve did not converge");
    float* xs = lwork(c, G, level, LW_XS);
    float* x = lwork(c, G, level, LW_X);
    float* e = lwork(c, G, level, LW_E);
    CK(launch_convert<double, float>(n, x64, xs, c->stream));
    CK(cudaMemsetAsync(x, 0, n * sizeof(float), c->stream));
    int stored = 0;
    auto hook = [&](const float* xk) {
      if (stored >= iters) return;
      copy32(c, level, xs, e);
      CK(launch_axpby<float>(n, -1.f, xk, 1.f, e, c->stream));  // e_k = x* - x_k
      store_pair(c, level, e, nullptr);
      ++stored;
    };
    if (st)
      fgcr(c, level, f, x, 1e-7, iters, false, hook);
    else
      fcg(c, level, f, x, 1e-7, iters, false, hook);
    wait_stream(c);
    if (count) *count = S.pair_count;
  });
}

hhg_status hhg_learn_get_pair(hhg_ctx* c, int64_t index, float* in_host, float* target_host) {
  return guard(c, [&] {
    LearnState& S = state(c);
    if (index < 0 || index >= S.pair_count) THROW(HHG_ERR_ARG, "pair %lld not stored", (long long)index);
    LearnGrid& G = grid(c, S.pair_level - S.pair_coarsen);
    const int nc = S.pair_nc, pin = ln_pair_in(nc), cin = ln_cin(nc);
    if (in_host) {
      std::vector<uint16_t> h((size_t)G.V * pin);
      CK(cudaMemcpyAsync(h.data(), (const char*)S.pin.p + (size_t)index * G.V * pin * 2, h.size() * 2,
                         cudaMemcpyDeviceToHost, c->stream));
      wait_stream(c);
      for (int64_t g = 0; g < G.V; ++g)
        for (int q = 0; q < cin; ++q) {
          const uint32_t u = (uint32_t)h[(size_t)g * pin + q] << 16;
          std::memcpy(&in_host[(size_t)g * cin + q], &u, 4);
        }
    }
    if (target_host) {
      CK(cudaMemcpyAsync(target_host, S.ptg.as<float>() + (size_t)index * G.V * nc, (size_t)G.V * nc * sizeof(float),
                         cudaMemcpyDeviceToHost, c->stream));
      wait_stream(c);
    }
  });
}

hhg_status hhg_learn_train(hhg_ctx* c, const hhg_learn_train_opts* o, hhg_learn_train_report* rep) {
  return guard(c, [&] {
    LearnState& S = state(c);
    need_params(S);
    if (!o || o->steps < 1 || o->batch < 1 || o->crop < 1 || !(o->lr > 0.0)) THROW(HHG_ERR_ARG, "bad options");
    if (S.pair_count < 1) THROW(HHG_ERR_STATE, "no training pairs (hhg_learn_collect)");
    LearnGrid& G = grid(c, S.pair_level - S.pair_coarsen);
    const int Sc = o->crop;
    if (Sc > G.D || Sc > G.H || Sc > G.W) THROW(HHG_ERR_ARG, "crop %d larger than the pair grid", Sc);
    const auto t0 = std::chrono::steady_clock::now();
    const GridShape s{o->batch, Sc, Sc, Sc};
    const int64_t V = s.voxels();
    ensure_acts(c, S, V);
    ensure_grad_scratch(c, S, s);
    // crop choices for every step
    std::vector<int32_t> idx((size_t)o->steps * o->batch), org((size_t)o->steps * o->batch * 3);
    uint64_t rs = o->seed ^ 0x747261696E696E67ull;
    for (size_t q = 0; q < idx.size(); ++q) {
      idx[q] = (int32_t)(splitmix64(rs) % (uint64_t)S.pair_count);
      org[3 * q] = (int32_t)(splitmix64(rs) % (uint64_t)(G.D - Sc + 1));
      org[3 * q + 1] = (int32_t)(splitmix64(rs) % (uint64_t)(G.H - Sc + 1));
      org[3 * q + 2] = (int32_t)(splitmix64(rs) % (uint64_t)(G.W - Sc + 1));
    }
    DevMem didx, dorg, dloss, dts;
    upload(didx, idx);
    upload(dorg, org);
    std::vector<float> ts(S.pair_tscale.begin(), S.pair_tscale.begin() + S.pair_count);
    upload(dts, ts);
    CK(dloss.alloc((size_t)o->steps * sizeof(double)));
    for (int st = 0; st < o->steps; ++st) {
      CK(launch_crop(S.pair_nc, S.pin.p, S.ptg.as<float>(), dts.as<float>(), G.D, G.H, G.W, didx.as<int32_t>() + (size_t)st * o->batch,
                     dorg.as<int32_t>() + (size_t)st * o->batch * 3, o->batch, Sc, S.act[0].p, S.tgt.as<float>(),
                     c->stream));
      forward(c, S, s, S.out.as<float>(), S.pair_nc);
      backward(c, S, s, S.out.as<float>(), S.tgt.as<float>(), S.pair_nc, dloss.as<double>() + st);
      const double lr = o->lr * (0.05 + 0.95 * 0.5 * (1.0 + std::cos(3.141592653589793 * st / o->steps)));
      CK(launch_adam(S.params.as<float>(), S.grad.as<float>(), S.m.as<float>(), S.v.as<float>(), LN_NPARAM, (float)lr,
                     ++S.adam_step, c->stream));
      repack(c, S);
    }
    std::vector<double> hl(o->steps);
    CK(cudaMemcpyAsync(hl.data(), dloss.p, o->steps * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    wait_stream(c);
    check_conv(S);
    for (double v : hl)
      if (!std::isfinite(v)) THROW(HHG_ERR_NUMERIC, "training diverged");
    if (rep) {
      const int tail = std::max(1, o->steps / 10);
      double a = 0.0, b = 0.0;
      for (int q = 0; q < tail; ++q) {
        a += hl[q];
        b += hl[o->steps - tail + q];
      }
      rep->loss_first = a / tail;
      rep->loss_last = b / tail;
      rep->pairs = S.pair_count;
      rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
  });
}

hhg_status hhg_learn_precondition(hhg_ctx* c, int level, int use_net, const void* r, void* z, double* alpha) {
  return guard(c, [&] {
    need_ready(c, true);
    mg_ready_check(c);
    if (!r || !z) THROW(HHG_ERR_ARG, "null vector");
    LearnGrid& G = grid(c, level);
    float* az = lwork(c, G, level, LW_AZ);
    const double a = precondition(c, level, (const float*)r, (float*)z, az, use_net != 0);
    wait_stream(c);
    check_conv(state(c));
    if (alpha) *alpha = a;
  });
}

hhg_status hhg_learn_stats(hhg_ctx* c, hhg_learn_stats_report* rep, int reset) {
  return guard(c, [&] {
    LearnState& S = state(c);
    if (rep) {
      rep->applications = S.applications;
      rep->fallbacks = S.fallbacks;
      rep->alpha_mean = S.applications ? S.alpha_sum / S.applications : 0.0;
      rep->alpha_min = S.alpha_min;
      rep->alpha_max = S.alpha_max;
      rep->gain_mean = S.applications ? S.gain_sum / S.applications : 0.0;
    }
    if (reset) {
      S.applications = S.fallbacks = 0;
      S.alpha_sum = S.alpha_min = S.alpha_max = S.gain_sum = 0.0;
    }
  });
}

}  // extern "C"
