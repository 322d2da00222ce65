// Launchers of the learned-preconditioner kernels (internal, C++ linkage).  Each returns
// a cudaError_t as int.
//
// The network: 4 layers of 3x3x3 convolutions with 16 channels on the structured node
// grid (z, y, x) of a mesh whose nodes lie on an axis-aligned uniform lattice, zero
// padding, ReLU after layers 0..2.  Activations are channels-last BF16 (16 channels,
// 32 bytes per voxel); weights are BF16 copies of FP32 master weights, biases FP32;
// accumulation in FP32.  Parameter layout (FP32, LN_NPARAM values): for layer l,
// W_l[t][i][o] at l*LN_LSIZE + (t*16 + i)*16 + o, then b_l[o] at l*LN_LSIZE + LN_WSIZE + o,
// tap t = (dz+1)*9 + (dy+1)*3 + (dx+1).
//
// The system has nc = 3 unknowns per node (elasticity) or nc = 4 (Stokes: velocity and
// pressure).  Input features (2 nc + 1 channels, see k_features): r1/s (nc), D z0/s (nc),
// log k - mean (1), with z0 the multigrid correction of the residual r, r1 = r - K z0,
// D the point diagonal of the velocity block (and, for the pressure, the diagonal Schur
// surrogate m / mu + (-C)_ii) and s the RMS of D z0 over the free DoFs.  Output (nc
// channels): D c / s, c the correction added to z0.
#pragma once
#include <cstdint>

namespace hhg {

constexpr int LN_C = 16;
constexpr int LN_LAYERS = 4;
constexpr int LN_CIN = 7;   // elasticity: 2 * 3 + 1
constexpr int LN_COUT = 3;
constexpr int ln_cin(int nc) { return 2 * nc + 1; }
constexpr int LN_TAPS = 27;
constexpr int LN_WSIZE = LN_TAPS * LN_C * LN_C;   // 6912
constexpr int LN_LSIZE = LN_WSIZE + LN_C;         // 6928
constexpr int LN_NPARAM = LN_LAYERS * LN_LSIZE;   // 27712
constexpr int LN_PACK = LN_TAPS * 2 * 32 * 2;     // 32-bit words of one layer's packed B fragments
constexpr int LN_PAIR_IN = 8;                     // BF16 input channels stored per pair voxel (nc = 3)
constexpr int ln_pair_in(int nc) { return nc == 4 ? 16 : LN_PAIR_IN; }

struct GridShape {
  int B, D, H, W;
  int64_t voxels() const { return (int64_t)B * D * H * W; }
};

// Y = act(conv(X, W) + bias) on 16-channel BF16 tensors; Wp = packed fragments of W
// (launch_pack).  Y (BF16, 16 channels) and Yf (FP32, the first nf channels) are optional.
// mask (BF16, 16 channels, optional): outputs where mask <= 0 are set to 0 (the ReLU
// derivative in the backward pass).  relu: apply max(., 0) before the mask.
// Wu (nullable): the layer's tcgen05 operands (launch_pack_umma); when given, the
// tensor-memory kernel runs instead of the warp-MMA one, its wait for the MMAs bounded by
// wait_polls polls (negative: the default bound).
int launch_conv(const void* X, const uint32_t* Wp, const void* Wu, const float* bias, void* Y, float* Yf, int nf,
                const void* mask, GridShape s, int relu, void* stream,
                int64_t wait_polls = -1);
// The same convolution as a persistent TMA + tcgen05 pipeline (Wu required)
int launch_conv_tma(const void* X, const void* Wu, const float* bias, void* Y, float* Yf, int nf, const void* mask,
                    GridShape s, int relu, void* stream);
// tcgen05 operands of every layer (LN_UMMA bytes each, forward and input-gradient weights)
constexpr int LN_UMMA = LN_TAPS * 256 * 2;
int launch_pack_umma(const float* params, void* fwd, void* bwd, void* stream);
// *flag = whether a tensor-core convolution's bounded wait ran out since the last call (resets it)
int conv_take_error(int* flag);

// dW[t][i][o] = sum_v A[v + off(t)][i] G[v][o] for all taps: per-block partial sums into
// partial (wgrad_partials() blocks x LN_WSIZE floats), then their ordered sum into dW.
int64_t wgrad_partials(GridShape s);
int launch_wgrad(const void* A, const void* G, float* partial, float* dW, GridShape s, void* stream);
// db[o] = sum_v G[v][o] (partial: bgrad_partials() x 16 floats)
int64_t bgrad_partials(int64_t V);
int launch_bgrad(const void* G, int64_t V, float* partial, float* db, void* stream);

// loss = mean over voxels and nc (3 or 4) channels of (out - target)^2 (written to *loss via
// partial sums); G = d loss / d out as BF16 16-channel tensor (channels >= nc zero)
int64_t mse_partials(int64_t V);
int launch_mse(const float* out, const float* target, int64_t V, int nc, void* G, double* partial, double* loss,
               void* stream);

// Adam (beta1 0.9, beta2 0.999, eps 1e-8) on n parameters, step >= 1
int launch_adam(float* p, const float* g, float* m, float* v, int n, float lr, int step, void* stream);

// packed B fragments of every layer: fwd (conv) and bwd (input gradient, W'[t][o][i] = W[26-t][i][o]),
// LN_PACK words per layer each
int launch_pack(const float* params, uint32_t* fwd, uint32_t* bwd, void* stream);

// FP32 [V][cin] -> BF16 [V][16] (zero padded)
int launch_to_bf16(int64_t V, int cin, const float* src, void* X, void* stream);

// In the feature kernels, nc = 3 or 4 components per node (vectors of nc * E values, component
// c of entry e at [e + c E]); velocity components count only at free nodes, the pressure
// (component 3) at every node.
// sum over voxels of sum_c (z0[e + c E] / dinv[e + c E])^2 over the free components c in
// [c0, c1), e = gent[g], written to *out (partial: mse_partials(V) doubles)
int launch_feature_norm(int64_t V, int64_t E, int nc, int c0, int c1, const int64_t* gent, const uint8_t* gfree,
                        const float* z0, const float* dinv, double* partial, double* out, void* stream);

// features of the library-layout vectors r1, z0 on the grid with the scales
// s = sqrt(*sumsq / count) for the velocity-like components and s_p = sqrt(*sumsq_p /
// count_p) for the pressure (nc = 4; 1 if zero).  X (16-channel BF16, inference) or pin
// (ln_pair_in(nc)-channel BF16) and target = D e1 / s (FP32, nc channels; e1 nullable ->
// no target), whichever is non-null.
int launch_features(int64_t V, int64_t E, int nc, const int64_t* gent, const uint8_t* gfree, const float* logk,
                    const float* r1, const float* z0, const float* e1, const float* dinv, const double* sumsq,
                    double count, const double* sumsq_p, double count_p, void* X, void* pin, float* target,
                    void* stream);

// library layout from an nc-channel FP32 grid field: z[e + c E] = (component free) ?
// s * out[g][c] * dinv[e + c E] : 0, with s (s_p for the pressure) as in launch_features
// (dinv and sumsq nullable: factor 1)
int launch_grid_to_lib(int64_t E, int nc, const int64_t* e2g, const uint8_t* efree, const float* out,
                       const float* dinv, const double* sumsq, double count, const double* sumsq_p, double count_p,
                       float* z, void* stream);

// training crops of S^3 voxels: sample b takes pair idx[b] at origin org[3b..3b+2] (z, y, x)
// of the PD x PH x PW pair grids (ln_pair_in(nc) input and nc target channels per voxel),
// its target multiplied by tscale[idx[b]] (tscale nullable: 1)
int launch_crop(int nc, const void* pin, const float* ptg, const float* tscale, int PD, int PH, int PW,
                const int32_t* idx, const int32_t* org, int B, int S, void* X, float* target, void* stream);

// *out = sum of x[i]^2, i < n (partial: mse_partials(n) doubles)
int launch_sumsq(int64_t n, const float* x, double* partial, double* out, void* stream);

}  // namespace hhg
