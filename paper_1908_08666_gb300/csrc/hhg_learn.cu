// Kernels of the learned preconditioner (not part of the paper): the 3x3x3 convolution
// of the 16-channel network on BF16 tensor cores with FP32 accumulation (warp-level
// mma.sync m16n8k16), its weight and bias gradients, the MSE loss, Adam, weight
// packing, and the transfers between the library's vector layout and the node grid.
// Layouts and conventions are those of hhg_learn.h.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "hhg_learn.h"

namespace hhg {

namespace {

constexpr int WARPS = 4;          // warps per block of the convolution kernels
constexpr int WG_ROWS = 32;       // 16-voxel row segments per warp in the weight gradient
constexpr int RED_BLOCK = 256;
constexpr int RED_MAX_BLOCKS = 1024;

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__device__ __forceinline__ uint32_t pack_raw(unsigned short lo, unsigned short hi) {
  return (uint32_t)lo | ((uint32_t)hi << 16);
}

// D += A * B, A 16x16 (row), B 16x8 (col), BF16 inputs, FP32 accumulators
__device__ __forceinline__ void mma_bf16(float d[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// a BF16 value packed in the low (hi = 0) or high half of w is > 0
__device__ __forceinline__ bool bf16_positive(uint32_t w, int hi) {
  const uint32_t h = hi ? (w >> 16) : (w & 0xFFFFu);
  return (h & 0x8000u) == 0 && (h & 0x7FFFu) != 0;
}

// Convolution as an implicit GEMM on a shared-memory tile.  A block computes an output
// tile of CT_Z x CT_Y x CT_X voxels (all 16 output channels): it stages the layer's packed
// B fragments and the input tile with its one-voxel halo (zero outside the grid) in
// shared memory with cp.async, then every warp takes two x-rows of 32 voxels (four m16
// tiles) and, per tap, loads the four A fragments with ldmatrix (rows = 16 voxels shifted
// by the tap, columns = 16 input channels) and the two B fragments (16 inputs x 8
// outputs) once for all four tiles: 8 mma.sync m16n8k16 per 4 ldmatrix.x4 + 2 LDS.64.
// A voxel's 16 channels are 32 bytes; its two 16-byte halves are stored swapped when bit
// 2 of the tile-voxel index is set, so the 8 rows of every ldmatrix phase (8 consecutive
// voxels) fall into distinct banks.
// Fragment layouts of m16n8k16 (lane = 4 * gid + tig):
//   A: a0 (row gid, cols 2 tig, +1), a1 (row gid + 8), a2 (cols + 8), a3 (row + 8, cols + 8)
//   B: b0 (rows 2 tig, +1; col gid), b1 (rows + 8)
//   D: d0, d1 (row gid, cols 2 tig, +1), d2, d3 (row gid + 8)
// ldmatrix.x4: lane l addresses row (l & 15) of the 16-row block, channel half (l >> 4),
// so that the four matrices are exactly a0..a3.
constexpr int CT_X = 32, CT_Y = 4, CT_Z = 4;
constexpr int CI_X = CT_X + 2, CI_Y = CT_Y + 2, CI_Z = CT_Z + 2;
constexpr int CI_VOX = CI_X * CI_Y * CI_Z;
constexpr int CONV_WARPS = 8;  // = CT_Y * CT_Z / 2 rows per warp
constexpr int CONV_SMEM = LN_PACK * 4 + CI_VOX * 32;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__global__ void __launch_bounds__(CONV_WARPS * 32) k_conv(const uint4* __restrict__ X, const uint4* __restrict__ Wp,
                                                          const float* __restrict__ bias, uint32_t* __restrict__ Y,
                                                          float* __restrict__ Yf, int nf,
                                                          const uint32_t* __restrict__ mask, int D, int H, int W,
                                                          int ntz, int relu) {
  extern __shared__ uint4 smem[];
  uint4* ws = smem;                  // LN_PACK / 4 chunks
  uint4* xs = smem + LN_PACK / 4;    // CI_VOX * 2 chunks
  const int b = blockIdx.z / ntz;
  const int x0 = blockIdx.x * CT_X, y0 = blockIdx.y * CT_Y, z0 = (blockIdx.z % ntz) * CT_Z;
  for (int q = threadIdx.x; q < LN_PACK / 4; q += blockDim.x) cp_async16(smem_u32(ws + q), Wp + q, true);
  for (int q = threadIdx.x; q < CI_VOX * 2; q += blockDim.x) {
    const int v = q >> 1, h = q & 1;
    const int ix = v % CI_X, iy = (v / CI_X) % CI_Y, iz = v / (CI_X * CI_Y);
    const int gx = x0 - 1 + ix, gy = y0 - 1 + iy, gz = z0 - 1 + iz;
    const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H && gz >= 0 && gz < D;
    const uint4* src = in ? X + ((((int64_t)b * D + gz) * H + gy) * W + gx) * 2 + h : X;
    cp_async16(smem_u32(xs + v * 2 + (h ^ ((v >> 2) & 1))), src, in);
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, tg = lane & 3;
  const int lrow = lane & 15, lhalf = lane >> 4;
  const uint32_t xs_base = smem_u32(xs);
  const uint2* wsl = reinterpret_cast<const uint2*>(ws) + lane;
  // rows of this warp: r = 2 warp + s (s = 0, 1); r -> (oz, oy) = (r / CT_Y, r % CT_Y)
  float acc[4][2][4];
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[m][nt][q] = 0.f;
#pragma unroll 1
  for (int dz = 0; dz < 3; ++dz)
#pragma unroll 1
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const int t = dz * 9 + dy * 3 + dx;
        const uint2 b0 = wsl[(t * 2) * 32], b1 = wsl[(t * 2 + 1) * 32];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int r = 2 * warp + (m >> 1);
          const int oz = r / CT_Y, oy = r % CT_Y;
          const int v = ((oz + dz) * CI_Y + (oy + dy)) * CI_X + (m & 1) * 16 + dx + lrow;
          uint32_t a0, a1, a2, a3;
          ldmatrix_x4(xs_base + (uint32_t)(v * 2 + (lhalf ^ ((v >> 2) & 1))) * 16u, a0, a1, a2, a3);
          mma_bf16(acc[m][0], a0, a1, a2, a3, b0.x, b0.y);
          mma_bf16(acc[m][1], a0, a1, a2, a3, b1.x, b1.y);
        }
      }
  float bv[2][2];
#pragma unroll
  for (int nt = 0; nt < 2; ++nt) {
    bv[nt][0] = bias ? bias[nt * 8 + 2 * tg] : 0.f;
    bv[nt][1] = bias ? bias[nt * 8 + 2 * tg + 1] : 0.f;
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int r = 2 * warp + (m >> 1);
    const int z = z0 + r / CT_Y, y = y0 + r % CT_Y;
    if (z >= D || y >= H) continue;
    const int64_t rowo = (((int64_t)b * D + z) * H + y) * W;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int x = x0 + (m & 1) * 16 + g + 8 * half;
      if (x >= W) continue;
      const int64_t v = rowo + x;
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int co = nt * 8 + 2 * tg;
        float v0 = acc[m][nt][2 * half] + bv[nt][0];
        float v1 = acc[m][nt][2 * half + 1] + bv[nt][1];
        if (relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        if (mask) {
          const uint32_t mw = mask[v * 8 + (co >> 1)];
          if (!bf16_positive(mw, 0)) v0 = 0.f;
          if (!bf16_positive(mw, 1)) v1 = 0.f;
        }
        if (Y) Y[v * 8 + (co >> 1)] = pack_bf16x2(v0, v1);
        if (Yf) {
          if (co < nf) Yf[v * nf + co] = v0;
          if (co + 1 < nf) Yf[v * nf + co + 1] = v1;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Convolution on the 5th-generation tensor cores (tcgen05, accumulators in tensor memory).
// A block owns an output tile of UX x UY x UZ voxels and stages the input tile with its
// one-voxel halo (UPX x UPY x UPZ voxels, zero outside the grid) in shared memory as two
// planes of 16-byte rows (channels 0-7 and 8-15 of every voxel), the K-major no-swizzle
// layout: 8 consecutive voxels form one 128-byte core matrix.  The implicit GEMM takes
// M = 128 consecutive padded positions starting at the first interior one, N = 16 output
// channels and K = 16 input channels per tap; tap (dz, dy, dx) shifts the A operand by
// ((dz UPY + dy) UPX + dx) rows, i.e. its descriptor start address by 16 bytes per row.
// Six such M tiles cover every interior position of the tile (rows at halo positions are
// computed and discarded).  One thread issues the 6 x 27 MMAs into six 16-column TMEM
// accumulators and commits them to an mbarrier; after a bounded wait every warp reads its
// 32 TMEM lanes (one output row per thread, 16 channels) and runs the epilogue.
constexpr int UX = 32, UY = 4, UZ = 4;
constexpr int UPX = UX + 2, UPY = UY + 2, UPZ = UZ + 2;
constexpr int U_VOX = UPX * UPY * UPZ;                  // staged voxels (1224)
constexpr int U_P0 = (UPY + 1) * UPX + 1;               // first interior padded position
constexpr int U_MT = 6;                                 // M tiles of 128 rows
constexpr int U_PLANE_VOX = 1280;                       // >= U_P0 + 128 U_MT + U_P0: rows any tap reads
constexpr int U_PLANE = U_PLANE_VOX * 16;               // bytes per channel-half plane
constexpr int U_WBYTES = LN_TAPS * 512;                 // B operands: [tap][k half][n 16][8 bf16]
constexpr int U_BAR = 2 * U_PLANE + U_WBYTES;           // mbarrier and TMEM-address slot
constexpr int U_SMEM = U_BAR + 64;
constexpr int U_TMEM_COLS = 128;                        // 6 accumulators x 16 columns, rounded up
constexpr uint32_t U_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
constexpr long long U_SPIN_LIMIT = 1ll << 24;           // bound of the mbarrier wait (polls, 100 ns apart)

static_assert(U_P0 + 128 * U_MT - 1 + U_P0 < U_PLANE_VOX, "plane too small for the shifted rows");
static_assert((UZ * UPY + UY) * UPX + UX <= U_P0 + 128 * U_MT - 1, "M tiles do not cover the tile");

__device__ int g_conv_error = 0;  // set when a tensor-core convolution's wait ran out

// shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte
// offsets of the core matrices, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

__global__ void __launch_bounds__(128) k_conv_umma(const uint4* __restrict__ X, const uint4* __restrict__ Wu,
                                                   const float* __restrict__ bias, uint4* __restrict__ Y,
                                                   float* __restrict__ Yf, int nf, const uint4* __restrict__ mask,
                                                   int D, int H, int W, int ntz, int relu, long long wait_polls) {
  extern __shared__ __align__(1024) unsigned char usm[];
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(usm);
  const uint32_t bar = sbase + U_BAR;
  const uint32_t slot = sbase + U_BAR + 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.z / ntz;
  const int x0 = blockIdx.x * UX, y0 = blockIdx.y * UY, z0 = (blockIdx.z % ntz) * UZ;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(U_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // B operands of the layer, then the input tile (two channel-half planes)
  for (int q = threadIdx.x; q < U_WBYTES / 16; q += blockDim.x) cp_async16(sbase + 2 * U_PLANE + 16 * q, Wu + q, true);
  for (int q = threadIdx.x; q < U_VOX * 2; q += blockDim.x) {
    const int v = q >> 1, h = q & 1;
    const int ix = v % UPX, iy = (v / UPX) % UPY, iz = v / (UPX * UPY);
    const int gx = x0 - 1 + ix, gy = y0 - 1 + iy, gz = z0 - 1 + iz;
    const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H && gz >= 0 && gz < D;
    const uint4* src = in ? X + ((((int64_t)b * D + gz) * H + gy) * W + gx) * 2 + h : X;
    cp_async16(sbase + h * U_PLANE + 16 * v, src, in);
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  uint32_t tmem;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(tmem) : "r"(slot));
  if (threadIdx.x == 0) {
    const uint64_t a0 = umma_desc(sbase + 16u * U_P0, U_PLANE, 128);
    const uint64_t b0 = umma_desc(sbase + 2 * U_PLANE, 256, 128);
    for (int mt = 0; mt < U_MT; ++mt) {
      const uint64_t am = a0 + (uint64_t)(128 * mt);
#pragma unroll
      for (int t = 0; t < LN_TAPS; ++t) {
        const int off = ((t / 9 - 1) * UPY + ((t / 3) % 3 - 1)) * UPX + (t % 3 - 1);
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem + 16u * mt),
            "l"(am + (uint64_t)(int64_t)off), "l"(b0 + (uint64_t)(32 * t)), "r"(U_IDESC), "r"((uint32_t)(t > 0)));
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
  }
  // bounded wait for the MMAs; a short sleep between polls leaves the issue slots to the
  // other blocks on the SM (their staging and epilogues)
  uint32_t done = 0;
  for (long long it = 0; it < wait_polls && !done; ++it) {
    asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(done)
                 : "r"(bar), "r"(0)
                 : "memory");
    if (!done) __nanosleep(100);
  }
  done = __all_sync(0xffffffffu, done);
  if (!done) {
    if (lane == 0) atomicExch(&g_conv_error, 1);
    // drain: the MMAs this CTA issued must have completed before their tensor memory is
    // freed below; this wait keeps the full bound whatever wait_polls was
    uint32_t drained = 0;
    for (long long it = 0; it < U_SPIN_LIMIT && !drained; ++it) {
      asm volatile(
          "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
          : "=r"(drained)
          : "r"(bar), "r"(0)
          : "memory");
      if (!drained) __nanosleep(100);
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  float bv[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) bv[c] = bias ? bias[c] : 0.f;
  for (int mt = 0; mt < U_MT && done; ++mt) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(tmem + ((uint32_t)(32 * warp) << 16) + 16u * mt));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int p = U_P0 + 128 * mt + 32 * warp + lane;
    const int iz = p / (UPX * UPY), rem = p % (UPX * UPY), iy = rem / UPX, ix = rem % UPX;
    const int gx = x0 + ix - 1, gy = y0 + iy - 1, gz = z0 + iz - 1;
    if (ix < 1 || ix > UX || iy < 1 || iy > UY || iz < 1 || iz > UZ || gx >= W || gy >= H || gz >= D) continue;
    const int64_t v = (((int64_t)b * D + gz) * H + gy) * W + gx;
    float o[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      o[c] = __uint_as_float(r[c]) + bv[c];
      if (relu) o[c] = fmaxf(o[c], 0.f);
    }
    if (mask) {
      const uint4 m0 = mask[2 * v], m1 = mask[2 * v + 1];
      const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (!bf16_positive(mw[q], 0)) o[2 * q] = 0.f;
        if (!bf16_positive(mw[q], 1)) o[2 * q + 1] = 0.f;
      }
    }
    if (Y) {
      Y[2 * v] = make_uint4(pack_bf16x2(o[0], o[1]), pack_bf16x2(o[2], o[3]), pack_bf16x2(o[4], o[5]),
                            pack_bf16x2(o[6], o[7]));
      Y[2 * v + 1] = make_uint4(pack_bf16x2(o[8], o[9]), pack_bf16x2(o[10], o[11]), pack_bf16x2(o[12], o[13]),
                                pack_bf16x2(o[14], o[15]));
    }
    if (Yf) {
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c < nf) Yf[v * nf + c] = o[c];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(U_TMEM_COLS));
}

// ---------------------------------------------------------------------------------------
// The same convolution as a persistent, warp-specialised pipeline: warp 0 loads input
// tiles with the tensor memory accelerator (one 5-D tiled copy per channel half straight
// into the plane layout; the halo outside the grid is zero-filled by the copy) into two
// shared-memory stages, warp 1 issues the tile's 6 x 27 MMAs into one of two TMEM
// accumulator sets, and warps 2-5 drain the other set through the epilogue, so loading,
// tensor-core work and stores of consecutive tiles overlap.  Stage and accumulator hand-off
// use mbarriers (full / empty per stage, tmem-full / tmem-empty per accumulator set); every
// wait is bounded and, once one runs out, all roles leave their loops (error flag set).
constexpr int P_STAGES = 2;
constexpr int P_THREADS = 192;
constexpr int P_WOFF = P_STAGES * 2 * U_PLANE;
constexpr int P_BAR = P_WOFF + U_WBYTES;
constexpr int P_FULL = P_BAR, P_EMPTY = P_BAR + 16, P_TFULL = P_BAR + 32, P_TEMPTY = P_BAR + 48;
constexpr int P_WBAR = P_BAR + 64, P_SLOT = P_BAR + 72, P_ABORT = P_BAR + 76;
constexpr int P_SMEM = P_BAR + 128;
constexpr int P_TMEM_COLS = 256;
constexpr uint32_t P_TX = 2u * U_VOX * 16u;  // bytes of one stage (two halves of 8 channels)

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
  for (long long it = 0; it < U_SPIN_LIMIT; ++it) {
    uint32_t ok;
    asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    if (ok) return true;
    if (*abort) return false;
    __nanosleep(64);
  }
  *abort = 1;
  atomicExch(&g_conv_error, 1);
  return false;
}

// bounded wait that ignores the abort flag: used to drain a block's own copies and MMAs
__device__ __forceinline__ void bar_drain(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < U_SPIN_LIMIT; ++it) {
    uint32_t ok;
    asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    if (ok) return;
    __nanosleep(64);
  }
  atomicExch(&g_conv_error, 1);
}

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar), "r"(bytes)
               : "memory");
}

__global__ void __launch_bounds__(P_THREADS, 1) k_conv_tma(const __grid_constant__ CUtensorMap tmap,
                                                           const uint4* __restrict__ Wu,
                                                           const float* __restrict__ bias, uint4* __restrict__ Y,
                                                           float* __restrict__ Yf, int nf,
                                                           const uint4* __restrict__ mask, int D, int H, int W,
                                                           int ntx, int nty, int ntz, int ntiles, int relu) {
  extern __shared__ __align__(1024) unsigned char psm[];
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(psm);
  volatile int* abort = (volatile int*)(psm + P_ABORT);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    *abort = 0;
    for (int q = 0; q < P_STAGES; ++q) {
      bar_init(sbase + P_FULL + 8 * q, 1);
      bar_init(sbase + P_EMPTY + 8 * q, 1);
      bar_init(sbase + P_TFULL + 8 * q, 1);
      bar_init(sbase + P_TEMPTY + 8 * q, 4);
    }
    bar_init(sbase + P_WBAR, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sbase + P_SLOT),
                 "r"(P_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  uint32_t tmem;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(tmem) : "r"(sbase + P_SLOT));
  const int ntile_mine = blockIdx.x < (unsigned)ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (warp == 0) {
    if (lane == 0) {
      bar_expect_tx(sbase + P_WBAR, U_WBYTES);
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       sbase + P_WOFF),
                   "l"(Wu), "r"(U_WBYTES), "r"(sbase + P_WBAR)
                   : "memory");
      int last[P_STAGES] = {-1, -1};
      for (int k = 0; k < ntile_mine; ++k) {
        const int st = k & 1;
        if (k >= 2 && !bar_wait(sbase + P_EMPTY + 8 * st, ((k >> 1) - 1) & 1, abort)) break;
        last[st] = k;
        const int tile = (int)blockIdx.x + k * (int)gridDim.x;
        const int tx = tile % ntx, ty = (tile / ntx) % nty, tzb = tile / (ntx * nty);
        const int b = tzb / ntz, tz = tzb % ntz;
        const int cx = tx * UX - 1, cy = ty * UY - 1, cz = tz * UZ - 1;
        const uint32_t full = sbase + P_FULL + 8 * st;
        bar_expect_tx(full, P_TX);
        for (int h = 0; h < 2; ++h)
          asm volatile(
              "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
              "%5, %6}], [%7];" ::"r"(sbase + (2 * st + h) * U_PLANE),
              "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(8 * h), "r"(cx), "r"(cy), "r"(cz), "r"(b), "r"(full)
              : "memory");
      }
      // no tensor copy of this block may still be writing shared memory when it exits
      if (*abort)
        for (int st = 0; st < P_STAGES; ++st)
          if (last[st] >= 0) bar_drain(sbase + P_FULL + 8 * st, (last[st] >> 1) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0 && bar_wait(sbase + P_WBAR, 0, abort)) {
      int last[P_STAGES] = {-1, -1};
      for (int k = 0; k < ntile_mine; ++k) {
        const int st = k & 1;
        if (!bar_wait(sbase + P_FULL + 8 * st, (k >> 1) & 1, abort)) break;
        if (k >= 2 && !bar_wait(sbase + P_TEMPTY + 8 * st, ((k >> 1) - 1) & 1, abort)) break;
        last[st] = k;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // descriptors as base + offset in 16-byte units (the start-address field): an M tile
        // is 128 rows further, a tap shifts by its row offset, a B operand is 512 bytes further
        const uint64_t a0 = umma_desc(sbase + 2 * st * U_PLANE + 16u * U_P0, U_PLANE, 128);
        const uint64_t b0 = umma_desc(sbase + P_WOFF, 256, 128);
        for (int mt = 0; mt < U_MT; ++mt) {
          const uint64_t am = a0 + (uint64_t)(128 * mt);
          const uint32_t d = tmem + 128u * st + 16u * mt;
#pragma unroll
          for (int t = 0; t < LN_TAPS; ++t) {
            const int off = ((t / 9 - 1) * UPY + ((t / 3) % 3 - 1)) * UPX + (t % 3 - 1);
            const uint64_t ad = am + (uint64_t)(int64_t)off;
            const uint64_t bd = b0 + (uint64_t)(32 * t);
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::
                    "r"(d),
                "l"(ad), "l"(bd), "r"(U_IDESC), "r"((uint32_t)(t > 0)));
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         sbase + P_EMPTY + 8 * st)
                     : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         sbase + P_TFULL + 8 * st)
                     : "memory");
      }
      // no MMA of this block may still be running when its tensor memory is freed
      if (*abort)
        for (int st = 0; st < P_STAGES; ++st)
          if (last[st] >= 0) bar_drain(sbase + P_EMPTY + 8 * st, (last[st] >> 1) & 1);
    }
    __syncwarp();
  } else {
    const int quarter = warp & 3;  // TMEM lanes 32 quarter .. of this warp
    float bv[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) bv[c] = bias ? bias[c] : 0.f;
    for (int k = 0; k < ntile_mine; ++k) {
      const int st = k & 1;
      const bool ok = __all_sync(0xffffffffu, bar_wait(sbase + P_TFULL + 8 * st, (k >> 1) & 1, abort));
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int tile = (int)blockIdx.x + k * (int)gridDim.x;
      const int tx = tile % ntx, ty = (tile / ntx) % nty, tzb = tile / (ntx * nty);
      const int b = tzb / ntz, tz = tzb % ntz;
      const int x0 = tx * UX, y0 = ty * UY, z0 = tz * UZ;
      for (int mt = 0; mt < U_MT; ++mt) {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(tmem + ((uint32_t)(32 * quarter) << 16) + 128u * st + 16u * mt));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int p = U_P0 + 128 * mt + 32 * quarter + lane;
        const int iz = p / (UPX * UPY), rem = p % (UPX * UPY), iy = rem / UPX, ix = rem % UPX;
        const int gx = x0 + ix - 1, gy = y0 + iy - 1, gz = z0 + iz - 1;
        if (ix < 1 || ix > UX || iy < 1 || iy > UY || iz < 1 || iz > UZ || gx >= W || gy >= H || gz >= D) continue;
        const int64_t v = (((int64_t)b * D + gz) * H + gy) * W + gx;
        float o[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          o[c] = __uint_as_float(r[c]) + bv[c];
          if (relu) o[c] = fmaxf(o[c], 0.f);
        }
        if (mask) {
          const uint4 m0 = mask[2 * v], m1 = mask[2 * v + 1];
          const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if (!bf16_positive(mw[q], 0)) o[2 * q] = 0.f;
            if (!bf16_positive(mw[q], 1)) o[2 * q + 1] = 0.f;
          }
        }
        if (Y) {
          Y[2 * v] = make_uint4(pack_bf16x2(o[0], o[1]), pack_bf16x2(o[2], o[3]), pack_bf16x2(o[4], o[5]),
                                pack_bf16x2(o[6], o[7]));
          Y[2 * v + 1] = make_uint4(pack_bf16x2(o[8], o[9]), pack_bf16x2(o[10], o[11]), pack_bf16x2(o[12], o[13]),
                                    pack_bf16x2(o[14], o[15]));
        }
        if (Yf) {
#pragma unroll
          for (int c = 0; c < 16; ++c)
            if (c < nf) Yf[v * nf + c] = o[c];
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) bar_arrive(sbase + P_TEMPTY + 8 * st);
    }
  }
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P_TMEM_COLS));
  }
}

// tcgen05 B operands of every layer: fwd[t][h][n][j] = W[t][8h+j][n] (forward),
// bwd[t][h][n][j] = W[26-t][n][8h+j] (input gradient), BF16, LN_TAPS * 256 values per layer
__global__ void k_pack_umma(const float* __restrict__ params, __nv_bfloat16* __restrict__ fwd,
                            __nv_bfloat16* __restrict__ bwd) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= LN_LAYERS * LN_TAPS * 256) return;
  const int l = q / (LN_TAPS * 256), r = q % (LN_TAPS * 256);
  const int t = r / 256, h = (r / 128) % 2, n = (r / 8) % 16, j = r % 8;
  const int k = 8 * h + j;
  const float* Wl = params + (int64_t)l * LN_LSIZE;
  fwd[q] = __float2bfloat16_rn(Wl[t * 256 + k * 16 + n]);
  bwd[q] = __float2bfloat16_rn(Wl[(26 - t) * 256 + n * 16 + k]);
}

// Weight gradient of tap t = blockIdx.y: dW[t][i][o] = sum_v A[v + off(t)][i] G[v][o] as a
// tensor-core product with the voxels as the k dimension (A fragment: input channels x
// 16 voxels, B fragment: 16 voxels x 8 output channels).  Each warp covers WG_ROWS row
// segments, the block sums its warps in a fixed order and writes one partial tile.
__global__ void __launch_bounds__(WARPS * 32) k_wgrad(const unsigned short* __restrict__ A,
                                                      const unsigned short* __restrict__ G, float* __restrict__ partial,
                                                      int B, int D, int H, int W) {
  __shared__ float red[WARPS][256];
  const int t = blockIdx.y;
  const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, tg = lane & 3;
  const int nxs = (W + 15) / 16;
  const int64_t nseg = (int64_t)B * D * H * nxs;
  const int64_t seg0 = ((int64_t)blockIdx.x * WARPS + warp) * WG_ROWS;
  float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  for (int r = 0; r < WG_ROWS; ++r) {
    const int64_t seg = seg0 + r;
    if (seg >= nseg) break;  // warp-uniform
    const int xs = (int)(seg % nxs);
    int64_t rest = seg / nxs;
    const int y = (int)(rest % H);
    rest /= H;
    const int z = (int)(rest % D);
    const int b = (int)(rest / D);
    const int x0 = xs * 16;
    const int64_t rowo = (((int64_t)b * D + z) * H + y) * W;
    const int zz = z + dz, yy = y + dy;
    const bool rin = zz >= 0 && zz < D && yy >= 0 && yy < H;
    const int64_t rowi = (((int64_t)b * D + zz) * H + yy) * W;
    // k index (voxel of the segment) of the four values this lane holds: 2tg, 2tg+1, 2tg+8, 2tg+9
    unsigned short av[4][2], gv[4][2];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int x = x0 + 2 * tg + (q & 1) + 8 * (q >> 1);
      const bool vin = x < W;
      const int xi = x + dx;
      const bool ain = vin && rin && xi >= 0 && xi < W;
      av[q][0] = ain ? A[(rowi + xi) * 16 + g] : (unsigned short)0;
      av[q][1] = ain ? A[(rowi + xi) * 16 + g + 8] : (unsigned short)0;
      gv[q][0] = vin ? G[(rowo + x) * 16 + g] : (unsigned short)0;
      gv[q][1] = vin ? G[(rowo + x) * 16 + g + 8] : (unsigned short)0;
    }
    const uint32_t a0 = pack_raw(av[0][0], av[1][0]);  // row (input channel) g, k = 2tg, 2tg+1
    const uint32_t a1 = pack_raw(av[0][1], av[1][1]);  // row g + 8
    const uint32_t a2 = pack_raw(av[2][0], av[3][0]);  // row g, k = 2tg+8, 2tg+9
    const uint32_t a3 = pack_raw(av[2][1], av[3][1]);  // row g + 8
    mma_bf16(acc[0], a0, a1, a2, a3, pack_raw(gv[0][0], gv[1][0]), pack_raw(gv[2][0], gv[3][0]));
    mma_bf16(acc[1], a0, a1, a2, a3, pack_raw(gv[0][1], gv[1][1]), pack_raw(gv[2][1], gv[3][1]));
  }
#pragma unroll
  for (int nt = 0; nt < 2; ++nt) {
    const int o = nt * 8 + 2 * tg;
    red[warp][g * 16 + o] = acc[nt][0];
    red[warp][g * 16 + o + 1] = acc[nt][1];
    red[warp][(g + 8) * 16 + o] = acc[nt][2];
    red[warp][(g + 8) * 16 + o + 1] = acc[nt][3];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 256; e += blockDim.x) {
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) s += red[w][e];
    partial[(int64_t)blockIdx.x * LN_WSIZE + t * 256 + e] = s;
  }
}

// out[c] = sum over rows r (in order) of partial[r * ncol + c]
__global__ void k_colsum(const float* __restrict__ partial, int64_t rows, int ncol, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncol) return;
  float s = 0.f;
  for (int64_t r = 0; r < rows; ++r) s += partial[r * ncol + c];
  out[c] = s;
}

__global__ void __launch_bounds__(RED_BLOCK) k_bgrad(const uint32_t* __restrict__ G, int64_t V,
                                                     float* __restrict__ partial) {
  __shared__ float s[16][RED_BLOCK / 32];
  float acc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) acc[c] = 0.f;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    const uint4* p = reinterpret_cast<const uint4*>(G + v * 8);
    const uint4 w0 = p[0], w1 = p[1];
    const uint32_t w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      acc[2 * q] += __uint_as_float(w[q] << 16);
      acc[2 * q + 1] += __uint_as_float(w[q] & 0xFFFF0000u);
    }
  }
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    float x = acc[c];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) s[c][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x < 16) {
    float x = 0.f;
    for (int w = 0; w < RED_BLOCK / 32; ++w) x += s[threadIdx.x][w];
    partial[blockIdx.x * 16 + threadIdx.x] = x;
  }
}

// NC = output channels of the network (3 elasticity, 4 Stokes)
template <int NC>
__global__ void __launch_bounds__(RED_BLOCK) k_mse(const float* __restrict__ out, const float* __restrict__ target,
                                                   int64_t V, double inv_n, uint32_t* __restrict__ G,
                                                   double* __restrict__ partial) {
  __shared__ double s[RED_BLOCK / 32];
  double acc = 0.0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    float gr[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double d = (double)out[v * NC + c] - (double)target[v * NC + c];
      acc += d * d;
      gr[c] = (float)(2.0 * d * inv_n);
    }
    uint4* p = reinterpret_cast<uint4*>(G + v * 8);
    p[0] = make_uint4(pack_bf16x2(gr[0], gr[1]), pack_bf16x2(gr[2], gr[3]), 0u, 0u);
    p[1] = make_uint4(0u, 0u, 0u, 0u);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0;
    for (int w = 0; w < RED_BLOCK / 32; ++w) x += s[w];
    partial[blockIdx.x] = x * inv_n;
  }
}

// *out = sum of partial[0..n) (one block, fixed order)
__global__ void __launch_bounds__(RED_BLOCK) k_sum_into(const double* __restrict__ partial, int n,
                                                        double* __restrict__ out) {
  __shared__ double s[RED_BLOCK];
  double x = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) x += partial[q];
  s[threadIdx.x] = x;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const float g = gr[q];
  const float mm = b1 * m[q] + (1.f - b1) * g;
  const float vv = b2 * v[q] + (1.f - b2) * g * g;
  m[q] = mm;
  v[q] = vv;
  p[q] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// one thread per (layer, tap, n-tile, lane): the lane's b0, b1 words of the forward
// fragments (B[k][n] = W[t][k][n]) and of the input-gradient fragments (B[k][n] = W[26-t][n][k])
__global__ void k_pack(const float* __restrict__ params, uint32_t* __restrict__ fwd, uint32_t* __restrict__ bwd) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= LN_LAYERS * LN_TAPS * 64) return;
  const int l = q / (LN_TAPS * 64);
  const int r = q % (LN_TAPS * 64);
  const int lane = r & 31, nt = (r >> 5) & 1, t = r >> 6;
  const int g = lane >> 2, tg = lane & 3;
  const int n = nt * 8 + g;
  const float* Wl = params + (int64_t)l * LN_LSIZE;
  auto wf = [&](int k) { return Wl[t * 256 + k * 16 + n]; };
  auto wb = [&](int k) { return Wl[(26 - t) * 256 + n * 16 + k]; };
  uint32_t* F = fwd + (int64_t)l * LN_PACK + r * 2;
  uint32_t* Bk = bwd + (int64_t)l * LN_PACK + r * 2;
  F[0] = pack_bf16x2(wf(2 * tg), wf(2 * tg + 1));
  F[1] = pack_bf16x2(wf(2 * tg + 8), wf(2 * tg + 9));
  Bk[0] = pack_bf16x2(wb(2 * tg), wb(2 * tg + 1));
  Bk[1] = pack_bf16x2(wb(2 * tg + 8), wb(2 * tg + 9));
}

__global__ void k_to_bf16(int64_t V, int cin, const float* __restrict__ src, uint32_t* __restrict__ X) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    float f[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) f[c] = c < cin ? src[v * cin + c] : 0.f;
    uint4* p = reinterpret_cast<uint4*>(X + v * 8);
    p[0] = make_uint4(pack_bf16x2(f[0], f[1]), pack_bf16x2(f[2], f[3]), pack_bf16x2(f[4], f[5]),
                      pack_bf16x2(f[6], f[7]));
    p[1] = make_uint4(pack_bf16x2(f[8], f[9]), pack_bf16x2(f[10], f[11]), pack_bf16x2(f[12], f[13]),
                      pack_bf16x2(f[14], f[15]));
  }
}

__device__ __forceinline__ double feature_scale(const double* sumsq, double count) {
  if (!sumsq) return 1.0;
  const double s2 = *sumsq / count;
  return (s2 > 0.0 && s2 < 1e300) ? sqrt(s2) : 1.0;
}

// Feature kernels, NC = components of the system's unknowns: 3 (elasticity: velocity-like
// displacement, zero on Dirichlet nodes) or 4 (Stokes: velocity, zero on velocity-Dirichlet
// nodes, then the pressure, free at every node).  dinv holds NC * E values.
template <int NC>
__global__ void __launch_bounds__(RED_BLOCK) k_feature_norm(int64_t V, int64_t E, int c0, int c1,
                                                            const int64_t* __restrict__ gent,
                                                            const uint8_t* __restrict__ gfree,
                                                            const float* __restrict__ z0,
                                                            const float* __restrict__ dinv,
                                                            double* __restrict__ partial) {
  __shared__ double s[RED_BLOCK / 32];
  double acc = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < V; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = gent[g];
    if (e < 0) continue;
    const bool fr = gfree[g] != 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (c < c0 || c >= c1 || (c < 3 && !fr)) continue;
      const double w = (double)z0[e + c * E] / (double)dinv[e + c * E];
      acc += w * w;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0;
    for (int w = 0; w < RED_BLOCK / 32; ++w) x += s[w];
    partial[blockIdx.x] = x;
  }
}

// channels: r1 / s (NC), D z0 / s (NC), log k - mean (1); X holds 16 channels per voxel,
// pin the first 8 * PW (PW = 1 for NC = 3, 2 for NC = 4).  The pressure (component 3) has
// its own scale s_p = sqrt(*sumsq_p / count_p).
template <int NC>
__global__ void k_features(int64_t V, int64_t E, const int64_t* __restrict__ gent, const uint8_t* __restrict__ gfree,
                           const float* __restrict__ logk, const float* __restrict__ r1,
                           const float* __restrict__ z0, const float* __restrict__ e1,
                           const float* __restrict__ dinv, const double* __restrict__ sumsq, double count,
                           const double* __restrict__ sumsq_p, double count_p, uint32_t* __restrict__ X,
                           uint32_t* __restrict__ pin, float* __restrict__ target) {
  constexpr int PW = NC == 4 ? 2 : 1;
  const float inv_u = (float)(1.0 / feature_scale(sumsq, count));
  const float inv_p = NC == 4 ? (float)(1.0 / feature_scale(sumsq_p, count_p)) : inv_u;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < V; g += (int64_t)gridDim.x * blockDim.x) {
    float f[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) f[q] = 0.f;
    float tg[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) tg[c] = 0.f;
    f[2 * NC] = logk[g];
    const int64_t e = gent[g];
    if (e >= 0) {
      const bool fr = gfree[g] != 0;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (c < 3 && !fr) continue;
        const float inv = c < 3 ? inv_u : inv_p;
        const float d = 1.f / dinv[e + c * E];
        f[c] = r1[e + c * E] * inv;
        f[NC + c] = z0[e + c * E] * d * inv;
        if (e1) tg[c] = e1[e + c * E] * d * inv;
      }
    }
    const uint4 w0 = make_uint4(pack_bf16x2(f[0], f[1]), pack_bf16x2(f[2], f[3]), pack_bf16x2(f[4], f[5]),
                                pack_bf16x2(f[6], f[7]));
    const uint4 w1 = make_uint4(pack_bf16x2(f[8], f[9]), pack_bf16x2(f[10], f[11]), pack_bf16x2(f[12], f[13]),
                                pack_bf16x2(f[14], f[15]));
    if (X) {
      uint4* p = reinterpret_cast<uint4*>(X + g * 8);
      p[0] = w0;
      p[1] = w1;
    }
    if (pin) {
      uint4* p = reinterpret_cast<uint4*>(pin) + g * PW;
      p[0] = w0;
      if (PW == 2) p[1] = w1;
    }
    if (target) {
#pragma unroll
      for (int c = 0; c < NC; ++c) target[g * NC + c] = tg[c];
    }
  }
}

template <int NC>
__global__ void k_grid_to_lib(int64_t E, const int64_t* __restrict__ e2g, const uint8_t* __restrict__ efree,
                              const float* __restrict__ out, const float* __restrict__ dinv,
                              const double* __restrict__ sumsq, double count, const double* __restrict__ sumsq_p,
                              double count_p, float* __restrict__ z) {
  const float s_u = (float)feature_scale(sumsq, count);
  const float s_p = NC == 4 ? (float)feature_scale(sumsq_p, count_p) : s_u;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const bool f = efree[e] != 0;
    const int64_t g = e2g[e];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const bool on = c < 3 ? f : g >= 0;
      const float s = c < 3 ? s_u : s_p;
      z[e + c * E] = on ? s * out[g * NC + c] * (dinv ? dinv[e + c * E] : 1.f) : 0.f;
    }
  }
}

template <int NC>
__global__ void k_crop(const uint4* __restrict__ pin, const float* __restrict__ ptg, const float* __restrict__ tscale,
                       int PD, int PH, int PW_, const int32_t* __restrict__ idx, const int32_t* __restrict__ org,
                       int B, int S, uint4* __restrict__ X, float* __restrict__ target) {
  constexpr int PW = NC == 4 ? 2 : 1;
  const int64_t V = (int64_t)B * S * S * S;
  const int64_t N3 = (int64_t)PD * PH * PW_;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(v % S);
    const int y = (int)((v / S) % S);
    const int z = (int)((v / ((int64_t)S * S)) % S);
    const int b = (int)(v / ((int64_t)S * S * S));
    const int64_t src = (int64_t)idx[b] * N3 + ((int64_t)(org[3 * b] + z) * PH + (org[3 * b + 1] + y)) * PW_ +
                        (org[3 * b + 2] + x);
    X[2 * v] = pin[src * PW];
    X[2 * v + 1] = PW == 2 ? pin[src * PW + 1] : make_uint4(0u, 0u, 0u, 0u);
    const float ts = tscale ? tscale[idx[b]] : 1.f;
#pragma unroll
    for (int c = 0; c < NC; ++c) target[v * NC + c] = ts * ptg[src * NC + c];
  }
}

// partial[block] = sum of x[i]^2 over the block's grid-stride share
__global__ void __launch_bounds__(RED_BLOCK) k_sumsq(const float* __restrict__ x, int64_t n,
                                                     double* __restrict__ partial) {
  __shared__ double s[RED_BLOCK / 32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    acc += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < RED_BLOCK / 32; ++w) t += s[w];
    partial[blockIdx.x] = t;
  }
}

inline unsigned blocks_for(int64_t n, int block, int64_t cap) {
  int64_t g = (n + block - 1) / block;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

inline int64_t red_blocks(int64_t V) { return blocks_for(V, RED_BLOCK, RED_MAX_BLOCKS); }

}  // namespace

int launch_conv(const void* X, const uint32_t* Wp, const void* Wu, const float* bias, void* Y, float* Yf, int nf,
                const void* mask, GridShape s, int relu, void* stream, int64_t wait_polls) {
  if (s.voxels() == 0) return 0;
  if (Wu) {
    static bool uattr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
    if (!uattr[dev]) {
      e = cudaFuncSetAttribute(k_conv_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, U_SMEM);
      if (e != cudaSuccess) return (int)e;
      uattr[dev] = true;
    }
    const int ntz = (s.D + UZ - 1) / UZ;
    dim3 grid((unsigned)((s.W + UX - 1) / UX), (unsigned)((s.H + UY - 1) / UY), (unsigned)(ntz * s.B));
    k_conv_umma<<<grid, 128, U_SMEM, (cudaStream_t)stream>>>((const uint4*)X, (const uint4*)Wu, bias, (uint4*)Y, Yf,
                                                             nf, (const uint4*)mask, s.D, s.H, s.W, ntz, relu,
                                                             wait_polls < 0 ? U_SPIN_LIMIT : (long long)wait_polls);
    return (int)cudaGetLastError();
  }
  static bool attr[64] = {};  // per device: dynamic shared memory above 48 KB
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
  if (!attr[dev]) {
    e = cudaFuncSetAttribute(k_conv, cudaFuncAttributeMaxDynamicSharedMemorySize, CONV_SMEM);
    if (e != cudaSuccess) return (int)e;
    attr[dev] = true;
  }
  const int ntz = (s.D + CT_Z - 1) / CT_Z;
  dim3 grid((unsigned)((s.W + CT_X - 1) / CT_X), (unsigned)((s.H + CT_Y - 1) / CT_Y), (unsigned)(ntz * s.B));
  k_conv<<<grid, CONV_WARPS * 32, CONV_SMEM, (cudaStream_t)stream>>>((const uint4*)X, (const uint4*)Wp, bias,
                                                                     (uint32_t*)Y, Yf, nf, (const uint32_t*)mask, s.D,
                                                                     s.H, s.W, ntz, relu);
  return (int)cudaGetLastError();
}

int64_t wgrad_partials(GridShape s) {
  const int64_t nseg = (int64_t)s.B * s.D * s.H * ((s.W + 15) / 16);
  const int64_t nb = (nseg + WARPS * WG_ROWS - 1) / (WARPS * WG_ROWS);
  return nb < 1 ? 1 : nb;
}

int launch_wgrad(const void* A, const void* G, float* partial, float* dW, GridShape s, void* stream) {
  const int64_t nb = wgrad_partials(s);
  dim3 grid((unsigned)nb, LN_TAPS);
  k_wgrad<<<grid, WARPS * 32, 0, (cudaStream_t)stream>>>((const unsigned short*)A, (const unsigned short*)G, partial,
                                                         s.B, s.D, s.H, s.W);
  k_colsum<<<(LN_WSIZE + 255) / 256, 256, 0, (cudaStream_t)stream>>>(partial, nb, LN_WSIZE, dW);
  return (int)cudaGetLastError();
}

int64_t bgrad_partials(int64_t V) { return red_blocks(V); }

int launch_bgrad(const void* G, int64_t V, float* partial, float* db, void* stream) {
  const int64_t nb = red_blocks(V);
  k_bgrad<<<(unsigned)nb, RED_BLOCK, 0, (cudaStream_t)stream>>>((const uint32_t*)G, V, partial);
  k_colsum<<<1, 32, 0, (cudaStream_t)stream>>>(partial, nb, 16, db);
  return (int)cudaGetLastError();
}

int64_t mse_partials(int64_t V) { return red_blocks(V); }

int launch_mse(const float* out, const float* target, int64_t V, int nc, void* G, double* partial, double* loss,
               void* stream) {
  if (nc != 3 && nc != 4) return (int)cudaErrorInvalidValue;
  const int64_t nb = red_blocks(V);
  (nc == 4 ? k_mse<4> : k_mse<3>)<<<(unsigned)nb, RED_BLOCK, 0, (cudaStream_t)stream>>>(
      out, target, V, 1.0 / ((double)V * nc), (uint32_t*)G, partial);
  k_sum_into<<<1, RED_BLOCK, 0, (cudaStream_t)stream>>>(partial, (int)nb, loss);
  return (int)cudaGetLastError();
}

int launch_adam(float* p, const float* g, float* m, float* v, int n, float lr, int step, void* stream) {
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - std::pow(b1, step)), c2 = (float)(1.0 - std::pow(b2, step));
  k_adam<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(p, g, m, v, n, lr, (float)b1, (float)b2, 1e-8f, c1, c2);
  return (int)cudaGetLastError();
}

// 5-D tensor map of a [B][D][H][W][16] BF16 activation tensor with a box of 8 channels x the
// padded tile (encoded through the driver entry point; no link to the driver library)
static int encode_act_map(CUtensorMap* map, const void* X, GridShape s) {
  typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                               const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return (int)e;
    if (q != cudaDriverEntryPointSuccess || !p) return (int)cudaErrorNotSupported;
    fn = (EncodeFn)p;
  }
  const cuuint64_t dims[5] = {16, (cuuint64_t)s.W, (cuuint64_t)s.H, (cuuint64_t)s.D, (cuuint64_t)s.B};
  const cuuint64_t strides[4] = {32, 32ull * s.W, 32ull * s.W * s.H, 32ull * s.W * s.H * s.D};
  const cuuint32_t box[5] = {8, UPX, UPY, UPZ, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(X), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : (int)cudaErrorInvalidValue;
}

int launch_conv_tma(const void* X, const void* Wu, const float* bias, void* Y, float* Yf, int nf, const void* mask,
                    GridShape s, int relu, void* stream) {
  if (s.voxels() == 0) return 0;
  static bool pattr[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
  if (!pattr[dev]) {
    e = cudaFuncSetAttribute(k_conv_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, P_SMEM);
    if (e != cudaSuccess) return (int)e;
    pattr[dev] = true;
  }
  CUtensorMap map;
  const int er = encode_act_map(&map, X, s);
  if (er) return er;
  const int ntx = (s.W + UX - 1) / UX, nty = (s.H + UY - 1) / UY, ntz = (s.D + UZ - 1) / UZ;
  const int ntiles = ntx * nty * ntz * s.B;
  const int grid = ntiles < 2 * 152 ? ntiles : 2 * 152;
  k_conv_tma<<<grid, P_THREADS, P_SMEM, (cudaStream_t)stream>>>(map, (const uint4*)Wu, bias, (uint4*)Y, Yf, nf,
                                                                 (const uint4*)mask, s.D, s.H, s.W, ntx, nty, ntz,
                                                                 ntiles, relu);
  return (int)cudaGetLastError();
}

int launch_pack_umma(const float* params, void* fwd, void* bwd, void* stream) {
  const int n = LN_LAYERS * LN_TAPS * 256;
  k_pack_umma<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, (__nv_bfloat16*)fwd, (__nv_bfloat16*)bwd);
  return (int)cudaGetLastError();
}

int conv_take_error(int* flag) {
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_conv_error, sizeof(int));
  if (e != cudaSuccess) return (int)e;
  if (v) {
    const int zero = 0;
    e = cudaMemcpyToSymbol(g_conv_error, &zero, sizeof(int));
    // landed before a kernel on a (non-blocking) library stream can read the flag
    if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
  }
  *flag = v;
  return (int)e;
}

int launch_pack(const float* params, uint32_t* fwd, uint32_t* bwd, void* stream) {
  const int n = LN_LAYERS * LN_TAPS * 64;
  k_pack<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(params, fwd, bwd);
  return (int)cudaGetLastError();
}

int launch_to_bf16(int64_t V, int cin, const float* src, void* X, void* stream) {
  k_to_bf16<<<blocks_for(V, 256, 152 * 16), 256, 0, (cudaStream_t)stream>>>(V, cin, src, (uint32_t*)X);
  return (int)cudaGetLastError();
}

int launch_feature_norm(int64_t V, int64_t E, int nc, int c0, int c1, const int64_t* gent, const uint8_t* gfree,
                        const float* z0, const float* dinv, double* partial, double* out, void* stream) {
  if (nc != 3 && nc != 4) return (int)cudaErrorInvalidValue;
  const int64_t nb = red_blocks(V);
  (nc == 4 ? k_feature_norm<4> : k_feature_norm<3>)<<<(unsigned)nb, RED_BLOCK, 0, (cudaStream_t)stream>>>(
      V, E, c0, c1, gent, gfree, z0, dinv, partial);
  k_sum_into<<<1, RED_BLOCK, 0, (cudaStream_t)stream>>>(partial, (int)nb, out);
  return (int)cudaGetLastError();
}

int launch_features(int64_t V, int64_t E, int nc, const int64_t* gent, const uint8_t* gfree, const float* logk,
                    const float* r1, const float* z0, const float* e1, const float* dinv, const double* sumsq,
                    double count, const double* sumsq_p, double count_p, void* X, void* pin, float* target,
                    void* stream) {
  if (nc != 3 && nc != 4) return (int)cudaErrorInvalidValue;
  (nc == 4 ? k_features<4> : k_features<3>)<<<blocks_for(V, 256, 152 * 16), 256, 0, (cudaStream_t)stream>>>(
      V, E, gent, gfree, logk, r1, z0, e1, dinv, sumsq, count, sumsq_p, count_p, (uint32_t*)X, (uint32_t*)pin,
      target);
  return (int)cudaGetLastError();
}

int launch_grid_to_lib(int64_t E, int nc, const int64_t* e2g, const uint8_t* efree, const float* out,
                       const float* dinv, const double* sumsq, double count, const double* sumsq_p, double count_p,
                       float* z, void* stream) {
  if (nc != 3 && nc != 4) return (int)cudaErrorInvalidValue;
  (nc == 4 ? k_grid_to_lib<4> : k_grid_to_lib<3>)<<<blocks_for(E, 256, 152 * 16), 256, 0, (cudaStream_t)stream>>>(
      E, e2g, efree, out, dinv, sumsq, count, sumsq_p, count_p, z);
  return (int)cudaGetLastError();
}

int launch_crop(int nc, const void* pin, const float* ptg, const float* tscale, int PD, int PH, int PW,
                const int32_t* idx, const int32_t* org, int B, int S, void* X, float* target, void* stream) {
  if (nc != 3 && nc != 4) return (int)cudaErrorInvalidValue;
  const int64_t V = (int64_t)B * S * S * S;
  (nc == 4 ? k_crop<4> : k_crop<3>)<<<blocks_for(V, 256, 152 * 16), 256, 0, (cudaStream_t)stream>>>(
      (const uint4*)pin, ptg, tscale, PD, PH, PW, idx, org, B, S, (uint4*)X, target);
  return (int)cudaGetLastError();
}

int launch_sumsq(int64_t n, const float* x, double* partial, double* out, void* stream) {
  const int64_t nb = red_blocks(n);
  k_sumsq<<<(unsigned)nb, RED_BLOCK, 0, (cudaStream_t)stream>>>(x, n, partial);
  k_sum_into<<<1, RED_BLOCK, 0, (cudaStream_t)stream>>>(partial, (int)nb, out);
  return (int)cudaGetLastError();
}

}  // namespace hhg
