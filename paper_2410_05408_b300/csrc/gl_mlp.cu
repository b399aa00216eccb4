// gl_mlp.cu -- surrogate network kernels (tcgen05 on sm_103a) and their C-ABI.
//
// Network: 7 -> 256 -> 256 -> 256 -> 256 -> 1, SiLU between layers, linear
// output, mean-squared-error loss, Adam.  The surrogate is not part of the paper;
// it predicts the oblate-minus-spherical flux residual of the light-curve path.
//
// Precision: FP32 master parameters, BF16 copies of the three 256x256 weight
// matrices and BF16 activations for the tensor-core layers, FP32 accumulation
// in tensor memory.  The 7-wide input layer, the 1-wide output layer, the
// biases, the loss and Adam run on CUDA cores in FP32.
//
// Tensor-core kernels (one CTA per SM, accumulators in TMEM, operands moved by
// TMA in the 128-byte-swizzled K-major layout, warp specialised: loads, MMA
// issue, eight epilogue warps):
//   gl_mlp_fwd3_kernel   the three hidden layers of the forward pass per 128-row
//                        tile, each layer's activations kept in shared memory
//                        for the next (batches of at most one tile per SM)
//   gl_mlp_gemm_kernel   D[128 x 256] = A[128 x 256] B[256 x 256] per row tile,
//                        one layer, weights resident in shared memory while the
//                        tiles overlap; epilogue: forward (z = D + b, h = SiLU(z);
//                        larger batches) or backward (dz_prev = D * SiLU'(z_prev))
//   gl_mlp_wgrad_kernel  dW[256 x 256] += A^T dZ over row tiles (two M = 128
//                        accumulators, 512 TMEM columns; operands staged in the
//                        K-major no-swizzle core-matrix layout), then added to
//                        the FP32 gradient
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/gl.h"
#include "gl_shuffle.cuh"

namespace {

constexpr int W = 256;          // hidden width
constexpr int NIN = 7;          // input features
constexpr int TILE_M = 128;     // rows (samples) per tensor-core tile
constexpr int NTHREADS = 128;

// parameter layout (FP32): W1[7][256], b1, W2[256][256], b2, W3, b3, W4, b4, w5[256], b5
constexpr int64_t OFF_W1 = 0;
constexpr int64_t OFF_B1 = OFF_W1 + NIN * W;
constexpr int64_t OFF_W2 = OFF_B1 + W;
constexpr int64_t LAYER_STRIDE = (int64_t)W * W + W;
__host__ __device__ constexpr int64_t off_w(int l) { return OFF_W2 + (l - 2) * LAYER_STRIDE; }   // l = 2, 3, 4
__host__ __device__ constexpr int64_t off_b(int l) { return off_w(l) + (int64_t)W * W; }
constexpr int64_t OFF_W5 = OFF_W2 + 3 * LAYER_STRIDE;
constexpr int64_t OFF_B5 = OFF_W5 + W;
constexpr int64_t NPARAM = OFF_B5 + 1;   // 199,681

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: K-major, no swizzle.  LBO = byte
// step between core matrices along K, SBO = byte step between 8-row groups.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version
  return d;
}
// instruction descriptor, kind::f16: BF16 A and B, FP32 D, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
// byte offset of element (r, k) in a K-major no-swizzle tile with kgroups
// core matrices along K
__device__ __forceinline__ uint32_t kmaj_off(int r, int k, int kgroups) {
  return (uint32_t)((((r >> 3) * kgroups + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      smem_u32(mbar)));
}
// tcgen05 shared-memory matrix descriptor: K-major, 128-byte swizzle (the layout
// a TMA box of 64 bf16 x rows with CU_TENSOR_MAP_SWIZZLE_128B writes): rows of
// 128 B, 8-row atoms of 1024 B (SBO), 1024-byte-aligned atoms; the leading byte
// offset is not used by this layout.  A K = 16 slice inside the 64-element row
// starts 32 B further (the hardware applies the swizzle to the final address).
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(16 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version
  d |= (uint64_t)2 << 61;   // 128-byte swizzle
  return d;
}
__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}
// Bulk copy of `bytes` contiguous bytes (both addresses 16-byte aligned, a
// multiple of 16 bytes) into shared memory, completion counted on the mbarrier
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(mbar))
      : "memory");
}
// TMA: a 2-D box of the tensor map at (x, y) into shared memory, completion
// counted in bytes on the mbarrier (x * 2 B is a multiple of 16 by construction)
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y,
                                            uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)tm), "r"(x), "r"(y), "r"(smem_u32(mbar))
      : "memory");
}

// bounded wait on an mbarrier phase (at most `limit` polls); returns 1 if the
// phase completed
__device__ __forceinline__ uint32_t mbar_wait(uint64_t* mbar, uint32_t parity,
                                              long limit = 1L << 22) {
  uint32_t done = 0;
  for (long it = 0; it < limit && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity));
  }
  return done;
}
// the same, giving up early once another role of the CTA has set *abort
__device__ __forceinline__ uint32_t mbar_wait_ab(uint64_t* mbar, uint32_t parity,
                                                 volatile int* abort, long limit = 1L << 22) {
  uint32_t done = 0;
  for (long it = 0; it < limit && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity));
    if (!done && (it & 255) == 255 && *abort) break;
  }
  return done;
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
}

// sigmoid as the fast reciprocal of 1 + e^-z (within 2 ulp of FP32, far below the
// BF16 rounding of the activations).  The epilogues apply it to 32 elements per
// thread at once: a branch-free form lets their chains interleave, where the
// correctly rounded reciprocal, with its branch to a slow path, ran them one
// after another (~5000 cycles per 32 elements).
__device__ __forceinline__ float sigmoid_(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }
__device__ __forceinline__ float silu(float z) { return z * sigmoid_(z); }
__device__ __forceinline__ float silu_grad(float z) {
  const float s = sigmoid_(z);
  return s * (1.0f + z * (1.0f - s));
}

enum : int { EPI_FWD_TRAIN = 0, EPI_FWD_INFER = 1, EPI_BWD = 2 };

struct GemmArgs {
  const __nv_bfloat16* a;     // [n][256] row-major (activations or dZ)
  const __nv_bfloat16* b;     // [256 (N)][256 (K)] row-major: the K-major B operand
  const float* bias;          // forward: [256]
  const float* zprev;         // backward: pre-activations of the previous layer [n][256]
  float* zout;                // forward-train: pre-activations [n][256]
  __nv_bfloat16* hout;        // forward: SiLU(z); backward: dz_prev  [n][256]
  int64_t n;
  int* status;
  int probe_polls;             // > 0: failure-detection probe (gl_mlp_wait_probe)
};

// Persistent, warp-specialised tensor-core layer D[128 x 256] = A[128 x 256] B^T
// per 128-row tile of A (B = [256 (N)][256 (K)], both K-major):
//   warp 0   TMA producer: B once (4 boxes of 64 x 256, 128 KB, one barrier
//            each, so that the first MMAs need only the first box), then per tile
//            the two K-halves of A (2 boxes of 64 x 128 each) into a two-stage
//            ring, 128-byte swizzle
//   warp 1   MMA issuer (one thread): 16 tcgen05.mma (K = 16 each) per tile into
//            one of two TMEM accumulators (2 x 256 columns), committing each
//            K-half's stage back to the producer and the finished accumulator to
//            the epilogue
//   warps 2-9 epilogue: warp w reads the 32-lane quarter w mod 4 of TMEM (its 32
//            rows) and one half of the 256 columns, applies bias + SiLU (or the
//            SiLU derivative) and stores; the accumulator is then released
// so that the loads of tile t + 1, its MMAs and the epilogue of tile t overlap.
// Every wait is bounded; a role that gives up sets the CTA's abort flag (the
// others then give up too), and before TMEM is freed the CTA waits, again with a
// bound, for the copies and MMAs it issued.
constexpr int GEMM_THREADS = 320;
constexpr uint32_t kAChunk = 16384;   // 128 rows x 64 bf16
constexpr uint32_t kBChunk = 32768;   // 256 rows x 64 bf16
constexpr size_t GEMM_SMEM = 4 * (size_t)kBChunk + 4 * (size_t)kAChunk + 1024;

template <int EPI>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    gl_mlp_gemm_kernel(GemmArgs g, const __grid_constant__ CUtensorMap tmA,
                       const __grid_constant__ CUtensorMap tmB) {
  extern __shared__ uint8_t sm_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sB = sm;                  // 4 x 32 KB
  uint8_t* sA = sm + 4 * kBChunk;    // stage h: 2 x 16 KB at sA + h * 2 * kAChunk
  __shared__ __align__(8) uint64_t bar_b[4], full[2], empty[2], tfull[2], tempty[2], drain;
  __shared__ __align__(16) float s_bias[8][128];   // each epilogue warp's copy of its half of the bias
  // per epilogue warp: 32 rows x 16 words (+1 against bank conflicts), through
  // which its global loads and stores go as contiguous row segments
  __shared__ __align__(16) uint32_t s_stage[8][32 * 17];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (g.n + TILE_M - 1) / TILE_M;
  if ((int64_t)blockIdx.x >= ntiles) return;
  const int my_tiles = (int)((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int c = 0; c < 4; ++c) mbar_init(&bar_b[c], 1);
    mbar_init(&drain, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 8);
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
        smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  int issued[2] = {0, 0};   // producer: A loads issued per stage
  bool b_issued = false;
  int committed = 0;        // MMA thread: tiles committed
  bool mma_open = false;    // MMA thread: MMAs issued since the last commit
  if (g.probe_polls > 0) {
    // Failure-detection probe: before any copy or MMA is issued, wait on the
    // first phase of an accumulator-release barrier, which nothing arrives on,
    // for probe_polls polls; the wait gives up and the CTA records the timeout
    // like any bounded wait that ran out, then leaves through the normal exit.
    const uint32_t done = mbar_wait(&tempty[0], 0, g.probe_polls);
    if (threadIdx.x == 0) {
      if (!done) atomicOr(g.status, 1);
      s_abort = 1;
    }
  } else if (warp == 0) {
    if (lane == 0) {
      for (int c = 0; c < 4; ++c) {
        mbar_expect_tx(&bar_b[c], kBChunk);
        tma_load_2d(sB + c * kBChunk, &tmB, c * 64, 0, &bar_b[c]);
      }
      b_issued = true;
      for (int t = 0; t < my_tiles && !s_abort; ++t) {
        const int row0 = (int)((blockIdx.x + (int64_t)t * gridDim.x) * TILE_M);
        for (int h = 0; h < 2; ++h) {
          if (t > 0 && !mbar_wait_ab(&empty[h], (t - 1) & 1, &s_abort)) {
            s_abort = 1;
            break;
          }
          uint8_t* st = sA + h * 2 * kAChunk;
          mbar_expect_tx(&full[h], 2 * kAChunk);
          tma_load_2d(st, &tmA, (2 * h) * 64, row0, &full[h]);
          tma_load_2d(st + kAChunk, &tmA, (2 * h + 1) * 64, row0, &full[h]);
          issued[h] = t + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(TILE_M, W);
      bool ok = true;
      for (int t = 0; ok && t < my_tiles && !s_abort; ++t) {
        const int buf = t & 1;
        if (t >= 2 && !mbar_wait_ab(&tempty[buf], ((t >> 1) - 1) & 1, &s_abort)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int h = 0; h < 2 && ok; ++h) {
          if (!mbar_wait_ab(&full[h], t & 1, &s_abort)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          for (int j = 0; j < 8; ++j) {
            const int ks = h * 8 + j, kc = ks >> 2;
            if (t == 0 && (ks & 3) == 0 && !mbar_wait_ab(&bar_b[kc], 0, &s_abort)) {
              ok = false;
              break;
            }
            const uint32_t within = (uint32_t)(ks & 3) * 32u;
            const uint32_t a_addr = smem_u32(sA) + h * 2 * kAChunk + (kc - 2 * h) * kAChunk + within;
            const uint32_t b_addr = smem_u32(sB) + kc * kBChunk + within;
            mma_bf16(tmem + (uint32_t)buf * 256u, umma_desc_sw128(a_addr), umma_desc_sw128(b_addr),
                     idesc, (h | j) != 0);
            mma_open = true;
          }
          if (!ok) break;
          mma_commit(&empty[h]);   // the stage is free once these MMAs have read it
        }
        if (!ok) break;
        mma_commit(&tfull[buf]);
        mma_open = false;
        committed = t + 1;
      }
      if (!ok) s_abort = 1;
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w mod 4) .. + 31, i.e. those rows,
    // columns 128 ((w - 2) / 4) .. + 127
    const int q = warp & 3, c0 = ((warp - 2) >> 2) * 128;
    float* bias = s_bias[warp - 2];
    if (EPI != EPI_BWD) {
      for (int j = lane; j < 128; j += 32) bias[j] = g.bias[c0 + j];
      __syncwarp();
    }
    for (int t = 0; t < my_tiles; ++t) {
      const int buf = t & 1;
      uint32_t done = 0;
      if (lane == 0) done = mbar_wait_ab(&tfull[buf], (t >> 1) & 1, &s_abort);
      done = __shfl_sync(0xffffffffu, done, 0);
      if (!done) {
        if (lane == 0) s_abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      // the warp's rows: row0w .. row0w + 31, this lane's row0w + lane
      const int64_t row0w = (blockIdx.x + (int64_t)t * gridDim.x) * TILE_M + q * 32;
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)buf * 256u;
      uint32_t* stg = s_stage[warp - 2];
      // 16 words of the lane's row out to global memory, 8 rows x 64 bytes per
      // instruction (lane: row 8 k + lane / 4, bytes 16 (lane mod 4) .. + 15)
      auto store16 = [&](const uint32_t* w16, char* dst_row0, int64_t row_bytes) {
#pragma unroll
        for (int j = 0; j < 16; ++j) stg[lane * 17 + j] = w16[j];
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int rr = 8 * k + (lane >> 2), cc = (lane & 3) * 4;
          if (row0w + rr < g.n)
            *(uint4*)(dst_row0 + (int64_t)rr * row_bytes + cc * 4) =
                make_uint4(stg[rr * 17 + cc], stg[rr * 17 + cc + 1], stg[rr * 17 + cc + 2],
                           stg[rr * 17 + cc + 3]);
        }
        __syncwarp();
      };
      // the converse: 16 words of each row in, the lane taking its own row's
      auto load16 = [&](uint32_t* w16, const char* src_row0, int64_t row_bytes) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int rr = 8 * k + (lane >> 2), cc = (lane & 3) * 4;
          const uint4 v = row0w + rr < g.n
                              ? *(const uint4*)(src_row0 + (int64_t)rr * row_bytes + cc * 4)
                              : make_uint4(0u, 0u, 0u, 0u);
          stg[rr * 17 + cc] = v.x;
          stg[rr * 17 + cc + 1] = v.y;
          stg[rr * 17 + cc + 2] = v.z;
          stg[rr * 17 + cc + 3] = v.w;
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 16; ++j) w16[j] = stg[lane * 17 + j];
        __syncwarp();
      };
      for (int c = c0; c < c0 + 128; c += 32) {
        uint32_t acc[32];
        tmem_ld32(taddr + (uint32_t)c, acc);
        // (pairs converted by one instruction, each half rounded to nearest)
        __align__(16) __nv_bfloat162 hv[16];
        if (EPI == EPI_BWD) {
          __align__(16) float zp[32];
          const char* z0 = (const char*)(g.zprev + row0w * W + c);
          load16((uint32_t*)zp, z0, (int64_t)W * 4);
          load16((uint32_t*)zp + 16, z0 + 64, (int64_t)W * 4);
#pragma unroll
          for (int v = 0; v < 16; ++v)
            hv[v] = __floats2bfloat162_rn(__uint_as_float(acc[2 * v]) * silu_grad(zp[2 * v]),
                                          __uint_as_float(acc[2 * v + 1]) * silu_grad(zp[2 * v + 1]));
        } else {
          __align__(16) float zv[32];
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            const float4 b4 = *(const float4*)(bias + c - c0 + 4 * v);
            zv[4 * v] = __uint_as_float(acc[4 * v]) + b4.x;
            zv[4 * v + 1] = __uint_as_float(acc[4 * v + 1]) + b4.y;
            zv[4 * v + 2] = __uint_as_float(acc[4 * v + 2]) + b4.z;
            zv[4 * v + 3] = __uint_as_float(acc[4 * v + 3]) + b4.w;
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) hv[j] = __floats2bfloat162_rn(silu(zv[2 * j]), silu(zv[2 * j + 1]));
          if (EPI == EPI_FWD_TRAIN) {
            char* z0 = (char*)(g.zout + row0w * W + c);
            store16((const uint32_t*)zv, z0, (int64_t)W * 4);
            store16((const uint32_t*)zv + 16, z0 + 64, (int64_t)W * 4);
          }
        }
        store16((const uint32_t*)hv, (char*)(g.hout + row0w * W + c), (int64_t)W * 2);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
    }
  }
  __syncthreads();
  // drain: nothing the CTA issued may still be in flight when TMEM is freed
  if (warp == 0 && lane == 0) {
    if (b_issued)
      for (int c = 0; c < 4; ++c) mbar_wait(&bar_b[c], 0);
    for (int h = 0; h < 2; ++h)
      if (issued[h] > 0) mbar_wait(&full[h], (issued[h] - 1) & 1);
  }
  if (warp == 1 && lane == 0 && mma_open) {
    mma_commit(&drain);
    mbar_wait(&drain, 0);
  }
  if (warp == 1 && lane == 0 && committed > 0 && s_abort)
    mbar_wait(&tfull[(committed - 1) & 1], ((committed - 1) >> 1) & 1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

// The three tensor-core layers of the forward pass in one kernel, one 128-row tile
// at a time:
//   warp 0   TMA producer: the tile's input activations (4 boxes of 64 x 128),
//            then each layer's weights (4 boxes of 64 x 256, 128 KB), the next
//            layer's as soon as the previous layer's MMAs have completed (the
//            weights buffer is then free), i.e. while its epilogue runs
//   warp 1   MMA issuer (one thread): 16 tcgen05.mma per layer into one TMEM
//            accumulator (256 columns), once the layer's input is in shared
//            memory and the previous epilogue has read the accumulator
//   warps 2-9 epilogue: bias + SiLU of the accumulator, written as BF16 into the
//            activation buffer in the same 128-byte-swizzled K-major layout the
//            TMA writes (row r, 16-byte unit u of a 64-column chunk at
//            r * 128 + ((u ^ (r mod 8)) * 16)), so that the next layer reads it
//            where it is; to global memory only what the caller keeps (training:
//            z and h of every layer; inference: h of the last layer)
// Layer L of the CTA (L = 3 t + l, tile t, layer l) completes each barrier once,
// so every wait is on the parity of a completion count; a barrier cannot run two
// completions ahead of its waiter, because each completion needs the waiter's
// own next step.  Every wait is bounded; a role that gives up sets the abort
// flag, and before TMEM is freed the CTA waits, again with a bound, for the
// copies and MMAs it issued.
struct Fwd3Args {
  const float* bias[3];       // b2, b3, b4
  float* zout[3];             // training: pre-activations of layers 2-4 [n][256]
  __nv_bfloat16* hout[3];     // SiLU of layers 2-4 [n][256] (inference: the last only)
  int64_t n;
  int* status;
  int probe_polls;            // > 0: failure-detection probe (gl_mlp_wait_probe)
};

template <bool TRAIN>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    gl_mlp_fwd3_kernel(Fwd3Args g, const __grid_constant__ CUtensorMap tmA,
                       const __grid_constant__ CUtensorMap tmB0,
                       const __grid_constant__ CUtensorMap tmB1,
                       const __grid_constant__ CUtensorMap tmB2) {
  extern __shared__ uint8_t sm_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sB = sm;                  // one layer's weights: 4 x 32 KB
  uint8_t* sA = sm + 4 * kBChunk;    // the tile's activations: 4 K-chunks of 16 KB
  __shared__ __align__(8) uint64_t bar_b[4], a_full, acc_full, epi_done, drain;
  __shared__ __align__(16) float s_bias[3][W];
  // per epilogue warp: 32 rows x 16 words (+1 against bank conflicts), through
  // which its global stores go out as contiguous row segments
  __shared__ __align__(16) uint32_t s_stage[8][32 * 17];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (g.n + TILE_M - 1) / TILE_M;
  if ((int64_t)blockIdx.x >= ntiles) return;
  const int my_tiles = (int)((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
  const int nlay = 3 * my_tiles;
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int c = 0; c < 4; ++c) mbar_init(&bar_b[c], 1);
    mbar_init(&a_full, 1);
    mbar_init(&acc_full, 1);
    mbar_init(&epi_done, 8);
    mbar_init(&drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
        smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  int a_loads = 0, b_loads = 0;   // producer: copies issued
  int committed = 0;              // MMA thread: layers committed
  bool mma_open = false;          // MMA thread: MMAs issued since the last commit
  if (g.probe_polls > 0) {
    // Failure-detection probe: before any copy or MMA is issued, wait on the
    // first phase of the epilogue barrier, which nothing completes, for
    // probe_polls polls; the CTA records the timeout like any bounded wait that
    // ran out and leaves through the normal exit.
    const uint32_t done = mbar_wait(&epi_done, 0, g.probe_polls);
    if (threadIdx.x == 0) {
      if (!done) atomicOr(g.status, 1);
      s_abort = 1;
    }
  } else if (warp == 0) {
    if (lane == 0) {
      const CUtensorMap* tmB[3] = {&tmB0, &tmB1, &tmB2};
      for (int L = 0; L < nlay && !s_abort; ++L) {
        const int t = L / 3, l = L % 3;
        // the weights buffer, and for a new tile the activations, are free once
        // the previous layer's MMAs have completed
        if (L > 0 && !mbar_wait_ab(&acc_full, (uint32_t)(L - 1) & 1u, &s_abort)) {
          s_abort = 1;
          break;
        }
        if (l == 0) {
          const int row0 = (int)((blockIdx.x + (int64_t)t * gridDim.x) * TILE_M);
          mbar_expect_tx(&a_full, 4 * kAChunk);
          for (int c = 0; c < 4; ++c) tma_load_2d(sA + c * kAChunk, &tmA, c * 64, row0, &a_full);
          ++a_loads;
        }
        for (int c = 0; c < 4; ++c) {
          mbar_expect_tx(&bar_b[c], kBChunk);
          tma_load_2d(sB + c * kBChunk, tmB[l], c * 64, 0, &bar_b[c]);
        }
        ++b_loads;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(TILE_M, W);
      bool ok = true;
      for (int L = 0; ok && L < nlay && !s_abort; ++L) {
        const int t = L / 3, l = L % 3;
        // input: by TMA for a tile's first layer, else by the previous epilogue,
        // which has also read the accumulator by the time it signals
        if (l == 0 && !mbar_wait_ab(&a_full, (uint32_t)t & 1u, &s_abort)) {
          ok = false;
          break;
        }
        if (L > 0 && !mbar_wait_ab(&epi_done, (uint32_t)(L - 1) & 1u, &s_abort)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int ks = 0; ks < 16; ++ks) {
          const int kc = ks >> 2;
          if ((ks & 3) == 0 && !mbar_wait_ab(&bar_b[kc], (uint32_t)L & 1u, &s_abort)) {
            ok = false;
            break;
          }
          const uint32_t within = (uint32_t)(ks & 3) * 32u;
          mma_bf16(tmem, umma_desc_sw128(smem_u32(sA) + kc * kAChunk + within),
                   umma_desc_sw128(smem_u32(sB) + kc * kBChunk + within), idesc, ks != 0);
          mma_open = true;
        }
        if (!ok) break;
        mma_commit(&acc_full);
        mma_open = false;
        committed = L + 1;
      }
      if (!ok) s_abort = 1;
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w mod 4) .. + 31 (those rows of the
    // tile) and columns 128 ((w - 2) / 4) .. + 127
    const int q = warp & 3, c0 = ((warp - 2) >> 2) * 128;
    const int r = q * 32 + lane;
    const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16);
    // the biases, staged by the epilogue warps alone (the copies and the MMAs
    // start meanwhile), then a barrier among these eight warps
    for (int i = threadIdx.x - 64; i < 3 * W; i += 256) s_bias[i / W][i % W] = g.bias[i / W][i % W];
    asm volatile("bar.sync 1, 256;" ::: "memory");
    for (int L = 0; L < nlay; ++L) {
      const int t = L / 3, l = L % 3;
      uint32_t done = 0;
      if (lane == 0) done = mbar_wait_ab(&acc_full, (uint32_t)L & 1u, &s_abort);
      done = __shfl_sync(0xffffffffu, done, 0);
      if (!done) {
        if (lane == 0) s_abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int64_t row = (blockIdx.x + (int64_t)t * gridDim.x) * TILE_M + r;
      const float* bias = s_bias[l];
      for (int c = c0; c < c0 + 128; c += 32) {
        uint32_t acc[32];
        tmem_ld32(taddr + (uint32_t)c, acc);
        __align__(16) float zv[32];
        __align__(16) __nv_bfloat162 hv[16];
        // (the bias four at a time: fewer shared-memory loads beside the copies
        // landing there)
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          const float4 b4 = *(const float4*)(bias + c + 4 * v);
          zv[4 * v] = __uint_as_float(acc[4 * v]) + b4.x;
          zv[4 * v + 1] = __uint_as_float(acc[4 * v + 1]) + b4.y;
          zv[4 * v + 2] = __uint_as_float(acc[4 * v + 2]) + b4.z;
          zv[4 * v + 3] = __uint_as_float(acc[4 * v + 3]) + b4.w;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) hv[j] = __floats2bfloat162_rn(silu(zv[2 * j]), silu(zv[2 * j + 1]));
        // global stores through the warp's staging rows: each lane writes its
        // row's 16 words, then the warp stores 8 rows x 64 bytes per instruction
        // (lane: row 8 k + lane / 4, bytes 16 (lane mod 4) .. + 15)
        auto store16 = [&](const uint32_t* w16, char* dst_row0, int64_t row_bytes) {
          uint32_t* stg = s_stage[warp - 2];
#pragma unroll
          for (int j = 0; j < 16; ++j) stg[lane * 17 + j] = w16[j];
          __syncwarp();
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int rr = 8 * k + (lane >> 2), cc = (lane & 3) * 4;
            if (row - r + q * 32 + rr < g.n) {
              const uint4 v = make_uint4(stg[rr * 17 + cc], stg[rr * 17 + cc + 1],
                                         stg[rr * 17 + cc + 2], stg[rr * 17 + cc + 3]);
              *(uint4*)(dst_row0 + (int64_t)rr * row_bytes + cc * 4) = v;
            }
          }
          __syncwarp();
        };
        // (row - r + q * 32 is the warp's first row)
        if (TRAIN) {
          char* z0 = (char*)(g.zout[l] + (row - r + q * 32) * W + c);
          store16((const uint32_t*)zv, z0, (int64_t)W * 4);
          store16((const uint32_t*)zv + 16, z0 + 64, (int64_t)W * 4);
        }
        if (TRAIN || l == 2)
          store16((const uint32_t*)hv, (char*)(g.hout[l] + (row - r + q * 32) * W + c), (int64_t)W * 2);
        if (l < 2) {
          // the next layer's input, in place (rows past n are never stored)
          uint8_t* rb = sA + (c >> 6) * kAChunk + r * 128;
          const int u0 = (c & 63) >> 3;
#pragma unroll
          for (int j = 0; j < 4; ++j)
            *(uint4*)(rb + (((u0 + j) ^ (r & 7)) << 4)) = *(const uint4*)(hv + 4 * j);
        }
      }
      // the generic-proxy stores become visible to the tensor cores' reads
      if (l < 2) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(&epi_done);
    }
  }
  __syncthreads();
  // drain: nothing the CTA issued may still be in flight when TMEM is freed
  // (each barrier has at most its last copy outstanding: a copy is issued only
  // after the previous one on that barrier was consumed)
  if (warp == 0 && lane == 0) {
    if (b_loads > 0)
      for (int c = 0; c < 4; ++c) mbar_wait(&bar_b[c], (uint32_t)(b_loads - 1) & 1u);
    if (a_loads > 0) mbar_wait(&a_full, (uint32_t)(a_loads - 1) & 1u);
  }
  if (warp == 1 && lane == 0 && mma_open) {
    mma_commit(&drain);
    mbar_wait(&drain, 0);
  }
  if (warp == 1 && lane == 0 && committed > 0 && s_abort)
    mbar_wait(&acc_full, (uint32_t)(committed - 1) & 1u);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

struct WgradArgs {
  const __nv_bfloat16* a;    // layer input activations [n][256]
  const __nv_bfloat16* dz;   // layer output gradient [n][256]
  float* part;               // per-CTA partial gradients [gridDim.x][256 (in)][256 (out)],
                             // summed in CTA order by gl_mlp_partsum_kernel
  int64_t n;
  int* status;
};

// dW = A^T dZ: M = input features (two halves of 128), N = outputs, K = samples
// (128 per tile); the two accumulators use all 512 TMEM columns.
__global__ void __launch_bounds__(NTHREADS, 1) gl_mlp_wgrad_kernel(WgradArgs g) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t* sA = sm;             // 256 (features) x 128 (samples) bf16 = 64 KB
  uint8_t* sB = sm + 65536;     // 256 (outputs)  x 128 (samples) bf16 = 64 KB
  uint8_t* sT = sm + 131072;    // staging: 128 (samples) x 256 bf16, row-major = 64 KB
  __shared__ __align__(8) uint64_t mbar, lbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = (g.n + TILE_M - 1) / TILE_M;
  if ((int64_t)blockIdx.x >= ntiles) return;
  if (tid == 0) {
    s_abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&lbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
        smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_bf16(128, W);
  uint32_t phase = 0, lphase = 0;
  bool lpending = false;   // a bulk copy issued and not seen complete
  bool first = true;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row0 = tile * TILE_M;
    // transpose on the way in: element (sample s, feature f) -> (f, s) of a K-major
    // tile with K = samples (16 core matrices along K).  Each operand's rows (one
    // contiguous block of global memory) arrive row-major in the staging buffer
    // by one bulk copy, the rows past n as zeros; then each thread gathers eight
    // consecutive samples of one feature (2-byte loads, consecutive features on
    // consecutive lanes) and writes them as one 16-byte row of a core matrix.
    const int valid = (int)(g.n - row0 < TILE_M ? g.n - row0 : TILE_M);
    for (int op = 0; op < 2; ++op) {
      const __nv_bfloat16* src = op ? g.dz : g.a;
      uint8_t* dst = op ? sB : sA;
      for (int v = valid * 32 + tid; v < TILE_M * 32; v += NTHREADS)
        *(uint4*)(sT + v * 16) = make_uint4(0, 0, 0, 0);
      if (tid == 0) {
        // (the previous gather's reads of the buffer are ordered before the copy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const uint32_t bytes = (uint32_t)valid * (W * 2);
        mbar_expect_tx(&lbar, bytes);
        bulk_load(sT, src + row0 * W, bytes, &lbar);
      }
      lpending = true;
      const uint32_t got = mbar_wait(&lbar, lphase);
      if (got) {
        lpending = false;
        lphase ^= 1;
      } else {   // (any thread whose wait gave up stops the CTA)
        atomicOr(g.status, 1);
        s_abort = 1;
      }
      __syncthreads();
      if (s_abort) break;
      for (int v = tid; v < W * (TILE_M / 8); v += NTHREADS) {
        const int f = v & (W - 1), sg = v >> 8;   // feature, group of 8 samples
        __align__(16) __nv_bfloat16 e[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
          e[j] = *(const __nv_bfloat16*)(sT + (sg * 8 + j) * (W * 2) + f * 2);
        *(uint4*)(dst + kmaj_off(f, sg * 8, 16)) = *(const uint4*)e;
      }
      __syncthreads();
    }
    if (s_abort) break;
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      for (int h = 0; h < 2; ++h) {
        for (int ks = 0; ks < TILE_M / 16; ++ks) {
          uint64_t ad = umma_desc(smem_u32(sA) + h * 16 * 16 * 128 + ks * 256, 128, 16 * 128);
          uint64_t bd = umma_desc(smem_u32(sB) + ks * 256, 128, 16 * 128);
          mma_bf16(tmem + (uint32_t)(h * W), ad, bd, idesc, (first && ks == 0) ? 0u : 1u);
        }
      }
      mma_commit(&mbar);
    }
    first = false;
    uint32_t done = mbar_wait(&mbar, phase);
    done = __shfl_sync(0xffffffffu, done, 0);
    phase ^= 1;
    if (!done && lane == 0) {
      atomicOr(g.status, 1);
      s_abort = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (s_abort) break;
  }
  if (!s_abort) {
    // the partial out through the (now free) staging buffer: the warp's 32 rows
    // x 32 columns at a time, then 4 rows x 128 bytes per store instruction
    float* stg = (float*)sT + warp * (32 * 33);
    for (int h = 0; h < 2; ++h) {
      const int f0 = h * 128 + warp * 32;
      for (int c = 0; c < W; c += 32) {
        uint32_t acc[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(h * W + c), acc);
#pragma unroll
        for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = __uint_as_float(acc[j]);
        __syncwarp();
        float* dst0 = g.part + (int64_t)blockIdx.x * W * W + (int64_t)f0 * W + c;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int rr = 4 * k + (lane >> 3), cc = (lane & 7) * 4;
          *(float4*)(dst0 + (int64_t)rr * W + cc) =
              make_float4(stg[rr * 33 + cc], stg[rr * 33 + cc + 1], stg[rr * 33 + cc + 2],
                          stg[rr * 33 + cc + 3]);
        }
        __syncwarp();
      }
    }
  }
  if (tid == 0 && lpending) mbar_wait(&lbar, lphase);   // no copy in flight at exit
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

// ---- CUDA-core kernels
// layer 1: z1 = x W1 + b1, h1 = SiLU(z1); one thread per (sample, output)
// Input layer: lane l of a warp owns outputs 8 l .. 8 l + 7 and keeps their
// weights and biases in registers; the warp walks over samples (its 7 inputs one
// broadcast load each), with 16-byte stores of z and h.  Launched with a grid of
// a few blocks per SM, so that each warp's weight loads serve several samples.
__global__ void __launch_bounds__(128) gl_mlp_in_kernel(const float* __restrict__ x,
                                                        const float* __restrict__ p,
                                                        float* __restrict__ z1,
                                                        __nv_bfloat16* __restrict__ h1,
                                                        int64_t n) {
  const int o = (threadIdx.x & 31) * 8;
  float w[NIN][8], b[8];
  {
    const float4 b0 = *(const float4*)(p + OFF_B1 + o), b1 = *(const float4*)(p + OFF_B1 + o + 4);
    b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
    b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
  }
#pragma unroll
  for (int k = 0; k < NIN; ++k) {
    const float4 w0 = *(const float4*)(p + OFF_W1 + k * W + o);
    const float4 w1 = *(const float4*)(p + OFF_W1 + k * W + o + 4);
    w[k][0] = w0.x; w[k][1] = w0.y; w[k][2] = w0.z; w[k][3] = w0.w;
    w[k][4] = w1.x; w[k][5] = w1.y; w[k][6] = w1.z; w[k][7] = w1.w;
  }
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  // the next sample's inputs are loaded while this one is computed
  float xn[NIN];
#pragma unroll
  for (int k = 0; k < NIN; ++k) xn[k] = s < n ? x[s * NIN + k] : 0.f;
  for (; s < n; s += nw) {
    float xs[NIN];
#pragma unroll
    for (int k = 0; k < NIN; ++k) {
      xs[k] = xn[k];
      xn[k] = s + nw < n ? x[(s + nw) * NIN + k] : 0.f;
    }
    float z[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) z[j] = b[j];
#pragma unroll
    for (int k = 0; k < NIN; ++k)
#pragma unroll
      for (int j = 0; j < 8; ++j) z[j] = fmaf(xs[k], w[k][j], z[j]);
    if (z1) {
      *(float4*)(z1 + s * W + o) = make_float4(z[0], z[1], z[2], z[3]);
      *(float4*)(z1 + s * W + o + 4) = make_float4(z[4], z[5], z[6], z[7]);
    }
    __align__(16) __nv_bfloat162 hv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) hv[j] = __floats2bfloat162_rn(silu(z[2 * j]), silu(z[2 * j + 1]));
    *(uint4*)(h1 + s * W + o) = *(const uint4*)hv;
  }
}
// Output layer: lane l keeps w5[8 l .. 8 l + 7] in registers and the warp walks
// over samples: one 16-byte load of 8 activations per lane, then the lanes'
// partial sums added by a fixed shuffle tree.
__global__ void __launch_bounds__(128) gl_mlp_out_kernel(const __nv_bfloat16* __restrict__ h4,
                                                         const float* __restrict__ p,
                                                         float* __restrict__ y, int64_t n) {
  const int lane = threadIdx.x & 31;
  const float4 w0 = *(const float4*)(p + OFF_W5 + 8 * lane);
  const float4 w1 = *(const float4*)(p + OFF_W5 + 8 * lane + 4);
  const float b5 = p[OFF_B5];
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  // the next sample's activations are loaded while this one is reduced
  uint4 hn = s < n ? *(const uint4*)(h4 + s * W + 8 * lane) : make_uint4(0u, 0u, 0u, 0u);
  for (; s < n; s += nw) {
    const uint4 hq = hn;
    if (s + nw < n) hn = *(const uint4*)(h4 + (s + nw) * W + 8 * lane);
    const __nv_bfloat162* hp = (const __nv_bfloat162*)&hq;
    const float2 h01 = __bfloat1622float2(hp[0]), h23 = __bfloat1622float2(hp[1]);
    const float2 h45 = __bfloat1622float2(hp[2]), h67 = __bfloat1622float2(hp[3]);
    float acc = h01.x * w0.x;
    acc = fmaf(h01.y, w0.y, acc);
    acc = fmaf(h23.x, w0.z, acc);
    acc = fmaf(h23.y, w0.w, acc);
    acc = fmaf(h45.x, w1.x, acc);
    acc = fmaf(h45.y, w1.y, acc);
    acc = fmaf(h67.x, w1.z, acc);
    acc = fmaf(h67.y, w1.w, acc);
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) y[s] = acc + b5;
  }
}

// output-layer backward, per sample: r = y - t, dy = 2 r / n, rr = r^2 / n,
// dz4 = dy w5 SiLU'(z4).  One warp per sample.
__global__ void gl_mlp_outgrad_kernel(const float* __restrict__ z4, const float* __restrict__ y,
                                      const float* __restrict__ t, const float* __restrict__ p,
                                      float* __restrict__ dy, float* __restrict__ rr,
                                      __nv_bfloat16* __restrict__ dz4, int64_t n) {
  int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (s >= n) return;
  float r = y[s] - t[s];
  float d = 2.0f * r / (float)n;
  if (lane == 0) {
    dy[s] = d;
    rr[s] = r * r / (float)n;
  }
  for (int k = lane; k < W; k += 32)
    dz4[s * W + k] = __float2bfloat16(d * p[OFF_W5 + k] * silu_grad(z4[s * W + k]));
}

// output-layer reductions: per block, sum_s h4[s][k] dy[s] (dw5), and in thread 0
// the sums of dy (db5) and rr (loss), over the samples s = block, block + grid, ...;
// the partials are summed over the blocks in block order afterwards.
__global__ void gl_mlp_outred_kernel(const __nv_bfloat16* __restrict__ h4,
                                     const float* __restrict__ dy, const float* __restrict__ rr,
                                     float* __restrict__ part, double* __restrict__ lpart,
                                     int64_t n) {
  int k = threadIdx.x;
  float acc = 0.f, sdy = 0.f;
  double sl = 0.0;
  for (int64_t s = blockIdx.x; s < n; s += gridDim.x) {
    float d = dy[s];
    acc = fmaf(__bfloat162float(h4[s * W + k]), d, acc);
    if (k == 0) {
      sdy += d;
      sl += (double)rr[s];
    }
  }
  part[(int64_t)blockIdx.x * (W + 1) + k] = acc;
  if (k == 0) {
    part[(int64_t)blockIdx.x * (W + 1) + W] = sdy;
    lpart[blockIdx.x] = sl;
  }
}

// bias gradient: per block, sum_s dz[s][o] over its samples; one thread per
// output column (partials summed in block order afterwards)
__global__ void gl_mlp_bgrad_kernel(const __nv_bfloat16* __restrict__ dz, float* __restrict__ part,
                                    int64_t n) {
  int o = threadIdx.x;
  float acc = 0.f;
  for (int64_t s = blockIdx.x; s < n; s += gridDim.x) acc += __bfloat162float(dz[s * W + o]);
  part[(int64_t)blockIdx.x * W + o] = acc;
}

// input-layer weight gradient: per block, sum_s x[s][k] dz1[s][o] (partials
// summed in block order afterwards)
__global__ void gl_mlp_w1grad_kernel(const float* __restrict__ x, const __nv_bfloat16* __restrict__ dz1,
                                     float* __restrict__ part, int64_t n) {
  int o = threadIdx.x;
  float acc[NIN] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t s = blockIdx.x; s < n; s += gridDim.x) {
    float d = __bfloat162float(dz1[s * W + o]);
#pragma unroll
    for (int k = 0; k < NIN; ++k) acc[k] = fmaf(x[s * NIN + k], d, acc[k]);
  }
#pragma unroll
  for (int k = 0; k < NIN; ++k) part[(int64_t)blockIdx.x * NIN * W + k * W + o] = acc[k];
}

// out[i] = sum over b < nb, in order, of part[b * stride + i]: the gradient sums
// over blocks in a fixed order, so that a training run is reproducible bit for bit
// (1024 threads per block, 32 consecutive outputs i per block: warp w sums the
// partials of the blocks b = w, w + 32, ... in that order for the 32 outputs,
// lane by lane, with coalesced loads; warp 0 then adds the 32 warp sums in warp
// order.  The order depends only on nb, so every run sums alike.)
__global__ void __launch_bounds__(1024) gl_mlp_partsum_kernel(const float* __restrict__ part,
                                                              int nb, int64_t stride,
                                                              int64_t count,
                                                              float* __restrict__ out) {
  __shared__ float s_w[32][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 32 + lane;
  float acc = 0.f;
  if (i < count)
    for (int b = warp; b < nb; b += 32) acc += part[(int64_t)b * stride + i];
  s_w[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && i < count) {
    float t = 0.f;
    for (int w = 0; w < 32; ++w) t += s_w[w][lane];
    out[i] = t;
  }
}

// sum of nb <= 1024 per-block losses: a fixed pairwise tree over one block
__global__ void __launch_bounds__(1024) gl_mlp_losssum_kernel(const double* __restrict__ lpart,
                                                              int nb,
                                                              double* __restrict__ loss) {
  __shared__ double s_l[1024];
  const int t = threadIdx.x;
  s_l[t] = t < nb ? lpart[t] : 0.0;
  __syncthreads();
  for (int h = 512; h > 0; h >>= 1) {
    if (t < h) s_l[t] += s_l[t + h];
    __syncthreads();
  }
  if (t == 0) *loss = s_l[0];
}

// Adam on the FP32 master parameters (bias-corrected), then refresh the BF16
// operand copies: wt_l[o][i] = W_l[i][o] (forward), wk_l[i][o] = W_l[i][o] (backward).
__global__ void gl_mlp_adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                                   float* __restrict__ m, float* __restrict__ v, float lr,
                                   float b1, float b2, float eps, float c1, float c2) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.0f - b1) * gi;
  float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void gl_mlp_cast_kernel(const float* __restrict__ p, __nv_bfloat16* __restrict__ wt,
                                   __nv_bfloat16* __restrict__ wk) {
  // grid: 3 layers x 256 rows; thread o
  int l = blockIdx.x / W, i = blockIdx.x % W, o = threadIdx.x;
  float w = p[off_w(l + 2) + (int64_t)i * W + o];
  __nv_bfloat16 b = __float2bfloat16(w);
  wt[(int64_t)l * W * W + (int64_t)o * W + i] = b;
  wk[(int64_t)l * W * W + (int64_t)i * W + o] = b;
}

// blocks of the CUDA-core gradient reductions (samples strided over them)
constexpr int kRedBlocks = 1024;
// floats of the partial-gradient buffer: the larger of one 256 x 256 slab per
// tensor-core CTA (at most one per SM) and the CUDA-core reductions' partials
constexpr size_t part_floats(int sms) {
  return (size_t)sms * W * W > (size_t)kRedBlocks * NIN * W ? (size_t)sms * W * W
                                                             : (size_t)kRedBlocks * NIN * W;
}
constexpr size_t WGRAD_SMEM = 65536 + 65536 + 65536;

}  // namespace

struct gl_mlp {
  int device = 0;
  int sms = 0;
  float* p = nullptr;          // master parameters
  float* g = nullptr;          // gradients
  float* m = nullptr;          // Adam first moment
  float* v = nullptr;          // Adam second moment
  __nv_bfloat16* wt = nullptr; // [3][256][256] forward operands
  __nv_bfloat16* wk = nullptr; // [3][256][256] backward operands
  int64_t step = 0;
  // activation workspace (grow-only)
  int64_t cap = 0;
  float* z = nullptr;          // [4][cap][256]
  __nv_bfloat16* h = nullptr;  // [4][cap][256]
  __nv_bfloat16* dz = nullptr; // [2][cap][256]
  float* y = nullptr;          // [cap]
  float* dy = nullptr;         // [cap]
  float* rr = nullptr;         // [cap]
  double* d_loss = nullptr;
  int* d_status = nullptr;
  bool attr_set = false;
  int probe_polls = 0;         // gl_mlp_wait_probe
  float* part = nullptr;       // per-block partial gradients (largest: sms x 256 x 256)
  double* lpart = nullptr;     // per-block partial losses
  // training (gl_surrogate_train): the gathered mini-batch and the loss sum
  int64_t bcap = 0;
  float* xb = nullptr;         // [bcap][7]
  float* tb = nullptr;         // [bcap]
  double* d_lsum = nullptr;    // sum of the mini-batch losses of a call
  unsigned* d_table = nullptr; // per-bin maximum error, as float bits
  // encoded tensor maps of the layer GEMMs' operands, by (base, rows, box rows):
  // the buffers are reused from call to call, and an encode is host work in
  // front of every launch
  struct TmapEntry {
    CUtensorMap tm;   // (the type carries its own alignment)
    const void* base;
    int64_t rows;
    int box;
  };
  std::vector<TmapEntry> tmaps;
  // kernel timing (gl_mlp_profile): event pairs per kernel kind
  bool prof = false;
  std::vector<cudaEvent_t> pev[GL_MLP_KERNEL_KINDS];
  size_t pused[GL_MLP_KERNEL_KINDS] = {};
};

namespace {

int mlp_grow(gl_mlp* m, int64_t n) {
  if (n <= m->cap) return GL_OK;
  cudaFree(m->z);
  cudaFree(m->h);
  cudaFree(m->dz);
  cudaFree(m->y);
  cudaFree(m->dy);
  cudaFree(m->rr);
  m->z = nullptr;
  m->h = nullptr;
  m->dz = nullptr;
  m->y = nullptr;
  m->dy = nullptr;
  m->rr = nullptr;
  m->cap = 0;
  int64_t c = n + n / 4 + TILE_M;
  if (cudaMalloc(&m->z, (size_t)4 * c * W * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&m->h, (size_t)4 * c * W * sizeof(__nv_bfloat16)) != cudaSuccess ||
      cudaMalloc(&m->dz, (size_t)2 * c * W * sizeof(__nv_bfloat16)) != cudaSuccess ||
      cudaMalloc(&m->y, (size_t)c * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&m->dy, (size_t)c * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&m->rr, (size_t)c * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return GL_ENOMEM;
  }
  m->cap = c;
  return GL_OK;
}

int mlp_attrs(gl_mlp* m) {
  if (m->attr_set) return GL_OK;
  if (cudaFuncSetAttribute(gl_mlp_gemm_kernel<EPI_FWD_TRAIN>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEMM_SMEM) != cudaSuccess ||
      cudaFuncSetAttribute(gl_mlp_gemm_kernel<EPI_FWD_INFER>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEMM_SMEM) != cudaSuccess ||
      cudaFuncSetAttribute(gl_mlp_gemm_kernel<EPI_BWD>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEMM_SMEM) != cudaSuccess ||
      cudaFuncSetAttribute(gl_mlp_fwd3_kernel<true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEMM_SMEM) != cudaSuccess ||
      cudaFuncSetAttribute(gl_mlp_fwd3_kernel<false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEMM_SMEM) != cudaSuccess ||
      cudaFuncSetAttribute(gl_mlp_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)WGRAD_SMEM) != cudaSuccess)
    return GL_ECUDA;
  m->attr_set = true;
  return GL_OK;
}

// cuTensorMapEncodeTiled from the driver (through the runtime's entry-point query,
// so that the library needs no link against the driver library)
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    else
      cudaGetLastError();
  }
  return fn;
}

// Tensor map of a [rows][256] row-major BF16 matrix in boxes of 64 columns x
// box_rows rows with the 128-byte swizzle (the layout umma_desc_sw128 reads);
// rows beyond the matrix read as zeros.
int make_tmap(CUtensorMap* tm, const void* base, int64_t rows, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
  if (!enc) return GL_ECUDA;
  const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)W * sizeof(__nv_bfloat16)};
  const cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? GL_OK : GL_ECUDA;
}

// Kernel timing: the start event of a launch of `kind` (returns the pair index,
// or -1 when timing is off, the kind's pairs are used up or an event cannot be
// made), and its end event.
constexpr size_t kMlpMaxTimed = 65536;
long prof_begin(gl_mlp* m, int kind, cudaStream_t st) {
  if (!m->prof) return -1;
  const size_t i = m->pused[kind];
  if (i >= kMlpMaxTimed) return -1;
  auto& v = m->pev[kind];
  if (v.size() < 2 * (i + 1)) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return -1;
    }
    v.push_back(a);
    v.push_back(b);
  }
  cudaEventRecord(v[2 * i], st);
  m->pused[kind] = i + 1;
  return (long)i;
}
void prof_end(gl_mlp* m, int kind, long i, cudaStream_t st) {
  if (i >= 0) cudaEventRecord(m->pev[kind][2 * i + 1], st);
}

int grid_for(const gl_mlp* m, int64_t n) {
  int64_t tiles = (n + TILE_M - 1) / TILE_M;
  return (int)(tiles < m->sms ? tiles : m->sms);
}

// One tensor-core layer over n rows (g.a: [n][256] BF16, g.b: [256][256] BF16).
// The tensor map of (base, rows, box_rows) from the network's cache, encoded on
// first use (NULL on an encode failure).  A map depends on nothing but its key
// (the row stride, type and swizzle are fixed), so an entry stays valid when a
// buffer is freed and another one later takes its address.  The pointer is
// valid until the next call.
const CUtensorMap* cached_tmap(gl_mlp* m, const void* base, int64_t rows, int box_rows) {
  for (const auto& e : m->tmaps)
    if (e.base == base && e.rows == rows && e.box == box_rows) return &e.tm;
  gl_mlp::TmapEntry e;
  if (make_tmap(&e.tm, base, rows, box_rows)) return nullptr;
  e.base = base;
  e.rows = rows;
  e.box = box_rows;
  if (m->tmaps.size() >= 64) m->tmaps.clear();   // (shapes change rarely)
  m->tmaps.push_back(e);
  return &m->tmaps.back().tm;
}

template <int EPI>
int launch_gemm(gl_mlp* m, const GemmArgs& g, int64_t n, cudaStream_t st) {
  // (each map copied before the next lookup, which may grow the cache)
  alignas(64) CUtensorMap ta, tb;
  const CUtensorMap* pa = cached_tmap(m, g.a, n, TILE_M);
  if (!pa) return GL_ECUDA;
  ta = *pa;
  const CUtensorMap* pb = cached_tmap(m, g.b, W, W);
  if (!pb) return GL_ECUDA;
  tb = *pb;
  const int kind = EPI == EPI_BWD ? GL_MLP_KERNEL_GEMM_BWD : GL_MLP_KERNEL_GEMM_FWD;
  const long pe = prof_begin(m, kind, st);
  gl_mlp_gemm_kernel<EPI><<<grid_for(m, n), GEMM_THREADS, GEMM_SMEM, st>>>(g, ta, tb);
  prof_end(m, kind, pe, st);
  return GL_OK;
}

// The three tensor-core layers of the forward pass (f: biases and outputs; the
// input is the first layer's activations m->h, the weights m->wt).
int launch_fwd3(gl_mlp* m, const Fwd3Args& f, bool train, int64_t n, cudaStream_t st) {
  alignas(64) CUtensorMap ta, tb[3];
  const CUtensorMap* pm = cached_tmap(m, m->h, n, TILE_M);
  if (!pm) return GL_ECUDA;
  ta = *pm;
  for (int l = 0; l < 3; ++l) {
    if (!(pm = cached_tmap(m, m->wt + (int64_t)l * W * W, W, W))) return GL_ECUDA;
    tb[l] = *pm;
  }
  const long pe = prof_begin(m, GL_MLP_KERNEL_GEMM_FWD, st);
  if (train)
    gl_mlp_fwd3_kernel<true><<<grid_for(m, n), GEMM_THREADS, GEMM_SMEM, st>>>(f, ta, tb[0], tb[1],
                                                                             tb[2]);
  else
    gl_mlp_fwd3_kernel<false><<<grid_for(m, n), GEMM_THREADS, GEMM_SMEM, st>>>(f, ta, tb[0], tb[1],
                                                                              tb[2]);
  prof_end(m, GL_MLP_KERNEL_GEMM_FWD, pe, st);
  return GL_OK;
}

bool dev_ptr(const void* p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice && a.device == device) || a.type == cudaMemoryTypeManaged;
}

// forward through all layers; train = keep pre-activations for backward
int mlp_forward(gl_mlp* m, int64_t n, const float* x, float* y, bool train, cudaStream_t st) {
  int rc = mlp_grow(m, n);
  if (rc) return rc;
  if ((rc = mlp_attrs(m))) return rc;
  const int64_t cs = m->cap * W;
  // (a few resident blocks per SM: each warp's weight loads serve several samples)
  const unsigned lgrid = (unsigned)std::min<int64_t>((n + 3) / 4, (int64_t)m->sms * 6);
  long pe = prof_begin(m, GL_MLP_KERNEL_IN, st);
  gl_mlp_in_kernel<<<lgrid, 128, 0, st>>>(x, m->p, train ? m->z : nullptr, m->h, n);
  prof_end(m, GL_MLP_KERNEL_IN, pe, st);
  if ((n + TILE_M - 1) / TILE_M <= m->sms) {
    // at most one tile per SM: the three layers in one kernel, each layer's
    // activations kept on chip for the next
    Fwd3Args f;
    memset(&f, 0, sizeof f);
    for (int l = 0; l < 3; ++l) {
      f.bias[l] = m->p + off_b(l + 2);
      f.zout[l] = train ? m->z + (l + 1) * cs : nullptr;
      f.hout[l] = m->h + (l + 1) * cs;
    }
    f.n = n;
    f.status = m->d_status;
    f.probe_polls = m->probe_polls;
    if ((rc = launch_fwd3(m, f, train, n, st))) return rc;
  } else {
    // several tiles per SM: one kernel per layer, whose weights stay resident
    // while the tiles' loads, MMAs and epilogues overlap (the fused kernel would
    // load every layer's weights again for each tile)
    for (int l = 2; l <= 4; ++l) {
      GemmArgs g;
      memset(&g, 0, sizeof g);
      g.a = m->h + (l - 2) * cs;
      g.b = m->wt + (int64_t)(l - 2) * W * W;
      g.bias = m->p + off_b(l);
      g.zout = m->z + (l - 1) * cs;
      g.hout = m->h + (l - 1) * cs;
      g.n = n;
      g.status = m->d_status;
      g.probe_polls = m->probe_polls;
      rc = train ? launch_gemm<EPI_FWD_TRAIN>(m, g, n, st) : launch_gemm<EPI_FWD_INFER>(m, g, n, st);
      if (rc) return rc;
    }
  }
  pe = prof_begin(m, GL_MLP_KERNEL_OUT, st);
  gl_mlp_out_kernel<<<lgrid, 128, 0, st>>>(m->h + 3 * cs, m->p, y, n);
  prof_end(m, GL_MLP_KERNEL_OUT, pe, st);
  return cudaGetLastError() == cudaSuccess ? GL_OK : GL_ECUDA;
}

int mlp_loss_grad(gl_mlp* m, int64_t n, const float* x, const float* t, cudaStream_t st);
int surrogate_train(gl_mlp* m, int64_t n, const float* feat, const float* target,
                    const gl_train_config* cfg, int64_t first_step, int64_t n_steps,
                    double* mean_loss, void* stream);

}  // namespace

extern "C" {

int64_t gl_mlp_param_count(void) { return NPARAM; }

int gl_mlp_create(gl_mlp** out, int device) {
  if (!out) return GL_EINVAL;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return GL_EINVAL;
  gl_mlp* m = new gl_mlp();
  m->device = device;
  size_t pb = (size_t)NPARAM * sizeof(float);
  if (cudaDeviceGetAttribute(&m->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMalloc(&m->p, pb) != cudaSuccess || cudaMalloc(&m->g, pb) != cudaSuccess ||
      cudaMalloc(&m->m, pb) != cudaSuccess || cudaMalloc(&m->v, pb) != cudaSuccess ||
      cudaMalloc(&m->wt, (size_t)3 * W * W * 2) != cudaSuccess ||
      cudaMalloc(&m->wk, (size_t)3 * W * W * 2) != cudaSuccess ||
      cudaMalloc(&m->d_loss, sizeof(double)) != cudaSuccess ||
      cudaMalloc(&m->d_status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&m->part, part_floats(m->sms) * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&m->lpart, kRedBlocks * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return GL_ENOMEM;
  }
  cudaMemset(m->p, 0, pb);
  cudaMemset(m->g, 0, pb);
  cudaMemset(m->m, 0, pb);
  cudaMemset(m->v, 0, pb);
  cudaMemset(m->d_status, 0, sizeof(int));
  *out = m;
  return GL_OK;
}

int gl_mlp_destroy(gl_mlp* m) {
  if (!m) return GL_OK;
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  cudaFree(m->p);
  cudaFree(m->g);
  cudaFree(m->m);
  cudaFree(m->v);
  cudaFree(m->wt);
  cudaFree(m->wk);
  cudaFree(m->z);
  cudaFree(m->h);
  cudaFree(m->dz);
  cudaFree(m->y);
  cudaFree(m->dy);
  cudaFree(m->rr);
  cudaFree(m->d_loss);
  cudaFree(m->d_status);
  cudaFree(m->part);
  cudaFree(m->lpart);
  cudaFree(m->xb);
  cudaFree(m->tb);
  cudaFree(m->d_lsum);
  cudaFree(m->d_table);
  for (auto& v : m->pev)
    for (cudaEvent_t e : v) cudaEventDestroy(e);
  delete m;
  return GL_OK;
}

int gl_mlp_set_params(gl_mlp* m, const float* p, int64_t n) {
  if (!m || !p || n != NPARAM) return GL_EINVAL;
  if (cudaSetDevice(m->device) != cudaSuccess) return GL_ECUDA;
  if (cudaMemcpy(m->p, p, (size_t)NPARAM * sizeof(float), cudaMemcpyDefault) != cudaSuccess)
    return GL_ECUDA;
  gl_mlp_cast_kernel<<<3 * W, W>>>(m->p, m->wt, m->wk);
  size_t pb = (size_t)NPARAM * sizeof(float);
  cudaMemset(m->m, 0, pb);
  cudaMemset(m->v, 0, pb);
  m->step = 0;
  return cudaDeviceSynchronize() == cudaSuccess ? GL_OK : GL_ECUDA;
}

int gl_mlp_get_params(gl_mlp* m, float* p, int64_t n) {
  if (!m || !p || n != NPARAM) return GL_EINVAL;
  if (cudaSetDevice(m->device) != cudaSuccess) return GL_ECUDA;
  return cudaMemcpy(p, m->p, (size_t)NPARAM * sizeof(float), cudaMemcpyDefault) == cudaSuccess
             ? GL_OK : GL_ECUDA;
}

int gl_mlp_get_grads(gl_mlp* m, float* g, int64_t n) {
  if (!m || !g || n != NPARAM) return GL_EINVAL;
  if (cudaSetDevice(m->device) != cudaSuccess) return GL_ECUDA;
  return cudaMemcpy(g, m->g, (size_t)NPARAM * sizeof(float), cudaMemcpyDefault) == cudaSuccess
             ? GL_OK : GL_ECUDA;
}

int gl_mlp_forward(gl_mlp* m, int64_t n, const float* x, float* y, void* stream) {
  if (!m || n < 0 || (n > 0 && (!x || !y))) return GL_EINVAL;
  if (n == 0) return GL_OK;
  if (cudaSetDevice(m->device) != cudaSuccess) return GL_ECUDA;
  if (!dev_ptr(x, m->device) || !dev_ptr(y, m->device)) return GL_EINVAL;
  return mlp_forward(m, n, x, y, false, (cudaStream_t)stream);
}

int gl_mlp_loss_grad(gl_mlp* m, int64_t n, const float* x, const float* t, double* loss,
                     void* stream) {
  if (!m || n <= 0 || !x || !t) return GL_EINVAL;
  if (cudaSetDevice(m->device) != cudaSuccess) return GL_ECUDA;
  if (!dev_ptr(x, m->device) || !dev_ptr(t, m->device)) return GL_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = mlp_loss_grad(m, n, x, t, st);
  if (rc) return rc;
  if (loss) {
    if (cudaMemcpyAsync(loss, m->d_loss, sizeof(double), cudaMemcpyDefault, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return GL_ECUDA;
  }
  return GL_OK;
}

}  // extern "C"

namespace {

// Loss (left in m->d_loss) and gradients of the mean squared error on (x, t).
int mlp_loss_grad(gl_mlp* m, int64_t n, const float* x, const float* t, cudaStream_t st) {
  int rc = mlp_grow(m, n);
  if (rc) return rc;
  rc = mlp_forward(m, n, x, m->y, true, st);
  if (rc) return rc;
  const int64_t cs = m->cap * W;
  __nv_bfloat16* dzA = m->dz;
  __nv_bfloat16* dzB = m->dz + cs;
  const int bgrid = (int)(n < kRedBlocks ? n : kRedBlocks);
  // every gradient entry is the sum of per-block partials, taken in block order
  auto partsum = [&](int nb, int64_t stride, int64_t count, float* out) {
    gl_mlp_partsum_kernel<<<(unsigned)((count + 31) / 32), 1024, 0, st>>>(m->part, nb, stride,
                                                                         count, out);
  };
  gl_mlp_outgrad_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(
      m->z + 3 * cs, m->y, t, m->p, m->dy, m->rr, dzA, n);
  gl_mlp_outred_kernel<<<bgrid, W, 0, st>>>(m->h + 3 * cs, m->dy, m->rr, m->part, m->lpart, n);
  partsum(bgrid, W + 1, W + 1, m->g + OFF_W5);   // w5 and b5 are contiguous
  gl_mlp_losssum_kernel<<<1, 1024, 0, st>>>(m->lpart, bgrid, m->d_loss);
  for (int l = 4; l >= 2; --l) {
    // bias and weight gradients of layer l from dz_l (in dzA)
    gl_mlp_bgrad_kernel<<<bgrid, W, 0, st>>>(dzA, m->part, n);
    partsum(bgrid, W, W, m->g + off_b(l));
    WgradArgs wg;
    wg.a = m->h + (l - 2) * cs;
    wg.dz = dzA;
    wg.part = m->part;
    wg.n = n;
    wg.status = m->d_status;
    const int wgrid = grid_for(m, n);
    const long pw = prof_begin(m, GL_MLP_KERNEL_WGRAD, st);
    gl_mlp_wgrad_kernel<<<wgrid, NTHREADS, WGRAD_SMEM, st>>>(wg);
    prof_end(m, GL_MLP_KERNEL_WGRAD, pw, st);
    partsum(wgrid, (int64_t)W * W, (int64_t)W * W, m->g + off_w(l));
    // dz_{l-1} = (dz_l W_l^T) * SiLU'(z_{l-1})
    GemmArgs g;
    memset(&g, 0, sizeof g);
    g.a = dzA;
    g.b = m->wk + (int64_t)(l - 2) * W * W;
    g.zprev = m->z + (l - 2) * cs;
    g.hout = dzB;
    g.n = n;
    g.status = m->d_status;
    if ((rc = launch_gemm<EPI_BWD>(m, g, n, st))) return rc;
    __nv_bfloat16* tmp = dzA;
    dzA = dzB;
    dzB = tmp;
  }
  // layer 1 from dz_1 (in dzA)
  gl_mlp_bgrad_kernel<<<bgrid, W, 0, st>>>(dzA, m->part, n);
  partsum(bgrid, W, W, m->g + OFF_B1);
  gl_mlp_w1grad_kernel<<<bgrid, W, 0, st>>>(x, dzA, m->part, n);
  partsum(bgrid, (int64_t)NIN * W, (int64_t)NIN * W, m->g + OFF_W1);
  return cudaGetLastError() == cudaSuccess ? GL_OK : GL_ECUDA;
}

// One bias-corrected Adam step with the last gradient, then the BF16 copies.
int mlp_adam(gl_mlp* m, float lr, float beta1, float beta2, float eps, cudaStream_t st) {
  m->step++;
  float c1 = 1.0f - powf(beta1, (float)m->step), c2 = 1.0f - powf(beta2, (float)m->step);
  gl_mlp_adam_kernel<<<(unsigned)((NPARAM + 255) / 256), 256, 0, st>>>(m->p, m->g, m->m, m->v, lr,
                                                                       beta1, beta2, eps, c1, c2);
  gl_mlp_cast_kernel<<<3 * W, W, 0, st>>>(m->p, m->wt, m->wk);
  return cudaGetLastError() == cudaSuccess ? GL_OK : GL_ECUDA;
}

bool adam_args_ok(float lr, float beta1, float beta2, float eps) {
  return (lr > 0.f) && (beta1 >= 0.f && beta1 < 1.f) && (beta2 >= 0.f && beta2 < 1.f) &&
         (eps > 0.f);
}

}  // namespace

extern "C" {

int gl_mlp_adam(gl_mlp* m, float lr, float beta1, float beta2, float eps, void* stream) {
  if (!m || !adam_args_ok(lr, beta1, beta2, eps)) return GL_EINVAL;
  if (cudaSetDevice(m->device) != cudaSuccess) return GL_ECUDA;
  return mlp_adam(m, lr, beta1, beta2, eps, (cudaStream_t)stream);
}

int gl_mlp_profile(gl_mlp* m, int on) {
  if (!m || on < 0 || on > 1) return GL_EINVAL;
  m->prof = on == 1;
  for (size_t& u : m->pused) u = 0;
  return GL_OK;
}

int gl_mlp_profile_read(gl_mlp* m, int kind, double* ms, int64_t* launches) {
  if (!m || !ms || !launches || kind < 0 || kind >= GL_MLP_KERNEL_KINDS) return GL_EINVAL;
  if (cudaSetDevice(m->device) != cudaSuccess) return GL_ECUDA;
  double tot = 0.0;
  for (size_t i = 0; i < m->pused[kind]; ++i) {
    float t = 0.f;
    if (cudaEventSynchronize(m->pev[kind][2 * i + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&t, m->pev[kind][2 * i], m->pev[kind][2 * i + 1]) != cudaSuccess)
      return GL_ECUDA;
    tot += t;
  }
  *ms = tot;
  *launches = (int64_t)m->pused[kind];
  return GL_OK;
}

int gl_mlp_status(gl_mlp* m) {
  if (!m) return GL_EINVAL;
  int h = 0;
  if (cudaMemcpy(&h, m->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GL_ECUDA;
  cudaMemset(m->d_status, 0, sizeof(int));
  return h ? GL_ETIMEOUT : GL_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ training
// Initialisation, the shuffled mini-batches and the held-out error table of the
// surrogate, and its checkpoint.  Random numbers come from SplitMix64 keyed by a
// seed and a counter (gl_shuffle.cuh), so every draw can be recomputed from
// (seed, counter) alone: a run resumed from a checkpoint (which stores the seed
// and the step) draws what the uninterrupted run would have.
namespace {
using gl::splitmix64;
using gl::Shuffle;
using gl::make_shuffle;
using gl::shuffle_index;

// uniform in [0, 1) from the top 24 bits of the generator at (seed, i)
__device__ __forceinline__ float uniform01(uint64_t seed, uint64_t i) {
  return (float)(splitmix64(seed ^ splitmix64(i)) >> 40) * (1.0f / 16777216.0f);
}

// He-style uniform initialisation: weights U(-sqrt(6 / fan_in), +), biases U(-0.1, 0.1)
__global__ void gl_mlp_init_kernel(float* __restrict__ p, uint64_t seed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  int fan_in;
  bool bias;
  if (i < OFF_B1) {
    fan_in = NIN;
    bias = false;
  } else if (i < OFF_W2) {
    fan_in = NIN;
    bias = true;
  } else if (i < OFF_W5) {
    const int64_t r = (i - OFF_W2) % LAYER_STRIDE;
    fan_in = W;
    bias = r >= (int64_t)W * W;
  } else {
    fan_in = W;
    bias = i == OFF_B5;
  }
  const float lim = bias ? 0.1f : sqrtf(6.0f / (float)fan_in);
  p[i] = (2.0f * uniform01(seed, (uint64_t)i) - 1.0f) * lim;
}

// mini-batch rows [b0, b0 + nb) of the epoch's permutation gathered contiguously
__global__ void gl_mlp_gather_kernel(const float* __restrict__ feat, const float* __restrict__ target,
                                     int64_t n, Shuffle s, int64_t b0, int64_t nb,
                                     float* __restrict__ xb, float* __restrict__ tb) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const int64_t src = shuffle_index(s, b0 + j, n);
  tb[j] = target[src];
#pragma unroll
  for (int k = 0; k < NIN; ++k) xb[j * NIN + k] = feat[src * NIN + k];
}

__global__ void gl_mlp_addloss_kernel(const double* __restrict__ loss, double* __restrict__ sum) {
  *sum += *loss;
}

// per-bin maximum of |y - t| (non-negative floats order like their bit patterns;
// bit pattern + 1 is stored so that 0 marks a bin without samples)
__global__ void gl_mlp_binmax_kernel(const float* __restrict__ y, const float* __restrict__ t,
                                     const int32_t* __restrict__ bin, int64_t n,
                                     unsigned* __restrict__ table, float* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float e = fabsf(y[i] - t[i]);
  if (err) err[i] = e;
  const int b = bin[i];
  if (b >= 0 && b < GL_SURROGATE_BINS) atomicMax(&table[b], __float_as_uint(e) + 1u);
}

int train_grow(gl_mlp* m, int64_t batch) {
  if (!m->d_lsum && (cudaMalloc(&m->d_lsum, sizeof(double)) != cudaSuccess ||
                     cudaMalloc(&m->d_table, GL_SURROGATE_BINS * sizeof(unsigned)) != cudaSuccess)) {
    cudaGetLastError();
    return GL_ENOMEM;
  }
  if (batch <= m->bcap) return GL_OK;
  cudaFree(m->xb);
  cudaFree(m->tb);
  m->xb = m->tb = nullptr;
  m->bcap = 0;
  if (cudaMalloc(&m->xb, (size_t)batch * NIN * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&m->tb, (size_t)batch * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return GL_ENOMEM;
  }
  m->bcap = batch;
  return GL_OK;
}

// learning rate of step s of a cosine schedule over `total` steps
float cosine_lr(const gl_train_config* c, int64_t s, int64_t total) {
  const double frac = total > 1 ? (double)s / (double)(total - 1) : 0.0;
  return (float)(c->lr_end + 0.5 * ((double)c->lr - c->lr_end) * (1.0 + cos(3.14159265358979323846 * frac)));
}

}  // namespace

extern "C" {

int gl_mlp_wait_probe(gl_mlp* m, int polls) {
  if (!m || polls < 0) return GL_EINVAL;
  m->probe_polls = polls;
  return GL_OK;
}

int gl_mlp_init(gl_mlp* m, uint64_t seed) {
  if (!m) return GL_EINVAL;
  if (cudaSetDevice(m->device) != cudaSuccess) return GL_ECUDA;
  gl_mlp_init_kernel<<<(unsigned)((NPARAM + 255) / 256), 256>>>(m->p, seed);
  gl_mlp_cast_kernel<<<3 * W, W>>>(m->p, m->wt, m->wk);
  const size_t pb = (size_t)NPARAM * sizeof(float);
  cudaMemset(m->m, 0, pb);
  cudaMemset(m->v, 0, pb);
  m->step = 0;
  return cudaDeviceSynchronize() == cudaSuccess ? GL_OK : GL_ECUDA;
}

int gl_surrogate_train(gl_mlp* m, int64_t n, const float* feat, const float* target,
                       const gl_train_config* cfg, int64_t first_step, int64_t n_steps,
                       double* mean_loss, void* stream) {
  nvtxRangePushA("gl_surrogate_train");
  const int rc = surrogate_train(m, n, feat, target, cfg, first_step, n_steps, mean_loss, stream);
  nvtxRangePop();
  return rc;
}

}  // extern "C"

namespace {

int surrogate_train(gl_mlp* m, int64_t n, const float* feat, const float* target,
                    const gl_train_config* cfg, int64_t first_step, int64_t n_steps,
                    double* mean_loss, void* stream) {
  if (!m || !cfg || n <= 0 || !feat || !target || first_step < 0 || n_steps < 0) return GL_EINVAL;
  if (cfg->epochs < 1 || cfg->batch < 1 || cfg->batch > (1 << 24) || !(cfg->lr_end >= 0.f) ||
      !adam_args_ok(cfg->lr, cfg->beta1, cfg->beta2, cfg->eps))
    return GL_EINVAL;
  const int64_t spe = (n + cfg->batch - 1) / cfg->batch;   // steps per epoch
  const int64_t total = cfg->epochs * spe;
  if (first_step + n_steps > total) return GL_EINVAL;
  if (cudaSetDevice(m->device) != cudaSuccess) return GL_ECUDA;
  if (!dev_ptr(feat, m->device) || !dev_ptr(target, m->device)) return GL_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = train_grow(m, cfg->batch);
  if (rc) return rc;
  if (cudaMemsetAsync(m->d_lsum, 0, sizeof(double), st) != cudaSuccess) return GL_ECUDA;
  int64_t epoch = -1;
  Shuffle sh{};
  for (int64_t s = first_step; s < first_step + n_steps; ++s) {
    const int64_t e = s / spe, b0 = (s % spe) * cfg->batch;
    if (e != epoch) {
      epoch = e;
      sh = make_shuffle(cfg->seed, e, n);
    }
    const int64_t nb = b0 + cfg->batch <= n ? cfg->batch : n - b0;
    gl_mlp_gather_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(feat, target, n, sh, b0, nb,
                                                                      m->xb, m->tb);
    if ((rc = mlp_loss_grad(m, nb, m->xb, m->tb, st))) return rc;
    gl_mlp_addloss_kernel<<<1, 1, 0, st>>>(m->d_loss, m->d_lsum);
    if ((rc = mlp_adam(m, cosine_lr(cfg, s, total), cfg->beta1, cfg->beta2, cfg->eps, st)))
      return rc;
  }
  if (cudaGetLastError() != cudaSuccess) return GL_ECUDA;
  if (mean_loss) {
    double sum = 0.0;
    if (cudaMemcpyAsync(&sum, m->d_lsum, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return GL_ECUDA;
    *mean_loss = n_steps > 0 ? sum / (double)n_steps : 0.0;
  }
  return GL_OK;
}

}  // namespace

extern "C" {

int gl_surrogate_error_table(gl_mlp* m, int64_t n, const float* feat, const float* target,
                             const int32_t* bin, float* table, float* err, void* stream) {
  if (!m || n < 0 || !table || (n > 0 && (!feat || !target || !bin))) return GL_EINVAL;
  if (cudaSetDevice(m->device) != cudaSuccess) return GL_ECUDA;
  if (n > 0 && (!dev_ptr(feat, m->device) || !dev_ptr(target, m->device) ||
                !dev_ptr(bin, m->device) || (err && !dev_ptr(err, m->device))))
    return GL_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = train_grow(m, 1);
  if (rc) return rc;
  if (cudaMemsetAsync(m->d_table, 0, GL_SURROGATE_BINS * sizeof(unsigned), st) != cudaSuccess)
    return GL_ECUDA;
  const int64_t chunk = (int64_t)1 << 20;
  for (int64_t a = 0; a < n; a += chunk) {
    const int64_t nb = a + chunk <= n ? chunk : n - a;
    if ((rc = mlp_grow(m, nb))) return rc;
    if ((rc = mlp_forward(m, nb, feat + a * NIN, m->y, false, st))) return rc;
    gl_mlp_binmax_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(
        m->y, target + a, bin + a, nb, m->d_table, err ? err + a : nullptr);
  }
  unsigned h[GL_SURROGATE_BINS];
  if (cudaMemcpyAsync(h, m->d_table, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return GL_ECUDA;
  // bins with no sample get +inf: their items are always recomputed exactly
  float out[GL_SURROGATE_BINS];
  for (int b = 0; b < GL_SURROGATE_BINS; ++b) {
    const unsigned bits = h[b] - 1u;
    float v;
    memcpy(&v, &bits, sizeof v);
    out[b] = h[b] ? v : INFINITY;
  }
  return cudaMemcpy(table, out, sizeof out, cudaMemcpyDefault) == cudaSuccess ? GL_OK : GL_ECUDA;
}

}  // extern "C"

namespace {

// Checkpoint layout: this header, then NPARAM FP32 parameters, the Adam first
// and second moments (NPARAM FP32 each) and GL_SURROGATE_BINS FP32 error-table
// entries, little-endian as the host writes them.
struct CkptHeader {
  char magic[8];          // "GLSURR01"
  uint32_t version;       // 1
  uint32_t nbins;         // GL_SURROGATE_BINS
  int64_t nparam;         // gl_mlp_param_count()
  int64_t adam_step;      // Adam steps taken (bias correction)
  int64_t train_step;     // schedule position of the next gl_surrogate_train step
  gl_train_config cfg;    // the schedule, batch and shuffle seed
};
const char kCkptMagic[8] = {'G', 'L', 'S', 'U', 'R', 'R', '0', '1'};

}  // namespace

extern "C" {

int gl_surrogate_save(gl_mlp* m, const char* path, const float* table, const gl_train_config* cfg,
                      int64_t train_step) {
  if (!m || !path || !table || !cfg || train_step < 0) return GL_EINVAL;
  if (cudaSetDevice(m->device) != cudaSuccess) return GL_ECUDA;
  const size_t pb = (size_t)NPARAM * sizeof(float);
  std::vector<float> buf((size_t)3 * NPARAM + GL_SURROGATE_BINS);
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(buf.data(), m->p, pb, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(buf.data() + NPARAM, m->m, pb, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(buf.data() + 2 * NPARAM, m->v, pb, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(buf.data() + 3 * NPARAM, table, GL_SURROGATE_BINS * sizeof(float),
                 cudaMemcpyDefault) != cudaSuccess)
    return GL_ECUDA;
  CkptHeader hd;
  memset(&hd, 0, sizeof hd);
  memcpy(hd.magic, kCkptMagic, sizeof kCkptMagic);
  hd.version = 1;
  hd.nbins = GL_SURROGATE_BINS;
  hd.nparam = NPARAM;
  hd.adam_step = m->step;
  hd.train_step = train_step;
  hd.cfg = *cfg;
  FILE* f = fopen(path, "wb");
  if (!f) return GL_EIO;
  const bool ok = fwrite(&hd, sizeof hd, 1, f) == 1 &&
                  fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  return (fclose(f) == 0 && ok) ? GL_OK : GL_EIO;
}

int gl_surrogate_load(gl_mlp* m, const char* path, float* table, gl_train_config* cfg,
                      int64_t* train_step) {
  if (!m || !path) return GL_EINVAL;
  if (cudaSetDevice(m->device) != cudaSuccess) return GL_ECUDA;
  FILE* f = fopen(path, "rb");
  if (!f) return GL_EIO;
  CkptHeader hd;
  std::vector<float> buf((size_t)3 * NPARAM + GL_SURROGATE_BINS);
  bool ok = fread(&hd, sizeof hd, 1, f) == 1 && memcmp(hd.magic, kCkptMagic, 8) == 0 &&
            hd.version == 1 && hd.nbins == GL_SURROGATE_BINS && hd.nparam == NPARAM &&
            fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  fclose(f);
  if (!ok) return GL_EIO;
  const size_t pb = (size_t)NPARAM * sizeof(float);
  if (cudaMemcpy(m->p, buf.data(), pb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->m, buf.data() + NPARAM, pb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->v, buf.data() + 2 * NPARAM, pb, cudaMemcpyHostToDevice) != cudaSuccess)
    return GL_ECUDA;
  gl_mlp_cast_kernel<<<3 * W, W>>>(m->p, m->wt, m->wk);
  if (cudaDeviceSynchronize() != cudaSuccess) return GL_ECUDA;
  m->step = hd.adam_step;
  if (table && cudaMemcpy(table, buf.data() + 3 * NPARAM, GL_SURROGATE_BINS * sizeof(float),
                          cudaMemcpyDefault) != cudaSuccess)
    return GL_ECUDA;
  if (cfg) *cfg = hd.cfg;
  if (train_step) *train_step = hd.train_step;
  return GL_OK;
}

}  // extern "C"
