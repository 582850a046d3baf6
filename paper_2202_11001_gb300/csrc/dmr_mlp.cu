// Learned proposal network on the 5th-generation tensor cores (sm_103a).
//
// A small MLP (256 -> 128 -> 128 -> 128 -> 6, tanh-form GELU) proposes a Gaussian
// displacement for every (candidate, point) of the target mesh; RV-GOMEA
// mixes its samples into its own proposals.  The paper has no learned part;
// this is the one dense contraction of the path, so it runs as tcgen05.mma
// (BF16 operands in shared memory, FP32 accumulators in tensor memory):
//
//  * k_mlp_forward  persistent, two 128-row tiles in flight per CTA: the four
//                   layers fused, weights resident in shared memory, the
//                   input streamed by TMA through a ring of shared-memory
//                   chunks, hidden activations kept in tensor memory (the
//                   next layer's A operand);
//  * k_gemm_tc      C (+)= op(A) op(B) for the backward pass (any strides,
//                   transposes folded into the shared-memory staging);
//  * small CUDA-core kernels for features, the loss gradient, GELU', bias
//    gradients and Adam.
//
// Operand layout in shared memory: K-major, no swizzle.  Element (r, k) of an
// R x K BF16 operand lives at ((r/8)*(K/8) + k/8)*128 + (r%8)*16 + (k%8)*2
// bytes: 8x8 core matrices of 128 contiguous bytes, 128 B apart along K
// (leading byte offset) and K/8*128 B apart along the rows (stride byte
// offset).  Every wait on an mbarrier is bounded; on a timeout the kernel
// records an error code, waits once more (bounded), frees its tensor memory
// and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/dmr.h"
#include "dmr_device.cuh"
#include "dmr_internal.cuh"

namespace dmr {
namespace {

constexpr int kIn = 256, kHid = 128, kOutP = 16, kOut = 6;
constexpr long kWaitLimit = 1L << 22;  // try_wait polls before giving up
constexpr int kErrTimeout = 1;

// flat parameter layout: [W1 b1 W2 b2 W3 b3 W4 b4], weights [out][in]
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
              kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid * kHid, kOffW4 = kOffB3 + kHid,
              kOffB4 = kOffW4 + kOutP * kHid, kNParams = kOffB4 + kOutP;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t kmaj_off(int r, int k, int K) {
  return ((uint32_t)((r >> 3) * (K >> 3) + (k >> 3)) << 7) + ((uint32_t)(r & 7) << 4) + ((uint32_t)(k & 7) << 1);
}

// Shared-memory matrix descriptor: start, leading / stride byte offsets,
// descriptor version 1 (sm_100 family), no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// D (+)= A B with A (M x K, BF16 pairs per 32-bit column, row m in lane m)
// in tensor memory.
__device__ __forceinline__ void mma_bf16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                            uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* m, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity) {
  for (long i = 0; i < kWaitLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_u32(m)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// One mbarrier arrival that also expects `bytes` of asynchronous copies.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
// TMA: the box at (x, y, z) of a 3-D tensor map into shared memory,
// completing on mbarrier m.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint64_t* m) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(m))
      : "memory");
}
// TMA: the box at (x, y) of a 2-D tensor map into shared memory, completing
// on mbarrier m.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint64_t* m) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(m))
      : "memory");
}

// GELU in its tanh form (Hendrycks & Gimpel): 0.5 z (1 + tanh(c (z + a z^3))),
// c = sqrt(2/pi), a = 0.044715; tanh from the hardware approximation, whose
// error is below the BF16 rounding the activations receive.
__device__ __forceinline__ float tanh_hw(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
constexpr float kGeluC = 0.7978845608028654f, kGeluA = 0.044715f;
// c (z + a z^3) as z (c + c a z^2), and 0.5 z (1 + t) as h + h t with h = z / 2:
// five FP32 operations besides the tanh
constexpr float kGeluCA = kGeluC * kGeluA;
__device__ __forceinline__ float gelu(float z) {
  const float t = tanh_hw(z * fmaf(kGeluCA, z * z, kGeluC));
  const float h = 0.5f * z;
  return fmaf(h, t, h);
}
__device__ __forceinline__ float gelu_grad(float z) {
  const float t = tanh_hw(kGeluC * fmaf(kGeluA * z, z * z, z));
  return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * kGeluC * fmaf(3.0f * kGeluA, z * z, 1.0f);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// Load R x K BF16 weights [R][K] from global into the canonical layout.
__device__ void stage_weights(unsigned char* dst, const __nv_bfloat16* W, int R, int K) {
  const int chunks = R * (K / 8);
  for (int e = threadIdx.x; e < chunks; e += blockDim.x) {
    int r = e / (K / 8), c = e % (K / 8);
    uint4 v = *reinterpret_cast<const uint4*>(W + (size_t)r * K + c * 8);
    *reinterpret_cast<uint4*>(dst + kmaj_off(r, c * 8, K)) = v;
  }
}

// Fused forward.  X [n][256] BF16 (through the tensor map tmX); out [n][6]
// FP32 = (mean, log-variance).  Optional saves for training: Z [3][n][128]
// FP32 pre-activations and H [3][n][128] BF16 activations.
//
// Two 128-row tiles are in flight per CTA: warps 0-7 (group 0) and 8-15
// (group 1) take the CTA's tiles alternately (its i-th tile, i = 0, 1, ...,
// goes to group i % 2) and run them through the four layers, so the tensor
// core multiplies one group's layer while the other group's warps run their
// bias + GELU epilogue.  Each group owns 256 TMEM columns: the FP32
// accumulator (128) and the hidden activation as BF16 pairs (64), which the
// epilogue stores there and the next layer's MMAs read as their A operand.
// The input reaches shared memory by TMA in chunks of 128 rows x 32 K (8 KB,
// 8 per tile; column group q of 8 columns at 2 KB q, row r at 16 r within
// it: 8 x 8 core matrices 2 KB apart along K and 128 B apart along the
// rows) through a ring of kRing slots: chunk j of tile i is number
// 8 i + j, slot (8 i + j) % kRing, completing on that slot's mbarrier.  The
// first kRing chunks are loaded up front; when a tile's layer-1 MMAs have
// completed, its group loads the chunks kRing further on into the slots it
// freed, so the next tiles' inputs arrive while this tile runs layers 2-4.
// A tile's layer 1 starts only after the previous tile's layer 1 has
// completed, so every slot mbarrier a group waits on is at most one phase
// ahead of the last phase it completed (the parity wait is unambiguous).
// The weights (132 KB) stay resident.
constexpr int kRing = 11;
constexpr int kChunkK = 32, kChunks = kIn / kChunkK;
constexpr uint32_t kChunkBytes = 128u * kChunkK * 2u;
struct FwdSmem {
  static constexpr uint32_t W1 = 0, W2 = W1 + kHid * kIn * 2, W3 = W2 + kHid * kHid * 2, W4 = W3 + kHid * kHid * 2,
                            RING = W4 + kOutP * kHid * 2, BIAS = RING + kRing * kChunkBytes,
                            MBAR = BIAS + (3 * kHid + kOutP) * 4,  // acc[2], full[kRing]
                            FLAG = MBAR + 8 * (2 + kRing),          // layer-1 tiles done, highest chunk issued
                            SLOT = FLAG + 8, TOTAL = SLOT + 16;
};
static_assert(FwdSmem::RING % 1024 == 0 && FwdSmem::MBAR % 8 == 0, "forward shared-memory layout");

// 16 warps = two groups of 8; in a group, warp w reads TMEM lanes
// 32 (w % 4) .. + 31 (its rows) and accumulator columns 64 (w / 4) .. + 63.
constexpr int kFwdThreads = 512;
constexpr int kGroupThreads = 256;

__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kGroupThreads) : "memory");
}
// Group barrier that returns the AND of `pred` over the group's threads.
__device__ __forceinline__ bool group_all(int g, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
      "barrier.cta.red.and.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(1 + g), "r"(kGroupThreads)
      : "memory");
  return r != 0;
}

__global__ void __launch_bounds__(kFwdThreads, 1)
    k_mlp_forward(const __grid_constant__ CUtensorMap tmX, int map3d, int n, const __nv_bfloat16* __restrict__ Wb,
                  const float* __restrict__ P, float* __restrict__ out, float* __restrict__ Zs,
                  __nv_bfloat16* __restrict__ Hs, int* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = warp >> 3, gt = tid & (kGroupThreads - 1), wl = warp & 7;
  uint64_t* accb = reinterpret_cast<uint64_t*>(sm + FwdSmem::MBAR) + g;
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + FwdSmem::MBAR) + 2;
  volatile int* l1done = reinterpret_cast<volatile int*>(sm + FwdSmem::FLAG);
  int* issued = reinterpret_cast<int*>(sm + FwdSmem::FLAG) + 1;
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + FwdSmem::SLOT);
  float* bias = reinterpret_cast<float*>(sm + FwdSmem::BIAS);
  const uint32_t sRing = smem_u32(sm + FwdSmem::RING);
  const int tiles = (n + 127) / 128;
  // this CTA's tiles: blockIdx.x + i gridDim.x, i < my_tiles
  const int my_tiles = (int)blockIdx.x < tiles ? (tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  const int n_chunks = my_tiles * kChunks;
  auto load_chunk = [&](int seq) {
    const int i = seq / kChunks, j = seq % kChunks;
    const int sl = seq % kRing;
    const int y = ((int)blockIdx.x + i * (int)gridDim.x) * 128;
    mbar_expect_tx(full + sl, kChunkBytes);
    if (map3d) {
      // (8 columns, 128 rows, 4 column groups): the whole chunk in one copy
      tma_load_3d(sRing + (uint32_t)sl * kChunkBytes, &tmX, 0, y, (kChunkK / 8) * j, full + sl);
    } else {
      for (int q = 0; q < kChunkK / 8; ++q)  // 8 columns x 128 rows (2 KB) per copy
        tma_load_2d(sRing + (uint32_t)sl * kChunkBytes + 2048u * q, &tmX, kChunkK * j + 8 * q, y, full + sl);
    }
  };
  if (warp == 0) tmem_alloc(slot, 512);
  if (tid == 0) {
    mbar_init(accb, 1);
    mbar_init(accb + 1, 1);
    for (int r = 0; r < kRing; ++r) mbar_init(full + r, 1);
    *l1done = 0;
    *issued = min(kRing, n_chunks);
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmX)) : "memory");
    for (int q = 0; q < min(kRing, n_chunks); ++q) load_chunk(q);
  }
  stage_weights(sm + FwdSmem::W1, Wb + kOffW1, kHid, kIn);
  stage_weights(sm + FwdSmem::W2, Wb + kOffW2, kHid, kHid);
  stage_weights(sm + FwdSmem::W3, Wb + kOffW3, kHid, kHid);
  stage_weights(sm + FwdSmem::W4, Wb + kOffW4, kOutP, kHid);
  for (int i = tid; i < kHid; i += kFwdThreads) {
    bias[i] = P[kOffB1 + i];
    bias[kHid + i] = P[kOffB2 + i];
    bias[2 * kHid + i] = P[kOffB3 + i];
  }
  if (tid < kOutP) bias[3 * kHid + tid] = P[kOffB4 + tid];
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tacc = *slot + 256u * (uint32_t)g;  // this group's accumulator columns
  const uint32_t thid = tacc + 128u;                  // and its hidden activation (64 columns of BF16 pairs)
  const uint32_t sW[4] = {smem_u32(sm + FwdSmem::W1), smem_u32(sm + FwdSmem::W2), smem_u32(sm + FwdSmem::W3),
                          smem_u32(sm + FwdSmem::W4)};
  const int quarter = wl & 3, cgrp = wl >> 2;
  const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
  uint32_t phase = 0;
  bool ok = true;
  bool pending = false;  // the group's issuer committed MMAs nobody has waited for
  // Every wait's outcome is made uniform over the group (a barrier with an
  // AND) before any branch on it, so all 256 threads pass the same barriers.
  auto wait_acc = [&]() -> bool {
    const bool w = group_all(g, mbar_wait(accb, phase));
    if (w) {
      phase ^= 1u;
      pending = false;
    }
    tc_fence_after();
    return w;
  };
  for (int i = g; i < my_tiles && ok; i += 2) {
    const int m0 = ((int)blockIdx.x + i * (int)gridDim.x) * 128;
    // layer 1: the tile's 8 input chunks from the ring (the accumulator is
    // free: the group finished the previous tile)
    bool good = true;
    if (gt == 0) {
      long w = 0;
      while (*l1done < i && w < kWaitLimit) ++w;
      good = *l1done >= i;
      bool any = false;
      for (int j = 0; j < kChunks && good; ++j) {
        const int seq = i * kChunks + j, sl = seq % kRing;
        good = mbar_wait(full + sl, (uint32_t)((seq / kRing) & 1));
        if (!good) break;
        if (j == 0) tc_fence_after();
#pragma unroll
        for (int s2 = 0; s2 < kChunkK / 16; ++s2)
          mma_bf16(tacc, sdesc(sRing + (uint32_t)sl * kChunkBytes + 4096u * s2, 2048u, 128u),
                   sdesc(sW[0] + 256u * (2 * j + s2), 128u, (kIn / 8) * 128u), idesc_bf16(128, kHid),
                   (j > 0 || s2 > 0) ? 1u : 0u);
        any = true;
      }
      if (any) {
        mma_commit(accb);  // also after a failed wait: the exit path waits for it
        pending = true;
      }
    }
    if (!(ok = group_all(g, good))) break;
    if (!(ok = wait_acc())) break;
    if (gt == 0) {
      // the chunks of this tile are consumed: load the ones kRing further on
      // into their slots, then let the next tile's layer 1 start
      for (int j = 0; j < kChunks; ++j) {
        const int seq = i * kChunks + j + kRing;
        if (seq < n_chunks) load_chunk(seq);
      }
      atomicMax(issued, min(i * kChunks + kChunks + kRing, n_chunks));
      __threadfence_block();
      *l1done = i + 1;
    }
    const int row = 32 * quarter + lane;
    const int grow = m0 + row;
    for (int layer = 0; layer < 4; ++layer) {
      if (layer > 0) {
        // the hidden activation is in tensor memory (every thread waited for
        // its stores) and the accumulator has been read
        tmem_wait_st();
        tc_fence_before();
        group_sync(g);
        if (gt == 0) {
          tc_fence_after();
          const int N = layer == 3 ? kOutP : kHid;
          for (int s = 0; s < kHid / 16; ++s)
            mma_bf16_ta(tacc, thid + 8u * s, sdesc(sW[layer] + 256u * s, 128u, (kHid / 8) * 128u), idesc_bf16(128, N),
                        s > 0 ? 1u : 0u);
          mma_commit(accb);
          pending = true;
        }
        if (!(ok = wait_acc())) break;
      }
      if (layer < 3) {
        // bias + GELU -> the next layer's A operand in tensor memory
        for (int half = 0; half < 2; ++half) {
          const int c0 = 64 * cgrp + 32 * half;
          float v[32];
          tmem_ld32(tacc + lane_off + (uint32_t)c0, v);
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] += bias[layer * kHid + c0 + j];
          if (Zs && grow < n)
            for (int j = 0; j < 32; ++j) Zs[((size_t)layer * n + grow) * kHid + c0 + j] = v[j];
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = gelu(v[j]);
          uint32_t pk[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) pk[q] = pack_bf16(v[2 * q], v[2 * q + 1]);
          tmem_st16(thid + lane_off + (uint32_t)(c0 / 2), pk);
          if (Hs && grow < n)
#pragma unroll
            for (int q = 0; q < 4; ++q)
              *reinterpret_cast<uint4*>(Hs + ((size_t)layer * n + grow) * kHid + c0 + 8 * q) =
                  make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
        }
      } else if (cgrp == 0) {
        float v[16];
        tmem_ld16(tacc + lane_off, v);
        if (grow < n)
          for (int j = 0; j < kOut; ++j) out[(size_t)grow * kOut + j] = v[j] + bias[3 * kHid + j];
      }
    }
    if (!ok) break;
    // the next tile's layer 1 overwrites the accumulator: every warp of the
    // group is done with it
    tc_fence_before();
    group_sync(g);
  }
  if (!ok && gt == 0) {
    atomicExch(err, kErrTimeout);
    if (pending) (void)mbar_wait(accb, phase);  // give an outstanding commit one more bounded chance
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    // no copy may be in flight when the CTA leaves: the last kRing chunks
    // issued occupy distinct slots, so each slot's latest phase is theirs
    const int hi = *issued;
    for (int seq = max(0, hi - kRing); seq < hi; ++seq) (void)mbar_wait(full + seq % kRing, (uint32_t)((seq / kRing) & 1));
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(*slot, 512);
  }
}

// C (+)= op(A) op(B): A(m,k) = A[m*sam + k*sak], B(n,k) = B[n*sbn + k*sbk]
// (BF16 or FP32 sources, rounded to BF16), C(m,n) = C[m*scm + n*scn] FP32.
// CTA (x, y) computes rows 128 x .. + 127, all N (<= 256) columns, over the
// y-th of gridDim.y contiguous K ranges of kspan (a multiple of 64), in
// chunks of 64 staged by the CTA's threads into two shared-memory buffers:
// the tensor core multiplies chunk c while chunk c + 1 is staged.  Operands
// are read along their contiguous index (coalesced).  With one K range the
// result goes to C; with several, range y writes its partial product to
// part[y][M][N] and k_splitk_reduce adds the ranges in order.
template <typename TA, typename TB>
__global__ void __launch_bounds__(128) k_gemm_tc(int M, int N, int K, int kspan, const TA* __restrict__ A, long sam,
                                                 long sak, const TB* __restrict__ B, long sbn, long sbk, float* C,
                                                 long scm, long scn, int accumulate, float* part, int* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int Np = (N + 15) & ~15;
  const uint32_t ncols = Np <= 32 ? 32u : (Np <= 64 ? 64u : (Np <= 128 ? 128u : 256u));
  constexpr uint32_t kStage = 16384 + 32768;  // A 128 x 64 + B <= 256 x 64, BF16
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + 2 * kStage);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + 2 * kStage + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128;
  const int kb = blockIdx.y * kspan, ke = min(K, kb + kspan);
  const int nch = ke > kb ? (ke - kb + 63) / 64 : 0;
  if (warp == 0) tmem_alloc(slot, ncols);
  if (tid == 0) {
    mbar_init(mbar, 1);
    mbar_init(mbar + 1, 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *slot;
  bool ok = true;
  for (int c = 0; c < nch && ok; ++c) {
    const int buf = c & 1;
    unsigned char* sA = sm + buf * kStage;
    unsigned char* sB = sA + 16384;
    // the buffer was last read by the MMAs of chunk c - 2
    if (c >= 2) ok = __syncthreads_and(mbar_wait(mbar + buf, (uint32_t)(((c - 2) >> 1) & 1))) != 0;
    if (!ok) break;
    tc_fence_after();
    const int k0 = kb + 64 * c;
    if (sak == 1) {
      for (int e = tid; e < 128 * 64; e += 128) {
        const int r = e >> 6, kk = e & 63, m = m0 + r, k = k0 + kk;
        const float v = (m < M && k < ke) ? (float)A[(size_t)m * sam + (size_t)k] : 0.f;
        *reinterpret_cast<__nv_bfloat16*>(sA + kmaj_off(r, kk, 64)) = __float2bfloat16_rn(v);
      }
    } else {
      for (int e = tid; e < 128 * 64; e += 128) {
        const int r = e & 127, kk = e >> 7, m = m0 + r, k = k0 + kk;
        const float v = (m < M && k < ke) ? (float)A[(size_t)m * sam + (size_t)k * sak] : 0.f;
        *reinterpret_cast<__nv_bfloat16*>(sA + kmaj_off(r, kk, 64)) = __float2bfloat16_rn(v);
      }
    }
    if (sbk == 1) {
      for (int e = tid; e < Np * 64; e += 128) {
        const int r = e >> 6, kk = e & 63, k = k0 + kk;
        const float v = (r < N && k < ke) ? (float)B[(size_t)r * sbn + (size_t)k] : 0.f;
        *reinterpret_cast<__nv_bfloat16*>(sB + kmaj_off(r, kk, 64)) = __float2bfloat16_rn(v);
      }
    } else {
      for (int e = tid; e < Np * 64; e += 128) {
        const int r = e % Np, kk = e / Np, k = k0 + kk;
        const float v = (r < N && k < ke) ? (float)B[(size_t)r * sbn + (size_t)k * sbk] : 0.f;
        *reinterpret_cast<__nv_bfloat16*>(sB + kmaj_off(r, kk, 64)) = __float2bfloat16_rn(v);
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      for (int s = 0; s < 4; ++s)
        mma_bf16(tbase, sdesc(smem_u32(sA) + 256u * s, 128u, 1024u), sdesc(smem_u32(sB) + 256u * s, 128u, 1024u),
                 idesc_bf16(128, Np), (c > 0 || s > 0) ? 1u : 0u);
      mma_commit(mbar + buf);  // tracks every MMA issued so far
    }
  }
  // the last chunk's commit covers all earlier MMAs
  if (ok && nch > 0) {
    const int last = nch - 1;
    ok = __syncthreads_and(mbar_wait(mbar + (last & 1), (uint32_t)((last >> 1) & 1))) != 0;
    tc_fence_after();
  }
  if (ok) {
    const int m = m0 + 32 * warp + lane;
    const uint32_t lb = tbase + ((uint32_t)(32 * warp) << 16);
    for (int c0 = 0; c0 < Np; c0 += 16) {
      float v[16];
      if (nch > 0) {
        tmem_ld16(lb + (uint32_t)c0, v);
      } else {
        for (int j = 0; j < 16; ++j) v[j] = 0.f;
      }
      if (m < M)
        for (int j = 0; j < 16; ++j) {
          const int n = c0 + j;
          if (n < N) {
            if (gridDim.y > 1) {
              part[((size_t)blockIdx.y * M + m) * N + n] = v[j];
            } else {
              float* dst = C + (size_t)m * scm + (size_t)n * scn;
              *dst = accumulate ? *dst + v[j] : v[j];
            }
          }
        }
    }
  } else {
    if (tid == 0) atomicExch(err, kErrTimeout);
    // give outstanding commits one more bounded chance before the tensor
    // memory is released
    if (nch > 0) (void)mbar_wait(mbar + ((nch - 1) & 1), (uint32_t)(((nch - 1) >> 1) & 1));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, ncols);
  }
}

// C (+)= sum over the K ranges of their partial products part[S][M][N], in
// range order (deterministic).
__global__ void k_splitk_reduce(int M, int N, int S, const float* __restrict__ part, float* C, long scm, long scn,
                                int accumulate) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= (long)M * N) return;
  const int m = (int)(i / N), n = (int)(i % N);
  float acc = 0.f;
  for (int y = 0; y < S; ++y) acc += part[((size_t)y * M + m) * N + n];
  float* dst = C + (size_t)m * scm + (size_t)n * scn;
  *dst = accumulate ? *dst + acc : acc;
}

// Features of (candidate, point) rows: 5x5x5 trilinear samples of the source
// image around the source point and of the target image around the target
// point (offsets -2..2 voxels), the correspondence offset t - s / 8 and the
// source point over the image size.  X [C*P][256] BF16.
__global__ void k_mlp_features(const DevProblem* probs, const double* __restrict__ coords, int C,
                               __nv_bfloat16* __restrict__ X) {
  const DevProblem& pr = probs[0];
  const long row = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (row >= (long)C * pr.P) return;
  const int c = (int)(row / pr.P), p = (int)(row % pr.P);
  float pt[2][3];
  for (int mesh = 0; mesh < 2; ++mesh)
    for (int a = 0; a < 3; ++a) pt[mesh][a] = (float)coords[((size_t)c * 6 + mesh * 3 + a) * pr.P + p];
  __nv_bfloat16* out = X + (size_t)row * kIn;
  int f = 0;
  for (int mesh = 0; mesh < 2; ++mesh) {
    const int* n = pr.n[mesh];
    for (int dz = -2; dz <= 2; ++dz)
      for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
          float q[3] = {pt[mesh][0] + dx, pt[mesh][1] + dy, pt[mesh][2] + dz};
          int i0[3], i1[3];
          float fr[3];
          for (int a = 0; a < 3; ++a) {
            float x = fminf(fmaxf(q[a], -1.0f), (float)n[a]);
            if (!(x == x)) x = -1.0f;
            float fl = floorf(x);
            fr[a] = x - fl;
            int i = (int)fl;
            i0[a] = min(max(i, 0), n[a] - 1);
            i1[a] = min(max(i + 1, 0), n[a] - 1);
          }
          float s = 0.f;
          for (int cz = 0; cz < 2; ++cz)
            for (int cy = 0; cy < 2; ++cy)
              for (int cx = 0; cx < 2; ++cx) {
                float wgt = (cx ? fr[0] : 1 - fr[0]) * (cy ? fr[1] : 1 - fr[1]) * (cz ? fr[2] : 1 - fr[2]);
                long li = ((long)(cz ? i1[2] : i0[2]) * n[1] + (cy ? i1[1] : i0[1])) * n[0] + (cx ? i1[0] : i0[0]);
                s += wgt * load_plain_dyn(pr.plain[mesh], pr.dtype, li);
              }
          out[f++] = __float2bfloat16_rn(s);
        }
  }
  for (int a = 0; a < 3; ++a) out[f++] = __float2bfloat16_rn((pt[1][a] - pt[0][a]) * 0.125f);
  for (int a = 0; a < 3; ++a) out[f++] = __float2bfloat16_rn(pt[0][a] / (float)pr.n[0][a]);
}

// Gaussian NLL gradient w.r.t. the output layer's pre-activation (padded to
// 16 columns) and the loss sum.
__global__ void k_nll_grad(const float* __restrict__ out, const float* __restrict__ Y, int n, float* dZ4,
                           double* loss_sum) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double l = 0.0;
  for (int d = 0; d < 3; ++d) {
    float mu = out[(size_t)i * kOut + d], s = out[(size_t)i * kOut + 3 + d];
    float r = Y[(size_t)i * 3 + d] - mu;
    float e = expf(-s);
    dZ4[(size_t)i * kOutP + d] = -r * e / (float)n;
    dZ4[(size_t)i * kOutP + 3 + d] = 0.5f * (1.0f - r * r * e) / (float)n;
    l += 0.5 * ((double)r * r * e + s);
  }
  for (int d = kOut; d < kOutP; ++d) dZ4[(size_t)i * kOutP + d] = 0.f;
  atomicAdd(loss_sum, l);
}

// dZ = dH * GELU'(Z), element-wise over [n][128].
__global__ void k_gelu_back(const float* __restrict__ dH, const float* __restrict__ Z, float* dZ, long count) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < count) dZ[i] = dH[i] * gelu_grad(Z[i]);
}

// Column sums of dZ [n][cols] into g[cols], in two passes: CTA b adds rows
// 128 b .. 128 b + 127 of every column (thread c takes column c, so a warp
// reads consecutive columns of a row) into part[b][cols]; k_colsum_fin adds
// the partial sums of a column in order of b (deterministic).
constexpr int kColRows = 128;
__global__ void k_colsum_part(const float* __restrict__ dZ, int n, int cols, float* part) {
  const int c = threadIdx.x, r0 = blockIdx.x * kColRows;
  if (c >= cols) return;
  float s = 0.f;
  const int r1 = min(n, r0 + kColRows);
  for (int i = r0; i < r1; ++i) s += dZ[(size_t)i * cols + c];
  part[(size_t)blockIdx.x * cols + c] = s;
}
__global__ void k_colsum_fin(const float* __restrict__ part, int groups, int cols, float* g) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double s = 0.0;
  for (int b = 0; b < groups; ++b) s += part[(size_t)b * cols + c];
  g[c] = (float)s;
}

__global__ void k_adam(float* P, const float* G, float* m, float* v, int count, float lr, float b1, float b2,
                       float eps, float c1, float c2, __nv_bfloat16* Wb) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  float g = G[i];
  float mi = b1 * m[i] + (1.f - b1) * g;
  float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  float p = P[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  // padding rows of the output layer stay zero
  if ((i >= kOffW4 + kOut * kHid && i < kOffB4) || i >= kOffB4 + kOut) p = 0.f;
  P[i] = p;
  Wb[i] = __float2bfloat16_rn(p);
}

__global__ void k_to_bf16(const float* P, __nv_bfloat16* Wb, int count) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) Wb[i] = __float2bfloat16_rn(P[i]);
}

// Largest number of K ranges a product is split into, and the partial-product
// workspace it needs (ranges x 128 x 256 FP32 for the weight gradients; the
// column sums of the bias gradients use it too).
constexpr int kMaxSplit = 64;
constexpr size_t kSplitWs = (size_t)kMaxSplit * 128 * 256;

// C (+)= op(A) op(B) on the tensor cores.  A product with few row tiles and a
// long K (the weight gradients: M = 128 outputs, K = batch rows) is split
// into K ranges so that about two CTAs per SM work on it; the ranges' partial
// products are added by k_splitk_reduce.
template <typename TA, typename TB>
void gemm(int M, int N, int K, const TA* A, long sam, long sak, const TB* B, long sbn, long sbk, float* C, long scm,
          long scn, int acc, int* err, float* ws, int n_sm, cudaStream_t st) {
  const size_t smem = 2 * (16384 + 32768) + 32;
  // per launch: the attribute belongs to the current device
  cudaFuncSetAttribute(k_gemm_tc<TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int mt = (M + 127) / 128, chunks = (K + 63) / 64;
  int S = std::min(std::max(1, (2 * n_sm + mt - 1) / mt), chunks);
  if ((size_t)S * M * N > kSplitWs) S = std::max(1, (int)(kSplitWs / ((size_t)M * N)));
  S = std::min(S, kMaxSplit);
  const int kspan = 64 * ((chunks + S - 1) / S);
  S = (K + kspan - 1) / kspan;
  if (S < 1) S = 1;
  k_gemm_tc<TA, TB><<<dim3(mt, S), 128, smem, st>>>(M, N, K, kspan, A, sam, sak, B, sbn, sbk, C, scm, scn, acc,
                                                     S > 1 ? ws : nullptr, err);
  if (S > 1) {
    const long cnt = (long)M * N;
    k_splitk_reduce<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(M, N, S, ws, C, scm, scn, acc);
  }
}

void colsum(const float* dZ, int n, int cols, float* g, float* ws, cudaStream_t st) {
  const int groups = (n + kColRows - 1) / kColRows;
  k_colsum_part<<<groups, cols, 0, st>>>(dZ, n, cols, ws);
  k_colsum_fin<<<(cols + 127) / 128, 128, 0, st>>>(ws, groups, cols, g);
}

}  // namespace
}  // namespace dmr

using namespace dmr;

struct dmr_mlp {
  cudaStream_t st = nullptr;
  int n_sm = 1;
  float* P = nullptr;   // FP32 master parameters
  float* G = nullptr;   // gradients
  float* m = nullptr;   // Adam moments
  float* v = nullptr;
  __nv_bfloat16* Wb = nullptr;  // BF16 copy for the tensor cores
  int* err = nullptr;
  double* loss = nullptr;
  int t = 0;
  // training workspace
  int cap = 0;
  float *out = nullptr, *Zs = nullptr, *dZ4 = nullptr, *dH = nullptr, *dZ = nullptr;
  __nv_bfloat16* Hs = nullptr;
  float* split = nullptr;  // partial products of split-K weight gradients
};

namespace {

template <class T>
int mlp_alloc(T** p, size_t count) {
  if (cudaMalloc((void**)p, sizeof(T) * (count ? count : 1)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return set_error(DMR_ENOMEM, "cudaMalloc failed (mlp)");
  }
  return DMR_OK;
}

int check_err(dmr_mlp* M) {
  int e = 0;
  if (cudaMemcpyAsync(&e, M->err, sizeof(int), cudaMemcpyDeviceToHost, M->st) != cudaSuccess ||
      cudaStreamSynchronize(M->st) != cudaSuccess)
    return set_error(DMR_ECUDA, std::string("mlp: ") + cudaGetErrorString(cudaGetLastError()));
  if (e) {
    cudaMemsetAsync(M->err, 0, sizeof(int), M->st);
    return set_error(DMR_ETIMEOUT, "mlp: a tensor-core wait gave up");
  }
  return DMR_OK;
}

int ensure_ws(dmr_mlp* M, int n) {
  if (n <= M->cap) return DMR_OK;
  cudaFree(M->out); cudaFree(M->Zs); cudaFree(M->dZ4); cudaFree(M->dH); cudaFree(M->dZ); cudaFree(M->Hs);
  M->out = M->Zs = M->dZ4 = M->dH = M->dZ = nullptr;
  M->Hs = nullptr;
  M->cap = 0;
  int rc;
  if ((rc = mlp_alloc(&M->out, (size_t)n * kOut)) || (rc = mlp_alloc(&M->Zs, (size_t)3 * n * kHid)) ||
      (rc = mlp_alloc(&M->dZ4, (size_t)n * kOutP)) || (rc = mlp_alloc(&M->dH, (size_t)n * kIn)) ||
      (rc = mlp_alloc(&M->dZ, (size_t)n * kHid)) || (rc = mlp_alloc(&M->Hs, (size_t)3 * n * kHid)))
    return rc;
  M->cap = n;
  return DMR_OK;
}

// The driver's tensor-map encoder, looked up once through the runtime.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// X BF16 [n][256] as a tensor map whose boxes land in the ring's layout:
// 3-D (column within a group of 8, row, group of 8 columns; strides 512 and
// 16 bytes), box 8 x 128 x 4 = one chunk; where the driver does not take
// that view, 2-D (column, row), box 8 x 128, four per chunk.  Rows past n
// read as 0.
int make_input_map(const __nv_bfloat16* X, int n, CUtensorMap* map, int* map3d) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return set_error(DMR_ECUDA, "mlp: cuTensorMapEncodeTiled not available");
  if (((uintptr_t)X & 15u) != 0) return set_error(DMR_EINVAL, "mlp: X must be 16-byte aligned");
  {
    const cuuint64_t dims[3] = {8, (cuuint64_t)n, (cuuint64_t)kIn / 8};
    const cuuint64_t strides[2] = {(cuuint64_t)kIn * 2, 16};
    const cuuint32_t box[3] = {8, 128, (cuuint32_t)kChunkK / 8};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)X, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
        CUDA_SUCCESS) {
      *map3d = 1;
      return DMR_OK;
    }
  }
  const cuuint64_t dims[2] = {(cuuint64_t)kIn, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)kIn * 2};
  const cuuint32_t box[2] = {8, 128};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)X, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(DMR_ECUDA, "mlp: input tensor map rejected (" + std::to_string((int)r) + ")");
  *map3d = 0;
  return DMR_OK;
}

int launch_forward(dmr_mlp* M, const __nv_bfloat16* X, int n, float* out, float* Zs, __nv_bfloat16* Hs) {
  // per launch: the attribute belongs to the current device
  cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FwdSmem::TOTAL);
  CUtensorMap map;
  int map3d = 0;
  const int rc = make_input_map(X, n, &map, &map3d);
  if (rc) return rc;
  int tiles = (n + 127) / 128;
  // two tiles in flight per CTA once there are more tiles than SMs; with
  // fewer (training batches) one tile per CTA, on more SMs
  int grid = tiles <= M->n_sm ? tiles : std::min((tiles + 1) / 2, M->n_sm);
  k_mlp_forward<<<grid, kFwdThreads, FwdSmem::TOTAL, M->st>>>(map, map3d, n, M->Wb, M->P, out, Zs, Hs, M->err);
  return DMR_OK;
}

// SplitMix64, a published counter-based generator, for the initial weights.
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int dmr_mlp_create(unsigned long long seed, void* stream, dmr_mlp** out) {
  if (!out) return set_error(DMR_EINVAL, "null argument");
  *out = nullptr;
  dmr_mlp* M = new dmr_mlp();
  M->st = (cudaStream_t)stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&M->n_sm, cudaDevAttrMultiProcessorCount, dev);
  int rc;
  if ((rc = mlp_alloc(&M->P, kNParams)) || (rc = mlp_alloc(&M->G, kNParams)) || (rc = mlp_alloc(&M->m, kNParams)) ||
      (rc = mlp_alloc(&M->v, kNParams)) || (rc = mlp_alloc(&M->Wb, kNParams)) || (rc = mlp_alloc(&M->err, 1)) ||
      (rc = mlp_alloc(&M->loss, 1)) || (rc = mlp_alloc(&M->split, kSplitWs))) {
    dmr_mlp_destroy(M);
    return rc;
  }
  // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases
  std::vector<float> h(kNParams, 0.f);
  uint64_t s = seed;
  auto fill = [&](int off, int rows, int cols, int live_rows) {
    float bound = 1.0f / std::sqrt((float)cols);
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < cols; ++c) {
        double u = (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
        h[off + r * cols + c] = r < live_rows ? (float)((2.0 * u - 1.0) * bound) : 0.f;
      }
  };
  fill(kOffW1, kHid, kIn, kHid);
  fill(kOffW2, kHid, kHid, kHid);
  fill(kOffW3, kHid, kHid, kHid);
  fill(kOffW4, kOutP, kHid, kOut);
  cudaMemcpy(M->P, h.data(), sizeof(float) * kNParams, cudaMemcpyHostToDevice);
  cudaMemset(M->m, 0, sizeof(float) * kNParams);
  cudaMemset(M->v, 0, sizeof(float) * kNParams);
  cudaMemset(M->err, 0, sizeof(int));
  k_to_bf16<<<(kNParams + 255) / 256, 256, 0, M->st>>>(M->P, M->Wb, kNParams);
  if (cudaStreamSynchronize(M->st) != cudaSuccess) {
    dmr_mlp_destroy(M);
    return set_error(DMR_ECUDA, "mlp create failed");
  }
  *out = M;
  return DMR_OK;
}

int dmr_mlp_destroy(dmr_mlp* M) {
  if (!M) return DMR_OK;
  cudaStreamSynchronize(M->st);
  cudaFree(M->P); cudaFree(M->G); cudaFree(M->m); cudaFree(M->v); cudaFree(M->Wb); cudaFree(M->err);
  cudaFree(M->loss); cudaFree(M->out); cudaFree(M->Zs); cudaFree(M->dZ4); cudaFree(M->dH); cudaFree(M->dZ);
  cudaFree(M->Hs);
  cudaFree(M->split);
  delete M;
  return DMR_OK;
}

int dmr_mlp_n_params(void) { return kNParams; }

int dmr_mlp_params(dmr_mlp* M, float* get, const float* set) {
  if (!M) return set_error(DMR_EINVAL, "null mlp");
  if (set) {
    if (cudaMemcpy(M->P, set, sizeof(float) * kNParams, cudaMemcpyDefault) != cudaSuccess)
      return set_error(DMR_ECUDA, "mlp set params");
    k_to_bf16<<<(kNParams + 255) / 256, 256, 0, M->st>>>(M->P, M->Wb, kNParams);
    cudaMemsetAsync(M->m, 0, sizeof(float) * kNParams, M->st);
    cudaMemsetAsync(M->v, 0, sizeof(float) * kNParams, M->st);
    M->t = 0;
  }
  if (get) {
    const int rc = check_err(M);  // synchronises; reports an earlier step's timeout
    if (rc) return rc;
    if (cudaMemcpy(get, M->P, sizeof(float) * kNParams, cudaMemcpyDefault) != cudaSuccess)
      return set_error(DMR_ECUDA, "mlp get params");
  }
  return DMR_OK;
}

int dmr_mlp_features(dmr_problem* p, const double* coords, int C, void* X) {
  if (!p || !coords || !X || C < 1) return set_error(DMR_EINVAL, "bad mlp feature arguments");
  DevProblem hp;
  int storage, warps, n_sm;
  cudaStream_t st;
  int rc = problem_view(p, &hp, &storage, &warps, &n_sm, &st);
  if (rc) return rc;
  // the problem's own device descriptor (first element of its array)
  const DevProblem* d = problem_device(p);
  long rows = (long)C * hp.P;
  k_mlp_features<<<(unsigned)((rows + 127) / 128), 128, 0, st>>>(d, coords, C, (__nv_bfloat16*)X);
  if (cudaGetLastError() != cudaSuccess) return set_error(DMR_ECUDA, "mlp features launch");
  return DMR_OK;
}

int dmr_mlp_forward(dmr_mlp* M, const void* X, int n, float* out) {
  if (!M || !X || !out || n < 1) return set_error(DMR_EINVAL, "bad mlp forward arguments");
  int rc = launch_forward(M, (const __nv_bfloat16*)X, n, out, nullptr, nullptr);
  if (rc) return rc;
  if (cudaGetLastError() != cudaSuccess) return set_error(DMR_ECUDA, "mlp forward launch");
  return check_err(M);
}

// One gradient evaluation (and, if lr > 0, one Adam step) on a batch.
int dmr_mlp_train_step(dmr_mlp* M, const void* Xv, const float* Y, int n, float lr, float* loss_out,
                       float* grad_out) {
  if (!M || !Xv || !Y || n < 1) return set_error(DMR_EINVAL, "bad mlp train arguments");
  if ((size_t)((n + kColRows - 1) / kColRows) * kHid > kSplitWs)
    return set_error(DMR_EINVAL, "mlp train: batch above " + std::to_string(kSplitWs / kHid * kColRows) + " rows");
  int rc = ensure_ws(M, n);
  if (rc) return rc;
  const __nv_bfloat16* X = (const __nv_bfloat16*)Xv;
  cudaStream_t st = M->st;
  cudaMemsetAsync(M->loss, 0, sizeof(double), st);
  if ((rc = launch_forward(M, X, n, M->out, M->Zs, M->Hs))) return rc;
  k_nll_grad<<<(n + 127) / 128, 128, 0, st>>>(M->out, Y, n, M->dZ4, M->loss);
  float* G = M->G;
  const __nv_bfloat16* W = M->Wb;
  const __nv_bfloat16* H[3] = {M->Hs, M->Hs + (size_t)n * kHid, M->Hs + 2 * (size_t)n * kHid};
  const float* Z[3] = {M->Zs, M->Zs + (size_t)n * kHid, M->Zs + 2 * (size_t)n * kHid};
  // layer 4: dW4^T = H3^T dZ4 (M=128 in, N=16 out, K=n); b4; dH3 = dZ4 W4
  float* ws = M->split;
  const int nsm = M->n_sm;
  gemm(kHid, kOutP, n, H[2], 1, kHid, M->dZ4, 1, kOutP, G + kOffW4, 1, kHid, 0, M->err, ws, nsm, st);
  colsum(M->dZ4, n, kOutP, G + kOffB4, ws, st);
  gemm(n, kHid, kOutP, M->dZ4, kOutP, 1, W + kOffW4, 1, kHid, M->dH, kHid, 1, 0, M->err, ws, nsm, st);
  // layers 3..1
  const int offW[3] = {kOffW1, kOffW2, kOffW3}, offB[3] = {kOffB1, kOffB2, kOffB3};
  for (int l = 2; l >= 0; --l) {
    long cnt = (long)n * kHid;
    k_gelu_back<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(M->dH, Z[l], M->dZ, cnt);
    colsum(M->dZ, n, kHid, G + offB[l], ws, st);
    const int in = l == 0 ? kIn : kHid;
    // dW_l = dZ^T * input (M=128 out, N=in, K=n)
    if (l == 0)
      gemm(kHid, kIn, n, M->dZ, 1, kHid, X, 1, kIn, G + offW[l], kIn, 1, 0, M->err, ws, nsm, st);
    else
      gemm(kHid, kHid, n, M->dZ, 1, kHid, H[l - 1], 1, kHid, G + offW[l], kHid, 1, 0, M->err, ws, nsm, st);
    // dH_{l-1} = dZ W_l (M=n, N=in, K=128)
    if (l > 0) gemm(n, in, kHid, M->dZ, kHid, 1, W + offW[l], 1, in, M->dH, in, 1, 0, M->err, ws, nsm, st);
  }
  if (cudaGetLastError() != cudaSuccess) return set_error(DMR_ECUDA, "mlp backward launch");
  if (lr > 0) {
    M->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.f - std::pow(b1, (float)M->t), c2 = 1.f - std::pow(b2, (float)M->t);
    k_adam<<<(kNParams + 255) / 256, 256, 0, st>>>(M->P, G, M->m, M->v, kNParams, lr, b1, b2, 1e-8f, c1, c2, M->Wb);
  }
  if (!loss_out && !grad_out) {
    // nothing to return to the host: no synchronisation; a tensor-core wait
    // that gave up is reported by the next call that synchronises
    return cudaGetLastError() == cudaSuccess ? DMR_OK : set_error(DMR_ECUDA, "mlp train launch");
  }
  rc = check_err(M);
  if (rc) return rc;
  if (loss_out) {
    double l = 0;
    cudaMemcpy(&l, M->loss, sizeof(double), cudaMemcpyDeviceToHost);
    *loss_out = (float)(l / n);
  }
  if (grad_out && cudaMemcpy(grad_out, G, sizeof(float) * kNParams, cudaMemcpyDeviceToHost) != cudaSuccess)
    return set_error(DMR_ECUDA, "mlp grad copy");
  return DMR_OK;
}

}  // extern "C"
