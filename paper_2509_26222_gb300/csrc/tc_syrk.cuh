// Tensor-core (tcgen05) trailing update of the mixed-precision Cholesky.
//
// One CTA computes one 128 x 128 tile (ti >= tj) of
//     C -= P_i P_j^T,   P = Ph + Pm + Pl   (three bfloat16 slices of the
//                                           float32 panel, 24 bits in all)
// as the six slice products whose sum keeps every term down to 2^-24 of
// |P_i| |P_j|:  hh + hm + mh + hl + mm + lh, accumulated in float32 in tensor
// memory (TMEM) and subtracted from the float32 working matrix C in the
// epilogue (float64 arithmetic here would run on GB300's narrow FP64 pipe).
//
// Operand tiles are 128 rows x 64 bf16 (one 128-byte swizzle row per matrix
// row), K-major, 128-byte swizzled, written by the CTA's threads with plain
// shared-memory stores and read by tcgen05.mma through shared-memory
// descriptors.  One thread issues the 24 MMAs (6 products x 4 k-steps of 16),
// commits them to an mbarrier, and every thread waits with a bounded spin.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "tc_util.cuh"

namespace rbf {
namespace tc {

constexpr int TILE = 128;             // M = N = 128
constexpr int KB = 64;                // panel width (bf16 elements per row)
constexpr int SLICE_BYTES = TILE * KB * 2;   // 16 KiB per operand slice tile
constexpr int SMEM_BYTES = 6 * SLICE_BYTES + 1024;  // 3 A + 3 B slices, 1 KiB alignment slack
// Instruction descriptor: kind::f16, A = B = bf16, D = f32, K-major A and B,
// N = 128 (bits 17-22: N >> 3), M = 128 (bits 24-28: M >> 4).
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TILE >> 3) << 17) |
                           ((uint32_t)(TILE >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %3, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %4, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(accum), "r"(IDESC));
}

// Copy rows [r0, r0 + 128) of a bf16 slice (row-major, KB elements per row,
// rows >= m read as zero) into a swizzled tile with asynchronous 16-byte
// copies (all in flight at once; the caller waits with cp_async_wait_all).
__device__ __forceinline__ void load_tile(uint8_t* tile, const __nv_bfloat16* __restrict__ P, int64_t r0,
                                          int64_t m) {
  uint32_t base = smem_u32(tile);
  for (int e = threadIdx.x; e < TILE * 8; e += blockDim.x) {
    int r = e >> 3, chunk = e & 7;
    int64_t gr = r0 + r;
    const __nv_bfloat16* src = P + (gr < m ? gr : 0) * KB + chunk * 8;
    uint32_t bytes = gr < m ? 16u : 0u;  // 0: fill the 16 bytes with zeros
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(base + sw128_offset(r, chunk)), "l"(src),
                 "r"(bytes)
                 : "memory");
  }
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// C[i][j] -= sum over the six slice products, for the lower tile pairs of the
// m x m float32 block C (row-major, leading dimension ldc; ldc % 4 == 0 and a
// 16-byte aligned C take the vectorized path).  grid = T (T + 1) / 2
// CTAs with T = ceil(m / 128), 128 threads, SMEM_BYTES dynamic shared memory.
__global__ void __launch_bounds__(128) k_syrk_tc(float* __restrict__ Cm, int64_t ldc, int64_t m,
                                                 const __nv_bfloat16* __restrict__ Ph,
                                                 const __nv_bfloat16* __restrict__ Pm,
                                                 const __nv_bfloat16* __restrict__ Pl, int* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* tA[3] = {sm, sm + SLICE_BYTES, sm + 2 * SLICE_BYTES};
  uint8_t* tB[3] = {sm + 3 * SLICE_BYTES, sm + 4 * SLICE_BYTES, sm + 5 * SLICE_BYTES};

  int64_t b = blockIdx.x;
  int64_t ti = (int64_t)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
  while ((ti + 1) * (ti + 2) / 2 <= b) ++ti;
  while (ti * (ti + 1) / 2 > b) --ti;
  int64_t tj = b - ti * (ti + 1) / 2;
  int64_t i0 = ti * TILE, j0 = tj * TILE;

  const __nv_bfloat16* S[3] = {Ph, Pm, Pl};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    load_tile(tA[q], S[q], i0, m);
    load_tile(tB[q], S[q], j0, m);
  }
  cp_async_wait_all();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) tmem_alloc(&tmem_slot, TILE);
  if (threadIdx.x == 0) mbar_init(&mbar, 1);
  fence_proxy_async();
  fence_before();
  __syncthreads();
  fence_after();
  uint32_t tmem = tmem_slot;

  if (threadIdx.x == 0) {
    // (A slice, B slice) of the six products
    const int pa[6] = {0, 0, 1, 0, 1, 2};
    const int pb[6] = {0, 1, 0, 2, 1, 0};
    uint32_t accum = 0;
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      uint64_t ad = sdesc_sw128(smem_u32(tA[pa[p]]));
      uint64_t bd = sdesc_sw128(smem_u32(tB[pb[p]]));
#pragma unroll
      for (int kk = 0; kk < KB / 16; ++kk) {
        // advance 16 elements (32 bytes) along K inside the swizzle row
        mma_bf16(tmem, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), accum);
        accum = 1;
      }
    }
    mma_commit(&mbar);
  }
  // one thread waits (bounded) for the MMAs, then the whole CTA proceeds
  __shared__ int done_s;
  if (threadIdx.x == 0) {
    long long it = 0;
    bool ok;
    while (!(ok = mbar_try_wait(&mbar, 0)) && ++it < WAIT_LIMIT) {
    }
    done_s = ok ? 1 : 0;
    if (!ok) atomicOr(status, 2);
  }
  __syncthreads();
  fence_after();
  const bool done = done_s != 0;

  // epilogue: warp w owns TMEM lanes (rows) 32 w .. 32 w + 31
  int64_t row = i0 + warp * 32 + lane;
  if (done) {
#pragma unroll 1
    for (int cb = 0; cb < TILE / 32; ++cb) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 32), v);
      if (row < m) {
        float* crow = Cm + row * ldc + j0 + cb * 32;
        int ncol = (int)(m - (j0 + cb * 32));
        if (ncol >= 32 && ((ldc & 3) == 0)) {
#pragma unroll
          for (int k = 0; k < 32; k += 4) {
            float4 o = *reinterpret_cast<float4*>(crow + k);
            o.x -= v[k];
            o.y -= v[k + 1];
            o.z -= v[k + 2];
            o.w -= v[k + 3];
            *reinterpret_cast<float4*>(crow + k) = o;
          }
        } else {
          for (int k = 0; k < ncol && k < 32; ++k) crow[k] -= v[k];
        }
      }
    }
  } else if (threadIdx.x == 0) {
    // give the MMAs one more bounded chance to drain before TMEM is freed
    long long it = 0;
    while (!mbar_try_wait(&mbar, 0) && ++it < WAIT_LIMIT) {
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TILE);
}

}  // namespace tc
}  // namespace rbf
