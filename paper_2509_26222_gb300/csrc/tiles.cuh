// Device helpers of the 64 x 64 tile factorizations (mixed.cu, batch.cu):
// the cross-CTA flag protocol, the 32 x 32 warp-level Cholesky and inverse,
// k-major staging of tiles in shared memory and the 64 x 64 x 64 product.
#pragma once

#include "common.cuh"

namespace rbf {

constexpr int MB = 64;          // tile edge of the float32 factorizations (= tc::KB)
constexpr int TL_THREADS = 256; // threads of the kernels that use the staging helpers

// flag protocol of the launches whose CTAs wait on one another
__device__ __forceinline__ int ld_acq(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr int MXS_LD = MB + 1;

// Cholesky of the 32 x 32 lower block T[o.., o..] in place (one full warp;
// lane i holds row i in registers, a[p] = entry (i, k + p) at step k).  The
// finished column k goes through shared memory (col) to every lane; the
// rank-1 update is applied to every lane and column without masks: entries
// above the diagonal (and past column 31) collect finite values that are
// never read, because the column written at step k is masked to zero above
// the diagonal.  rd[o + k] = 1 / L_kk.
__device__ __forceinline__ void mx_chol32(float* T, float* rd, float* col, int o, int* flag) {
  const int lane = threadIdx.x & 31;
  float a[32];
#pragma unroll
  for (int p = 0; p < 32; ++p) a[p] = (p <= lane) ? T[(o + lane) * MXS_LD + o + p] : 0.f;
  col[32 + lane] = 0.f;
  bool bad = false;
  // unrolled by 4: the pivot of step k + 1 overlaps the update of step k
#pragma unroll 4
  for (int k = 0; k < 32; ++k) {
    float d = __shfl_sync(0xffffffffu, a[0], k);
    bad |= !(d > 0.f);
    float r = rsqrtf(d);
    float lik = (lane >= k) ? a[0] * r : 0.f;
    T[(o + lane) * MXS_LD + o + k] = lik;  // column k of L (zero above the diagonal)
    col[lane] = lik;
    if (lane == 0) rd[o + k] = r;
    __syncwarp();
    const float* cb = col + k;
#pragma unroll
    for (int p = 1; p < 32; ++p) a[p - 1] = fmaf(-lik, cb[p], a[p]);
    a[31] = 0.f;
    __syncwarp();
  }
  if (bad && lane == 0) atomicOr(flag, DEV_NOT_SPD);
}

// Z[o.., o..] = inverse of the 32 x 32 factor in T[o.., o..] (one full warp):
// column `lane` by forward substitution, four partial sums per row.
__device__ __forceinline__ void mx_inv32(const float* T, float* Z, const float* rd, int o) {
  const int lane = threadIdx.x & 31;
  float x[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const float* Lr = T + (o + i) * MXS_LD + o;
    float s0 = (i == lane) ? 1.f : 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
    for (int t = 0; t + 3 < i; t += 4) {
      s0 = fmaf(-Lr[t], x[t], s0);
      s1 = fmaf(-Lr[t + 1], x[t + 1], s1);
      s2 = fmaf(-Lr[t + 2], x[t + 2], s2);
      s3 = fmaf(-Lr[t + 3], x[t + 3], s3);
    }
#pragma unroll
    for (int t = i & ~3; t < i; ++t) s0 = fmaf(-Lr[t], x[t], s0);
    x[i] = ((s0 + s1) + (s2 + s3)) * rd[o + i];
    Z[(o + i) * MXS_LD + o + lane] = x[i];
  }
}

// L21 = A21 L11^{-T} by substitution, row 32 + lane per lane (one full warp).
__device__ __forceinline__ void mx_l21(float* T, const float* rd) {
  const int lane = threadIdx.x & 31;
  float* row = T + (32 + lane) * MXS_LD;
  float l[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const float* Lj = T + j * MXS_LD;
    float s0 = row[j], s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
    for (int t = 0; t + 3 < j; t += 4) {
      s0 = fmaf(-l[t], Lj[t], s0);
      s1 = fmaf(-l[t + 1], Lj[t + 1], s1);
      s2 = fmaf(-l[t + 2], Lj[t + 2], s2);
      s3 = fmaf(-l[t + 3], Lj[t + 3], s3);
    }
#pragma unroll
    for (int t = j & ~3; t < j; ++t) s0 = fmaf(-l[t], Lj[t], s0);
    l[j] = ((s0 + s1) + (s2 + s3)) * rd[j];
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) row[j] = l[j];
}

// band tiles (i, l), l <= i <= l + bwb, of an nb x nb tile grid are numbered
// column by column
// first band tile of block column l (column-major enumeration of the band)
__device__ __forceinline__ int df_colstart(int l, int nb, int bwb) {
  const int full = nb - bwb > 0 ? nb - bwb : 0;  // columns holding bwb + 1 tiles
  if (l <= full) return l * (bwb + 1);
  const int m = l - full, s0 = nb - full;
  return full * (bwb + 1) + m * s0 - m * (m - 1) / 2;
}

// k-major staging with the float4 columns xor-swizzled by k: S[kk][r] holds
// element (r, kk) of a 64 x 64 row-major tile
__device__ __forceinline__ int df_swz(int kk, int r) { return kk * 64 + (r ^ (((kk >> 2) & 7) << 2)); }

// from global memory (rows < nr, columns < nc; zeros elsewhere)
__device__ __forceinline__ void df_stage(float* S, const float* src, int64_t ld, int nr, int nc) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int q = tid + TL_THREADS * e, r = q >> 4, c4 = (q & 15) * 4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < nr) {
      const float* p = src + (int64_t)r * ld + c4;
      if (c4 + 3 < nc) {
        v = __ldcg(reinterpret_cast<const float4*>(p));
      } else {
        if (c4 < nc) v.x = __ldcg(p);
        if (c4 + 1 < nc) v.y = __ldcg(p + 1);
        if (c4 + 2 < nc) v.z = __ldcg(p + 2);
      }
    }
    S[df_swz(c4, r)] = v.x;
    S[df_swz(c4 + 1, r)] = v.y;
    S[df_swz(c4 + 2, r)] = v.z;
    S[df_swz(c4 + 3, r)] = v.w;
  }
}

// from a row-major 64 x 64 accumulator in shared memory
__device__ __forceinline__ void df_stage_smem(float* S, const float* A) {
  for (int e = threadIdx.x; e < 64 * 64; e += TL_THREADS) S[df_swz(e & 63, e >> 6)] = A[e];
}

// acc[u][v] += sum_kk A(r, kk) B(c, kk), r = 4 ty + u, c = 4 tx + v
__device__ __forceinline__ void df_mma(float (&acc)[4][4], const float* As, const float* Bs, int ty, int tx) {
#pragma unroll 8
  for (int kk = 0; kk < 64; ++kk) {
    const int sw = ((kk >> 2) & 7) << 2;
    const float4 a = *reinterpret_cast<const float4*>(As + kk * 64 + ((ty * 4) ^ sw));
    const float4 b = *reinterpret_cast<const float4*>(Bs + kk * 64 + ((tx * 4) ^ sw));
    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
  }
}


// L = chol(T) in place and Z = L^{-1} for a 64 x 64 tile in shared memory,
// blocked 2 x 2 with 32 x 32 blocks: L11 and Z11 (one warp), L21 = A21 Z11^T,
// S = A22 - L21 L21^T, L22 and Z22 (one warp), Z21 = -Z22 (L21 Z11).  T and Z
// have row stride MXS_LD (Z zero on entry); Y is 32 x 33, rd and col 64
// floats.  All TL_THREADS threads call it after a barrier; it ends with one.
__device__ __forceinline__ void tile_chol_inv(float* T, float* Z, float* Y, float* rd, float* col, int* flag) {
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) mx_chol32(T, rd, col, 0, flag);
  __syncthreads();
  if (warp == 0) mx_inv32(T, Z, rd, 0);
  else if (warp == 1) mx_l21(T, rd);
  __syncthreads();
  const int bi = tid >> 3, bj = tid & 7;
  {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
    for (int t = 0; t < 32; ++t) {
      const float lv = T[(32 + bi) * MXS_LD + t];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fmaf(lv, T[(32 + bj + 8 * u) * MXS_LD + t], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = bj + 8 * u;
      if (j <= bi) T[(32 + bi) * MXS_LD + 32 + j] -= acc[u];
    }
  }
  __syncthreads();
  if (warp == 0) {
    mx_chol32(T, rd, col, 32, flag);
    mx_inv32(T, Z, rd, 32);
  }
  {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
    for (int t = 0; t < 32; ++t) {
      const float lv = T[(32 + bi) * MXS_LD + t];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fmaf(lv, Z[t * MXS_LD + bj + 8 * u], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) Y[bi * 33 + bj + 8 * u] = acc[u];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = 0.f;
#pragma unroll 8
    for (int t = 0; t < 32; ++t) {
      const float zv = Z[(32 + bi) * MXS_LD + 32 + t];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fmaf(zv, Y[t * 33 + bj + 8 * u], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) Z[(32 + bi) * MXS_LD + bj + 8 * u] = -acc[u];
    __syncthreads();
  }
}

// Float-float arithmetic (a value as hi + lo, two float32), used where a
// result needs more than float32 but GB300's float64 rate (a small fraction of
// its float32 rate) would bound the kernel.  Error-free transforms:
// the sum by Knuth's TwoSum, the product by one fused multiply-add; the square
// root by one Newton (Heron) correction of the float32 root.  About 2^-46
// relative, against 2^-53 for float64.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ FF ff_fast_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_add(FF x, FF y) {
  FF s = ff_two_sum(x.hi, y.hi);
  return ff_fast_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ FF ff_mul(FF x, FF y) {
  const float p = __fmul_rn(x.hi, y.hi), e = fmaf(x.hi, y.hi, -p);
  return ff_fast_sum(p, fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e)));
}
__device__ __forceinline__ FF ff_sqrt(FF x) {
  if (!(x.hi > 0.f)) return {0.f, 0.f};
  const float y = __fsqrt_rn(x.hi);
  const float p = __fmul_rn(y, y), pe = fmaf(y, y, -p);  // y^2 = p + pe exactly
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), pe), x.lo);
  return ff_fast_sum(y, __fdiv_rn(r, __fmul_rn(2.f, y)));
}
__device__ __forceinline__ FF ff_of(double v) {
  const float hi = (float)v;
  return {hi, (float)(v - (double)hi)};
}

// x = hi + lo to about 2^-48 (one float64 subtraction)
__device__ __forceinline__ FF ff_split(double v) { return ff_of(v); }
// acc + x y
__device__ __forceinline__ FF ff_mac(FF acc, FF x, FF y) {
  const float p = __fmul_rn(x.hi, y.hi);
  const float e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, fmaf(x.hi, y.hi, -p)));
  const FF sum = ff_two_sum(acc.hi, p);
  return ff_fast_sum(sum.hi, __fadd_rn(sum.lo, __fadd_rn(acc.lo, e)));
}
__device__ __forceinline__ double ff_to_double(FF x) { return (double)x.hi + (double)x.lo; }

}  // namespace rbf
