// Mixed-precision factorization and solves for the active-block update.
//
// The information matrix H of the active block (Eq. H_update restricted to
// the active rows) is kept exactly in float64.  Its Cholesky factor is
// computed in float32 with the O(a^3) trailing updates on the tensor cores
// (tcgen05, three-way bfloat16 split, see tc_syrk.cuh), and the float64
// accuracy of every solve H x = b is recovered by iterative refinement with
// float64 residuals r = b - H x.  GB300 executes float64 at about 1 TFLOP/s,
// float32 at about 70 TFLOP/s and bfloat16 on the tensor cores at about
// 1.9 PFLOP/s; float64 is therefore spent only on H itself and on the
// residuals.
//
// Blocked right-looking Cholesky, block 64, on a float32 working copy W of H:
//   k_mx_diag  : one CTA factors W_kk in float32 and inverts the factor
//                (Z_kk = L_kk^{-1}, kept for the solves);
//   k_mx_panel : L_ik = W_ik Z_kk^T for the rows below, written to W and as
//                three bfloat16 slices;
//   k_syrk_tc  : W_ij -= L_ik L_jk^T on the tensor cores (lower tiles).
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "tc_syrk.cuh"
#include "tiles.cuh"

namespace rbf {


__global__ void k_mx_to_f32(const double* __restrict__ H, int64_t ldh, int64_t n, float* __restrict__ W,
                            int64_t ldw) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  int64_t i = e / n, j = e % n;
  W[i * ldw + j] = (float)H[i * ldh + j];
}

// ---------------------------------------------------------------------------
// One block column of the factorization in one launch.  Every CTA factors the
// 64 x 64 diagonal tile W_kk itself (L_kk, and Z_kk = L_kk^{-1}), then
// computes its 64 panel rows L_ik = W_ik Z_kk^T as a small matrix product,
// writes them to W and as three bfloat16 slices for the tensor-core trailing
// update.  CTA 0 stores Z_kk for the triangular solves.  Repeating the 64 x 64
// factorization in every CTA replaces a separate launch and a row-by-row
// substitution with work that runs in parallel on otherwise idle SMs.
//
// The 64 x 64 factorization is blocked 2 x 2 with 32 x 32 blocks:
//   L11 = chol(A11), Z11 = L11^{-1}           (one warp, registers + shuffles)
//   L21 = A21 Z11^T, S = A22 - L21 L21^T      (all warps)
//   L22 = chol(S),   Z22 = L22^{-1}           (one warp)
//   Z21 = -Z22 (L21 Z11)                      (all warps)
// The diagonal tile of W itself is left as it was: the solves read the
// diagonal blocks only through Z.
// ---------------------------------------------------------------------------
constexpr size_t MXS_SMEM = (size_t)(5 * MB * MXS_LD + 32 * 33 + MB + 64) * sizeof(float);

__global__ void __launch_bounds__(256) k_mx_step(float* __restrict__ W, int64_t ldw, int64_t n, int64_t k,
                                                 int kb, int prev, float* __restrict__ Zk,
                                                 __nv_bfloat16* __restrict__ Ph, __nv_bfloat16* __restrict__ Pm,
                                                 __nv_bfloat16* __restrict__ Pl, int* __restrict__ flag) {
  extern __shared__ float mxs[];
  float* T = mxs;                     // diagonal tile -> L_kk
  float* Z = T + MB * MXS_LD;         // Z_kk = L_kk^{-1}
  float* X = Z + MB * MXS_LD;         // this CTA's panel rows
  float* Y = X + MB * MXS_LD;         // 32 x 33 temporary
  float* rd = Y + 32 * 33;            // 1 / L_jj
  float* Lk = rd + MB;                // L_{k,k-1} (look-ahead update)
  float* Lr = Lk + MB * MXS_LD;       // L_{rows,k-1}
  float* col = Lr + MB * MXS_LD;      // column broadcast of the 32 x 32 Cholesky
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t k0 = k + kb;
  const int64_t r0 = k0 + (int64_t)blockIdx.x * MB;
  {
    // every load of a thread is issued before the first one is used
    float tv[MB * MB / 256], xv[MB * MB / 256], lkv[MB * MB / 256], lrv[MB * MB / 256];
#pragma unroll
    for (int q = 0; q < MB * MB / 256; ++q) {
      int e = tid + 256 * q, i = e / MB, j = e % MB;
      int64_t r = r0 + i;
      tv[q] = (i < kb && j <= i) ? W[(k + i) * ldw + k + j] : 0.f;
      xv[q] = (r < n && j < kb) ? W[r * ldw + k + j] : 0.f;
      // this block column has every update but the one of the previous
      // panel: W_kk -= L_{k,k-1} L_{k,k-1}^T, W_{rows,k} -= L_{rows,k-1} L_{k,k-1}^T
      lkv[q] = (prev && i < kb) ? W[(k + i) * ldw + (k - MB) + j] : 0.f;
      lrv[q] = (prev && r < n) ? W[r * ldw + (k - MB) + j] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < MB * MB / 256; ++q) {
      int e = tid + 256 * q, i = e / MB, j = e % MB;
      T[i * MXS_LD + j] = (i >= kb && i == j) ? 1.f : tv[q];  // identity beyond a ragged last block
      Z[i * MXS_LD + j] = 0.f;
      X[i * MXS_LD + j] = xv[q];
      Lk[i * MXS_LD + j] = lkv[q];
      Lr[i * MXS_LD + j] = lrv[q];
    }
  }
  __syncthreads();
  if (prev) {
    // T -= Lk Lk^T (lower part), 4 x 4 blocks: rows 4 pr + u, columns pc + 16 q
    const int pr = tid >> 4, pc = tid & 15;
    float at[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int q = 0; q < 4; ++q) at[u][q] = 0.f;
#pragma unroll 4
    for (int t = 0; t < MB; ++t) {
      float kv[4], cv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) kv[u] = Lk[(4 * pr + u) * MXS_LD + t];
#pragma unroll
      for (int q = 0; q < 4; ++q) cv[q] = Lk[(pc + 16 * q) * MXS_LD + t];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < 4; ++q) at[u][q] = fmaf(kv[u], cv[q], at[u][q]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int i = 4 * pr + u, j = pc + 16 * q;
        if (j <= i && i < kb) T[i * MXS_LD + j] -= at[u][q];
      }
    __syncthreads();
  }
  if (warp == 0) {
    mx_chol32(T, rd, col, 0, flag);
  } else if (prev) {
    // X -= Lr Lk^T by warps 1-7 while warp 0 factors: rows w - 1 + 7 m, columns lane and lane + 32
    float ax[10][2];
#pragma unroll
    for (int m = 0; m < 10; ++m) ax[m][0] = ax[m][1] = 0.f;
#pragma unroll 2
    for (int t = 0; t < MB; ++t) {
      float c0 = Lk[lane * MXS_LD + t], c1 = Lk[(lane + 32) * MXS_LD + t];
#pragma unroll
      for (int m = 0; m < 10; ++m) {
        int i = warp - 1 + 7 * m;
        if (i < MB) {
          float rv = Lr[i * MXS_LD + t];
          ax[m][0] = fmaf(rv, c0, ax[m][0]);
          ax[m][1] = fmaf(rv, c1, ax[m][1]);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < 10; ++m) {
      int i = warp - 1 + 7 * m;
      if (i < MB) {
        X[i * MXS_LD + lane] -= ax[m][0];
        X[i * MXS_LD + lane + 32] -= ax[m][1];
      }
    }
  }
  __syncthreads();
  // Z11 (warp 0) while warp 1 forms L21 = A21 L11^{-T} by substitution
  if (warp == 0) mx_inv32(T, Z, rd, 0);
  else if (warp == 1) mx_l21(T, rd);
  __syncthreads();
  const int bi = tid >> 3, bj = tid & 7;  // 32 x 32 products: row bi, columns bj + 8q
  {
    // S = A22 - L21 L21^T (lower part)
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
    for (int t = 0; t < 32; ++t) {
      float lv = T[(32 + bi) * MXS_LD + t];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(lv, T[(32 + bj + 8 * q) * MXS_LD + t], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int j = bj + 8 * q;
      if (j <= bi) T[(32 + bi) * MXS_LD + 32 + j] -= acc[q];
    }
    __syncthreads();
  }
  if (warp == 0) {
    mx_chol32(T, rd, col, 32, flag);
    mx_inv32(T, Z, rd, 32);
  }
  {
    // Y = L21 Z11 (all warps but the first; the first joins after its factorization)
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
    for (int t = 0; t < 32; ++t) {
      float lv = T[(32 + bi) * MXS_LD + t];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(lv, Z[t * MXS_LD + bj + 8 * q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) Y[bi * 33 + bj + 8 * q] = acc[q];
    __syncthreads();
    // Z21 = -Z22 Y
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = 0.f;
#pragma unroll 8
    for (int t = 0; t < 32; ++t) {
      float zv = Z[(32 + bi) * MXS_LD + 32 + t];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(zv, Y[t * 33 + bj + 8 * q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) Z[(32 + bi) * MXS_LD + bj + 8 * q] = -acc[q];
    __syncthreads();
  }
  if (blockIdx.x == 0)
    for (int e = tid; e < MB * MB; e += blockDim.x) Zk[e] = Z[(e / MB) * MXS_LD + e % MB];
  if (r0 >= n) return;
  // panel rows: X <- X Z^T, each thread a 4 x 4 block (rows 4 pr.., columns pc + 16 q)
  const int pr = tid >> 4, pc = tid & 15;
  float acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[u][q] = 0.f;
#pragma unroll 4
  for (int t = 0; t < MB; ++t) {
    float xv[4], zv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) xv[u] = X[(4 * pr + u) * MXS_LD + t];
#pragma unroll
    for (int q = 0; q < 4; ++q) zv[q] = Z[(pc + 16 * q) * MXS_LD + t];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[u][q] = fmaf(xv[u], zv[q], acc[u][q]);
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int q = 0; q < 4; ++q) X[(4 * pr + u) * MXS_LD + pc + 16 * q] = acc[u][q];
  __syncthreads();
  for (int e = tid; e < MB * MB; e += blockDim.x) {
    int i = e / MB, j = e % MB;
    int64_t r = r0 + i;
    if (r >= n) continue;
    float x = X[i * MXS_LD + j];
    if (j < kb) W[r * ldw + k + j] = x;
    else x = 0.f;
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    float rem = x - __bfloat162float(h);
    __nv_bfloat16 mm = __float2bfloat16_rn(rem);
    float rem2 = rem - __bfloat162float(mm);
    __nv_bfloat16 l = __float2bfloat16_rn(rem2);
    int64_t prr = r - k0;
    Ph[prr * MB + j] = h;
    Pm[prr * MB + j] = mm;
    Pl[prr * MB + j] = l;
  }
}

// ---------------------------------------------------------------------------
// The whole factorization in one persistent launch (dataflow over tiles).
//
// The band of H' is cut into 64 x 64 tiles (i, l), l <= i <= l + bwb, owned
// round-robin (column-major order) by the CTAs of one cooperative launch.  A
// tile's owner applies the updates W_il -= L_ik L_lk^T of the columns k < l
// as their panels become ready, then finishes the tile:
//   diagonal tile   D(l): L_ll = chol(W_ll), Z_ll = L_ll^{-1}  (-> Zd, W)
//   panel tile      P(i,l): L_il = W_il Z_ll^T                  (-> W)
// and publishes a per-tile ready flag (release store; readers acquire).  All
// CTAs walk the same global task order
//   stage s: U(., s+1; s)   D(s+1)   P(., s+1)   U(., l >= s+2; s)
// -- the updates of the next block column first, so that its factorization
// overlaps the rest of stage s (look-ahead) -- and every wait is for a task
// earlier in that order, which some co-resident CTA finishes without waiting
// on anything later: the launch cannot deadlock.  Waits are bounded; a wait
// that runs out sets DEV_TIMEOUT and an abort word that ends every other
// wait, and the CTAs return.
//
// Each tile's updates are applied in ascending k by its one owner, so the
// result does not depend on timing.  The diagonal tile of W receives L_ll
// (the solves read the diagonal blocks through Zd).
// ---------------------------------------------------------------------------
constexpr int DF_THREADS = 256;
constexpr int DF_MAXOWN = 64;            // band tiles one CTA may own
constexpr int DF_NACC = 8;               // owned tiles whose running sums stay in shared memory
constexpr int64_t DF_NMAX = 16384;       // largest block factored by the dataflow launch (64 size buckets of 256)
constexpr long long DF_SPIN = 1LL << 22;
// dynamic shared memory (floats): two k-major staged tiles, or the diagonal
// factorization's T, Z (64 x 65), Y (32 x 33), 1 / L_jj and the column buffer;
// then DF_NACC tile accumulators (64 x 64, row-major); then the bitmap of the
// ready flags this CTA has already seen
constexpr int DF_STAGE_FLOATS = 2 * 64 * 64;
constexpr int DF_DIAG_FLOATS = 2 * MB * MXS_LD + 32 * 33 + MB + 64;
constexpr int DF_R0 = DF_STAGE_FLOATS > DF_DIAG_FLOATS ? DF_STAGE_FLOATS : DF_DIAG_FLOATS;
constexpr size_t DF_SMEM_BASE = (size_t)(DF_R0 + DF_NACC * 64 * 64) * sizeof(float);

struct DfParams {
  float* W;
  int64_t ldw, n;
  int nb, bwb, ntiles;
  float* Zd;
  int* flags;  // ntiles ready flags, then the abort word
  int epoch;
  int* status;
  long long spin;
  int wait_xor;
};

// Bounded waits for the ready flags a and b (b < 0: none), thread 0 for a and
// thread 32 for b; flags seen ready once are remembered in `seen`.  False if
// this or another CTA gave up.
__device__ __forceinline__ bool df_wait2(const DfParams& P, unsigned* seen, int a, int b, int* bail) {
  const int tid = threadIdx.x;
  if (tid == 0 || tid == 32) {
    const int idx = tid == 0 ? a : b;
    if (idx >= 0 && !(seen[idx >> 5] & (1u << (idx & 31)))) {
      const int want = P.epoch ^ P.wait_xor;
      long long it = 0;
      bool ok = true;
      while (ld_acq(P.flags + idx) != want) {
        if (ld_acq(P.flags + P.ntiles) == P.epoch) {
          ok = false;
          break;
        }
        if (++it > P.spin) {
          atomicOr(P.status, DEV_TIMEOUT);
          st_rel(P.flags + P.ntiles, P.epoch);
          ok = false;
          break;
        }
        __nanosleep(32);
      }
      if (ok) atomicOr(seen + (idx >> 5), 1u << (idx & 31));
      else *bail = 1;
    }
  }
  __syncthreads();
  return *bail == 0;
}

__device__ __forceinline__ void df_publish(const DfParams& P, int idx) {
  __syncthreads();  // every thread's stores of the tile are done
  if (threadIdx.x == 0) {
    __threadfence();
    st_rel(P.flags + idx, P.epoch);
  }
}

__global__ void __launch_bounds__(DF_THREADS) k_chol_df(DfParams P) {
  extern __shared__ float dfs[];
  __shared__ int own_i[DF_MAXOWN], own_l[DF_MAXOWN];
  __shared__ int bail;
  float* R0 = dfs;
  float* ACC = dfs + DF_R0;
  unsigned* seen = reinterpret_cast<unsigned*>(ACC + DF_NACC * 64 * 64);
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int nb = P.nb, bwb = P.bwb;
  if (tid == 0) {
    bail = 0;
    int l = 0, no = 0;
    for (int t = blockIdx.x; t < P.ntiles && no < DF_MAXOWN; t += gridDim.x, ++no) {
      while (df_colstart(l + 1, nb, bwb) <= t) ++l;
      own_l[no] = l;
      own_i[no] = l + (t - df_colstart(l, nb, bwb));
    }
  }
  for (int e = tid; e < (P.ntiles + 31) / 32; e += DF_THREADS) seen[e] = 0u;
  __syncthreads();
  int nown = 0;
  for (int t = blockIdx.x; t < P.ntiles && nown < DF_MAXOWN; t += gridDim.x) ++nown;
  float* As = R0;
  float* Bs = R0 + 64 * 64;
  auto rows_of = [&](int b) { return (int)min((int64_t)64, P.n - (int64_t)b * 64); };
  auto tile = [&](int i, int l) { return P.W + (int64_t)i * 64 * P.ldw + (int64_t)l * 64; };
  auto tid_of = [&](int i, int l) { return df_colstart(l, nb, bwb) + (i - l); };
  // running sums of the first DF_NACC owned tiles live in shared memory
  const int nacc = nown < DF_NACC ? nown : DF_NACC;
  for (int q = 0; q < nacc; ++q) {
    const int ri = rows_of(own_i[q]), rl = rows_of(own_l[q]);
    const float* src = tile(own_i[q], own_l[q]);
    float* A = ACC + q * 64 * 64;
    for (int e = tid; e < 64 * 64; e += DF_THREADS) {
      const int r = e >> 6, cc = e & 63;
      A[e] = (r < ri && cc < rl) ? __ldcg(src + (int64_t)r * P.ldw + cc) : 0.f;
    }
  }
  __syncthreads();

  // U(i, l; k): tile q -= L_ik L_lk^T
  auto update = [&](int q, int k) -> bool {
    const int i = own_i[q], l = own_l[q];
    if (!df_wait2(P, seen, tid_of(i, k), i != l ? tid_of(l, k) : -1, &bail)) return false;
    const int ri = rows_of(i), rl = rows_of(l), ck = rows_of(k);
    df_stage(As, tile(i, k), P.ldw, ri, ck);
    if (i != l) df_stage(Bs, tile(l, k), P.ldw, rl, ck);
    __syncthreads();
    float acc[4][4] = {};
    df_mma(acc, As, i != l ? Bs : As, ty, tx);
    if (q < DF_NACC) {
      float* A = ACC + q * 64 * 64;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float4* p = reinterpret_cast<float4*>(A + (ty * 4 + u) * 64 + tx * 4);
        float4 v = *p;
        v.x -= acc[u][0];
        v.y -= acc[u][1];
        v.z -= acc[u][2];
        v.w -= acc[u][3];
        *p = v;
      }
    } else {
      float* dst = tile(i, l);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = ty * 4 + u;
        if (r >= ri) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int cc = tx * 4 + v;
          if (cc < rl) __stcg(dst + (int64_t)r * P.ldw + cc, __ldcg(dst + (int64_t)r * P.ldw + cc) - acc[u][v]);
        }
      }
    }
    __syncthreads();  // the staged tiles are read before the next task restages them
    return true;
  };

  // P(i, l): L_il = W_il Z_ll^T
  auto panel = [&](int q) -> bool {
    const int i = own_i[q], l = own_l[q];
    if (!df_wait2(P, seen, tid_of(l, l), -1, &bail)) return false;
    const int ri = rows_of(i);
    if (q < DF_NACC) df_stage_smem(As, ACC + q * 64 * 64);
    else df_stage(As, tile(i, l), P.ldw, ri, 64);
    df_stage(Bs, P.Zd + (int64_t)l * 64 * 64, 64, 64, 64);
    __syncthreads();
    float acc[4][4] = {};
    df_mma(acc, As, Bs, ty, tx);
    float* dst = tile(i, l);
    const int cl = rows_of(l);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = ty * 4 + u;
      if (r >= ri) continue;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int cc = tx * 4 + v;
        if (cc < cl) __stcg(dst + (int64_t)r * P.ldw + cc, acc[u][v]);
      }
    }
    df_publish(P, tid_of(i, l));
    return true;
  };

  // D(l): L_ll = chol(W_ll) and Z_ll = L_ll^{-1} (2 x 2 blocks of 32, as k_mx_step)
  auto diag = [&](int q) {
    const int l = own_l[q];
    float* T = R0;
    float* Z = T + MB * MXS_LD;
    float* Y = Z + MB * MXS_LD;
    float* rd = Y + 32 * 33;
    float* col = rd + MB;
    const int kb = rows_of(l);
    const float* src = tile(l, l);
    const float* A = q < DF_NACC ? ACC + q * 64 * 64 : nullptr;
    for (int e = tid; e < MB * MB; e += DF_THREADS) {
      const int i = e / MB, j = e % MB;
      float v = 0.f;
      if (i < kb && j <= i) v = A ? A[e] : __ldcg(src + (int64_t)i * P.ldw + j);
      if (i >= kb && i == j) v = 1.f;  // identity beyond a ragged last block
      T[i * MXS_LD + j] = v;
      Z[i * MXS_LD + j] = 0.f;
    }
    __syncthreads();
    tile_chol_inv(T, Z, Y, rd, col, P.status);
    float* zd = P.Zd + (int64_t)l * MB * MB;
    float* dst = tile(l, l);
    for (int e = tid; e < MB * MB; e += DF_THREADS) {
      const int i = e / MB, j = e % MB;
      __stcg(zd + e, Z[i * MXS_LD + j]);
      if (i < kb && j < kb) __stcg(dst + (int64_t)i * P.ldw + j, j <= i ? T[i * MXS_LD + j] : 0.f);
    }
    df_publish(P, tid_of(l, l));
  };

  int p0 = 0;  // first owned tile of a block column >= s + 1
  for (int s = -1; s < nb - 1; ++s) {
    while (p0 < nown && own_l[p0] < s + 1) ++p0;
    const int c = s + 1;
    // U(., s+1; s): the next block column first
    if (s >= 0)
      for (int q = p0; q < nown && own_l[q] == c; ++q)
        if (own_i[q] - s <= bwb && !update(q, s)) return;
    // D(s+1), then P(., s+1)
    for (int q = p0; q < nown && own_l[q] == c; ++q)
      if (own_i[q] == c) diag(q);
    for (int q = p0; q < nown && own_l[q] == c; ++q)
      if (own_i[q] > c && !panel(q)) return;
    // U(., l >= s+2; s)
    if (s >= 0)
      for (int q = p0; q < nown && own_l[q] <= s + bwb; ++q) {
        const int l = own_l[q], i = own_i[q];
        if (l >= s + 2 && i - s <= bwb && !update(q, s)) return;
      }
  }
}

// The factorization by k_chol_df.  Returns RBF_ERANGE (and launches nothing)
// when the band has more tiles than the co-resident CTAs can own.
static rbf_status potrf_df(Ctx* c, int64_t n, float* W, int64_t ldw, float* Zd, cudaStream_t s, int64_t bw) {
  const int nb = (int)((n + MB - 1) / MB);
  int bwb = nb - 1;
  if (bw < n) {
    int64_t b = (bw + MB - 1) / MB + 1;
    if (b < bwb) bwb = (int)b;
  }
  const int full = nb - bwb > 0 ? nb - bwb : 0;
  const int m = nb - full, s0 = nb - full;
  const int64_t ntiles = (int64_t)full * (bwb + 1) + (int64_t)m * s0 - (int64_t)m * (m - 1) / 2;
  // shared memory: staging, accumulators and the bitmap of seen flags (at
  // most DF_MAXOWN tiles per CTA on up to 1024 SMs)
  constexpr size_t smem_max = DF_SMEM_BASE + (size_t)(DF_MAXOWN * 1024 / 32) * sizeof(unsigned);
  static int max_blocks[64] = {0};
  const int dev = c->device & 63;
  if (!max_blocks[dev]) {
    int per_sm = 0, sms = 0;
    RBF_CUDA(cudaFuncSetAttribute(k_chol_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
    RBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chol_df, DF_THREADS, smem_max));
    RBF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    max_blocks[dev] = (per_sm > 0 ? 1 : 0) * (sms < 1024 ? sms : 1024);  // one CTA per SM
  }
  int64_t grid = ntiles < max_blocks[dev] ? ntiles : max_blocks[dev];
  if (grid < 1 || (ntiles + grid - 1) / grid > DF_MAXOWN) return RBF_ERANGE;
  const size_t smem = DF_SMEM_BASE + (size_t)((ntiles + 31) / 32) * sizeof(unsigned);
  if (c->df_flags.bytes < (size_t)(ntiles + 1) * sizeof(int)) {
    RBF_TRY(c->df_flags.ensure((size_t)(ntiles + 1) * sizeof(int)));
    RBF_CUDA(cudaMemsetAsync(c->df_flags.p, 0, c->df_flags.bytes, s));
    c->df_epoch = 0;
  }
  DfParams P;
  P.W = W;
  P.ldw = ldw;
  P.n = n;
  P.nb = nb;
  P.bwb = bwb;
  P.ntiles = (int)ntiles;
  P.Zd = Zd;
  P.flags = c->df_flags.as<int>();
  P.epoch = (int)(++c->df_epoch & 0x3fffffff);
  if (P.epoch == 0) P.epoch = (int)(++c->df_epoch & 0x3fffffff);
  P.status = c->dflag.as<int>();
  P.spin = c->spin_limit > 0 ? c->spin_limit : DF_SPIN;
  P.wait_xor = c->wait_xor;
  void* args[] = {(void*)&P};
  StageTimer st(c, RBF_STAGE_PANEL, s, (double)n * n * n / 3.0);
  RBF_CUDA(cooperative_launch((const void*)k_chol_df, dim3((unsigned)grid), dim3(DF_THREADS), args, smem, s));
  return RBF_OK;
}

static rbf_status potrf_chain(Ctx* c, int64_t n, float* W, int64_t ldw, float* Zd, cudaStream_t s, int64_t bw);

static rbf_status to_f32(const double* H, int64_t ldh, int64_t n, float* W, int64_t ldw, cudaStream_t s) {
  int64_t tot = n * n;
  { k_mx_to_f32<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(H, ldh, n, W, ldw); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  return RBF_OK;
}

// Float32 factor of H (with the diagonal-block inverses Zd) by the dataflow
// launch or by the launch chain.  Which is faster depends on the size (the
// chain's tensor-core trailing updates win for large blocks): the first
// factorization of each size bucket of 256 runs both, timed, and the bucket
// keeps the faster.  Stream capture, batched sub-contexts and blocks beyond
// DF_NMAX use the chain.
rbf_status potrf_mixed(Ctx* c, const double* H, int64_t ldh, int64_t n, float* W, int64_t ldw, float* Zd,
                       cudaStream_t s, int64_t bw) {
  if (n <= 0) return RBF_OK;
  cudaStreamCaptureStatus cap0 = cudaStreamCaptureStatusNone;
  RBF_CUDA(cudaStreamIsCapturing(s, &cap0));
  if (!(c->la_ok && c->df_ok && n <= DF_NMAX && cap0 == cudaStreamCaptureStatusNone)) {
    RBF_TRY(to_f32(H, ldh, n, W, ldw, s));
    return potrf_chain(c, n, W, ldw, Zd, s, bw);
  }
  const int b = (int)(n / 256);
  int8_t& pick = c->fchoice[b < 64 ? b : 63];
  if (pick == 1) {
    RBF_TRY(to_f32(H, ldh, n, W, ldw, s));
    return potrf_chain(c, n, W, ldw, Zd, s, bw);
  }
  if (pick == 2) {
    RBF_TRY(to_f32(H, ldh, n, W, ldw, s));
    rbf_status st = potrf_df(c, n, W, ldw, Zd, s, bw);
    if (st != RBF_ERANGE) return st;
    RBF_TRY(to_f32(H, ldh, n, W, ldw, s));
    return potrf_chain(c, n, W, ldw, Zd, s, bw);
  }
  // first block of this size: time both (the dataflow result is kept)
  cudaEvent_t ev[3];
  for (auto& e : ev) RBF_CUDA(cudaEventCreate(&e));
  RBF_CUDA(cudaEventRecord(ev[0], s));
  RBF_TRY(to_f32(H, ldh, n, W, ldw, s));
  RBF_TRY(potrf_chain(c, n, W, ldw, Zd, s, bw));
  RBF_CUDA(cudaEventRecord(ev[1], s));
  RBF_TRY(to_f32(H, ldh, n, W, ldw, s));
  rbf_status st = potrf_df(c, n, W, ldw, Zd, s, bw);
  RBF_CUDA(cudaEventRecord(ev[2], s));
  RBF_CUDA(cudaEventSynchronize(ev[2]));
  float t_chain = 0.f, t_df = 0.f;
  RBF_CUDA(cudaEventElapsedTime(&t_chain, ev[0], ev[1]));
  RBF_CUDA(cudaEventElapsedTime(&t_df, ev[1], ev[2]));
  for (auto& e : ev) cudaEventDestroy(e);
  if (st == RBF_ERANGE) {
    pick = 1;
    RBF_TRY(to_f32(H, ldh, n, W, ldw, s));
    return potrf_chain(c, n, W, ldw, Zd, s, bw);
  }
  RBF_TRY(st);
  pick = t_df <= t_chain ? 2 : 1;
  return RBF_OK;
}

static rbf_status potrf_chain(Ctx* c, int64_t n, float* W, int64_t ldw, float* Zd, cudaStream_t s, int64_t bw) {
  int* flag = c->dflag.as<int>();
  // bf16 slices of the panel, two sets (panel k is read by the trailing
  // update of step k while step k + 1 writes the next one)
  const size_t slice = (size_t)(n + MB) * MB;
  Buf& pb = c->scratch(26);
  RBF_TRY(pb.ensure(2 * 3 * slice * sizeof(__nv_bfloat16)));
  static bool attr_set[64] = {false};
  if (!attr_set[c->device & 63]) {
    RBF_CUDA(cudaFuncSetAttribute(tc::k_syrk_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES));
    RBF_CUDA(cudaFuncSetAttribute(k_mx_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MXS_SMEM));
    attr_set[c->device & 63] = true;
  }
  // Look-ahead: step k applies the previous panel to its own block column,
  // so the tensor-core update of the rest of the trailing matrix (columns
  // beyond k + 1) runs on a side stream while step k + 1 factors.  Not used
  // while the stream is being captured into a graph, nor where the eager and
  // captured runs must give identical bits (batched patches): the update of
  // the next block column then runs on the tensor cores with the rest.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  RBF_CUDA(cudaStreamIsCapturing(s, &cap));
  const bool la = c->la_ok && cap == cudaStreamCaptureStatusNone;
  if (la && !c->la_stream) {
    RBF_CUDA(cudaStreamCreateWithFlags(&c->la_stream, cudaStreamNonBlocking));
    for (auto& ev : c->la_ev) RBF_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  }
  cudaStream_t side = la ? c->la_stream : s;
  bool r_pending[2] = {false, false};
  bool any_side = false;
  for (int64_t k = 0, step = 0; k < n; k += MB, ++step) {
    int kb = (int)((n - k) < MB ? (n - k) : MB);
    // rows beyond the band are zero in this panel and untouched by its update
    int64_t rows = ((k + kb + bw) < n ? (k + kb + bw) : n) - k - kb;
    const int par = (int)(step & 1);
    __nv_bfloat16* Ph = pb.as<__nv_bfloat16>() + (size_t)par * 3 * slice;
    __nv_bfloat16* Pm = Ph + slice;
    __nv_bfloat16* Pl = Pm + slice;
    if (la && r_pending[par]) {  // trailing update of step - 2: done with this slice set and column
      RBF_CUDA(cudaStreamWaitEvent(s, c->la_ev[2 + par], 0));
      r_pending[par] = false;
    }
    {
      StageTimer st(c, RBF_STAGE_PANEL, s, (double)kb * kb * kb / 3.0 + (double)rows * kb * kb);
      unsigned g = rows > 0 ? (unsigned)((rows + MB - 1) / MB) : 1u;
      int prev = (la && step > 0) ? 1 : 0;
      { k_mx_step<<<g, 256, MXS_SMEM, s>>>(W, ldw, n, k, kb, prev, Zd + step * MB * MB, Ph, Pm, Pl, flag); ::rbf::note_launch(); }
      RBF_CUDA(cudaGetLastError());
    }
    const int64_t off = la ? MB : 0;  // with look-ahead the next block column is left to the next step
    if (rows > off) {
      const int64_t tr = rows - off;
      if (la) {
        RBF_CUDA(cudaEventRecord(c->la_ev[par], s));
        RBF_CUDA(cudaStreamWaitEvent(side, c->la_ev[par], 0));
      }
      {
        StageTimer st(c, RBF_STAGE_TRAILING, side, (double)tr * (double)(tr + 1) * kb);
        int64_t T = (tr + tc::TILE - 1) / tc::TILE;
        const int64_t o = k + kb + off;
        { tc::k_syrk_tc<<<(unsigned)(T * (T + 1) / 2), 128, tc::SMEM_BYTES, side>>>(W + o * ldw + o, ldw, tr,
                                                                                   Ph + off * MB, Pm + off * MB,
                                                                                   Pl + off * MB, flag); ::rbf::note_launch(); }
        RBF_CUDA(cudaGetLastError());
      }
      if (la) {
        RBF_CUDA(cudaEventRecord(c->la_ev[2 + par], side));
        r_pending[par] = true;
        any_side = true;
      }
    }
  }
  if (la && any_side) {
    RBF_CUDA(cudaEventRecord(c->la_ev[4], side));
    RBF_CUDA(cudaStreamWaitEvent(s, c->la_ev[4], 0));
  }
  return RBF_OK;
}

// ---------------------------------------------------------------------------
// float32 sync-free triangular solve (block 64) with the stored inverses of
// the diagonal blocks: op(L) X = B for up to 160 right-hand sides per launch.
// ---------------------------------------------------------------------------
constexpr int T32_MC = 160;
constexpr long long T32_SPIN = 1LL << 22;


__global__ void __launch_bounds__(256) k_trsm32(const float* __restrict__ L, int64_t ldl, int64_t n,
                                                const float* __restrict__ Zd, float* B, int64_t ldb, int c0,
                                                int mc, bool transpose, int bwb, int* flags, int epoch,
                                                int* status, long long spin_limit, int wait_xor) {
  // acc and Xs (64 x (T32_MC + 1) floats each) in dynamic shared memory
  extern __shared__ float t32_dyn[];
  float (*acc)[T32_MC + 1] = reinterpret_cast<float (*)[T32_MC + 1]>(t32_dyn);
  float (*Xs)[T32_MC + 1] = reinterpret_cast<float (*)[T32_MC + 1]>(t32_dyn + MB * (T32_MC + 1));
  __shared__ float Zs[MB][MB + 1];
  __shared__ int bail;
  const int tid = threadIdx.x, ti = tid >> 2, tg = tid & 3;
  int64_t nblk = (n + MB - 1) / MB;
  for (int64_t lk = blockIdx.x; lk < nblk; lk += gridDim.x) {
    int64_t r = transpose ? (nblk - 1 - lk) : lk;
    int64_t r0 = r * MB;
    int rb = (int)((n - r0) < MB ? (n - r0) : MB);
    const float* Zr = Zd + r * MB * MB;
    for (int e = tid; e < MB * MB; e += blockDim.x) {
      int i = e / MB, t = e % MB;
      Zs[i][t] = transpose ? Zr[t * MB + i] : Zr[e];  // inverse of op(L)_rr
    }
    for (int e = tid; e < MB * T32_MC; e += blockDim.x) {
      int i = e / T32_MC, j = e % T32_MC;
      acc[i][j] = (i < rb && j < mc) ? B[(r0 + i) * ldb + c0 + j] : 0.f;
    }
    if (tid == 0) bail = 0;
    __syncthreads();
    for (int64_t lc = (lk - bwb) > 0 ? (lk - bwb) : 0; lc < lk; ++lc) {  // blocks outside the band are zero
      int64_t cb = transpose ? (nblk - 1 - lc) : lc;
      int64_t cc0 = cb * MB;
      int cbs = (int)((n - cc0) < MB ? (n - cc0) : MB);
      float lv[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        int t = 16 * tg + u;
        float v = 0.f;
        if (ti < rb && t < cbs) v = transpose ? L[(cc0 + t) * ldl + r0 + ti] : L[(r0 + ti) * ldl + cc0 + t];
        lv[u] = v;
      }
      if (tid == 0) {
        long long it = 0;
        while (ld_acq(flags + cb) != (epoch ^ wait_xor)) {
          if (++it > spin_limit) {
            atomicOr(status, DEV_TIMEOUT);
            bail = 1;
            break;
          }
          __nanosleep(20);
        }
      }
      __syncthreads();
      if (bail) break;
      for (int e = tid; e < MB * mc; e += blockDim.x) {
        int t = e / mc, j = e % mc;
        Xs[t][j] = (t < cbs) ? __ldcg(B + (cc0 + t) * ldb + c0 + j) : 0.f;
      }
      __syncthreads();
      for (int j = 0; j < mc; ++j) {
        float pp = 0.f;
#pragma unroll
        for (int u = 0; u < 16; ++u) pp = fmaf(lv[u], Xs[16 * tg + u][j], pp);
        pp += __shfl_xor_sync(0xffffffffu, pp, 1);
        pp += __shfl_xor_sync(0xffffffffu, pp, 2);
        if (tg == 0) acc[ti][j] -= pp;
      }
      __syncthreads();
    }
    __syncthreads();
    for (int j = 0; j < mc; ++j) {
      float pp = 0.f;
#pragma unroll
      for (int u = 0; u < 16; ++u) pp = fmaf(Zs[ti][16 * tg + u], acc[16 * tg + u][j], pp);
      pp += __shfl_xor_sync(0xffffffffu, pp, 1);
      pp += __shfl_xor_sync(0xffffffffu, pp, 2);
      if (tg == 0 && ti < rb) B[(r0 + ti) * ldb + c0 + j] = pp;
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();  // cumulative: orders the block's stores (seen through the barrier) before the flag
      st_rel(flags + r, epoch);
    }
  }
}

rbf_status trsm32(Ctx* c, const float* L, int64_t n, int64_t ldl, const float* Zd, float* B, int64_t m,
                  int64_t ldb, bool transpose, cudaStream_t s, int64_t bw) {
  if (n <= 0 || m <= 0) return RBF_OK;
  int64_t nblk = (n + MB - 1) / MB;
  if (c->sync_flags.bytes < (size_t)nblk * sizeof(int)) {
    RBF_TRY(c->sync_flags.ensure((size_t)nblk * sizeof(int)));
    RBF_CUDA(cudaMemsetAsync(c->sync_flags.p, 0, c->sync_flags.bytes, s));
    c->epoch = 0;
  }
  static int max_blocks[64] = {0};
  const size_t dyn = (size_t)2 * MB * (T32_MC + 1) * sizeof(float);
  int dev = c->device & 63;
  if (!max_blocks[dev]) {
    int per_sm = 0, sms = 0;
    RBF_CUDA(cudaFuncSetAttribute(k_trsm32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    RBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trsm32, 256, dyn));
    RBF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    max_blocks[dev] = per_sm * sms;
  }
  int64_t grid = nblk < max_blocks[dev] ? nblk : max_blocks[dev];
  if (grid < 1) return fail(RBF_ECUDA, "trsm32: no co-resident blocks");
  int* flags = c->sync_flags.as<int>();
  int* status = c->dflag.as<int>();
  for (int64_t c0 = 0; c0 < m; c0 += T32_MC) {
    int mc = (int)((m - c0) < T32_MC ? (m - c0) : T32_MC);
    int epoch = (int)(++c->epoch);
    int c0i = (int)c0;
    int bwb = (int)(bw >= n ? nblk : bw / MB + 2);
    long long lim = c->spin_limit > 0 ? c->spin_limit : T32_SPIN;
    int wx = c->wait_xor;
    void* args[] = {(void*)&L, (void*)&ldl, (void*)&n, (void*)&Zd, (void*)&B, (void*)&ldb, (void*)&c0i,
                    (void*)&mc, (void*)&transpose, (void*)&bwb, (void*)&flags, (void*)&epoch, (void*)&status,
                    (void*)&lim, (void*)&wx};
    StageTimer st(c, RBF_STAGE_TRSM32, s, (double)n * (double)n * (double)mc);
    RBF_CUDA(cooperative_launch((const void*)k_trsm32, dim3((unsigned)grid), dim3(256), args, dyn, s));
  }
  return RBF_OK;
}

// ---------------------------------------------------------------------------
// Refined solves H X = B (float64, n x m, row-major ld m) with the float32
// factor.  X overwrites B.  Each sweep: R = B - H X (float64), C = factor
// solve of R (float32), X += C.
// ---------------------------------------------------------------------------
__global__ void k_f64_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
__global__ void k_f32_to_f64(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}
__global__ void k_add_f32_to_f64(double* __restrict__ x, const float* __restrict__ c, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] += (double)c[i];
}

// R = B - H X for m right-hand sides (row-major n x m): one warp per row of H,
// 8 right-hand sides per pass, lanes stride over the row.
__global__ void __launch_bounds__(256) k_residual_multi(const double* __restrict__ H, int64_t n, int64_t ldh,
                                                        const double* __restrict__ X, const double* __restrict__ Bm,
                                                        int64_t m, double* __restrict__ R) {
  int lane = threadIdx.x & 31;
  int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  const double* hr = H + row * ldh;
  for (int64_t j0 = 0; j0 < m; j0 += 8) {
    int q = (int)((m - j0) < 8 ? (m - j0) : 8);
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t t = lane; t < n; t += 32) {
      double h = hr[t];
      const double* xr = X + t * m + j0;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (u < q) acc[u] = fma(h, xr[u], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      double v = acc[u];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0 && u < q) R[row * m + j0 + u] = Bm[row * m + j0 + u] - v;
    }
  }
}

rbf_status mixed_solve(Ctx* c, const double* H, int64_t ldh, const SpH* Hs, const float* W, int64_t ldw,
                       const float* Zd, const float* Zi, int64_t n, double* B, int64_t m, int sweeps,
                       cudaStream_t s, int64_t bw) {
  if (Hs && !(Hs->valid && Hs->n == n)) Hs = nullptr;
  if (n <= 0 || m <= 0) return RBF_OK;
  int64_t tot = n * m;
  Buf& xb = c->scratch(59);
  Buf& rb = c->scratch(60);
  Buf& fb = c->scratch(61);
  Buf& bb = c->scratch(62);
  RBF_TRY(xb.ensure((size_t)tot * sizeof(double)));
  RBF_TRY(rb.ensure((size_t)tot * sizeof(double)));
  RBF_TRY(fb.ensure((size_t)tot * sizeof(float)));
  RBF_TRY(bb.ensure((size_t)tot * sizeof(double)));
  double* X = xb.as<double>();
  double* Rr = rb.as<double>();
  float* F = fb.as<float>();
  RBF_CUDA(cudaMemcpyAsync(bb.p, B, (size_t)tot * sizeof(double), cudaMemcpyDeviceToDevice, s));
  RBF_CUDA(cudaMemsetAsync(X, 0, (size_t)tot * sizeof(double), s));
  const double* R = B;  // first sweep: X = 0, so R = B
  unsigned nb = (unsigned)((tot + 255) / 256);
  for (int it = 0; it < sweeps; ++it) {
    if (Zi && m <= 8) {
      // X += Z^T Z R, the roundings inside the two matrix-vector launches
      RBF_TRY(inv_solve_acc(c, Zi, ldw, n, R, X, m, s));
    } else {
      { k_f64_to_f32<<<nb, 256, 0, s>>>(R, F, tot); ::rbf::note_launch(); }
      RBF_CUDA(cudaGetLastError());
      if (Zi) {
        RBF_TRY(inv_solve(c, Zi, ldw, n, F, m, s));
      } else {
        RBF_TRY(trsm32(c, W, n, ldw, Zd, F, m, m, false, s, bw));
        RBF_TRY(trsm32(c, W, n, ldw, Zd, F, m, m, true, s, bw));
      }
      { k_add_f32_to_f64<<<nb, 256, 0, s>>>(X, F, tot); ::rbf::note_launch(); }
      RBF_CUDA(cudaGetLastError());
    }
    if (it + 1 < sweeps) {
      if (Hs) {
        RBF_TRY(csr_residual(*Hs, X, bb.as<double>(), m, Rr, s));
      } else if (m == 1) {
        RBF_TRY(symv_residual(H, n, ldh, X, bb.as<double>(), Rr, s));
      } else {
        unsigned nw = (unsigned)((n * 32 + 255) / 256);
        { k_residual_multi<<<nw, 256, 0, s>>>(H, n, ldh, X, bb.as<double>(), m, Rr); ::rbf::note_launch(); }
        RBF_CUDA(cudaGetLastError());
      }
      R = Rr;
    }
  }
  RBF_CUDA(cudaMemcpyAsync(B, X, (size_t)tot * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return RBF_OK;
}

// Block P[D, D] = E_D^T H^{-1} E_D of the covariance for the columns B = E_D
// (unit vectors at positions pos, overwritten).  X comes from sweeps - 1
// refined solves; then one residual R = E_D - H X (float-float products,
// float64 result) gives the second-order estimate
//   P = E_D^T X + X^T R    (error -(X - H^{-1}E_D)^T H (X - H^{-1}E_D)),
// symmetrised.  With the float32 factor accurate to eps, one solve already
// gives P to about eps^2, where one more refinement sweep would need a
// second solve.
__global__ void k_sym_gather(const double* __restrict__ X, int64_t k, const int32_t* __restrict__ pos,
                             double* __restrict__ P) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * k) return;
  int64_t u = e / k, v = e % k;
  P[e] = 0.5 * (X[(int64_t)pos[u] * k + v] + X[(int64_t)pos[v] * k + u]);
}

// P = sym(X[pos, :]) + sym(G), G = X^T R
__global__ void k_cov_second_order(const double* __restrict__ X, int64_t k, const int32_t* __restrict__ pos,
                                   const double* __restrict__ G, double* __restrict__ P) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * k) return;
  int64_t u = e / k, v = e % k;
  P[e] = 0.5 * (X[(int64_t)pos[u] * k + v] + X[(int64_t)pos[v] * k + u]) + 0.5 * (G[u * k + v] + G[v * k + u]);
}

rbf_status mixed_cov(Ctx* c, const double* H, int64_t ldh, const SpH* Hs, const float* W, int64_t ldw,
                     const float* Zd, const float* Zi, int64_t n, double* B, int64_t k, const int32_t* pos,
                     int sweeps, double* P, cudaStream_t s, int64_t bw) {
  if (n <= 0 || k <= 0) return RBF_OK;
  if (Hs && !(Hs->valid && Hs->n == n)) Hs = nullptr;
  if (sweeps <= 1) {
    RBF_TRY(mixed_solve(c, H, ldh, Hs, W, ldw, Zd, Zi, n, B, k, 1, s, bw));
    { k_sym_gather<<<(unsigned)((k * k + 255) / 256), 256, 0, s>>>(B, k, pos, P); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    return RBF_OK;
  }
  int64_t tot = n * k;
  Buf& e0 = c->scratch(57);
  Buf& rr = c->scratch(58);
  RBF_TRY(e0.ensure((size_t)tot * sizeof(double)));
  RBF_TRY(rr.ensure((size_t)tot * sizeof(double)));
  RBF_CUDA(cudaMemcpyAsync(e0.p, B, (size_t)tot * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (Zi && sweeps == 2) {
    // X = Z^T Z E_D: the first product is a gather of columns of Z
    Buf& fb = c->scratch(61);
    RBF_TRY(fb.ensure((size_t)tot * sizeof(float)));
    RBF_TRY(inv_solve_unit(c, Zi, ldw, n, pos, k, fb.as<float>(), s));
    { k_f32_to_f64<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(fb.as<float>(), B, tot); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  } else {
    RBF_TRY(mixed_solve(c, H, ldh, Hs, W, ldw, Zd, Zi, n, B, k, sweeps - 1, s, bw));
  }
  double* R = rr.as<double>();
  if (bw >= n) {
    // H filled in by earlier departures: a tiled product over the dense H
    RBF_CUDA(cudaMemcpyAsync(R, e0.p, (size_t)tot * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RBF_TRY(gemm_ff(c, false, false, n, k, n, -1.0, H, ldh, B, k, 1.0, R, k, s, 97));
  } else if (Hs) {
    RBF_TRY(csr_residual_ff(c, *Hs, B, e0.as<double>(), k, R, s, 97));
  } else {
    unsigned nw = (unsigned)((n * 32 + 255) / 256);
    { k_residual_multi<<<nw, 256, 0, s>>>(H, n, ldh, B, e0.as<double>(), k, R); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }
  Buf& gq = c->scratch(86);
  RBF_TRY(gq.ensure((size_t)k * k * sizeof(double)));
  RBF_TRY(gemm_ff(c, true, false, k, k, n, 1.0, B, k, R, k, 0.0, gq.as<double>(), k, s, 96));
  { k_cov_second_order<<<(unsigned)((k * k + 255) / 256), 256, 0, s>>>(B, k, pos, gq.as<double>(), P); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  return RBF_OK;
}

}  // namespace rbf
