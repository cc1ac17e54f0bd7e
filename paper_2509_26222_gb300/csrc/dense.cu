// Dense FP64 linear algebra for the active-block update (Sec. III-C).
//
// The update needs the Cholesky factor of the information matrix of the
// active rows (the matrix whose inverse Eq. kf_w_update applies), triangular
// solves with it, a partial factorization (Schur complement) to drop centers
// that leave the active block, and a few small products.  All matrices are
// row-major with a leading dimension; only lower triangles are referenced
// where a matrix is symmetric.
//
//  potrf_lower: right-looking blocked Cholesky, block NB = 32.  Per block
//    column: one kernel factors the 32 x 32 diagonal tile (every CTA redoes it
//    in shared memory) and solves its share of the panel rows; one kernel
//    applies the rank-32 update to the lower trailing tiles.  Stopping after
//    nfactor columns leaves the Schur complement in the trailing block.
//  trsm_lower: L X = B or L^T X = B for many right-hand sides with one
//    cooperative launch: CTA b owns block rows b, b + G, ... and waits on a
//    per-block-row flag (bounded spin; a timeout sets a status bit) before
//    consuming a solved block.
#include <math.h>

#include "common.cuh"

namespace rbf {

constexpr int NB = 32;

// ---------------------------------------------------------------------------
// Diagonal tile factorization in shared memory (kb <= 32), all threads of the
// CTA participate.  T is [32][33].  Returns through T (lower triangle).
// ---------------------------------------------------------------------------
__device__ void chol_tile_smem(double (*T)[NB + 1], int kb, int* flag) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, ny = blockDim.x >> 5;
  __shared__ double rinv;
  for (int j = 0; j < kb; ++j) {
    if (threadIdx.x == 0) {
      double d = T[j][j];
      if (!(d > 0.0)) {
        atomicOr(flag, DEV_NOT_SPD);
        d = 1.0;
      }
      double r = sqrt(d);
      T[j][j] = r;
      rinv = 1.0 / r;
    }
    __syncthreads();
    if (threadIdx.x < 32 && tx > j && tx < kb) T[tx][j] *= rinv;
    __syncthreads();
    if (tx > j) {
      double tkj = T[tx][j];
      for (int i = ty; i < kb; i += ny)
        if (i >= tx) T[i][tx] -= T[i][j] * tkj;
    }
    __syncthreads();
  }
}

// Panel kernel of step k: factor A[k:k+kb, k:k+kb], then solve rows
// [k+kb, n) of the block column: X L_kk^T = A[rows, k:k+kb].
__global__ void __launch_bounds__(256) k_potrf_panel(double* __restrict__ A, int64_t lda, int64_t n,
                                                     int64_t k, int kb, int rows_per_cta,
                                                     double* __restrict__ dtile,
                                                     int* __restrict__ flag) {
  __shared__ double T[NB][NB + 1];
  __shared__ double inv_d[NB];
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    int i = e / NB, j = e % NB;
    T[i][j] = (i < kb && j <= i) ? A[(k + i) * lda + k + j] : 0.0;
  }
  __syncthreads();
  chol_tile_smem(T, kb, flag);
  if (threadIdx.x < NB) inv_d[threadIdx.x] = threadIdx.x < kb ? 1.0 / T[threadIdx.x][threadIdx.x] : 0.0;
  __syncthreads();
  // every CTA reads the unfactored tile from A, so the factored tile goes to
  // scratch and k_copy_tile writes it back after this kernel
  if (blockIdx.x == 0) {
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
      int i = e / NB, j = e % NB;
      dtile[e] = (j <= i) ? T[i][j] : 0.0;
    }
  }
  // panel rows: one warp per row, lane c holds column c
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t r0 = k + kb + (int64_t)blockIdx.x * rows_per_cta;
  int64_t r1 = r0 + rows_per_cta;
  if (r1 > n) r1 = n;
  for (int64_t r = r0 + wid; r < r1; r += nw) {
    double* row = A + r * lda + k;
    double b = lane < kb ? row[lane] : 0.0;
    for (int t = 0; t < kb; ++t) {
      double xt = __shfl_sync(0xffffffffu, b, t) * inv_d[t];
      if (lane == t) b = xt;
      else if (lane > t) b -= xt * T[lane][t];
    }
    if (lane < kb) row[lane] = b;
  }
}

__global__ void k_copy_tile(double* __restrict__ A, int64_t lda, int64_t k, int kb,
                            const double* __restrict__ dtile) {
  for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
    int i = e / kb, j = e % kb;
    A[(k + i) * lda + k + j] = dtile[i * NB + j];
  }
}

// Trailing update of step k: for lower tiles (ti >= tj) of the block
// A[k0:n, k0:n] (k0 = k + kb): C -= P P^T with P = A[k0:n, k:k+kb].
constexpr int ST = 64;  // output tile
__global__ void __launch_bounds__(256) k_syrk_trailing(double* __restrict__ A, int64_t lda, int64_t n,
                                                       int64_t k, int kb) {
  int64_t k0 = k + kb;
  int64_t b = blockIdx.x;
  int64_t ti = (int64_t)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
  while ((ti + 1) * (ti + 2) / 2 <= b) ++ti;
  while (ti * (ti + 1) / 2 > b) --ti;
  int64_t tj = b - ti * (ti + 1) / 2;
  int64_t i0 = k0 + ti * ST, j0 = k0 + tj * ST;
  __shared__ double Pi[NB][ST + 1];
  __shared__ double Pj[NB][ST + 1];
  for (int e = threadIdx.x; e < ST * NB; e += blockDim.x) {
    int r = e / NB, t = e % NB;
    double vi = 0.0, vj = 0.0;
    if (t < kb) {
      if (i0 + r < n) vi = A[(i0 + r) * lda + k + t];
      if (j0 + r < n) vj = A[(j0 + r) * lda + k + t];
    }
    Pi[t][r] = vi;
    Pj[t][r] = vj;
  }
  __syncthreads();
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int t = 0; t < kb; ++t) {
    double a[4], bb[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] = Pi[t][ty * 4 + u];
      bb[u] = Pj[t][tx * 4 + u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], bb[v], acc[u][v]);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int64_t i = i0 + ty * 4 + u;
    if (i >= n) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int64_t j = j0 + tx * 4 + v;
      if (j < n && j <= i) A[i * lda + j] -= acc[u][v];
    }
  }
}

rbf_status potrf_lower(Ctx* c, double* A, int64_t n, int64_t lda, int64_t nfactor, bool mixed,
                       cudaStream_t s, int64_t bw) {
  (void)mixed;
  if (n <= 0 || nfactor <= 0) return RBF_OK;
  int* flag = c->dflag.as<int>();
  Buf& dt = c->scratch(30);
  RBF_TRY(dt.ensure(NB * NB * sizeof(double)));
  for (int64_t k = 0; k < nfactor; k += NB) {
    int kb = (int)((nfactor - k) < NB ? (nfactor - k) : NB);
    // rows beyond the band are zero in this panel and untouched by its update
    const int64_t ne = (k + kb + bw) < n ? (k + kb + bw) : n;
    int64_t rows = ne - k - kb;
    int rows_per_cta = 16;
    int64_t ctas = rows > 0 ? (rows + rows_per_cta - 1) / rows_per_cta : 1;
    {
      StageTimer st(c, RBF_STAGE_PANEL, s, (double)kb * kb * kb / 3.0 + (double)rows * kb * kb);
      { k_potrf_panel<<<(unsigned)ctas, 256, 0, s>>>(A, lda, ne, k, kb, rows_per_cta, dt.as<double>(),
                                                   flag); ::rbf::note_launch(); }
      RBF_CUDA(cudaGetLastError());
      { k_copy_tile<<<1, 256, 0, s>>>(A, lda, k, kb, dt.as<double>()); ::rbf::note_launch(); }
      RBF_CUDA(cudaGetLastError());
    }
    if (rows > 0) {
      StageTimer st(c, RBF_STAGE_TRAILING, s, (double)rows * (double)(rows + 1) * kb);
      int64_t T = (rows + ST - 1) / ST;
      int64_t tiles = T * (T + 1) / 2;
      { k_syrk_trailing<<<(unsigned)tiles, 256, 0, s>>>(A, lda, ne, k, kb); ::rbf::note_launch(); }
      RBF_CUDA(cudaGetLastError());
    }
  }
  return RBF_OK;
}

// ---------------------------------------------------------------------------
// Sync-free blocked triangular solve with many right-hand sides.
// ---------------------------------------------------------------------------
constexpr int TS_MC = 32;          // right-hand sides per launch
constexpr int TS_THREADS = 256;
constexpr long long TS_SPIN_LIMIT = 1LL << 22;

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Solves op(L) X = B in place for columns [c0, c0 + mc) of B.
// transpose = false: forward (block rows in order 0..nblk-1)
// transpose = true : backward with L^T (block rows nblk-1..0)
// Before waiting on anything, a CTA inverts the diagonal block of its block
// row; each dependency is then a 32 x 32 x mc product from a shared-memory
// copy of the solved block, and the final step is x = D^{-1} acc.
__global__ void __launch_bounds__(TS_THREADS) k_trsm_syncfree(const double* __restrict__ L, int64_t ldl,
                                                              int64_t n, double* B, int64_t ldb,
                                                              int c0, int mc, bool transpose, int64_t bwb,
                                                              int* flags, int epoch, int* status,
                                                              long long spin_limit, int wait_xor) {
  __shared__ double acc[NB][TS_MC + 1];
  __shared__ double Xs[NB][TS_MC + 1];
  __shared__ double Dinv[NB][NB + 1];
  __shared__ double Dg[NB][NB + 1];
  __shared__ int bail;
  const int tid = threadIdx.x, ti = tid >> 3, tg = tid & 7;
  const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  int64_t nblk = (n + NB - 1) / NB;
  for (int64_t lk = blockIdx.x; lk < nblk; lk += gridDim.x) {
    int64_t r = transpose ? (nblk - 1 - lk) : lk;
    int64_t r0 = r * NB;
    int rb = (int)((n - r0) < NB ? (n - r0) : NB);
    // diagonal block op(L)_rr (lower for forward, upper for transpose) and its inverse
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      int i = e / NB, j = e % NB;
      double v = (i == j) ? 1.0 : 0.0;
      if (i < rb && j < rb) v = transpose ? L[(r0 + j) * ldl + r0 + i] : L[(r0 + i) * ldl + r0 + j];
      Dg[i][j] = v;
    }
    for (int e = tid; e < NB * TS_MC; e += blockDim.x) {
      int i = e / TS_MC, j = e % TS_MC;
      acc[i][j] = (i < rb && j < mc) ? B[(r0 + i) * ldb + c0 + j] : 0.0;
    }
    if (tid == 0) bail = 0;
    __syncthreads();
    // column c of D^{-1}: solve D x = e_c by substitution, lane = row
    for (int cidx = wid; cidx < NB; cidx += nw) {
      double b = (lane == cidx) ? 1.0 : 0.0;
      if (!transpose) {
        for (int t = 0; t < NB; ++t) {
          double xt = __shfl_sync(0xffffffffu, b, t) / Dg[t][t];
          if (lane == t) b = xt;
          else if (lane > t) b -= Dg[lane][t] * xt;
        }
      } else {
        for (int t = NB - 1; t >= 0; --t) {
          double xt = __shfl_sync(0xffffffffu, b, t) / Dg[t][t];
          if (lane == t) b = xt;
          else if (lane < t) b -= Dg[lane][t] * xt;
        }
      }
      Dinv[lane][cidx] = b;
    }
    for (int64_t lc = (lk - bwb) > 0 ? (lk - bwb) : 0; lc < lk; ++lc) {  // blocks outside the band are zero
      int64_t cb = transpose ? (nblk - 1 - lc) : lc;
      int64_t cc0 = cb * NB;
      int cbs = (int)((n - cc0) < NB ? (n - cc0) : NB);
      double lv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int t = 4 * tg + u;
        double v = 0.0;
        if (ti < rb && t < cbs)
          v = transpose ? L[(cc0 + t) * ldl + r0 + ti] : L[(r0 + ti) * ldl + cc0 + t];
        lv[u] = v;
      }
      if (tid == 0) {
        long long it = 0;
        while (ld_acquire(flags + cb) != (epoch ^ wait_xor)) {
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
      for (int e = tid; e < NB * mc; e += blockDim.x) {
        int t = e / mc, j = e % mc;
        Xs[t][j] = (t < cbs) ? __ldcg(B + (cc0 + t) * ldb + c0 + j) : 0.0;
      }
      __syncthreads();
      for (int j = 0; j < mc; ++j) {
        double pp = 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u) pp = fma(lv[u], Xs[4 * tg + u][j], pp);
        pp += __shfl_xor_sync(0xffffffffu, pp, 1);
        pp += __shfl_xor_sync(0xffffffffu, pp, 2);
        pp += __shfl_xor_sync(0xffffffffu, pp, 4);
        if (tg == 0) acc[ti][j] -= pp;
      }
      __syncthreads();
    }
    __syncthreads();
    // x = D^{-1} acc
    for (int j = 0; j < mc; ++j) {
      double pp = 0.0;
#pragma unroll
      for (int u = 0; u < 4; ++u) pp = fma(Dinv[ti][4 * tg + u], acc[4 * tg + u][j], pp);
      pp += __shfl_xor_sync(0xffffffffu, pp, 1);
      pp += __shfl_xor_sync(0xffffffffu, pp, 2);
      pp += __shfl_xor_sync(0xffffffffu, pp, 4);
      if (tg == 0 && ti < rb) B[(r0 + ti) * ldb + c0 + j] = pp;
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();  // cumulative: orders the block's stores (seen through the barrier) before the flag
      st_release(flags + r, epoch);
    }
  }
}

rbf_status trsm_lower(Ctx* c, const double* L, int64_t n, int64_t ldl, double* B, int64_t m,
                      int64_t ldb, bool transpose, cudaStream_t s, int64_t bw) {
  if (n <= 0 || m <= 0) return RBF_OK;
  int64_t nblk = (n + NB - 1) / NB;
  if (c->sync_flags.bytes < (size_t)nblk * sizeof(int)) {
    RBF_TRY(c->sync_flags.ensure((size_t)nblk * sizeof(int)));
    RBF_CUDA(cudaMemsetAsync(c->sync_flags.p, 0, c->sync_flags.bytes, s));
    c->epoch = 0;
  }
  static int max_blocks_dev[64] = {0};
  int dev = c->device;
  if (!max_blocks_dev[dev & 63]) {
    int per_sm = 0, sms = 0;
    RBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trsm_syncfree, TS_THREADS, 0));
    RBF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    max_blocks_dev[dev & 63] = per_sm * sms;
  }
  int64_t grid = nblk < max_blocks_dev[dev & 63] ? nblk : max_blocks_dev[dev & 63];
  if (grid < 1) return fail(RBF_ECUDA, "trsm: no co-resident blocks");
  int* flags = c->sync_flags.as<int>();
  int* status = c->dflag.as<int>();
  for (int64_t c0 = 0; c0 < m; c0 += TS_MC) {
    int mc = (int)((m - c0) < TS_MC ? (m - c0) : TS_MC);
    int epoch = (int)(++c->epoch);
    int c0i = (int)c0;
    int64_t bwb = bw >= n ? nblk : bw / NB + 2;
    long long lim = c->spin_limit > 0 ? c->spin_limit : TS_SPIN_LIMIT;
    int wx = c->wait_xor;
    void* args[] = {(void*)&L, (void*)&ldl, (void*)&n, (void*)&B, (void*)&ldb, (void*)&c0i,
                    (void*)&mc, (void*)&transpose, (void*)&bwb, (void*)&flags, (void*)&epoch, (void*)&status,
                    (void*)&lim, (void*)&wx};
    RBF_CUDA(cooperative_launch((const void*)k_trsm_syncfree, dim3((unsigned)grid),
                                         dim3(TS_THREADS), args, 0, s));
  }
  return RBF_OK;
}

// ---------------------------------------------------------------------------
// Inverse of a small SPD matrix (m <= 64) in one CTA by Gauss-Jordan
// elimination without pivoting (the pivots are the diagonals of successive
// Schur complements, positive for an SPD matrix).  Each of the m steps is one
// parallel update of all m^2 entries between two barriers.  In place,
// row-major m x m, symmetrised on output.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_spd_inverse_small(double* __restrict__ G, int m, int* __restrict__ flag) {
  extern __shared__ double gj[];  // A (m x (m + 1)), then the pivot column and row
  const int ld = m + 1;
  double* A = gj;
  double* fcol = gj + (int64_t)m * ld;
  double* prow = fcol + m;
  const int tid = threadIdx.x;
  for (int e = tid; e < m * m; e += blockDim.x) A[(e / m) * ld + e % m] = G[e];
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    if (tid < m) {
      fcol[tid] = A[tid * ld + k];
      prow[tid] = A[k * ld + tid];
    }
    __syncthreads();
    double p = prow[k];
    if (!(p > 0.0)) {
      if (tid == 0) atomicOr(flag, DEV_NOT_SPD);
      p = 1.0;
    }
    const double rp = 1.0 / p;
    for (int i = tid >> 4; i < m; i += 16) {  // 16 x 16 threads, no index division
      const double fi = -fcol[i] * rp;
      for (int j = tid & 15; j < m; j += 16) {
        double v;
        if (i == k) v = (j == k) ? rp : prow[j] * rp;
        else v = (j == k) ? fi : fma(fi, prow[j], A[i * ld + j]);
        A[i * ld + j] = v;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < m * m; e += blockDim.x) {
    int i = e / m, j = e % m;
    G[e] = 0.5 * (A[i * ld + j] + A[j * ld + i]);
  }
}

rbf_status spd_inverse_small(Ctx* c, double* G, int64_t m, cudaStream_t s) {
  if (m <= 0 || m > SPD_SMALL_MAX) return fail(RBF_EINVAL, "spd_inverse_small: m must be in [1, %d]", SPD_SMALL_MAX);
  size_t smem = (size_t)(m * (m + 1) + 2 * m) * sizeof(double);
  static bool attr[64] = {false};
  if (!attr[c->device & 63]) {
    size_t mx = (size_t)(SPD_SMALL_MAX * (SPD_SMALL_MAX + 1) + 2 * SPD_SMALL_MAX) * sizeof(double);
    RBF_CUDA(cudaFuncSetAttribute(k_spd_inverse_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx));
    attr[c->device & 63] = true;
  }
  { k_spd_inverse_small<<<1, 256, smem, s>>>(G, (int)m, c->dflag.as<int>()); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  return RBF_OK;
}

// ---------------------------------------------------------------------------
// Small FP64 GEMM: C = alpha op(A) op(B) + beta C (row-major).
// ---------------------------------------------------------------------------
constexpr int GT = 32;
__global__ void __launch_bounds__(256) k_gemm_f64(bool ta, bool tb, int64_t m, int64_t n, int64_t k,
                                                  double alpha, const double* __restrict__ A,
                                                  int64_t lda, const double* __restrict__ B,
                                                  int64_t ldb, double beta, double* __restrict__ Cm,
                                                  int64_t ldc) {
  __shared__ double As[GT][GT + 1];
  __shared__ double Bs[GT][GT + 1];
  int64_t i0 = (int64_t)blockIdx.y * GT, j0 = (int64_t)blockIdx.x * GT;
  int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of threads, 4 outputs each
  double acc[4] = {0, 0, 0, 0};
  for (int64_t k0 = 0; k0 < k; k0 += GT) {
    for (int e = threadIdx.x; e < GT * GT; e += blockDim.x) {
      int r = e / GT, q = e % GT;
      int64_t ia = i0 + r, ka = k0 + q;
      double va = 0.0;
      if (ia < m && ka < k) va = ta ? A[ka * lda + ia] : A[ia * lda + ka];
      As[r][q] = va;
      int64_t kb = k0 + r, jb = j0 + q;
      double vb = 0.0;
      if (kb < k && jb < n) vb = tb ? B[jb * ldb + kb] : B[kb * ldb + jb];
      Bs[r][q] = vb;
    }
    __syncthreads();
#pragma unroll 8
    for (int t = 0; t < GT; ++t) {
      double b = Bs[t][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fma(As[ty * 4 + u][t], b, acc[u]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int64_t i = i0 + ty * 4 + u, j = j0 + tx;
    if (i < m && j < n) {
      double prev = beta != 0.0 ? Cm[i * ldc + j] : 0.0;
      Cm[i * ldc + j] = alpha * acc[u] + beta * prev;
    }
  }
}

// Partial products over a slice of k (split-K) for small outputs with long k.
__global__ void __launch_bounds__(256) k_gemm_splitk(bool ta, bool tb, int64_t m, int64_t n, int64_t k,
                                                     int64_t kchunk, const double* __restrict__ A,
                                                     int64_t lda, const double* __restrict__ B,
                                                     int64_t ldb, double* __restrict__ part) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * n) return;
  int64_t i = e / n, j = e % n;
  int64_t k0 = (int64_t)blockIdx.y * kchunk, k1 = k0 + kchunk < k ? k0 + kchunk : k;
  double acc = 0.0;
  for (int64_t t = k0; t < k1; ++t) {
    double a = ta ? A[t * lda + i] : A[i * lda + t];
    double b = tb ? B[j * ldb + t] : B[t * ldb + j];
    acc = fma(a, b, acc);
  }
  part[(int64_t)blockIdx.y * m * n + e] = acc;
}

__global__ void k_gemm_reduce(int64_t m, int64_t n, int nsplit, const double* __restrict__ part, double alpha,
                              double beta, double* __restrict__ Cm, int64_t ldc) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * n) return;
  double acc = 0.0;
  for (int q = 0; q < nsplit; ++q) acc += part[(int64_t)q * m * n + e];
  int64_t i = e / n, j = e % n;
  double prev = beta != 0.0 ? Cm[i * ldc + j] : 0.0;
  Cm[i * ldc + j] = alpha * acc + beta * prev;
}

rbf_status gemm_f64(Ctx* c, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                    int64_t lda, const double* B, int64_t ldb, double beta, double* Cm, int64_t ldc,
                    cudaStream_t s, int slot) {
  if (m <= 0 || n <= 0) return RBF_OK;
  int64_t tiles = ((m + GT - 1) / GT) * ((n + GT - 1) / GT);
  if (tiles < 64 && k > 512) {
    int64_t kchunk = 64;
    int64_t nsplit = (k + kchunk - 1) / kchunk;
    if (nsplit > 4096) {
      nsplit = 4096;
      kchunk = (k + nsplit - 1) / nsplit;
      nsplit = (k + kchunk - 1) / kchunk;
    }
    Buf& part = c->scratch(slot);
    RBF_TRY(part.ensure((size_t)nsplit * m * n * sizeof(double)));
    dim3 grid((unsigned)((m * n + 255) / 256), (unsigned)nsplit);
    { k_gemm_splitk<<<grid, 256, 0, s>>>(ta, tb, m, n, k, kchunk, A, lda, B, ldb, part.as<double>()); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    { k_gemm_reduce<<<(unsigned)((m * n + 255) / 256), 256, 0, s>>>(m, n, (int)nsplit, part.as<double>(), alpha,
                                                                 beta, Cm, ldc); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    return RBF_OK;
  }
  dim3 grid((unsigned)((n + GT - 1) / GT), (unsigned)((m + GT - 1) / GT));
  { k_gemm_f64<<<grid, 256, 0, s>>>(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  return RBF_OK;
}

// r = b - H x for a symmetric H stored in full (one warp per row).
__global__ void __launch_bounds__(256) k_symv_residual(const double* __restrict__ H, int64_t n, int64_t ld,
                                                       const double* __restrict__ x,
                                                       const double* __restrict__ b,
                                                       double* __restrict__ r) {
  int lane = threadIdx.x & 31;
  int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  double acc = 0.0;
  for (int64_t j = lane; j < n; j += 32) acc = fma(H[row * ld + j], x[j], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) r[row] = b[row] - acc;
}

rbf_status symv_residual(const double* H, int64_t n, int64_t ld, const double* x, const double* b,
                         double* r, cudaStream_t s) {
  if (n <= 0) return RBF_OK;
  { k_symv_residual<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(H, n, ld, x, b, r); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  return RBF_OK;
}

}  // namespace rbf
