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

namespace rbf {

constexpr int MB = 64;  // block size of the mixed factorization (= tc::KB)

__global__ void k_mx_to_f32(const double* __restrict__ H, int64_t ldh, int64_t n, float* __restrict__ W,
                            int64_t ldw) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  int64_t i = e / n, j = e % n;
  W[i * ldw + j] = (float)H[i * ldh + j];
}

// Cholesky of the 64 x 64 diagonal block (float32, one CTA of 256 threads),
// right-looking with one barrier per column: every thread computes the
// pivot's reciprocal square root itself, the trailing update uses
// T_ik -= T_ij T_kj / T_jj with unscaled columns, and the columns are scaled
// once at the end.  rd[j] = 1 / L_jj is kept for the panel solve.
__global__ void __launch_bounds__(256) k_mx_diag(float* __restrict__ W, int64_t ldw, int64_t k, int kb,
                                                 float* __restrict__ rd_out, int* __restrict__ flag) {
  __shared__ float T[MB][MB + 1];
  __shared__ float rv[MB];
  const int tid = threadIdx.x;
  for (int e = tid; e < MB * MB; e += blockDim.x) {
    int i = e / MB, j = e % MB;
    float v;
    if (i < kb && j < kb) v = (j <= i) ? W[(k + i) * ldw + k + j] : 0.f;
    else v = (i == j) ? 1.f : 0.f;
    T[i][j] = v;
  }
  __syncthreads();
  const int tx = tid & (MB - 1), ty = tid >> 6;
  for (int j = 0; j < MB; ++j) {
    float d = T[j][j];
    float ri = rsqrtf(d);
    if (tid == 0) {
      if (!(d > 0.f)) atomicOr(flag, DEV_NOT_SPD);
      rv[j] = ri;
    }
    if (tx > j) {
      float ckj = T[tx][j] * ri * ri;
      float tij[MB / 4], tik[MB / 4];
#pragma unroll
      for (int q = 0; q < MB / 4; ++q) {
        int i = ty + 4 * q;
        tij[q] = T[i][j];
        tik[q] = T[i][tx];
      }
#pragma unroll
      for (int q = 0; q < MB / 4; ++q) {
        int i = ty + 4 * q;
        if (i >= tx) T[i][tx] = fmaf(-tij[q], ckj, tik[q]);
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < MB * MB; e += blockDim.x) {
    int i = e / MB, j = e % MB;
    if (i < kb && j < kb) W[(k + i) * ldw + k + j] = (j <= i) ? T[i][j] * rv[j] : 0.f;
  }
  if (tid < MB) rd_out[tid] = rv[tid];
}

// Panel rows [k + kb, n): solve X L_kk^T = W[rows, k:k+kb] row by row (four
// threads per row share each dot product), write X to W and as bf16 slices
// (row index relative to k + kb, 64 columns, zero beyond kb).
__global__ void __launch_bounds__(256) k_mx_panel(float* __restrict__ W, int64_t ldw, int64_t n, int64_t k,
                                                  int kb, const float* __restrict__ rd,
                                                  __nv_bfloat16* __restrict__ Ph, __nv_bfloat16* __restrict__ Pm,
                                                  __nv_bfloat16* __restrict__ Pl) {
  __shared__ float Ls[MB][MB + 1];  // L_kk (lower)
  __shared__ float X[MB][MB + 1];   // this CTA's 64 rows
  __shared__ float rds[MB];
  const int tid = threadIdx.x;
  const int64_t k0 = k + kb;
  const int64_t r0 = k0 + (int64_t)blockIdx.x * MB;
  for (int e = tid; e < MB * MB; e += blockDim.x) {
    int i = e / MB, t = e % MB;
    Ls[i][t] = (i < kb && t <= i) ? W[(k + i) * ldw + k + t] : 0.f;
    int64_t r = r0 + i;
    X[i][t] = (r < n && t < kb) ? W[r * ldw + k + t] : 0.f;
  }
  if (tid < MB) rds[tid] = tid < kb ? rd[tid] : 0.f;
  __syncthreads();
  const int ri = tid >> 2, g = tid & 3;
  const unsigned gm = 0xfu << (tid & 28);
  for (int j = 0; j < kb; ++j) {
    float s = 0.f;
    for (int t = g; t < j; t += 4) s = fmaf(X[ri][t], Ls[j][t], s);
    s += __shfl_xor_sync(gm, s, 1);
    s += __shfl_xor_sync(gm, s, 2);
    if (g == 0) X[ri][j] = (X[ri][j] - s) * rds[j];
    __syncwarp(gm);
  }
  __syncthreads();
  for (int e = tid; e < MB * MB; e += blockDim.x) {
    int i = e / MB, j = e % MB;
    int64_t r = r0 + i;
    if (r >= n) continue;
    float x = X[i][j];
    if (j < kb) W[r * ldw + k + j] = x;
    else x = 0.f;
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    float rem = x - __bfloat162float(h);
    __nv_bfloat16 mm = __float2bfloat16_rn(rem);
    float rem2 = rem - __bfloat162float(mm);
    __nv_bfloat16 l = __float2bfloat16_rn(rem2);
    int64_t pr = r - k0;
    Ph[pr * MB + j] = h;
    Pm[pr * MB + j] = mm;
    Pl[pr * MB + j] = l;
  }
}

// Inverses of every 64 x 64 diagonal block of the finished factor, one CTA per
// block (all blocks at once, off the factorization's critical chain): a row
// sweep with one barrier per row, Z_ic -= L_ij Z_jc after row j is final.
__global__ void __launch_bounds__(256) k_mx_blockinv(const float* __restrict__ W, int64_t ldw, int64_t n,
                                                     float* __restrict__ Zd) {
  __shared__ float T[MB][MB + 1];
  __shared__ float Z[MB][MB + 1];
  __shared__ float rl[MB];
  const int tid = threadIdx.x;
  const int64_t k = (int64_t)blockIdx.x * MB;
  const int kb = (int)((n - k) < MB ? (n - k) : MB);
  for (int e = tid; e < MB * MB; e += blockDim.x) {
    int i = e / MB, j = e % MB;
    float v;
    if (i < kb && j < kb) v = (j <= i) ? W[(k + i) * ldw + k + j] : 0.f;
    else v = (i == j) ? 1.f : 0.f;
    T[i][j] = v;
    Z[i][j] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  if (tid < MB) rl[tid] = 1.f / T[tid][tid];
  __syncthreads();
  const int tx = tid & (MB - 1), ty = tid >> 6;
  for (int j = 0; j < MB; ++j) {
    float lj = rl[j];
    if (tx <= j) {
      float zjc = Z[j][tx] * lj;
      float lij[MB / 4], zic[MB / 4];
#pragma unroll
      for (int q = 0; q < MB / 4; ++q) {
        int i = ty + 4 * q;
        lij[q] = T[i][j];
        zic[q] = Z[i][tx];
      }
#pragma unroll
      for (int q = 0; q < MB / 4; ++q) {
        int i = ty + 4 * q;
        if (i > j) Z[i][tx] = fmaf(-lij[q], zjc, zic[q]);
      }
    }
    __syncthreads();
    if (ty == 0 && tx <= j) Z[j][tx] *= lj;
    __syncthreads();
  }
  float* out = Zd + (int64_t)blockIdx.x * MB * MB;
  for (int e = tid; e < MB * MB; e += blockDim.x) out[e] = Z[e / MB][e % MB];
}

rbf_status potrf_mixed(Ctx* c, const double* H, int64_t ldh, int64_t n, float* W, int64_t ldw, float* Zd,
                       cudaStream_t s) {
  if (n <= 0) return RBF_OK;
  int* flag = c->dflag.as<int>();
  {
    int64_t tot = n * n;
    { k_mx_to_f32<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(H, ldh, n, W, ldw); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }
  Buf& pb = c->scratch(26);
  RBF_TRY(pb.ensure((size_t)3 * (n + MB) * MB * sizeof(__nv_bfloat16)));
  __nv_bfloat16* Ph = pb.as<__nv_bfloat16>();
  __nv_bfloat16* Pm = Ph + (n + MB) * MB;
  __nv_bfloat16* Pl = Pm + (n + MB) * MB;
  Buf& rb = c->scratch(54);
  RBF_TRY(rb.ensure(MB * sizeof(float)));
  float* rdiag = rb.as<float>();
  static bool attr_set[64] = {false};
  if (!attr_set[c->device & 63]) {
    RBF_CUDA(cudaFuncSetAttribute(tc::k_syrk_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES));
    attr_set[c->device & 63] = true;
  }
  for (int64_t k = 0, step = 0; k < n; k += MB, ++step) {
    int kb = (int)((n - k) < MB ? (n - k) : MB);
    int64_t rows = n - k - kb;
    {
      StageTimer st(c, RBF_STAGE_PANEL, s, (double)kb * kb * kb / 3.0 + (double)rows * kb * kb);
      { k_mx_diag<<<1, 256, 0, s>>>(W, ldw, k, kb, rdiag, flag); ::rbf::note_launch(); }
      RBF_CUDA(cudaGetLastError());
      if (rows > 0) {
        { k_mx_panel<<<(unsigned)((rows + MB - 1) / MB), 256, 0, s>>>(W, ldw, n, k, kb, rdiag, Ph, Pm,
                                                                       Pl); ::rbf::note_launch(); }
        RBF_CUDA(cudaGetLastError());
      }
    }
    if (rows > 0) {
      StageTimer st(c, RBF_STAGE_TRAILING, s, (double)rows * (double)(rows + 1) * kb);
      int64_t T = (rows + tc::TILE - 1) / tc::TILE;
      { tc::k_syrk_tc<<<(unsigned)(T * (T + 1) / 2), 128, tc::SMEM_BYTES, s>>>(W + (k + kb) * ldw + (k + kb), ldw,
                                                                              rows, Ph, Pm, Pl, flag); ::rbf::note_launch(); }
      RBF_CUDA(cudaGetLastError());
    }
  }
  {
    StageTimer st(c, RBF_STAGE_PANEL, s, 0.0);
    int64_t nb = (n + MB - 1) / MB;
    { k_mx_blockinv<<<(unsigned)nb, 256, 0, s>>>(W, ldw, n, Zd); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }
  return RBF_OK;
}

// ---------------------------------------------------------------------------
// float32 sync-free triangular solve (block 64) with the stored inverses of
// the diagonal blocks: op(L) X = B for up to 160 right-hand sides per launch.
// ---------------------------------------------------------------------------
constexpr int T32_MC = 160;
constexpr long long T32_SPIN = 1LL << 22;

__device__ __forceinline__ int ld_acq(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__global__ void __launch_bounds__(256) k_trsm32(const float* __restrict__ L, int64_t ldl, int64_t n,
                                                const float* __restrict__ Zd, float* B, int64_t ldb, int c0,
                                                int mc, bool transpose, int* flags, int epoch, int* status) {
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
    for (int64_t lc = 0; lc < lk; ++lc) {
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
        while (ld_acq(flags + cb) != epoch) {
          if (++it > T32_SPIN) {
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
                  int64_t ldb, bool transpose, cudaStream_t s) {
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
    void* args[] = {(void*)&L, (void*)&ldl, (void*)&n, (void*)&Zd, (void*)&B, (void*)&ldb, (void*)&c0i,
                    (void*)&mc, (void*)&transpose, (void*)&flags, (void*)&epoch, (void*)&status};
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

rbf_status mixed_solve(Ctx* c, const double* H, int64_t ldh, const float* W, int64_t ldw, const float* Zd,
                       int64_t n, double* B, int64_t m, int sweeps, cudaStream_t s) {
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
    { k_f64_to_f32<<<nb, 256, 0, s>>>(R, F, tot); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    RBF_TRY(trsm32(c, W, n, ldw, Zd, F, m, m, false, s));
    RBF_TRY(trsm32(c, W, n, ldw, Zd, F, m, m, true, s));
    { k_add_f32_to_f64<<<nb, 256, 0, s>>>(X, F, tot); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    if (it + 1 < sweeps) {
      if (m == 1) {
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

}  // namespace rbf
