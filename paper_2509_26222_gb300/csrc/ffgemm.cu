// Float64 products computed in float-float arithmetic on the float32 pipes.
//
// The block stage of the update (the Schur complement of the leaving centers
// and the float64 residuals of their covariance block) multiplies float64
// matrices of a few thousand rows by blocks of tens to hundreds of columns.
// GB300 executes float64 at a small fraction of its float32 rate, so these
// products take each operand as hi + lo (two float32, about 2^-48 relative),
// multiply-accumulate with error-free transforms (about 12 float32
// operations per product term, accuracy about 2^-46 relative to the sum of
// |terms|) and return float64.
#include "common.cuh"
#include "tiles.cuh"

namespace rbf {
namespace {

constexpr int FK = 16;  // k chunk

// s + t += x y, with x, y as hi + lo: the leading product's rounding error
// and the cross terms go to t, which is only added into s at the end
__device__ __forceinline__ void ff_acc(float& sacc, float& tacc, FF x, FF y) {
  const float p = __fmul_rn(x.hi, y.hi);
  const float e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, fmaf(x.hi, y.hi, -p)));
  const FF sum = ff_two_sum(sacc, p);
  sacc = sum.hi;
  tacc = __fadd_rn(tacc, __fadd_rn(sum.lo, e));
}

// C = alpha op(A) op(B) + beta C, row-major; a TM x TN tile per CTA of
// TM TN / 16 threads, each a 4 x 4 block.  With part set, slice z of k
// ([z kc, (z + 1) kc)) writes its float64 partial product to part[z][m][n]
// instead.  With lower set only the tiles that reach the diagonal or below it
// are computed (a symmetric result read from its lower triangle).
template <int TM, int TN>
__global__ void __launch_bounds__(TM * TN / 16, 3) k_gemm_ff(bool ta, bool tb, bool lower, int64_t m, int64_t n,
                                                          int64_t k, int64_t kc, double alpha,
                                                          const double* __restrict__ A, int64_t lda,
                                                          const double* __restrict__ B, int64_t ldb, double beta,
                                                          double* __restrict__ Cm, int64_t ldc,
                                                          double* __restrict__ part) {
  constexpr int NT = TM * TN / 16, CX = TN / 4;
  const int64_t i0 = (int64_t)blockIdx.y * TM, j0 = (int64_t)blockIdx.x * TN;
  if (lower && j0 > i0 + TM - 1) return;
  // two stages: the global loads of chunk c + 1 are in flight while chunk c
  // is multiplied, then split into the other stage (one barrier per chunk)
  __shared__ __align__(16) float Ah[2][FK][TM + 4], Al[2][FK][TM + 4], Bh[2][FK][TN + 4], Bl[2][FK][TN + 4];
  const int tid = threadIdx.x, ty = tid / CX, tx = tid % CX;
  const int64_t kb = (int64_t)blockIdx.z * kc, ke = kb + kc < k ? kb + kc : k;
  constexpr int LA = TM * FK / NT, LB = TN * FK / NT;
  double ra[LA], rb[LB];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = tid + NT * q;
      const int r = ta ? e % TM : e / FK, kk = ta ? e / TM : e % FK;
      const int64_t gi = i0 + r, gk = k0 + kk;
      ra[q] = (gi < m && gk < ke) ? (ta ? A[gk * lda + gi] : A[gi * lda + gk]) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = tid + NT * q;
      const int cc = tb ? e / FK : e % TN, kk = tb ? e % FK : e / TN;
      const int64_t gj = j0 + cc, gk = k0 + kk;
      rb[q] = (gj < n && gk < ke) ? (tb ? B[gj * ldb + gk] : B[gk * ldb + gj]) : 0.0;
    }
  };
  auto store = [&](int st) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = tid + NT * q;
      const int r = ta ? e % TM : e / FK, kk = ta ? e / TM : e % FK;
      const FF f = ff_split(ra[q]);
      Ah[st][kk][r] = f.hi;
      Al[st][kk][r] = f.lo;
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = tid + NT * q;
      const int cc = tb ? e / FK : e % TN, kk = tb ? e % FK : e / TN;
      const FF f = ff_split(rb[q]);
      Bh[st][kk][cc] = f.hi;
      Bl[st][kk][cc] = f.lo;
    }
  };
  float sa[4][4], ta4[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) sa[u][v] = ta4[u][v] = 0.f;
  int st = 0;
  if (kb < ke) {
    load(kb);
    store(0);
  }
  __syncthreads();
  for (int64_t k0 = kb; k0 < ke; k0 += FK, st ^= 1) {
    const bool more = k0 + FK < ke;
    if (more) load(k0 + FK);
#pragma unroll 4
    for (int kk = 0; kk < FK; ++kk) {
      const float4 ah = *reinterpret_cast<const float4*>(&Ah[st][kk][ty * 4]);
      const float4 al = *reinterpret_cast<const float4*>(&Al[st][kk][ty * 4]);
      const float4 bh = *reinterpret_cast<const float4*>(&Bh[st][kk][tx * 4]);
      const float4 bl = *reinterpret_cast<const float4*>(&Bl[st][kk][tx * 4]);
      const FF av[4] = {{ah.x, al.x}, {ah.y, al.y}, {ah.z, al.z}, {ah.w, al.w}};
      const FF bv[4] = {{bh.x, bl.x}, {bh.y, bl.y}, {bh.z, bl.z}, {bh.w, bl.w}};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) ff_acc(sa[u][v], ta4[u][v], av[u], bv[v]);
    }
    if (more) store(st ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t i = i0 + ty * 4 + u;
    if (i >= m) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t j = j0 + tx * 4 + v;
      if (j >= n) continue;
      const double r = (double)sa[u][v] + (double)ta4[u][v];
      if (part) {
        part[((int64_t)blockIdx.z * m + i) * n + j] = r;
      } else {
        const double prev = beta != 0.0 ? Cm[i * ldc + j] : 0.0;
        Cm[i * ldc + j] = alpha * r + beta * prev;
      }
    }
  }
}

__global__ void k_gemm_ff_reduce(int64_t m, int64_t n, int nsplit, const double* __restrict__ part, double alpha,
                                 double beta, double* __restrict__ Cm, int64_t ldc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * n) return;
  double acc = 0.0;
  for (int q = 0; q < nsplit; ++q) acc += part[(int64_t)q * m * n + e];
  const int64_t i = e / n, j = e % n;
  const double prev = beta != 0.0 ? Cm[i * ldc + j] : 0.0;
  Cm[i * ldc + j] = alpha * acc + beta * prev;
}

// the float-float copy of X (n x m)
__global__ void k_split_ff(const double* __restrict__ X, int64_t cnt, float* __restrict__ hi, float* __restrict__ lo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) {
    const FF f = ff_split(X[i]);
    hi[i] = f.hi;
    lo[i] = f.lo;
  }
}

// R = B - H X for right-hand sides [c0, c0 + 32 U) of m: one warp per row of
// the compressed H, lanes over the right-hand sides; the row's values are
// split once per warp and broadcast
template <int U>
__global__ void __launch_bounds__(256) k_csr_resm_ff(int64_t n, int64_t m, int64_t c0, const int32_t* __restrict__ rp,
                                                     const int32_t* __restrict__ col, const double* __restrict__ val,
                                                     const float* __restrict__ Xh, const float* __restrict__ Xl,
                                                     const double* __restrict__ B, double* __restrict__ R) {
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  FF acc[U];
#pragma unroll
  for (int u = 0; u < U; ++u) acc[u] = {0.f, 0.f};
  const int p0 = rp[row], p1 = rp[row + 1];
  for (int pb = p0; pb < p1; pb += 32) {
    const int p = pb + lane;
    FF hv = {0.f, 0.f};
    int jv = 0;
    if (p < p1) {
      hv = ff_split(val[p]);
      jv = col[p];
    }
    const int cnt = p1 - pb < 32 ? p1 - pb : 32;
    for (int q = 0; q < cnt; ++q) {
      const FF h = {__shfl_sync(0xffffffffu, hv.hi, q), __shfl_sync(0xffffffffu, hv.lo, q)};
      const int64_t j = __shfl_sync(0xffffffffu, jv, q);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t cidx = c0 + lane + 32 * u;
        if (cidx < m) acc[u] = ff_mac(acc[u], h, {Xh[j * m + cidx], Xl[j * m + cidx]});
      }
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t cidx = c0 + lane + 32 * u;
    if (cidx < m) R[row * m + cidx] = B[row * m + cidx] - ff_to_double(acc[u]);
  }
}

// 1 / p to about 2^-46: the float32 reciprocal and one Newton-Raphson step
// r + r (1 - p r), with the residual 1 - p r formed in float-float
__device__ __forceinline__ FF ff_recip(FF p) {
  const float r = __frcp_rn(p.hi);
  const FF pr = ff_mul(p, {r, 0.f});
  const FF e = ff_add({1.f, 0.f}, {-pr.hi, -pr.lo});
  return ff_add({r, 0.f}, ff_mul({r, 0.f}, e));
}

// Inverse of a small SPD matrix (m <= SPD_SMALL_MAX) in one CTA of 512
// threads by Gauss-Jordan elimination without pivoting (the pivots are the
// diagonals of successive Schur complements, positive for an SPD matrix), in
// float-float arithmetic: each of the m steps is one parallel update of all
// m^2 entries between two barriers.  In place, row-major float64 in and out,
// symmetrised on output.
__global__ void __launch_bounds__(512) k_spd_inverse_small_ff(double* __restrict__ G, int m, int* __restrict__ flag) {
  extern __shared__ float gjf[];  // hi and lo of A (m x (m + 1)), then the pivot column and row (hi, lo)
  const int ld = m + 1;
  float* Ah = gjf;
  float* Al = Ah + m * ld;
  float* ch = Al + m * ld;
  float* cl = ch + m;
  float* rh = cl + m;
  float* rl = rh + m;
  const int tid = threadIdx.x;
  for (int e = tid; e < m * m; e += blockDim.x) {
    const FF v = ff_split(G[e]);
    Ah[(e / m) * ld + e % m] = v.hi;
    Al[(e / m) * ld + e % m] = v.lo;
  }
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    if (tid < m) {
      ch[tid] = Ah[tid * ld + k];
      cl[tid] = Al[tid * ld + k];
      rh[tid] = Ah[k * ld + tid];
      rl[tid] = Al[k * ld + tid];
    }
    __syncthreads();
    FF p = {rh[k], rl[k]};
    if (!(p.hi > 0.f)) {
      if (tid == 0) atomicOr(flag, DEV_NOT_SPD);
      p = {1.f, 0.f};
    }
    const FF rp = ff_recip(p);
    for (int i = tid >> 5; i < m; i += 16) {  // 16 x 32 threads
      const FF fi = ff_mul({-ch[i], -cl[i]}, rp);
      for (int j = tid & 31; j < m; j += 32) {
        const FF pj = {rh[j], rl[j]};
        FF v;
        if (i == k) v = (j == k) ? rp : ff_mul(pj, rp);
        else v = (j == k) ? fi : ff_add(ff_mul(fi, pj), {Ah[i * ld + j], Al[i * ld + j]});
        Ah[i * ld + j] = v.hi;
        Al[i * ld + j] = v.lo;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    G[e] = 0.5 * (ff_to_double({Ah[i * ld + j], Al[i * ld + j]}) + ff_to_double({Ah[j * ld + i], Al[j * ld + i]}));
  }
}

template <int TM, int TN>
rbf_status gemm_ff_tiles(Ctx* c, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                         int64_t lda, const double* B, int64_t ldb, double beta, double* Cm, int64_t ldc,
                         cudaStream_t s, int slot, bool lower) {
  constexpr int NT = TM * TN / 16;
  const int64_t tiles = ((m + TM - 1) / TM) * ((n + TN - 1) / TN);
  // Outputs with fewer tiles than co-resident CTAs split k into slices of at
  // least 64, their number chosen to fill whole waves: a partial last wave
  // costs a whole slice time for a few CTAs.
  static int cap[64] = {0};
  const int dev = c->device & 63;
  if (!cap[dev]) {
    int occ = 0, sms = 0;
    RBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gemm_ff<TM, TN>, NT, 0));
    RBF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    cap[dev] = (occ > 0 ? occ : 1) * (sms > 0 ? sms : 1);
  }
  int64_t nsplit = 1;
  if (!lower && tiles < cap[dev] && k >= 128) {
    // the number of waves (1 to 4) whose slots the slices fill best
    const int64_t most = k / 64;
    double best = 0.0;
    for (int w = 1; w <= 4; ++w) {
      int64_t ns = (int64_t)w * cap[dev] / tiles;
      if (ns > most) ns = most;
      if (ns < 1) ns = 1;
      const double eff = (double)(tiles * ns) / ((double)w * cap[dev]);
      if (eff > best + 0.03) {
        best = eff;
        nsplit = ns;
      }
    }
  }
  int64_t kc = (k + nsplit - 1) / nsplit;
  kc = (kc + FK - 1) / FK * FK;
  nsplit = (k + kc - 1) / kc;
  double* part = nullptr;
  if (nsplit > 1) {
    Buf& pb = c->scratch(slot);
    RBF_TRY(pb.ensure((size_t)nsplit * m * n * sizeof(double)));
    part = pb.as<double>();
  }
  dim3 grid((unsigned)((n + TN - 1) / TN), (unsigned)((m + TM - 1) / TM), (unsigned)nsplit);
  { k_gemm_ff<TM, TN><<<grid, NT, 0, s>>>(ta, tb, lower, m, n, k, kc, alpha, A, lda, B, ldb, beta, Cm, ldc, part); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  if (part) {
    { k_gemm_ff_reduce<<<(unsigned)((m * n + 255) / 256), 256, 0, s>>>(m, n, (int)nsplit, part, alpha, beta, Cm,
                                                                      ldc); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }
  return RBF_OK;
}

}  // namespace

rbf_status gemm_ff(Ctx* c, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                   int64_t lda, const double* B, int64_t ldb, double beta, double* Cm, int64_t ldc, cudaStream_t s,
                   int slot, bool lower) {
  if (m <= 0 || n <= 0) return RBF_OK;
  // the tile follows the output's shape: small, tall, wide or square
  if (!lower && m <= 32 && n <= 32)
    return gemm_ff_tiles<32, 32>(c, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc, s, slot, lower);
  if (!lower && n <= 32)
    return gemm_ff_tiles<128, 32>(c, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc, s, slot, lower);
  if (!lower && m <= 32)
    return gemm_ff_tiles<32, 128>(c, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc, s, slot, lower);
  return gemm_ff_tiles<64, 64>(c, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc, s, slot, lower);
}

rbf_status spd_inverse_small_ff(Ctx* c, double* G, int64_t m, cudaStream_t s) {
  if (m <= 0 || m > SPD_SMALL_MAX)
    return fail(RBF_EINVAL, "spd_inverse_small_ff: m must be in [1, %d]", SPD_SMALL_MAX);
  const size_t smem = (size_t)(2 * m * (m + 1) + 4 * m) * sizeof(float);
  static bool attr[64] = {false};
  if (!attr[c->device & 63]) {
    const size_t mx = (size_t)(2 * SPD_SMALL_MAX * (SPD_SMALL_MAX + 1) + 4 * SPD_SMALL_MAX) * sizeof(float);
    RBF_CUDA(cudaFuncSetAttribute(k_spd_inverse_small_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx));
    attr[c->device & 63] = true;
  }
  { k_spd_inverse_small_ff<<<1, 512, smem, s>>>(G, (int)m, c->dflag.as<int>()); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  return RBF_OK;
}

rbf_status csr_residual_ff(Ctx* c, const SpH& A, const double* X, const double* B, int64_t m, double* R,
                           cudaStream_t s, int slot) {
  const int64_t n = A.n;
  if (n <= 0 || m <= 0) return RBF_OK;
  Buf& xs = c->scratch(slot);
  RBF_TRY(xs.ensure((size_t)2 * n * m * sizeof(float)));
  float* Xh = xs.as<float>();
  float* Xl = Xh + n * m;
  { k_split_ff<<<(unsigned)((n * m + 255) / 256), 256, 0, s>>>(X, n * m, Xh, Xl); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  const int32_t* rp = A.rp.as<int32_t>();
  const int32_t* col = A.col.as<int32_t>();
  const double* val = A.val.as<double>();
  const unsigned g = (unsigned)((n * 32 + 255) / 256);
  for (int64_t c0 = 0; c0 < m; c0 += 128) {
    const int64_t w = m - c0;
    if (w <= 32) { k_csr_resm_ff<1><<<g, 256, 0, s>>>(n, m, c0, rp, col, val, Xh, Xl, B, R); ::rbf::note_launch(); }
    else if (w <= 64) { k_csr_resm_ff<2><<<g, 256, 0, s>>>(n, m, c0, rp, col, val, Xh, Xl, B, R); ::rbf::note_launch(); }
    else if (w <= 96) { k_csr_resm_ff<3><<<g, 256, 0, s>>>(n, m, c0, rp, col, val, Xh, Xl, B, R); ::rbf::note_launch(); }
    else { k_csr_resm_ff<4><<<g, 256, 0, s>>>(n, m, c0, rp, col, val, Xh, Xl, B, R); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }
  return RBF_OK;
}

}  // namespace rbf
