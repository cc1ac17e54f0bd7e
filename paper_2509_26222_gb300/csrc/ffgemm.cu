// Float64 products computed in float-float arithmetic on the float32 pipes.
//
// The block stage of the update (the Schur complement of the leaving centers
// and the float64 residuals of their covariance block) multiplies float64
// matrices of a few thousand rows by blocks of tens to hundreds of columns.
// GB300 executes float64 at a small fraction of its float32 rate, so these
// products take each operand as hi + lo (two float32, about 2^-48 relative),
// multiply-accumulate with error-free transforms (about 14 float32
// operations per product term, accuracy about 2^-46 relative to the sum of
// |terms|) and return float64.
#include "common.cuh"
#include "tiles.cuh"

namespace rbf {
namespace {

constexpr int FT = 64;  // output tile
constexpr int FK = 16;  // k chunk
constexpr int FLD = FT + 4;

// C = alpha op(A) op(B) + beta C, row-major; 256 threads, each a 4 x 4 block.
// With part set, slice z of k ([z kc, (z + 1) kc)) writes its float64 partial
// product to part[z][m][n] instead.  With lower set only the tiles on or below
// the diagonal are computed (a symmetric result read from its lower triangle).
__global__ void __launch_bounds__(256) k_gemm_ff(bool ta, bool tb, bool lower, int64_t m, int64_t n, int64_t k,
                                                 int64_t kc, double alpha, const double* __restrict__ A, int64_t lda,
                                                 const double* __restrict__ B, int64_t ldb, double beta,
                                                 double* __restrict__ Cm, int64_t ldc, double* __restrict__ part) {
  if (lower && blockIdx.x > blockIdx.y) return;
  __shared__ __align__(16) float Ah[FK][FLD], Al[FK][FLD], Bh[FK][FLD], Bl[FK][FLD];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int64_t i0 = (int64_t)blockIdx.y * FT, j0 = (int64_t)blockIdx.x * FT;
  const int64_t kb = (int64_t)blockIdx.z * kc, ke = kb + kc < k ? kb + kc : k;
  FF acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = {0.f, 0.f};
  for (int64_t k0 = kb; k0 < ke; k0 += FK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;  // 0 .. 1023
      // A: row r of the tile, k index kk
      int r, kk;
      if (ta) { r = e & 63; kk = e >> 6; }
      else { kk = e & 15; r = e >> 4; }
      const int64_t gi = i0 + r, gk = k0 + kk;
      double a = 0.0;
      if (gi < m && gk < ke) a = ta ? A[gk * lda + gi] : A[gi * lda + gk];
      const FF af = ff_split(a);
      Ah[kk][r] = af.hi;
      Al[kk][r] = af.lo;
      int cc;
      if (tb) { kk = e & 15; cc = e >> 4; }
      else { cc = e & 63; kk = e >> 6; }
      const int64_t gj = j0 + cc, gk2 = k0 + kk;
      double b = 0.0;
      if (gj < n && gk2 < ke) b = tb ? B[gj * ldb + gk2] : B[gk2 * ldb + gj];
      const FF bf = ff_split(b);
      Bh[kk][cc] = bf.hi;
      Bl[kk][cc] = bf.lo;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < FK; ++kk) {
      const float4 ah = *reinterpret_cast<const float4*>(&Ah[kk][ty * 4]);
      const float4 al = *reinterpret_cast<const float4*>(&Al[kk][ty * 4]);
      const float4 bh = *reinterpret_cast<const float4*>(&Bh[kk][tx * 4]);
      const float4 bl = *reinterpret_cast<const float4*>(&Bl[kk][tx * 4]);
      const FF av[4] = {{ah.x, al.x}, {ah.y, al.y}, {ah.z, al.z}, {ah.w, al.w}};
      const FF bv[4] = {{bh.x, bl.x}, {bh.y, bl.y}, {bh.z, bl.z}, {bh.w, bl.w}};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = ff_mac(acc[u][v], av[u], bv[v]);
    }
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
      if (part) {
        part[((int64_t)blockIdx.z * m + i) * n + j] = ff_to_double(acc[u][v]);
      } else {
        const double prev = beta != 0.0 ? Cm[i * ldc + j] : 0.0;
        Cm[i * ldc + j] = alpha * ff_to_double(acc[u][v]) + beta * prev;
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

}  // namespace

rbf_status gemm_ff(Ctx* c, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                   int64_t lda, const double* B, int64_t ldb, double beta, double* Cm, int64_t ldc, cudaStream_t s,
                   int slot, bool lower) {
  if (m <= 0 || n <= 0) return RBF_OK;
  const int64_t tiles = ((m + FT - 1) / FT) * ((n + FT - 1) / FT);
  // outputs that do not fill the GPU twice split k into slices of >= 128
  int64_t nsplit = 1;
  if (!lower && tiles < 2 * 152 && k > 256) {
    nsplit = (2 * 152 + tiles - 1) / tiles;
    const int64_t most = k / 128;
    if (nsplit > most) nsplit = most;
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
  dim3 grid((unsigned)((n + FT - 1) / FT), (unsigned)((m + FT - 1) / FT), (unsigned)nsplit);
  { k_gemm_ff<<<grid, 256, 0, s>>>(ta, tb, lower, m, n, k, kc, alpha, A, lda, B, ldb, beta, Cm, ldc, part); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  if (part) {
    if (lower) return fail(RBF_EINVAL, "gemm_ff: lower with split k");
    { k_gemm_ff_reduce<<<(unsigned)((m * n + 255) / 256), 256, 0, s>>>(m, n, (int)nsplit, part, alpha, beta, Cm,
                                                                      ldc); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }
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
