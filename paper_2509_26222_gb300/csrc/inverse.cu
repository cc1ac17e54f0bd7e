// Explicit inverse of the float32 Cholesky factor and solves by products.
//
// The refined solves of the mixed-precision update apply the float32 factor
// many times per frame (the weight increment, and the covariance columns of
// the centers that leave the active block).  A blocked substitution is a
// chain of a/64 dependent steps per application.  For active blocks of a few
// thousand centers it is cheaper to form Z = L^{-1} once per factorization,
// in log2(a/64) levels of independent products, and to apply
// H^{-1} ~ Z^T Z as two products that run on every SM at once:
//
//   level b (b = 128, 256, ...): for every diagonal pair of b/2-blocks
//     [L11 0; L21 L22]^{-1} = [Z11 0; -Z22 L21 Z11  Z22]
//   (T = L21 Z11, then Z21 = -Z22 T; Z11, Z22 come from the level below and
//   the 64 x 64 blocks from the factorization itself).
//
// Z has the factor's shape (row-major, leading dimension ldz) with zeros
// above the diagonal; its transpose follows it in the same buffer (rows
// n .. 2n - 1).  The solves are Y = Z F followed by F = Z^T Y.
#include <cuda_runtime.h>

#include "common.cuh"

namespace rbf {
namespace {

constexpr int TG = 64;       // output tile (rows and columns)
constexpr int TK = 32;       // K chunk staged in shared memory
constexpr int TLD = TG + 4;  // padded row of the staged chunks
constexpr int GEMV_M = 8;    // right-hand sides handled by the matrix-vector kernels

// Element (r, c) of a row-major matrix, or of the transpose of one.
struct Mat {
  const float* p;
  int64_t ld;
  bool t;
};

// acc += A[i0 + 0..63, kb..ke) * B[kb..ke, j0 + 0..63) for rows < M and
// columns < N; 256 threads, each a 4 x 4 block of the tile.  The next chunk
// is fetched into registers while the current one is multiplied.
__device__ __forceinline__ void tile_mma(float (&acc)[4][4], const Mat A, const Mat B, int64_t i0, int64_t j0,
                                         int64_t M, int64_t N, int64_t kb, int64_t ke, float (*As)[TLD],
                                         float (*Bs)[TLD]) {
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  float ra[8], rb[8];
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      int idx = tid + 256 * e;  // 0 .. 2047
      int r, kk;
      if (A.t) { r = idx & (TG - 1); kk = idx >> 6; }
      else { kk = idx & (TK - 1); r = idx >> 5; }
      int64_t gi = i0 + r, gk = k0 + kk;
      ra[e] = (gi < M && gk < ke) ? (A.t ? A.p[gk * A.ld + gi] : A.p[gi * A.ld + gk]) : 0.f;
      int cc;
      if (B.t) { kk = idx & (TK - 1); cc = idx >> 5; }
      else { cc = idx & (TG - 1); kk = idx >> 6; }
      int64_t gj = j0 + cc;
      gk = k0 + kk;
      rb[e] = (gj < N && gk < ke) ? (B.t ? B.p[gj * B.ld + gk] : B.p[gk * B.ld + gj]) : 0.f;
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      int idx = tid + 256 * e;
      int r, kk;
      if (A.t) { r = idx & (TG - 1); kk = idx >> 6; }
      else { kk = idx & (TK - 1); r = idx >> 5; }
      As[kk][r] = ra[e];
      int cc;
      if (B.t) { kk = idx & (TK - 1); cc = idx >> 5; }
      else { cc = idx & (TG - 1); kk = idx >> 6; }
      Bs[kk][cc] = rb[e];
    }
  };
  if (kb >= ke) return;
  fetch(kb);
  for (int64_t k0 = kb; k0 < ke; k0 += TK) {
    stash();
    __syncthreads();
    if (k0 + TK < ke) fetch(k0 + TK);
#pragma unroll 8
    for (int kk = 0; kk < TK; ++kk) {
      float4 a4 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      float4 b4 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      float av[4] = {a4.x, a4.y, a4.z, a4.w};
      float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
    }
    __syncthreads();
  }
}

// C = alpha acc, or C += alpha acc with atomics (the two halves of a K range
// split in two: 0 + a + b equals 0 + b + a exactly, so the result does not
// depend on which half lands first)
__device__ __forceinline__ void tile_store(const float (&acc)[4][4], float alpha, float* C, int64_t ldc, int64_t i0,
                                           int64_t j0, int64_t M, int64_t N, bool add = false) {
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int64_t i = i0 + ty * 4 + u;
    if (i >= M) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int64_t j = j0 + tx * 4 + v;
      if (j < N) {
        if (add) atomicAdd(C + i * ldc + j, alpha * acc[u][v]);
        else C[i * ldc + j] = alpha * acc[u][v];
      }
    }
  }
}

// Copy the 64 x 64 diagonal inverses into Z (whose other entries are zero).
__global__ void k_inv_diag(const float* __restrict__ Zd, int64_t n, float* __restrict__ Z, int64_t ldz) {
  int64_t q = blockIdx.x;
  int64_t k = q * 64;
  int kb = (int)((n - k) < 64 ? (n - k) : 64);
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    int i = e >> 6, t = e & 63;
    if (i < kb && t <= i) Z[(k + i) * ldz + k + t] = Zd[q * 64 * 64 + e];
  }
}

// One level of the doubling: pair p covers rows [p b, p b + b); its upper
// half has h1 = b/2 rows, its lower half h2 = min(b/2, n - p b - b/2).
// kind 0: T21 = L21 Z11 (Z11 lower: only k >= j contributes);
// kind 1: Z21 = -Z22 T21 (Z22 lower: only k <= i contributes).
// split = 2: blockIdx.z = 2 p + half, each half of the K range adds its
// partial product into the (zeroed) output.
__global__ void __launch_bounds__(256) k_trtri_level(int kind, int64_t b, int64_t n, const float* __restrict__ W,
                                                     int64_t ldw, float* __restrict__ Z, int64_t ldz,
                                                     float* __restrict__ T, int split) {
  __shared__ __align__(16) float As[TK][TLD];
  __shared__ __align__(16) float Bs[TK][TLD];
  const int64_t p = split == 2 ? (blockIdx.z >> 1) : blockIdx.z;
  const int half = split == 2 ? (int)(blockIdx.z & 1) : -1;
  const int64_t r1 = p * b, h1 = b / 2, r2 = r1 + h1;
  const int64_t h2 = (n - r2) < h1 ? (n - r2) : h1;
  if (h2 <= 0) return;
  const int64_t i0 = (int64_t)blockIdx.y * TG, j0 = (int64_t)blockIdx.x * TG;
  if (i0 >= h2 || j0 >= h1) return;
  float acc[4][4] = {};
  int64_t kb, ke;
  if (kind == 0) {
    kb = j0;
    ke = h1;
  } else {
    kb = 0;
    ke = (i0 + TG) < h2 ? (i0 + TG) : h2;
  }
  if (half >= 0) {
    int64_t mid = kb + ((ke - kb) / 2 + TK - 1) / TK * TK;
    if (mid > ke) mid = ke;
    if (half == 0) ke = mid;
    else kb = mid;
  }
  if (kind == 0) {
    Mat A{W + r2 * ldw + r1, ldw, false};
    Mat B{Z + r1 * ldz + r1, ldz, false};
    tile_mma(acc, A, B, i0, j0, h2, h1, kb, ke, As, Bs);
    tile_store(acc, 1.f, T + r2 * ldz + r1, ldz, i0, j0, h2, h1, half >= 0);
  } else {
    Mat A{Z + r2 * ldz + r2, ldz, false};
    Mat B{T + r2 * ldz + r1, ldz, false};
    tile_mma(acc, A, B, i0, j0, h2, h1, kb, ke, As, Bs);
    tile_store(acc, -1.f, Z + r2 * ldz + r1, ldz, i0, j0, h2, h1, half >= 0);
  }
}

// Y = Z F (forward, Z lower) or Y = Zt F (backward, Zt = Z^T upper) for
// m > GEMV_M right-hand sides; F, Y row-major n x m.  blockIdx.z splits K; partial
// products go to P[z] and are summed by k_sum_partials.
__global__ void __launch_bounds__(256) k_inv_apply(bool backward, int64_t n, int64_t m, const float* __restrict__ Z,
                                                   int64_t ldz, const float* __restrict__ F, float* __restrict__ P,
                                                   int nsplit) {
  __shared__ __align__(16) float As[TK][TLD];
  __shared__ __align__(16) float Bs[TK][TLD];
  const int64_t i0 = (int64_t)blockIdx.y * TG, j0 = (int64_t)blockIdx.x * TG;
  int64_t kb = backward ? i0 : 0;
  int64_t ke = backward ? n : ((i0 + TG) < n ? (i0 + TG) : n);
  int64_t len = ke - kb;
  int64_t chunk = ((len + nsplit - 1) / nsplit + TK - 1) / TK * TK;
  int64_t sb = kb + (int64_t)blockIdx.z * chunk;
  int64_t se = (sb + chunk) < ke ? (sb + chunk) : ke;
  float acc[4][4] = {};
  Mat A{Z, ldz, false};  // Z (forward) or its transpose stored row-major (backward)
  Mat B{F, m, false};
  if (sb < se) tile_mma(acc, A, B, i0, j0, n, m, sb, se, As, Bs);
  tile_store(acc, 1.f, P + (int64_t)blockIdx.z * n * m, m, i0, j0, n, m);
}

__global__ void k_sum_partials(const float* __restrict__ P, int nsplit, int64_t tot, float* __restrict__ Y) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= tot) return;
  float s = 0.f;
  for (int z = 0; z < nsplit; ++z) s += P[z * tot + e];
  Y[e] = s;
}

// Y = A F for m <= GEMV_M with A = Z (lower: row i over k <= i) or A = Z^T
// stored transposed (upper: row i over k >= i): one warp per row, lanes over
// the row, eight loads of A in flight per lane.  With Xd set, the result is
// added to the float64 Xd instead of stored to Y.
template <bool UPPER>
__global__ void __launch_bounds__(256) k_inv_gemv(int64_t n, int m, const float* __restrict__ A, int64_t lda,
                                                  const float* __restrict__ F, float* __restrict__ Y,
                                                  double* __restrict__ Xd = nullptr) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= n) return;
  const int64_t lo = UPPER ? i : 0, hi = UPPER ? n : i + 1;
  float acc[GEMV_M];
#pragma unroll
  for (int j = 0; j < GEMV_M; ++j) acc[j] = 0.f;
  const float* ar = A + i * lda;
  for (int64_t k0 = lo + lane; k0 < hi; k0 += 256) {
    float z[8], f[8][GEMV_M];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      int64_t k = k0 + 32 * u;
      bool ok = k < hi;
      z[u] = ok ? ar[k] : 0.f;
#pragma unroll
      for (int j = 0; j < GEMV_M; ++j) f[u][j] = (ok && j < m) ? F[k * m + j] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int j = 0; j < GEMV_M; ++j) acc[j] = fmaf(z[u], f[u][j], acc[j]);
  }
#pragma unroll
  for (int j = 0; j < GEMV_M; ++j) {
    if (j >= m) break;
    float v = acc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) {
      if (Xd) Xd[i * m + j] += (double)v;
      else Y[i * m + j] = v;
    }
  }
}

// Zt = Z^T (n x n, both with leading dimension ld), 32 x 32 tiles
__global__ void k_transpose32(const float* __restrict__ Z, int64_t n, int64_t ld, float* __restrict__ Zt) {
  __shared__ float t[32][33];
  const int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int r = ty; r < 32; r += 8) {
    int64_t i = by + r, j = bx + tx;
    t[r][tx] = (i < n && j < n) ? Z[i * ld + j] : 0.f;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    int64_t i = bx + r, j = by + tx;
    if (i < n && j < n) Zt[i * ld + j] = t[tx][r];
  }
}

// Y[i][u] = Z[i][pos[u]]: the product of Z with unit columns
__global__ void k_gather_cols(const float* __restrict__ Z, int64_t n, int64_t ld, const int32_t* __restrict__ pos,
                              int64_t m, float* __restrict__ Y) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * m) return;
  int64_t i = e / m, u = e % m;
  Y[e] = Z[i * ld + pos[u]];
}

unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

}  // namespace

// K slices of the inverse apply: as many as fill the co-resident CTAs of
// the GPU once (the tiles alone leave most SMs idle for a few right-hand
// sides), at least 4 chunks of K each and at most 8.
static int apply_split(Ctx* c, int64_t tiles, int64_t n) {
  static int cap[64] = {0};
  const int dev = c->device & 63;
  if (!cap[dev]) {
    int occ = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_inv_apply, 256, 0) != cudaSuccess || occ < 1) occ = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms < 1) sms = 1;
    cap[dev] = occ * sms;
  }
  int64_t ns = cap[dev] / (tiles > 0 ? tiles : 1);
  const int64_t most = n / (4 * TK);
  if (ns > most) ns = most;
  if (ns > 8) ns = 8;
  return ns < 1 ? 1 : (int)ns;
}

rbf_status trtri_mixed(Ctx* c, const float* W, int64_t ldw, int64_t n, const float* Zd, float* Z, int64_t ldz,
                       cudaStream_t s) {
  if (n <= 0) return RBF_OK;
  Buf& tb = c->scratch(65);
  RBF_TRY(tb.ensure((size_t)n * ldz * sizeof(float)));
  float* T = tb.as<float>();
  StageTimer st(c, RBF_STAGE_INVERSE, s, (double)n * n * n / 3.0);
  RBF_CUDA(cudaMemsetAsync(Z, 0, (size_t)n * ldz * sizeof(float), s));
  RBF_CUDA(cudaMemsetAsync(T, 0, (size_t)n * ldz * sizeof(float), s));  // levels write disjoint blocks
  { k_inv_diag<<<cdiv(n, 64), 256, 0, s>>>(Zd, n, Z, ldz); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  for (int64_t b = 128; b / 2 < n; b *= 2) {
    int64_t h = b / 2;
    // levels whose tiles do not fill the GPU twice split K in two halves
    const int64_t tiles = (int64_t)cdiv(h, TG) * cdiv(h, TG) * cdiv(n, b);
    const int split = (tiles < 2 * 152 && h >= 256) ? 2 : 1;
    dim3 grid(cdiv(h, TG), cdiv(h, TG), (unsigned)(cdiv(n, b) * split));
    for (int kind = 0; kind < 2; ++kind) {
      { k_trtri_level<<<grid, 256, 0, s>>>(kind, b, n, W, ldw, Z, ldz, T, split); ::rbf::note_launch(); }
      RBF_CUDA(cudaGetLastError());
    }
  }
  // Z^T stored row-major, so that products with Z^T read rows too
  { k_transpose32<<<dim3(cdiv(n, 32), cdiv(n, 32)), 256, 0, s>>>(Z, n, ldz, Z + n * ldz); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  return RBF_OK;
}

rbf_status inv_solve(Ctx* c, const float* Z, int64_t ldz, int64_t n, float* F, int64_t m, cudaStream_t s) {
  if (n <= 0 || m <= 0) return RBF_OK;
  Buf& yb = c->scratch(66);
  RBF_TRY(yb.ensure((size_t)n * m * sizeof(float)));
  float* Y = yb.as<float>();
  StageTimer st(c, RBF_STAGE_INVAPPLY, s, 2.0 * (double)n * n * m);
  const float* Zt = Z + n * ldz;
  if (m <= GEMV_M) {
    { k_inv_gemv<false><<<cdiv(n * 32, 256), 256, 0, s>>>(n, (int)m, Z, ldz, F, Y); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    { k_inv_gemv<true><<<cdiv(n * 32, 256), 256, 0, s>>>(n, (int)m, Zt, ldz, Y, F); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    return RBF_OK;
  }
  int64_t tiles = (int64_t)cdiv(n, TG) * cdiv(m, TG);
  int nsplit = apply_split(c, tiles, n);
  Buf& pb = c->scratch(67);
  RBF_TRY(pb.ensure((size_t)nsplit * n * m * sizeof(float)));
  float* P = pb.as<float>();
  dim3 grid(cdiv(m, TG), cdiv(n, TG), nsplit);
  unsigned nr = cdiv(n * m, 256);
  { k_inv_apply<<<grid, 256, 0, s>>>(false, n, m, Z, ldz, F, P, nsplit); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  { k_sum_partials<<<nr, 256, 0, s>>>(P, nsplit, n * m, Y); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  { k_inv_apply<<<grid, 256, 0, s>>>(true, n, m, Zt, ldz, Y, P, nsplit); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  { k_sum_partials<<<nr, 256, 0, s>>>(P, nsplit, n * m, F); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  return RBF_OK;
}

// X += Z^T (Z R) for m <= GEMV_M right-hand sides, R and X float64: R is
// rounded to float32 once (a float64 operand inside the matrix-vector loop
// would convert it once per row, on GB300's narrow float64 pipe), and the
// float64 accumulation happens in the second matrix-vector launch.
__global__ void k_round_f32(const double* __restrict__ R, int64_t cnt, float* __restrict__ F) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) F[i] = (float)R[i];
}

rbf_status inv_solve_acc(Ctx* c, const float* Z, int64_t ldz, int64_t n, const double* R, double* X, int64_t m,
                         cudaStream_t s) {
  if (n <= 0 || m <= 0) return RBF_OK;
  if (m > GEMV_M) return fail(RBF_EINVAL, "inv_solve_acc: at most %d right-hand sides", GEMV_M);
  Buf& yb = c->scratch(66);
  RBF_TRY(yb.ensure((size_t)2 * n * m * sizeof(float)));
  float* Y = yb.as<float>();
  float* F = Y + n * m;
  StageTimer st(c, RBF_STAGE_INVAPPLY, s, 2.0 * (double)n * n * m);
  const float* Zt = Z + n * ldz;
  { k_round_f32<<<cdiv(n * m, 256), 256, 0, s>>>(R, n * m, F); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  { k_inv_gemv<false><<<cdiv(n * 32, 256), 256, 0, s>>>(n, (int)m, Z, ldz, F, Y); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  { k_inv_gemv<true><<<cdiv(n * 32, 256), 256, 0, s>>>(n, (int)m, Zt, ldz, Y, nullptr, X); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  return RBF_OK;
}

// F = Z^T (Z E_P) for unit columns E_P at positions pos (n x m, row-major):
// the first product is a gather of columns of Z.
rbf_status inv_solve_unit(Ctx* c, const float* Z, int64_t ldz, int64_t n, const int32_t* pos, int64_t m, float* F,
                          cudaStream_t s) {
  if (n <= 0 || m <= 0) return RBF_OK;
  Buf& yb = c->scratch(66);
  RBF_TRY(yb.ensure((size_t)n * m * sizeof(float)));
  float* Y = yb.as<float>();
  StageTimer st(c, RBF_STAGE_INVAPPLY, s, (double)n * n * m);
  const float* Zt = Z + n * ldz;
  { k_gather_cols<<<cdiv(n * m, 256), 256, 0, s>>>(Z, n, ldz, pos, m, Y); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  if (m <= GEMV_M) {
    { k_inv_gemv<true><<<cdiv(n * 32, 256), 256, 0, s>>>(n, (int)m, Zt, ldz, Y, F); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    return RBF_OK;
  }
  int64_t tiles = (int64_t)cdiv(n, TG) * cdiv(m, TG);
  int nsplit = apply_split(c, tiles, n);
  Buf& pb = c->scratch(67);
  RBF_TRY(pb.ensure((size_t)nsplit * n * m * sizeof(float)));
  float* P = pb.as<float>();
  dim3 grid(cdiv(m, TG), cdiv(n, TG), nsplit);
  { k_inv_apply<<<grid, 256, 0, s>>>(true, n, m, Zt, ldz, Y, P, nsplit); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  { k_sum_partials<<<cdiv(n * m, 256), 256, 0, s>>>(P, nsplit, n * m, F); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  return RBF_OK;
}

}  // namespace rbf
