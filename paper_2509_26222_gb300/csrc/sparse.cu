// Compressed-row copy of the float64 information matrix for the residuals of
// the refined solves.
//
// The information matrix of the active block is the prior block of the
// centers that stayed (with the fill of Schur complements of the centers
// that left), lambda on the diagonal for fresh centers, and m~ m~^T, which
// only couples centers within two support radii.  On the staircase sequence
// 5-22 % of its entries are nonzero, so the float64 residuals r = b - H x of
// iterative refinement, bound by the GPU's float64 rate, run on the nonzero
// entries only.  The copy holds every exactly nonzero entry in ascending
// column order, so the products equal the dense ones up to the order of
// their sums.
#include <cuda_runtime.h>

#include "common.cuh"

namespace rbf {
namespace {

// nonzeros per row (one warp per row)
// nonzeros per row (one warp per row) and the half-bandwidth max |i - j|
// over the nonzero entries (atomicMax into *bw)
__global__ void __launch_bounds__(256) k_csr_count(const double* __restrict__ H, int64_t n, int64_t ld,
                                                   int32_t* __restrict__ cnt, int* __restrict__ bw) {
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  const double* hr = H + row * ld;
  int c = 0;
  int64_t far = 0;
  for (int64_t j0 = 0; j0 < n; j0 += 32) {
    int64_t j = j0 + lane;
    bool nz = j < n && hr[j] != 0.0;
    c += __popc(__ballot_sync(0xffffffffu, nz));
    if (nz) {
      int64_t dj = j > row ? j - row : row - j;
      far = dj > far ? dj : far;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    int64_t v = __shfl_xor_sync(0xffffffffu, far, o);
    far = v > far ? v : far;
  }
  if (lane == 0) {
    cnt[row] = c;
    atomicMax(bw, (int)far);
  }
}

// column indices and values in ascending column order (one warp per row)
__global__ void __launch_bounds__(256) k_csr_fill(const double* __restrict__ H, int64_t n, int64_t ld,
                                                  const int32_t* __restrict__ rp, int32_t* __restrict__ col,
                                                  double* __restrict__ val) {
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  const double* hr = H + row * ld;
  int base = rp[row];
  const unsigned below = (1u << lane) - 1u;
  for (int64_t j0 = 0; j0 < n; j0 += 32) {
    int64_t j = j0 + lane;
    double v = j < n ? hr[j] : 0.0;
    bool nz = v != 0.0;
    unsigned m = __ballot_sync(0xffffffffu, nz);
    if (nz) {
      int pos = base + __popc(m & below);
      col[pos] = (int32_t)j;
      val[pos] = v;
    }
    base += __popc(m);
  }
}

// r = b - H x (one right-hand side; one warp per row)
__global__ void __launch_bounds__(256) k_csr_res1(int64_t n, const int32_t* __restrict__ rp,
                                                  const int32_t* __restrict__ col, const double* __restrict__ val,
                                                  const double* __restrict__ x, const double* __restrict__ b,
                                                  double* __restrict__ r) {
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  double acc = 0.0;
  for (int p = rp[row] + lane; p < rp[row + 1]; p += 32) acc = fma(val[p], x[col[p]], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) r[row] = b[row] - acc;
}

// R = B - H X for the right-hand sides [c0, c0 + 32 U) of m (row-major
// n x m): one warp per row, lanes over the right-hand sides, the row's
// nonzeros in order, four in flight.
template <int U>
__global__ void __launch_bounds__(256) k_csr_resm(int64_t n, int64_t m, int64_t c0, const int32_t* __restrict__ rp,
                                                  const int32_t* __restrict__ col, const double* __restrict__ val,
                                                  const double* __restrict__ X, const double* __restrict__ B,
                                                  double* __restrict__ R) {
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  double acc[U];
#pragma unroll
  for (int u = 0; u < U; ++u) acc[u] = 0.0;
  const int p0 = rp[row], p1 = rp[row + 1];
  int p = p0;
  for (; p + 4 <= p1; p += 4) {
    int j[4];
    double h[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      j[q] = col[p + q];
      h[q] = val[p + q];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int u = 0; u < U; ++u) {
        int64_t cidx = c0 + lane + 32 * u;
        if (cidx < m) acc[u] = fma(h[q], X[(int64_t)j[q] * m + cidx], acc[u]);
      }
  }
  for (; p < p1; ++p) {
    int j = col[p];
    double h = val[p];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int64_t cidx = c0 + lane + 32 * u;
      if (cidx < m) acc[u] = fma(h, X[(int64_t)j * m + cidx], acc[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    int64_t cidx = c0 + lane + 32 * u;
    if (cidx < m) R[row * m + cidx] = B[row * m + cidx] - acc[u];
  }
}

unsigned warps_grid(int64_t n) { return (unsigned)((n * 32 + 255) / 256); }

}  // namespace

// The half-bandwidth is left in scratch slot 70 at index n (read by csr_bandwidth).
rbf_status build_csr(Ctx* c, const double* H, int64_t ld, int64_t n, SpH& out, cudaStream_t s) {
  out.valid = false;
  out.n = n;
  if (n <= 0 || n > SPH_MAX) return RBF_OK;
  RBF_TRY(out.rp.ensure((size_t)(n + 1) * sizeof(int32_t)));
  RBF_TRY(out.col.ensure((size_t)n * n * sizeof(int32_t)));
  RBF_TRY(out.val.ensure((size_t)n * n * sizeof(double)));
  Buf& cnt = c->scratch(70);
  RBF_TRY(cnt.ensure((size_t)(n + 1) * sizeof(int32_t)));
  RBF_CUDA(cudaMemsetAsync(cnt.as<int32_t>() + n, 0, sizeof(int32_t), s));
  { k_csr_count<<<warps_grid(n), 256, 0, s>>>(H, n, ld, cnt.as<int32_t>(), cnt.as<int32_t>() + n); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  RBF_TRY(scan_i32(c, cnt.as<int32_t>(), out.rp.as<int32_t>(), n, s, 71));
  { k_csr_fill<<<warps_grid(n), 256, 0, s>>>(H, n, ld, out.rp.as<int32_t>(), out.col.as<int32_t>(),
                                             out.val.as<double>()); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  out.valid = true;
  return RBF_OK;
}

// Half-bandwidth of the matrix of the last build_csr (one host read).
rbf_status csr_bandwidth(Ctx* c, int64_t n, int64_t* bw, cudaStream_t s) {
  int32_t* h32 = (int32_t*)c->host_small;
  RBF_CUDA(cudaMemcpyAsync(h32 + 6, c->scratch(70).as<int32_t>() + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  RBF_CUDA(cudaStreamSynchronize(s));
  *bw = h32[6];
  return RBF_OK;
}

// Half-bandwidth of a dense symmetric matrix (no compressed copy kept).
rbf_status dense_bandwidth(Ctx* c, const double* H, int64_t ld, int64_t n, int64_t* bw, cudaStream_t s) {
  Buf& cnt = c->scratch(70);
  RBF_TRY(cnt.ensure((size_t)(n + 1) * sizeof(int32_t)));
  RBF_CUDA(cudaMemsetAsync(cnt.as<int32_t>() + n, 0, sizeof(int32_t), s));
  { k_csr_count<<<warps_grid(n), 256, 0, s>>>(H, n, ld, cnt.as<int32_t>(), cnt.as<int32_t>() + n); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  return csr_bandwidth(c, n, bw, s);
}

rbf_status csr_residual(const SpH& A, const double* X, const double* B, int64_t m, double* R, cudaStream_t s) {
  const int64_t n = A.n;
  if (n <= 0 || m <= 0) return RBF_OK;
  const int32_t* rp = A.rp.as<int32_t>();
  const int32_t* col = A.col.as<int32_t>();
  const double* val = A.val.as<double>();
  unsigned g = warps_grid(n);
  if (m == 1) {
    { k_csr_res1<<<g, 256, 0, s>>>(n, rp, col, val, X, B, R); ::rbf::note_launch(); }
  } else {
    for (int64_t c0 = 0; c0 < m; c0 += 128) {
      int64_t w = m - c0;
      if (w <= 32) {
        { k_csr_resm<1><<<g, 256, 0, s>>>(n, m, c0, rp, col, val, X, B, R); ::rbf::note_launch(); }
      } else if (w <= 64) {
        { k_csr_resm<2><<<g, 256, 0, s>>>(n, m, c0, rp, col, val, X, B, R); ::rbf::note_launch(); }
      } else if (w <= 96) {
        { k_csr_resm<3><<<g, 256, 0, s>>>(n, m, c0, rp, col, val, X, B, R); ::rbf::note_launch(); }
      } else {
        { k_csr_resm<4><<<g, 256, 0, s>>>(n, m, c0, rp, col, val, X, B, R); ::rbf::note_launch(); }
      }
    }
  }
  RBF_CUDA(cudaGetLastError());
  return RBF_OK;
}

}  // namespace rbf
