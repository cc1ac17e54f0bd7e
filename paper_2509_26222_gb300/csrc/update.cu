// Recursive ridge update of the weights on the active rows (Sec. III-C).
//
// Per frame (n points, world frame):
//  1. neighbour lists: for every point the centers j with d2 < r^2 (float32
//     rule, ids ascending) -- the nonzero pattern of m~ in Eq. mfk_m_approx;
//  2. active rows A = sorted union of the lists, local index map;
//  3. m~ entries in float64 (Wendland phi, or the Gaussian moment row of
//     Sec. III-B) and the innovation e = z - m~^T w_A (Eq. kf_w_update);
//  4. the information matrix of the new block,
//        H' = (P[A, A])^{-1} + m~ m~^T           (Eq. H_update on the block),
//     where (P[A, A])^{-1} is assembled from the previous block's information
//     matrix (a Schur complement drops the centers that leave) and the stored
//     covariance of the centers that enter;
//  5. H' = L L^T, w_A += H'^{-1} m~ e (Eq. kf_w_update,
//     Eq. active_rows_weights_update);
//  6. the covariance of the centers that left is written to the outside store
//     and their coupling to everything else is zero: the covariance stays
//     block diagonal as in Eq. H_inverse_update.
// The covariance of the active block is thus kept in information form; it is
// the same matrix the Woodbury form of Eq. H_inverse_update produces.
#include <limits.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "common.cuh"

namespace rbf {

// ---------------------------------------------------------------------------
// Neighbour lists
// ---------------------------------------------------------------------------
struct NbrParams {
  Grid g;
  float r2;  // fl32(r) * fl32(r), rounded to float32
  float rc;  // radius in cell units
};

template <class F>
__device__ __forceinline__ void for_each_cand(const Grid& g, const int32_t* __restrict__ cell_start,
                                              float x, float y, float rc, F&& f) {
  float fx = (x - g.x0) * g.inv_cs, fy = (y - g.y0) * g.inv_cs;
  int jlo, jhi;
  if (!rows_range(g, fy, rc, jlo, jhi)) return;
  for (int j = jlo; j <= jhi; ++j) {
    int ilo, ihi;
    if (!row_range(g, fx, fy, rc, j, ilo, ihi)) continue;
    int s0 = cell_start[j * g.nx + ilo];
    int s1 = cell_start[j * g.nx + ihi + 1];
    for (int s = s0; s < s1; ++s) f(s);
  }
}

__global__ void __launch_bounds__(256) k_nbr_count(NbrParams P, const int32_t* __restrict__ cell_start,
                                                   const float4* __restrict__ xyw,
                                                   const float* __restrict__ pts, int stride,
                                                   int64_t n, int32_t* __restrict__ cnt,
                                                   int* __restrict__ status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x = pts[i * stride], y = pts[i * stride + 1];
  int c = 0;
  if (isfinite(x) && isfinite(y) && (stride < 3 || isfinite(pts[i * stride + 2]))) {
    for_each_cand(P.g, cell_start, x, y, P.rc, [&](int s) {
      float4 cc = xyw[s];
      if (d2_rn(x, y, cc.x, cc.y) < P.r2) ++c;
    });
  } else {
    atomicOr(status, DEV_BAD_INDEX);
  }
  cnt[i] = c;
}

__global__ void __launch_bounds__(256) k_nbr_fill(NbrParams P, const int32_t* __restrict__ cell_start,
                                                  const float4* __restrict__ xyw,
                                                  const int32_t* __restrict__ sorted_id,
                                                  const float* __restrict__ pts, int stride, int64_t n,
                                                  const int64_t* __restrict__ row_ptr,
                                                  int32_t* __restrict__ col, int64_t cap) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x = pts[i * stride], y = pts[i * stride + 1];
  int64_t a = row_ptr[i], b = row_ptr[i + 1];
  if (a == b || b > cap) return;  // past the capacity: the caller sees the total and retries
  int64_t p = a;
  for_each_cand(P.g, cell_start, x, y, P.rc, [&](int s) {
    float4 cc = xyw[s];
    if (d2_rn(x, y, cc.x, cc.y) < P.r2 && p < b) col[p++] = sorted_id[s];
  });
  // ascending ids (rows are short)
  for (int64_t u = a + 1; u < b; ++u) {
    int32_t v = col[u];
    int64_t k = u - 1;
    while (k >= a && col[k] > v) {
      col[k + 1] = col[k];
      --k;
    }
    col[k + 1] = v;
  }
}

rbf_status neighbor_lists(Ctx* c, const float* pts, int64_t n, int stride, double radius,
                          Buf& row_ptr, Buf& col, int64_t* nnz, cudaStream_t s, int64_t defer_cap) {
  NbrParams P;
  P.g = c->grid;
  float r32 = (float)radius;
  P.r2 = r32 * r32;
  P.rc = (float)(radius / (double)c->grid.cs);
  Buf& cnt = c->scratch(10);
  RBF_TRY(cnt.ensure((size_t)(n + 1) * sizeof(int32_t)));
  RBF_TRY(row_ptr.ensure((size_t)(n + 1) * sizeof(int64_t)));
  unsigned nb = (unsigned)((n + 255) / 256);
  { k_nbr_count<<<nb, 256, 0, s>>>(P, c->cell_start.as<int32_t>(), c->sorted_xyw.as<float4>(), pts,
                                 stride, n, cnt.as<int32_t>(), c->dflag.as<int>()); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  RBF_TRY(scan_i32_to_i64(c, cnt.as<int32_t>(), row_ptr.as<int64_t>(), n, s, 48));
  if (defer_cap > 0) {
    // the total and the non-finite flag are read by the caller with its next
    // host read; rows past the capacity are left unfilled
    RBF_TRY(col.ensure((size_t)defer_cap * sizeof(int32_t)));
    { k_nbr_fill<<<nb, 256, 0, s>>>(P, c->cell_start.as<int32_t>(), c->sorted_xyw.as<float4>(),
                                  c->sorted_id.as<int32_t>(), pts, stride, n, row_ptr.as<int64_t>(),
                                  col.as<int32_t>(), defer_cap); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    *nnz = -1;
    return RBF_OK;
  }
  RBF_CUDA(cudaMemcpyAsync(c->host_small, row_ptr.as<int64_t>() + n, sizeof(int64_t),
                           cudaMemcpyDeviceToHost, s));
  int flag = 0;
  RBF_TRY(read_dev_flag(c, s, &flag));
  if (flag & DEV_BAD_INDEX) return fail(RBF_EINVAL, "a point has a non-finite coordinate");
  *nnz = c->host_small[0];
  RBF_TRY(col.ensure((size_t)(*nnz > 0 ? *nnz : 1) * sizeof(int32_t)));
  if (*nnz > 0) {
    { k_nbr_fill<<<nb, 256, 0, s>>>(P, c->cell_start.as<int32_t>(), c->sorted_xyw.as<float4>(),
                                  c->sorted_id.as<int32_t>(), pts, stride, n, row_ptr.as<int64_t>(),
                                  col.as<int32_t>(), *nnz); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }
  return RBF_OK;
}

// ---------------------------------------------------------------------------
// Active set and block bookkeeping
// ---------------------------------------------------------------------------
__global__ void k_mark(const int32_t* __restrict__ col, int64_t nnz, int32_t* __restrict__ mark) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nnz) mark[col[k]] = 1;
}

// the same with the total read on the device (entries past cap were not filled)
__global__ void k_mark_dev(const int32_t* __restrict__ col, const int64_t* __restrict__ nnz_dev, int64_t cap,
                           int32_t* __restrict__ mark) {
  const int64_t nnz = *nnz_dev;
  if (nnz > cap) return;
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nnz) mark[col[k]] = 1;
}

// A[pos[j]] = j for marked j; g2l[j] = pos[j] or -1
__global__ void k_fill_i32(int32_t* __restrict__ a, int64_t n, int32_t v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

__global__ void k_compact(const int32_t* __restrict__ mark, const int32_t* __restrict__ pos, int64_t M,
                          int32_t* __restrict__ A, int32_t* __restrict__ g2l) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  if (mark[j]) {
    A[pos[j]] = (int32_t)j;
    g2l[j] = pos[j];
  } else {
    g2l[j] = -1;
  }
}

// ---------------------------------------------------------------------------
// m~ entries, innovation, transposed (center-major) lists
// ---------------------------------------------------------------------------
struct RowParams {
  int kernel;
  double inv_rho;
  double g_scale;   // sigma^2 / st^2
  double g_inv2s2;  // 1 / (2 st^2)
};

// One warp per point: lanes take the point's neighbour entries, write the
// regression values m_ij and local column ids, and reduce the prediction
// m_i^T w for the innovation e_i = z_i - m_i^T w (Eq. kf_w_update, G3).
__global__ void __launch_bounds__(256) k_rowvals(RowParams R, const float* __restrict__ pts, int64_t n,
                                                 const int64_t* __restrict__ row_ptr,
                                                 const int32_t* __restrict__ col,
                                                 const double* __restrict__ c64,
                                                 const double* __restrict__ w,
                                                 const int32_t* __restrict__ g2l,
                                                 double* __restrict__ val, int32_t* __restrict__ lcol,
                                                 double* __restrict__ e) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= n) return;
  double x = (double)pts[3 * i], y = (double)pts[3 * i + 1], z = (double)pts[3 * i + 2];
  double acc = 0.0;
  for (int64_t k = row_ptr[i] + lane; k < row_ptr[i + 1]; k += 32) {
    int j = col[k];
    double dx = x - c64[2 * j], dy = y - c64[2 * j + 1];
    double m = row_value(R.kernel, dx * dx + dy * dy, R.inv_rho, R.g_scale, R.g_inv2s2);
    val[k] = m;
    lcol[k] = g2l[j];
    acc = fma(m, w[j], acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) e[i] = z - acc;
}

// ---------------------------------------------------------------------------
// m~ m~^T and m~ e with order-independent exact accumulation.
//
// Every point adds m_{i,l1} m_{i,l2} to entry (l1, l2) and m_{i,l} e_i to
// u_l.  The products are rounded once to float64 (as in a plain float64 sum)
// and then accumulated exactly in integers with 64-bit atomics, so the
// result does not depend on the order in which points arrive and needs no
// center-major copy of the lists:
//   * Gram entries: products lie in [0, 1] and an entry has at most n terms,
//     so a signed 64-bit fixed point with 2^gs units per 1, gs = 62 -
//     ceil(log2(n + 1)), cannot overflow (resolution 2^-gs, at least 2^-46
//     for n < 65536);
//   * u: a 128-bit fixed point with 2^64 units per 1 (two words, the carry
//     of the low word added to the high word), exact for every product of
//     magnitude below 2^63.
// Only the lower triangle (l2 <= l1) is accumulated; k_gram_merge adds it to
// both triangles of H and clears the accumulator for the next frame.
// ---------------------------------------------------------------------------

// One warp per point: pairs (t1, t2 <= t1) of its neighbour entries.
__global__ void __launch_bounds__(256) k_gram_atomic(int64_t n, const int64_t* __restrict__ row_ptr,
                                                     const int32_t* __restrict__ lcol,
                                                     const double* __restrict__ val,
                                                     const double* __restrict__ e, int64_t a, double gscale,
                                                     unsigned long long* __restrict__ G,
                                                     unsigned long long* __restrict__ U) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= n) return;
  const int64_t ra = row_ptr[i];
  const int len = (int)(row_ptr[i + 1] - ra);
  const double ei = e[i];
  for (int t = lane; t < len; t += 32) add_u128(U + 2 * (int64_t)lcol[ra + t], val[ra + t] * ei);
  if (len <= 32) {
    int lt = lane < len ? lcol[ra + lane] : 0;
    double mt = lane < len ? val[ra + lane] : 0.0;
    for (int t1 = 0; t1 < len; ++t1) {
      int l1 = __shfl_sync(0xffffffffu, lt, t1);
      double m1 = __shfl_sync(0xffffffffu, mt, t1);
      if (lane <= t1) {
        int hi = l1 > lt ? l1 : lt, lo = l1 > lt ? lt : l1;  // lower triangle whatever the list order
        atomicAdd(G + (int64_t)hi * a + lo, (unsigned long long)__double2ll_rn(m1 * mt * gscale));
      }
    }
  } else {
    for (int t1 = 0; t1 < len; ++t1) {
      int l1 = lcol[ra + t1];
      double m1 = val[ra + t1];
      for (int t2 = lane; t2 <= t1; t2 += 32) {
        int l2 = lcol[ra + t2];
        int hi = l1 > l2 ? l1 : l2, lo = l1 > l2 ? l2 : l1;
        atomicAdd(G + (int64_t)hi * a + lo, (unsigned long long)__double2ll_rn(m1 * val[ra + t2] * gscale));
      }
    }
  }
}

// H[l1][l2] += G[l1][l2] / gscale for l2 <= l1 (and the mirror entry),
// u[l] = U[l]; both accumulators are cleared.
__global__ void k_gram_merge(int64_t a, double inv_gscale, unsigned long long* __restrict__ G,
                             unsigned long long* __restrict__ U, double* __restrict__ H, int64_t ldh,
                             double* __restrict__ u) {
  int64_t l1 = blockIdx.y;
  for (int64_t l2 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l2 <= l1; l2 += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long q = G[l1 * a + l2];
    if (q == 0ull) continue;
    G[l1 * a + l2] = 0ull;
    double v = (double)(long long)q * inv_gscale;
    H[l1 * ldh + l2] += v;
    if (l2 != l1) H[l2 * ldh + l1] += v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned long long lo = U[2 * l1], hi = U[2 * l1 + 1];
    u[l1] = (double)(long long)hi + ldexp((double)lo, -64);
    U[2 * l1] = 0ull;
    U[2 * l1 + 1] = 0ull;
  }
}

// ---------------------------------------------------------------------------
// Block assembly helpers
// ---------------------------------------------------------------------------
// T[u][v] = H[perm[u]][perm[v]] (symmetric, full)
__global__ void k_gather_sym(const double* __restrict__ H, int64_t ldh, const int32_t* __restrict__ perm,
                             int64_t m, double* __restrict__ T, int64_t ldt) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * m) return;
  int64_t u = e / m, v = e % m;
  T[u * ldt + v] = H[(int64_t)perm[u] * ldh + perm[v]];
}

// D = S (m x m, leading dimension m) from the lower triangle of S
__global__ void k_copy_lower_sym(const double* __restrict__ S, int64_t lds, int64_t m, double* __restrict__ D) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * m) return;
  int64_t u = e / m, v = e % m;
  D[e] = (v <= u) ? S[u * lds + v] : S[v * lds + u];
}

// Hn[pos[u]][pos[v]] = S[u][v] using the lower triangle of S (symmetric)
__global__ void k_scatter_sym(const double* __restrict__ S, int64_t lds, int64_t m,
                              const int32_t* __restrict__ pos, double* __restrict__ Hn, int64_t ldn) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * m) return;
  int64_t u = e / m, v = e % m;
  double x = (v <= u) ? S[u * lds + v] : S[v * lds + u];
  Hn[(int64_t)pos[u] * ldn + pos[v]] = x;
}

// Hn[pn[u]][pn[v]] = H[po[u]][po[v]] for a symmetric block (full copy)
__global__ void k_move_sym(const double* __restrict__ H, int64_t ldh, const int32_t* __restrict__ po,
                           const int32_t* __restrict__ pn, int64_t m, double* __restrict__ Hn, int64_t ldn) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * m) return;
  int64_t u = e / m, v = e % m;
  Hn[(int64_t)pn[u] * ldn + pn[v]] = H[(int64_t)po[u] * ldh + po[v]];
}

// cpl[q] = 1 if staying center q (previous-local row Sl[q]) has a nonzero
// entry in a column of a leaving center (isD over previous-local ids): only
// those rows change in the Schur complement H_SS - H_SD H_DD^{-1} H_DS.
__global__ void __launch_bounds__(256) k_coupled(const double* __restrict__ H, int64_t ldh, int64_t ap,
                                                 const int32_t* __restrict__ Sl, int64_t sN,
                                                 const int32_t* __restrict__ isD, int32_t* __restrict__ cpl) {
  const int lane = threadIdx.x & 31;
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (q >= sN) return;
  const double* hr = H + (int64_t)Sl[q] * ldh;
  bool any = false;
  for (int64_t j = lane; j < ap && !any; j += 32) any = isD[j] && hr[j] != 0.0;
  any = __any_sync(0xffffffffu, any);
  if (lane == 0) cpl[q] = any ? 1 : 0;
}

// the same flags from the compressed rows of H
__global__ void __launch_bounds__(256) k_coupled_csr(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                     const int32_t* __restrict__ Sl, int64_t sN,
                                                     const int32_t* __restrict__ isD, int32_t* __restrict__ cpl) {
  const int lane = threadIdx.x & 31;
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (q >= sN) return;
  const int row = Sl[q];
  bool any = false;
  for (int p = rp[row] + lane; p < rp[row + 1] && !any; p += 32) any = isD[col[p]] != 0;
  any = __any_sync(0xffffffffu, any);
  if (lane == 0) cpl[q] = any ? 1 : 0;
}

__global__ void k_pick(const int32_t* __restrict__ flag, const int32_t* __restrict__ pos, int64_t m,
                       const int32_t* __restrict__ a, const int32_t* __restrict__ b, int32_t* __restrict__ oa,
                       int32_t* __restrict__ ob) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m || !flag[q]) return;
  oa[pos[q]] = a[q];
  ob[pos[q]] = b[q];
}

// D[u][v] = S[u][v] for a rows x cols block
__global__ void k_copy_block(const double* __restrict__ S, int64_t lds, int64_t rows, int64_t cols,
                             double* __restrict__ D, int64_t ldd) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  int64_t u = e / cols, v = e % cols;
  D[u * ldd + v] = S[u * lds + v];
}

__global__ void k_scatter_diag(const int32_t* __restrict__ pos, int64_t m, double value,
                               double* __restrict__ Hn, int64_t ldn) {
  int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u < m) Hn[(int64_t)pos[u] * ldn + pos[u]] = value;
}

// B (m x q) = 0 except B[rowpos[c]][c] = 1
__global__ void k_unit_rhs(double* __restrict__ B, int64_t m, int64_t q, const int32_t* __restrict__ rowpos) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * q) return;
  int64_t r = e / q, cidx = e % q;
  B[e] = (rowpos[cidx] == r) ? 1.0 : 0.0;
}

// Entry (a, b) of the covariance of two centers outside the active block:
// nonzero only when both refer to the same stored block; a center that never
// left keeps the prior variance.
__device__ __forceinline__ double outside_entry(const BlkRef* __restrict__ ref, const double* __restrict__ arena,
                                                int a, int b, double prior) {
  const BlkRef ra = ref[a], rb = ref[b];
  if (ra.base < 0 || rb.base < 0) return a == b ? prior : 0.0;
  if (ra.base != rb.base) return 0.0;
  return arena[ra.base + (long long)ra.pos * ra.d + rb.pos];
}

// gather G[u][v] = P[ids[u]][ids[v]] of centers outside the block
__global__ void k_gather_outside(const BlkRef* __restrict__ ref, const double* __restrict__ arena, double prior,
                                 const int32_t* __restrict__ gids, const int32_t* __restrict__ lpos, int64_t m,
                                 double* __restrict__ G) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * m) return;
  int64_t u = e / m, v = e % m;
  G[e] = outside_entry(ref, arena, gids[lpos[u]], gids[lpos[v]], prior);
}

// base[q] = arena offset of the stored block of returning center q
__global__ void k_ret_base(const BlkRef* __restrict__ ref, const int32_t* __restrict__ gids,
                           const int32_t* __restrict__ lpos, int64_t r, long long* __restrict__ base) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < r) base[q] = ref[gids[lpos[q]]].base;
}

__global__ void k_identity(double* __restrict__ B, int64_t m) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m * m) B[e] = (e / m == e % m) ? 1.0 : 0.0;
}

__global__ void k_copy_lower(const double* __restrict__ S, double* __restrict__ D, int64_t m, int64_t ld) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * m) return;
  D[(e / m) * ld + e % m] = S[(e / m) * ld + e % m];
}

// the leaving centers refer to their new block (arena offset base, d x d)
// The commit kernels are issued before the host reads the device flags and
// do nothing when the factorization or a solve failed (the state stays as it
// was, as the failing update's contract requires).
__device__ __forceinline__ bool update_failed(const int* __restrict__ flag) {
  return (*flag & (DEV_NOT_SPD | DEV_TIMEOUT)) != 0;
}

__global__ void k_blk_assign(BlkRef* __restrict__ ref, const int32_t* __restrict__ ids,
                             const int32_t* __restrict__ lpos, int64_t d, long long base,
                             const int* __restrict__ flag) {
  if (update_failed(flag)) return;
  int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u < d) {
    BlkRef r;
    r.base = base;
    r.d = (int)d;
    r.pos = (int)u;
    ref[ids[lpos[u]]] = r;
  }
}

// P[u][v] = 0.5 (X[pos[u]][v] + X[pos[v]][u]) for X = H^{-1} E_pos (n x k)
// Exclusive scan of one int per thread over a CTA of SL_THREADS threads;
// returns the total.  Ends with a barrier, so ws can be reused right away.
constexpr int SL_THREADS = 1024;
__device__ __forceinline__ int sl_block_scan(int v, int& excl, int* ws) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) ws[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int t = ws[lane];
    int ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    ws[lane] = ti - t;
    if (lane == 31) ws[32] = ti;
  }
  __syncthreads();
  excl = ws[wid] + inc - v;
  const int tot = ws[32];
  __syncthreads();
  return tot;
}

// The leaving (D), staying (S) and entering (E) sets of one update in one
// CTA: previous-local positions of D and S and new-local positions of E and
// of the staying centers (Sn), each in ascending order, the leaving flags over
// the previous block, and cnt = {|D|, |S|, |E|, entering centers that left
// some earlier block}.  The new block's size is read from the device.
__global__ void __launch_bounds__(SL_THREADS) k_set_lists(const int32_t* __restrict__ Ap, int64_t ap,
                                                          const int32_t* __restrict__ An,
                                                          const int32_t* __restrict__ an_dev,
                                                          const int32_t* __restrict__ g2l_new,
                                                          const int32_t* __restrict__ g2l_prev,
                                                          const int32_t* __restrict__ departed, int64_t M,
                                                          int32_t* __restrict__ flD, int32_t* __restrict__ Dl,
                                                          int32_t* __restrict__ Sl, int32_t* __restrict__ El,
                                                          int32_t* __restrict__ Sn, int32_t* __restrict__ cnt) {
  __shared__ int ws[33];
  constexpr int PER = 8;
  const int64_t an = *an_dev;  // size of the new block (the compaction's total)
  int nS = 0;  // staying centers seen so far (uniform)
  for (int64_t c0 = 0; c0 < ap; c0 += (int64_t)SL_THREADS * PER) {
    const int64_t b = c0 + (int64_t)threadIdx.x * PER;
    int in[PER], k = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int64_t l = b + q;
      int v = 0;
      if (l < ap) {
        const int32_t id = Ap[l];
        v = (id >= 0 && id < M && g2l_new[id] >= 0) ? 1 : 0;
      }
      in[q] = v;
      k += v;
    }
    int ex;
    const int tot = sl_block_scan(k, ex, ws);
    int ps = nS + ex;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int64_t l = b + q;
      if (l >= ap) break;
      flD[l] = 1 - in[q];
      if (in[q]) Sl[ps++] = (int32_t)l;
      else Dl[l - ps] = (int32_t)l;
    }
    nS += tot;
  }
  int nSn = 0, nret = 0;
  for (int64_t c0 = 0; c0 < an; c0 += (int64_t)SL_THREADS * PER) {
    const int64_t b = c0 + (int64_t)threadIdx.x * PER;
    int in[PER], k = 0, r = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int64_t l = b + q;
      int v = 0;
      if (l < an) {
        const int32_t id = An[l];
        const bool ok = id >= 0 && id < M;
        v = (ok && g2l_prev[id] >= 0) ? 1 : 0;
        if (ok && !v && departed[id]) ++r;
      }
      in[q] = v;
      k += v;
    }
    int ex, exr;
    const int tot = sl_block_scan(k, ex, ws);
    nret += sl_block_scan(r, exr, ws);
    int ps = nSn + ex;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int64_t l = b + q;
      if (l >= an) break;
      if (in[q]) Sn[ps++] = (int32_t)l;
      else El[l - ps] = (int32_t)l;
    }
    nSn += tot;
  }
  if (threadIdx.x == 0) {
    cnt[0] = (int32_t)(ap - nS);
    cnt[1] = nS;
    cnt[2] = (int32_t)(an - nSn);
    cnt[3] = nret;
  }
}

// ret[q] = 1 if entering center q (new-local El[q]) left an earlier block
__global__ void k_ret_flags(const int32_t* __restrict__ ids, const int32_t* __restrict__ El, int64_t e,
                            const int32_t* __restrict__ departed, int32_t* __restrict__ ret) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= e) return;
  ret[q] = departed[ids[El[q]]] ? 1 : 0;
}

// split El into returning (flag set) and fresh lists, order kept
__global__ void k_split_flags(const int32_t* __restrict__ flag, const int32_t* __restrict__ pos, int64_t m,
                              const int32_t* __restrict__ src, int32_t* __restrict__ yes, int32_t* __restrict__ no) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m) return;
  if (flag[q]) yes[pos[q]] = src[q];
  else no[q - pos[q]] = src[q];
}

__global__ void k_mark_departed(const int32_t* __restrict__ ids, const int32_t* __restrict__ lpos, int64_t d,
                                int32_t* __restrict__ departed, const int* __restrict__ flag) {
  if (update_failed(flag)) return;
  int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u < d) departed[ids[lpos[u]]] = 1;
}

__global__ void k_w_add(double* __restrict__ w, const int32_t* __restrict__ A, int64_t a,
                        const double* __restrict__ delta, const int* __restrict__ flag) {
  if (update_failed(flag)) return;
  int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l < a) w[A[l]] += delta[l];
}

__global__ void k_copy_f64_guarded(double* __restrict__ dst, const double* __restrict__ src, int64_t n,
                                   const int* __restrict__ flag) {
  if (update_failed(flag)) return;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}

// test hook: H'[l][l] += shift
__global__ void k_diag_add(double* __restrict__ H, int64_t ld, int64_t n, double shift) {
  int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l < n) H[l * ld + l] += shift;
}

__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += x[i];
}

static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

static RowParams row_params(const rbf_config& cfg, double noise) {
  RowParams R;
  R.kernel = cfg.kernel;
  R.inv_rho = 1.0 / cfg.rho;
  double st2 = cfg.sigma * cfg.sigma + noise * noise;
  R.g_scale = cfg.sigma * cfg.sigma / st2;
  R.g_inv2s2 = 1.0 / (2.0 * st2);
  return R;
}

// Solve H x = b with the Cholesky factor L (x overwrites b).  In mixed mode
// the factor is only single-precision accurate, so the solution is refined
// with float64 residuals r = b - H x until the correction stops shrinking.
rbf_status chol_solve(Ctx* c, const double* H, const double* L, int64_t a, int64_t ld, double* b, bool refine,
                      cudaStream_t s, int64_t bw) {
  if (!refine) {
    RBF_TRY(trsm_lower(c, L, a, ld, b, 1, 1, false, s, bw));
    RBF_TRY(trsm_lower(c, L, a, ld, b, 1, 1, true, s, bw));
    return RBF_OK;
  }
  Buf& rb = c->scratch(31);
  Buf& xb = c->scratch(32);
  Buf& bb = c->scratch(33);
  RBF_TRY(rb.ensure((size_t)a * sizeof(double)));
  RBF_TRY(xb.ensure((size_t)a * sizeof(double)));
  RBF_TRY(bb.ensure((size_t)a * sizeof(double)));
  RBF_CUDA(cudaMemcpyAsync(bb.p, b, (size_t)a * sizeof(double), cudaMemcpyDeviceToDevice, s));
  RBF_CUDA(cudaMemcpyAsync(xb.p, b, (size_t)a * sizeof(double), cudaMemcpyDeviceToDevice, s));
  RBF_TRY(trsm_lower(c, L, a, ld, xb.as<double>(), 1, 1, false, s, bw));
  RBF_TRY(trsm_lower(c, L, a, ld, xb.as<double>(), 1, 1, true, s, bw));
  for (int it = 0; it < 6; ++it) {
    RBF_TRY(symv_residual(H, a, ld, xb.as<double>(), bb.as<double>(), rb.as<double>(), s));
    RBF_TRY(trsm_lower(c, L, a, ld, rb.as<double>(), 1, 1, false, s, bw));
    RBF_TRY(trsm_lower(c, L, a, ld, rb.as<double>(), 1, 1, true, s, bw));
    { k_axpy<<<nblk(a), 256, 0, s>>>(xb.as<double>(), rb.as<double>(), a); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }
  RBF_CUDA(cudaMemcpyAsync(b, xb.p, (size_t)a * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return RBF_OK;
}

// Room for `need` float64 entries in the arena of stored blocks, keeping its
// contents (a new buffer, a copy, the old one freed).
static rbf_status arena_reserve(Ctx* c, int64_t need, cudaStream_t s) {
  const size_t bytes = (size_t)need * sizeof(double);
  if (bytes <= c->arena.bytes) return RBF_OK;
  size_t want = 2 * c->arena.bytes;
  if (want < bytes) want = bytes;
  if (want < ((size_t)1 << 20)) want = (size_t)1 << 20;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, want);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
  if (c->arena_used > 0) {
    e = cudaMemcpyAsync(p, c->arena.p, (size_t)c->arena_used * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
      cudaFree(p);
      return cuda_fail(e, "cudaMemcpyAsync", __FILE__, __LINE__);
    }
  }
  c->arena.release();  // cudaFree waits for the copy
  c->arena.p = p;
  c->arena.bytes = want;
  return RBF_OK;
}

// Inverse of an SPD matrix G (m x m, in place): G = L L^T, Z = L^{-1}, G^{-1} = Z^T Z.
static rbf_status spd_inverse(Ctx* c, double* G, int64_t m, cudaStream_t s, int slot) {
  Buf& Zb = c->scratch(slot);
  RBF_TRY(Zb.ensure((size_t)m * m * sizeof(double)));
  RBF_TRY(potrf_lower(c, G, m, m, m, false, s));
  { k_identity<<<nblk(m * m), 256, 0, s>>>(Zb.as<double>(), m); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  RBF_TRY(trsm_lower(c, G, m, m, Zb.as<double>(), m, m, false, s));
  RBF_TRY(gemm_f64(c, true, false, m, m, m, 1.0, Zb.as<double>(), m, Zb.as<double>(), m, 0.0, G, m, s));
  return RBF_OK;
}

// The deferred neighbour total and the device flags, copied into the pinned
// words 8..9 (total) and 10 (flags) with the caller's next host read.
static rbf_status read_deferred_total(Ctx* c, const int64_t* total_dev, cudaStream_t s) {
  int32_t* h32 = (int32_t*)c->host_small;
  RBF_CUDA(cudaMemcpyAsync(h32 + 8, total_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  RBF_CUDA(cudaMemcpyAsync(h32 + 10, c->dflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  return RBF_OK;
}

// After that read: EINVAL for a non-finite point (flag cleared), ERANGE with
// the capacity raised when the lists did not fit.
static rbf_status check_deferred_total(Ctx* c, int64_t cap, cudaStream_t s) {
  int32_t* h32 = (int32_t*)c->host_small;
  const int flag = h32[10];
  int64_t total = 0;
  memcpy(&total, h32 + 8, sizeof(int64_t));
  if (flag & DEV_BAD_INDEX) {
    RBF_CUDA(cudaMemsetAsync(c->dflag.p, 0, sizeof(int), s));
    return fail(RBF_EINVAL, "a point has a non-finite coordinate");
  }
  if (total > cap) {
    c->nbr_cap = 2 * total;
    return RBF_ERANGE;
  }
  return RBF_OK;
}

}  // namespace rbf

using namespace rbf;

extern "C" rbf_status rbf_update(rbf_ctx* cx, const float* pts, int64_t n, double noise, void* stream) {
  RBF_TRY(check_ctx(cx, true));
  if (n < 0) return fail(RBF_EINVAL, "negative n");
  if (n == 0) return RBF_OK;
  if (!pts) return fail(RBF_EINVAL, "null points");
  if (!(noise >= 0) || !isfinite(noise)) return fail(RBF_EINVAL, "noise must be finite and >= 0");
  Ctx* c = C(cx);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t M = c->M;
  const bool mixed = c->cfg.update_precision == RBF_UPDATE_MIXED;

  // 1. neighbour lists.  After the first update their total is not read
  // here: the lists are filled up to a capacity (twice the largest total
  // seen) and the total comes with the set sizes' host read below; a total
  // past the capacity makes the update start over with the capacity raised.
  Buf& row_ptr = c->scratch(0);
  Buf& col = c->scratch(1);
  int64_t nnz = 0;
  const int64_t cap = c->nbr_cap;
  {
    StageTimer st(c, RBF_STAGE_NEIGHBORS, s, 12.0 * (double)n);
    RBF_TRY(neighbor_lists(c, pts, n, 3, assembly_radius(c->cfg, noise), row_ptr, col, &nnz, s, cap));
  }
  if (cap == 0) {
    if (nnz == 0) return RBF_OK;
    c->nbr_cap = 2 * nnz;
  }
  const int64_t nnz_buf = cap > 0 ? cap : nnz;  // entries the lists may hold

  // 2. active set
  Buf& mark = c->scratch(2);
  Buf& pos = c->scratch(3);
  Buf& An = c->scratch(4);
  Buf& g2ln = c->scratch(5);
  RBF_TRY(mark.ensure((size_t)M * sizeof(int32_t)));
  RBF_TRY(pos.ensure((size_t)(M + 1) * sizeof(int32_t)));
  RBF_TRY(An.ensure((size_t)M * sizeof(int32_t)));
  RBF_TRY(g2ln.ensure((size_t)M * sizeof(int32_t)));
  if (c->cfg.exact) {
    // exact recursion: every center is in the block of every update
    { k_fill_i32<<<nblk(M), 256, 0, s>>>(mark.as<int32_t>(), M, 1); ::rbf::note_launch(); }
  } else {
    RBF_CUDA(cudaMemsetAsync(mark.p, 0, (size_t)M * sizeof(int32_t), s));
    if (cap > 0) {
      { k_mark_dev<<<nblk(cap), 256, 0, s>>>(col.as<int32_t>(), row_ptr.as<int64_t>() + n, cap, mark.as<int32_t>()); ::rbf::note_launch(); }
    } else {
      { k_mark<<<nblk(nnz), 256, 0, s>>>(col.as<int32_t>(), nnz, mark.as<int32_t>()); ::rbf::note_launch(); }
    }
  }
  RBF_CUDA(cudaGetLastError());
  RBF_TRY(scan_i32(c, mark.as<int32_t>(), pos.as<int32_t>(), M, s, 48));
  { k_compact<<<nblk(M), 256, 0, s>>>(mark.as<int32_t>(), pos.as<int32_t>(), M, An.as<int32_t>(),
                                    g2ln.as<int32_t>()); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());

  // 3. relation to the previous block: S (stay), D (leave), E (enter)
  const int64_t ap = c->a;
  Buf& fl = c->scratch(6);
  Buf& Dl = c->scratch(8);   // prev-local positions of leaving centers
  Buf& Sl = c->scratch(9);   // prev-local positions of staying centers
  Buf& El = c->scratch(11);  // new-local positions of entering centers
  Buf& Sn = c->scratch(12);  // new-local positions of staying centers
  int64_t amax = (ap > M ? ap : M);
  RBF_TRY(fl.ensure((size_t)(amax + 1) * sizeof(int32_t)));
  RBF_TRY(Dl.ensure((size_t)(amax + 1) * sizeof(int32_t)));
  RBF_TRY(Sl.ensure((size_t)(amax + 1) * sizeof(int32_t)));
  RBF_TRY(El.ensure((size_t)(amax + 1) * sizeof(int32_t)));
  RBF_TRY(Sn.ensure((size_t)(amax + 1) * sizeof(int32_t)));
  int32_t* flD = fl.as<int32_t>();  // leaving flags over the previous block
  // sizes to the host: a, d, s, e (one read: the set lists take a from the device)
  int64_t* hs = c->host_small;
  int32_t* h32 = (int32_t*)hs;
  int64_t an = 0, d = 0, sN = 0, e = 0, e_returning = 0;
  if (ap > 0) {
    Buf& cnt = c->scratch(53);
    RBF_TRY(cnt.ensure(4 * sizeof(int32_t)));
    { k_set_lists<<<1, SL_THREADS, 0, s>>>(c->A.as<int32_t>(), ap, An.as<int32_t>(), pos.as<int32_t>() + M,
                                          g2ln.as<int32_t>(), c->g2l.as<int32_t>(), c->departed.as<int32_t>(), M,
                                          flD, Dl.as<int32_t>(), Sl.as<int32_t>(), El.as<int32_t>(),
                                          Sn.as<int32_t>(), cnt.as<int32_t>()); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    RBF_CUDA(cudaMemcpyAsync(h32, cnt.p, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaMemcpyAsync(h32 + 5, pos.as<int32_t>() + M, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (cap > 0) RBF_TRY(read_deferred_total(c, row_ptr.as<int64_t>() + n, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    if (cap > 0) {
      const rbf_status st = check_deferred_total(c, cap, s);
      if (st == RBF_ERANGE) return rbf_update(cx, pts, n, noise, stream);  // lists past the capacity
      RBF_TRY(st);
    }
    an = h32[5];
    d = h32[0];
    sN = h32[1];
    e = h32[2];
    e_returning = h32[3];
    if (an == 0) return RBF_OK;
    if (sN + e != an || sN + d != ap) return fail(RBF_ECUDA, "inconsistent active-set bookkeeping");
  } else {
    RBF_CUDA(cudaMemcpyAsync(h32 + 5, pos.as<int32_t>() + M, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (cap > 0) RBF_TRY(read_deferred_total(c, row_ptr.as<int64_t>() + n, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    if (cap > 0) {
      const rbf_status st = check_deferred_total(c, cap, s);
      if (st == RBF_ERANGE) return rbf_update(cx, pts, n, noise, stream);  // lists past the capacity
      RBF_TRY(st);
    }
    an = h32[5];
    if (an == 0) return RBF_OK;
    e = an;
    // every new center enters: El = 0..an-1
    std::vector<int32_t> iota((size_t)an);
    for (int64_t l = 0; l < an; ++l) iota[l] = (int32_t)l;
    RBF_CUDA(cudaMemcpyAsync(El.p, iota.data(), (size_t)an * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    RBF_CUDA(cudaStreamSynchronize(s));
  }

  // 4. m~ entries, innovation, center-major lists
  StageTimer* st_asm = new StageTimer(c, RBF_STAGE_ASSEMBLY, s, 0.0);
  Buf& val = c->scratch(15);
  Buf& lcol = c->scratch(16);
  Buf& ev = c->scratch(17);
  RBF_TRY(val.ensure((size_t)nnz_buf * sizeof(double)));
  RBF_TRY(lcol.ensure((size_t)nnz_buf * sizeof(int32_t)));
  RBF_TRY(ev.ensure((size_t)n * sizeof(double)));
  RowParams RP = row_params(c->cfg, noise);
  { k_rowvals<<<nblk(n * 32), 256, 0, s>>>(RP, pts, n, row_ptr.as<int64_t>(), col.as<int32_t>(),
                                    c->c64.as<double>(), c->w.as<double>(), g2ln.as<int32_t>(),
                                    val.as<double>(), lcol.as<int32_t>(), ev.as<double>()); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  delete st_asm;
  // 5. leaving centers: their covariance block and the Schur complement
  StageTimer* st_blk = new StageTimer(c, RBF_STAGE_BLOCK, s, 0.0);
  const int64_t ld = an;
  Buf& Hn = c->scratch(35);
  Buf& Ln = c->scratch(36);
  Buf& u = c->scratch(37);
  RBF_TRY(Hn.ensure((size_t)an * an * sizeof(double)));
  RBF_TRY(Ln.ensure((size_t)an * an * sizeof(double)));
  RBF_TRY(u.ensure((size_t)an * sizeof(double)));
  RBF_CUDA(cudaMemsetAsync(Hn.p, 0, (size_t)an * an * sizeof(double), s));
  Buf& Pdd = c->scratch(38);
  // The covariance block of the leaving centers, the information of the
  // entering ones and the Schur complement of the staying ones read only the
  // previous state and write disjoint outputs: they run on three streams.
  // (The FP64 path and large returning blocks keep one stream: their
  // cooperative substitution solves share one set of ready flags.)
  {
    Buf& G0 = c->scratch(68);
    Buf& U0 = c->scratch(69);
    size_t gbytes = (size_t)an * an * sizeof(unsigned long long);
    size_t ubytes = (size_t)2 * an * sizeof(unsigned long long);
    if (G0.bytes < gbytes || U0.bytes < ubytes || c->gacc_dirty) {
      RBF_TRY(G0.ensure(gbytes));
      RBF_TRY(U0.ensure(ubytes));
      RBF_CUDA(cudaMemsetAsync(G0.p, 0, G0.bytes, s));
      RBF_CUDA(cudaMemsetAsync(U0.p, 0, U0.bytes, s));
    }
  }
  // Schur complement, first part (caller's stream, before the other streams
  // are fed): H_SS moves over unchanged, the rows N of S coupled to some
  // leaving center are listed, and their count goes to the host, so that the
  // host reads it after the other streams' work has been issued.
  Buf& cpl = c->scratch(74);
  Buf& cpp = c->scratch(75);
  Buf& perm = c->scratch(40);
  Buf& Nn = c->scratch(76);

  if (d > 0 && sN > 0) {
    StageTimer st_sc0(c, RBF_STAGE_SCHUR, s, 0.0);
    { k_move_sym<<<nblk(sN * sN), 256, 0, s>>>(c->H.as<double>(), c->ldH, Sl.as<int32_t>(), Sn.as<int32_t>(),
                                             sN, Hn.as<double>(), ld); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    RBF_TRY(cpl.ensure((size_t)(sN + 1) * sizeof(int32_t)));
    RBF_TRY(cpp.ensure((size_t)(sN + 1) * sizeof(int32_t)));
    RBF_TRY(perm.ensure((size_t)(d + sN) * sizeof(int32_t)));
    RBF_TRY(Nn.ensure((size_t)(sN + 1) * sizeof(int32_t)));
    if (c->Hs.valid && c->Hs.n == ap) {
      { k_coupled_csr<<<nblk(sN * 32), 256, 0, s>>>(c->Hs.rp.as<int32_t>(), c->Hs.col.as<int32_t>(),
                                                   Sl.as<int32_t>(), sN, flD, cpl.as<int32_t>()); ::rbf::note_launch(); }
    } else {
      { k_coupled<<<nblk(sN * 32), 256, 0, s>>>(c->H.as<double>(), c->ldH, ap, Sl.as<int32_t>(), sN, flD,
                                              cpl.as<int32_t>()); ::rbf::note_launch(); }
    }
    RBF_CUDA(cudaGetLastError());
    RBF_TRY(scan_i32(c, cpl.as<int32_t>(), cpp.as<int32_t>(), sN, s, 77));
    RBF_CUDA(cudaMemcpyAsync(perm.p, Dl.p, (size_t)d * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    { k_pick<<<nblk(sN), 256, 0, s>>>(cpl.as<int32_t>(), cpp.as<int32_t>(), sN, Sl.as<int32_t>(),
                                    Sn.as<int32_t>(), perm.as<int32_t>() + d, Nn.as<int32_t>()); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    RBF_CUDA(cudaMemcpyAsync(h32 + 4, cpp.as<int32_t>() + sN, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  }
  const bool par = mixed && e_returning <= SPD_SMALL_MAX;
  // The Schur chain is the longest of the block stage; its stream has the
  // highest priority, so that its small kernels are not queued behind the
  // second wave of the covariance block's product.
  cudaStream_t sA = s, sB = s, sC = s;
  if (par) {
    for (int q = 0; q < 2; ++q)
      if (!c->bs[q]) RBF_CUDA(cudaStreamCreateWithFlags(&c->bs[q], cudaStreamNonBlocking));
    if (!c->bs[2]) {
      int least = 0, greatest = 0;
      RBF_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
      RBF_CUDA(cudaStreamCreateWithPriority(&c->bs[2], cudaStreamNonBlocking, greatest));
    }
    for (auto& ev : c->bev)
      if (!ev) RBF_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    sA = c->bs[0];
    sB = c->bs[2];
    sC = c->bs[1];
    RBF_CUDA(cudaEventRecord(c->bev[0], s));
    RBF_CUDA(cudaStreamWaitEvent(sA, c->bev[0], 0));
    RBF_CUDA(cudaStreamWaitEvent(sB, c->bev[0], 0));
    RBF_CUDA(cudaStreamWaitEvent(sC, c->bev[0], 0));
  }
  if (d > 0) {
    Buf& Y = c->scratch(39);
    RBF_TRY(Y.ensure((size_t)ap * d * sizeof(double)));
    RBF_TRY(Pdd.ensure((size_t)d * d * sizeof(double)));
    { k_unit_rhs<<<nblk(ap * d), 256, 0, sA>>>(Y.as<double>(), ap, d, Dl.as<int32_t>()); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    StageTimer st_cb(c, RBF_STAGE_COVBLOCK, sA, 0.0);
    if (mixed) {
      // X = H_prev^{-1} E_D by refined solves with the float32 factor; P_DD = X[D, :]
      RBF_TRY(mixed_cov(c, c->H.as<double>(), c->ldH, &c->Hs, c->Lf.as<float>(), c->ldw, c->Zd.as<float>(),
                        c->zi_valid ? c->Zi.as<float>() : nullptr, ap, Y.as<double>(), d, Dl.as<int32_t>(),
                        c->refine_sweeps_cov, Pdd.as<double>(), sA, c->bw_lf));
    } else {
      // Y = L_prev^{-1} E_D, P_DD = Y^T Y
      RBF_TRY(trsm_lower(c, c->L.as<double>(), ap, c->ldH, Y.as<double>(), d, d, false, s, c->bw_lf));
      RBF_TRY(gemm_f64(c, true, false, d, d, ap, 1.0, Y.as<double>(), d, Y.as<double>(), d, 0.0,
                       Pdd.as<double>(), d, s));
    }
  }
  // Schur complement, second part (stream sB), issued before the Gram
  // and the entering centers: its chain is the longest of the block stage
  if (d > 0) {
    StageTimer st_sc(c, RBF_STAGE_SCHUR, sB, 0.0);
    if (sN > 0) {
      // H_S = H_SS - H_SD H_DD^{-1} H_DS.  H_SS moves over unchanged; only the
      // rows N of S coupled to some leaving center change: T = H_prev on
      // [D; N], and d steps of Cholesky leave the new H_NN in T[d:, d:].
      // (the coupled rows N and their count were found before the fork)
      RBF_CUDA(cudaStreamSynchronize(s));
      const int64_t nN = h32[4];
      if (nN > 0) {
        const int64_t t = d + nN;
        Buf& T = c->scratch(41);
        RBF_TRY(T.ensure((size_t)t * t * sizeof(double)));
        { k_gather_sym<<<nblk(t * t), 256, 0, sB>>>(c->H.as<double>(), c->ldH, perm.as<int32_t>(), t,
                                                 T.as<double>(), t); ::rbf::note_launch(); }
        RBF_CUDA(cudaGetLastError());
        if (mixed) {
          // Block elimination of D in chunks of at most SPD_SMALL_MAX: each
          // chunk's Schur complement is taken in the block the previous
          // chunks left, T[r, r] -= T[r, q] T[q, q]^{-1} T[r, q]^T, with the
          // inverse and the products in float-float arithmetic.  Only the lower triangle of T
          // is kept current (the 64 x 64 tiles on or below the diagonal).
          Buf& Gd = c->scratch(84);
          Buf& Yb = c->scratch(85);
          const int64_t nc = (d + SPD_SMALL_MAX - 1) / SPD_SMALL_MAX;
          const int64_t cs = (d + nc - 1) / nc;
          RBF_TRY(Gd.ensure((size_t)cs * cs * sizeof(double)));
          RBF_TRY(Yb.ensure((size_t)cs * (t - 1) * sizeof(double)));
          double* Tp = T.as<double>();
          for (int64_t q0 = 0; q0 < d; q0 += cs) {
            const int64_t dq = cs < d - q0 ? cs : d - q0, r0 = q0 + dq, rest = t - r0;
            { k_copy_lower_sym<<<nblk(dq * dq), 256, 0, sB>>>(Tp + q0 * t + q0, t, dq, Gd.as<double>()); ::rbf::note_launch(); }
            RBF_CUDA(cudaGetLastError());
            RBF_TRY(spd_inverse_small_ff(c, Gd.as<double>(), dq, sB));
            RBF_TRY(gemm_ff(c, false, true, dq, rest, dq, 1.0, Gd.as<double>(), dq, Tp + r0 * t + q0, t, 0.0,
                            Yb.as<double>(), rest, sB, 87));
            RBF_TRY(gemm_ff(c, false, false, rest, rest, dq, -1.0, Tp + r0 * t + q0, t, Yb.as<double>(), rest, 1.0,
                            Tp + r0 * t + r0, t, sB, 87, true));
          }
        } else if (d <= SPD_SMALL_MAX) {
          // H_NN -= H_ND (H_DD^{-1} H_DN), with H_DD^{-1} by the one-CTA inverse
          Buf& Gd = c->scratch(84);
          Buf& Yb = c->scratch(85);
          RBF_TRY(Gd.ensure((size_t)d * d * sizeof(double)));
          RBF_TRY(Yb.ensure((size_t)d * nN * sizeof(double)));
          { k_copy_block<<<nblk(d * d), 256, 0, sB>>>(T.as<double>(), t, d, d, Gd.as<double>(), d); ::rbf::note_launch(); }
          RBF_CUDA(cudaGetLastError());
          RBF_TRY(spd_inverse_small(c, Gd.as<double>(), d, sB));
          RBF_TRY(gemm_f64(c, false, false, d, nN, d, 1.0, Gd.as<double>(), d, T.as<double>() + d, t, 0.0,
                           Yb.as<double>(), nN, sB, 87));
          RBF_TRY(gemm_f64(c, false, false, nN, nN, d, -1.0, T.as<double>() + d * t, t, Yb.as<double>(), nN, 1.0,
                           T.as<double>() + d * t + d, t, sB, 87));
        } else {
          RBF_TRY(potrf_lower(c, T.as<double>(), t, t, d, false, sB));
        }
        { k_scatter_sym<<<nblk(nN * nN), 256, 0, sB>>>(T.as<double>() + d * t + d, t, nN, Nn.as<int32_t>(),
                                                    Hn.as<double>(), ld); ::rbf::note_launch(); }
        RBF_CUDA(cudaGetLastError());
      }
    }
  } else if (sN > 0) {
    // nobody leaves: the staying block is the previous information matrix
    { k_move_sym<<<nblk(sN * sN), 256, 0, s>>>(c->H.as<double>(), c->ldH, Sl.as<int32_t>(), Sn.as<int32_t>(), sN,
                                             Hn.as<double>(), ld); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }
  // m~ m~^T and m~ e: exact integer accumulation into cleared accumulators
  // (added to H' once the block stage has written it)
  if (an > 65535) return fail(RBF_EINVAL, "active block of %lld centers exceeds 65535", (long long)an);
  Buf& G = c->scratch(68);
  Buf& U = c->scratch(69);
  const int gs = 62 - (int)ceil(log2((double)n + 1.0));
  const double gscale = ldexp(1.0, gs);
  {
    StageTimer st(c, RBF_STAGE_ASSEMBLY, sC, 0.0);
    c->gacc_dirty = true;
    { k_gram_atomic<<<nblk(n * 32), 256, 0, sC>>>(n, row_ptr.as<int64_t>(), lcol.as<int32_t>(), val.as<double>(),
                                                ev.as<double>(), an, gscale, G.as<unsigned long long>(),
                                                U.as<unsigned long long>()); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }

  // 6. entering centers: inverse of their stored covariance block
  if (e > 0) {
    StageTimer st_en(c, RBF_STAGE_ENTER, sC, 0.0);
    if (!c->pg_on || e_returning == 0) {
      // never-departed centers keep the prior P = I / lambda with no coupling
      { k_scatter_diag<<<nblk(e), 256, 0, sC>>>(El.as<int32_t>(), e, c->cfg.lambda, Hn.as<double>(), ld); ::rbf::note_launch(); }
      RBF_CUDA(cudaGetLastError());
    } else {
      // the stored covariance couples the returning centers R only among
      // themselves (fresh ones F keep the uncoupled prior), so the block's
      // inverse is diag(P_RR^{-1}, lambda I)
      const int64_t r = e_returning, f = e - e_returning;
      Buf& rf = c->scratch(80);
      Buf& rp = c->scratch(81);
      Buf& Rl = c->scratch(82);
      Buf& Fl = c->scratch(83);
      RBF_TRY(rf.ensure((size_t)(e + 1) * sizeof(int32_t)));
      RBF_TRY(rp.ensure((size_t)(e + 1) * sizeof(int32_t)));
      RBF_TRY(Rl.ensure((size_t)(r + 1) * sizeof(int32_t)));
      RBF_TRY(Fl.ensure((size_t)(f + 1) * sizeof(int32_t)));
      { k_ret_flags<<<nblk(e), 256, 0, sC>>>(An.as<int32_t>(), El.as<int32_t>(), e, c->departed.as<int32_t>(),
                                          rf.as<int32_t>()); ::rbf::note_launch(); }
      RBF_CUDA(cudaGetLastError());
      RBF_TRY(scan_i32(c, rf.as<int32_t>(), rp.as<int32_t>(), e, sC, 88));
      { k_split_flags<<<nblk(e), 256, 0, sC>>>(rf.as<int32_t>(), rp.as<int32_t>(), e, El.as<int32_t>(),
                                            Rl.as<int32_t>(), Fl.as<int32_t>()); ::rbf::note_launch(); }
      RBF_CUDA(cudaGetLastError());
      if (f > 0) {
        { k_scatter_diag<<<nblk(f), 256, 0, sC>>>(Fl.as<int32_t>(), f, c->cfg.lambda, Hn.as<double>(), ld); ::rbf::note_launch(); }
        RBF_CUDA(cudaGetLastError());
      }
      Buf& Gb = c->scratch(42);
      // P_RR is block-diagonal over the departures the centers came back from
      // (P[A, not A] = 0 at each departure), so many returning centers are
      // inverted block by block: their stored blocks' offsets go to the host,
      // which groups them (the block stage runs on one stream in that case).
      std::vector<int32_t> grp_list;
      std::vector<int64_t> grp_start{0};
      if (r > SPD_SMALL_MAX) {
        Buf& bb = c->scratch(98);
        RBF_TRY(bb.ensure((size_t)r * sizeof(long long)));
        { k_ret_base<<<nblk(r), 256, 0, sC>>>(c->blkref.as<BlkRef>(), An.as<int32_t>(), Rl.as<int32_t>(), r,
                                           bb.as<long long>()); ::rbf::note_launch(); }
        RBF_CUDA(cudaGetLastError());
        std::vector<long long> hb((size_t)r);
        std::vector<int32_t> hr((size_t)r);
        RBF_CUDA(cudaMemcpyAsync(hb.data(), bb.p, (size_t)r * sizeof(long long), cudaMemcpyDeviceToHost, sC));
        RBF_CUDA(cudaMemcpyAsync(hr.data(), Rl.p, (size_t)r * sizeof(int32_t), cudaMemcpyDeviceToHost, sC));
        RBF_CUDA(cudaStreamSynchronize(sC));
        std::vector<int64_t> ord((size_t)r);
        for (int64_t q = 0; q < r; ++q) ord[q] = q;
        std::stable_sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) { return hb[x] < hb[y]; });
        grp_list.resize((size_t)r);
        for (int64_t q = 0; q < r; ++q) {
          grp_list[q] = hr[ord[q]];
          if (q > 0 && hb[ord[q]] != hb[ord[q - 1]]) grp_start.push_back(q);
        }
        RBF_CUDA(cudaMemcpyAsync(Rl.p, grp_list.data(), (size_t)r * sizeof(int32_t), cudaMemcpyHostToDevice, sC));
        RBF_CUDA(cudaStreamSynchronize(sC));  // the host list is released at the end of this scope
      }
      grp_start.push_back(r);
      int64_t kmax = 0;
      for (size_t g = 0; g + 1 < grp_start.size(); ++g) kmax = std::max(kmax, grp_start[g + 1] - grp_start[g]);
      RBF_TRY(Gb.ensure((size_t)kmax * kmax * sizeof(double)));
      for (size_t g = 0; g + 1 < grp_start.size(); ++g) {
        const int64_t q0 = grp_start[g], k = grp_start[g + 1] - q0;
        const int32_t* lk = Rl.as<int32_t>() + q0;
        { k_gather_outside<<<nblk(k * k), 256, 0, sC>>>(c->blkref.as<BlkRef>(), c->arena.as<double>(),
                                                      1.0 / c->cfg.lambda, An.as<int32_t>(), lk, k,
                                                      Gb.as<double>()); ::rbf::note_launch(); }
        RBF_CUDA(cudaGetLastError());
        if (k <= SPD_SMALL_MAX && mixed) RBF_TRY(spd_inverse_small_ff(c, Gb.as<double>(), k, sC));
        else if (k <= SPD_SMALL_MAX) RBF_TRY(spd_inverse_small(c, Gb.as<double>(), k, sC));
        else RBF_TRY(spd_inverse(c, Gb.as<double>(), k, sC, 43));
        { k_scatter_sym<<<nblk(k * k), 256, 0, sC>>>(Gb.as<double>(), k, k, lk, Hn.as<double>(), ld); ::rbf::note_launch(); }
        RBF_CUDA(cudaGetLastError());
      }
    }
  }


  if (par) {
    RBF_CUDA(cudaEventRecord(c->bev[1], sA));
    RBF_CUDA(cudaEventRecord(c->bev[2], sC));
    RBF_CUDA(cudaEventRecord(c->bev[3], sB));
    RBF_CUDA(cudaStreamWaitEvent(s, c->bev[1], 0));
    RBF_CUDA(cudaStreamWaitEvent(s, c->bev[2], 0));
    RBF_CUDA(cudaStreamWaitEvent(s, c->bev[3], 0));
  }
  delete st_blk;
  // 7. + m~ m~^T and u = m~ e (accumulated above, beside the block stage)
  {
    StageTimer st(c, RBF_STAGE_ASSEMBLY, s, 0.0);
    dim3 mg((unsigned)((an + 255) / 256 < 8 ? (an + 255) / 256 : 8), (unsigned)an);
    { k_gram_merge<<<mg, 256, 0, s>>>(an, 1.0 / gscale, G.as<unsigned long long>(), U.as<unsigned long long>(),
                                      Hn.as<double>(), ld, u.as<double>()); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    c->gacc_dirty = false;
  }
  if (c->diag_shift != 0.0) {
    { k_diag_add<<<nblk(an), 256, 0, s>>>(Hn.as<double>(), ld, an, c->diag_shift); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }
  // Until a center has left some block there is no Schur-complement fill and
  // H' has the band structure of m~ m~^T: read its half-bandwidth then, and
  // skip the zero blocks outside the band in the factorization and solves.
  // Otherwise the compressed rows of H' (needed from the first residual of
  // the solve on) are built on a side stream beside the factorization.
  int64_t bw = BW_DENSE;
  const bool band_probe = !c->pg_on && d == 0;
  // Once a center has left, H' carries Schur fill and soon holds about a^2
  // nonzeros: its residuals then read the dense H' (8 bytes an entry against
  // 12 for the compressed rows) and no compressed copy is built.
  if (mixed) {
    if (band_probe) RBF_TRY(build_csr(c, Hn.as<double>(), ld, an, c->Hs_next, s));
    else c->Hs_next.valid = false;
  }
  if (band_probe) {
    if (mixed && c->Hs_next.valid) RBF_TRY(csr_bandwidth(c, an, &bw, s));
    else RBF_TRY(dense_bandwidth(c, Hn.as<double>(), ld, an, &bw, s));
    if (3 * bw >= an) bw = BW_DENSE;
  }

  // 8. factor H' and solve for the weight increment
  Buf& Wn = c->scratch(27);
  Buf& Zdn = c->scratch(63);
  Buf& Zin = c->scratch(64);
  const int64_t ldw = (an + 3) & ~(int64_t)3;
  // (the inverse of a banded factor is dense, but for blocks this small the
  // products with it still beat the chain of substitution steps)
  const bool use_inv = mixed && an <= c->inv_max;
  if (mixed) {
    RBF_TRY(Wn.ensure((size_t)an * ldw * sizeof(float)));
    RBF_TRY(Zdn.ensure((size_t)((an + 63) / 64) * 64 * 64 * sizeof(float)));
    RBF_TRY(potrf_mixed(c, Hn.as<double>(), ld, an, Wn.as<float>(), ldw, Zdn.as<float>(), s, bw));
    if (use_inv) {
      RBF_TRY(Zin.ensure((size_t)2 * an * ldw * sizeof(float)));  // L^{-1} and its transpose
      RBF_TRY(trtri_mixed(c, Wn.as<float>(), ldw, an, Zdn.as<float>(), Zin.as<float>(), ldw, s));
    }
  } else {
    RBF_CUDA(cudaMemcpyAsync(Ln.p, Hn.p, (size_t)an * an * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RBF_TRY(potrf_lower(c, Ln.as<double>(), an, ld, an, false, s, bw));
  }
  int flag = 0;
  {
    StageTimer st(c, RBF_STAGE_SOLVE, s, (mixed ? 2.0 * c->refine_sweeps + 2.0 * (c->refine_sweeps - 1) : 2.0) *
                                            (double)an * an);
    if (mixed)
      RBF_TRY(mixed_solve(c, Hn.as<double>(), ld, &c->Hs_next, Wn.as<float>(), ldw, Zdn.as<float>(),
                          use_inv ? Zin.as<float>() : nullptr, an, u.as<double>(), 1, c->refine_sweeps, s, bw));
    else
      RBF_TRY(chol_solve(c, Hn.as<double>(), Ln.as<double>(), an, ld, u.as<double>(), false, s, bw));
  }
  // 9. commit, issued before the one read of the device flags that covers the
  // factorization and the solves: the kernels skip their writes if it failed,
  // and the host's bookkeeping below happens only after a clean read
  const int* dflag = c->dflag.as<int>();
  { k_w_add<<<nblk(an), 256, 0, s>>>(c->w.as<double>(), An.as<int32_t>(), an, u.as<double>(), dflag); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  const long long base = c->arena_used;
  if (d > 0) {
    // the block P_DD goes to the arena; the leaving centers refer to it, which
    // also drops their coupling to every older block (P[D, not D] = 0)
    RBF_TRY(arena_reserve(c, base + d * d, s));
    { k_copy_f64_guarded<<<nblk(d * d), 256, 0, s>>>(c->arena.as<double>() + base, Pdd.as<double>(), d * d, dflag); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    { k_blk_assign<<<nblk(d), 256, 0, s>>>(c->blkref.as<BlkRef>(), c->A.as<int32_t>(), Dl.as<int32_t>(), d, base,
                                         dflag); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    { k_mark_departed<<<nblk(d), 256, 0, s>>>(c->A.as<int32_t>(), Dl.as<int32_t>(), d, c->departed.as<int32_t>(),
                                            dflag); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }
  // the evaluation tables follow the weights (unchanged if the update failed)
  RBF_TRY(refresh_center_weights(c, s));
  RBF_TRY(read_dev_flag(c, s, &flag));
  if (flag & DEV_NOT_SPD) return fail(RBF_ENOTSPD, "information matrix of the active block is not SPD");
  if (flag & DEV_TIMEOUT) return fail(RBF_ETIMEOUT, "triangular solve wait timed out");
  if (d > 0) {
    c->arena_used = base + d * d;
    c->pg_on = true;
  }
  std::swap(c->H, Hn);
  if (mixed) {
    std::swap(c->Lf, Wn);
    std::swap(c->Zd, Zdn);
    std::swap(c->Hs, c->Hs_next);
    if (use_inv) std::swap(c->Zi, Zin);
    c->zi_valid = use_inv;
    c->bw_lf = bw;
    c->ldw = ldw;
  } else {
    std::swap(c->L, Ln);
    c->bw_lf = bw;
  }
  std::swap(c->A, An);
  std::swap(c->g2l, g2ln);
  c->a = an;
  c->ldH = ld;
  return RBF_OK;
}

extern "C" rbf_status rbf_get_active(rbf_ctx* cx, int32_t* A, int64_t cap, int64_t* a_out, void* stream) {
  RBF_TRY(check_ctx(cx, true));
  if (!a_out) return fail(RBF_EINVAL, "null a_out");
  Ctx* c = C(cx);
  *a_out = c->a;
  if (c->a == 0) return RBF_OK;
  if (!A) return fail(RBF_EINVAL, "null A");
  if (cap < c->a) return fail(RBF_ERANGE, "capacity %lld < %lld", (long long)cap, (long long)c->a);
  cudaStream_t s = (cudaStream_t)stream;
  RBF_CUDA(cudaMemcpyAsync(A, c->A.p, (size_t)c->a * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  RBF_CUDA(cudaStreamSynchronize(s));
  return RBF_OK;
}

extern "C" rbf_status rbf_get_neighbors(rbf_ctx* cx, const float* pts, int64_t n, double noise,
                                        int64_t* row_ptr, int32_t* col, int64_t cap, int64_t* nnz_out,
                                        void* stream) {
  RBF_TRY(check_ctx(cx, true));
  if (n < 0 || !nnz_out || !row_ptr) return fail(RBF_EINVAL, "bad arguments");
  if (n > 0 && !pts) return fail(RBF_EINVAL, "null points");
  Ctx* c = C(cx);
  cudaStream_t s = (cudaStream_t)stream;
  Buf& rp = c->scratch(0);
  Buf& cl = c->scratch(1);
  int64_t nnz = 0;
  if (n == 0) {
    RBF_CUDA(cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), s));
    *nnz_out = 0;
    return RBF_OK;
  }
  RBF_TRY(neighbor_lists(c, pts, n, 3, assembly_radius(c->cfg, noise), rp, cl, &nnz, s));
  *nnz_out = nnz;
  RBF_CUDA(cudaMemcpyAsync(row_ptr, rp.p, (size_t)(n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  if (nnz > cap) {
    RBF_CUDA(cudaStreamSynchronize(s));
    return fail(RBF_ERANGE, "capacity %lld < %lld entries", (long long)cap, (long long)nnz);
  }
  if (nnz > 0) {
    if (!col) return fail(RBF_EINVAL, "null col");
    RBF_CUDA(cudaMemcpyAsync(col, cl.p, (size_t)nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  }
  RBF_CUDA(cudaStreamSynchronize(s));
  return RBF_OK;
}

// P[ids, ids]: active ids from the factor of the block's information matrix,
// the others from the outside store (or the prior), zero across the two.
__global__ void k_cov_assemble(int64_t k, const int32_t* __restrict__ ids, const int32_t* __restrict__ g2l,
                               const int32_t* __restrict__ rank_in_active, const double* __restrict__ Paa,
                               int64_t ka, const BlkRef* __restrict__ ref, const double* __restrict__ arena,
                               double prior, double* __restrict__ out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * k) return;
  int64_t u = e / k, v = e % k;
  int iu = ids[u], iv = ids[v];
  bool au = g2l[iu] >= 0, av = g2l[iv] >= 0;
  double x = 0.0;
  if (au && av) {
    x = Paa[(int64_t)rank_in_active[u] * ka + rank_in_active[v]];
  } else if (!au && !av) {
    x = outside_entry(ref, arena, iu, iv, prior);
  }
  out[e] = x;
}

extern "C" rbf_status rbf_get_cov(rbf_ctx* cx, const int32_t* ids, int64_t k, double* Pk, void* stream) {
  RBF_TRY(check_ctx(cx, true));
  if (k < 0) return fail(RBF_EINVAL, "negative k");
  if (k == 0) return RBF_OK;
  if (!ids || !Pk) return fail(RBF_EINVAL, "null argument");
  Ctx* c = C(cx);
  cudaStream_t s = (cudaStream_t)stream;
  for (int64_t u = 0; u < k; ++u)
    if (ids[u] < 0 || ids[u] >= c->M) return fail(RBF_EINVAL, "id %d out of range", ids[u]);
  // local indices of the active ids (host copy of g2l)
  std::vector<int32_t> g2l((size_t)c->M, -1);
  if (c->a > 0)
    RBF_CUDA(cudaMemcpyAsync(g2l.data(), c->g2l.p, (size_t)c->M * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  RBF_CUDA(cudaStreamSynchronize(s));
  std::vector<int32_t> rank((size_t)k, -1), lpos;
  for (int64_t u = 0; u < k; ++u) {
    int l = c->a > 0 ? g2l[ids[u]] : -1;
    if (l >= 0) {
      rank[u] = (int32_t)lpos.size();
      lpos.push_back(l);
    }
  }
  int64_t ka = (int64_t)lpos.size();
  Buf& ib = c->scratch(44);
  Buf& rb = c->scratch(45);
  Buf& lb = c->scratch(46);
  Buf& Y = c->scratch(47);
  Buf& Paa = c->scratch(39);
  RBF_TRY(ib.ensure((size_t)k * sizeof(int32_t)));
  RBF_TRY(rb.ensure((size_t)k * sizeof(int32_t)));
  RBF_CUDA(cudaMemcpyAsync(ib.p, ids, (size_t)k * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  RBF_CUDA(cudaMemcpyAsync(rb.p, rank.data(), (size_t)k * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  if (ka > 0) {
    RBF_TRY(lb.ensure((size_t)ka * sizeof(int32_t)));
    RBF_TRY(Y.ensure((size_t)c->a * ka * sizeof(double)));
    RBF_TRY(Paa.ensure((size_t)ka * ka * sizeof(double)));
    RBF_CUDA(cudaMemcpyAsync(lb.p, lpos.data(), (size_t)ka * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    { k_unit_rhs<<<nblk(c->a * ka), 256, 0, s>>>(Y.as<double>(), c->a, ka, lb.as<int32_t>()); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    if (c->cfg.update_precision == RBF_UPDATE_MIXED) {
      RBF_TRY(mixed_cov(c, c->H.as<double>(), c->ldH, &c->Hs, c->Lf.as<float>(), c->ldw, c->Zd.as<float>(),
                        c->zi_valid ? c->Zi.as<float>() : nullptr, c->a, Y.as<double>(), ka, lb.as<int32_t>(),
                        c->refine_sweeps_cov, Paa.as<double>(), s, c->bw_lf));
    } else {
      RBF_TRY(trsm_lower(c, c->L.as<double>(), c->a, c->ldH, Y.as<double>(), ka, ka, false, s, c->bw_lf));
      RBF_TRY(gemm_f64(c, true, false, ka, ka, c->a, 1.0, Y.as<double>(), ka, Y.as<double>(), ka, 0.0,
                       Paa.as<double>(), ka, s));
    }
  }
  { k_cov_assemble<<<nblk(k * k), 256, 0, s>>>(k, ib.as<int32_t>(), c->g2l.as<int32_t>(), rb.as<int32_t>(),
                                             ka > 0 ? Paa.as<double>() : nullptr, ka,
                                             c->blkref.as<BlkRef>(), c->arena.as<double>(), 1.0 / c->cfg.lambda,
                                             Pk); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  RBF_CUDA(cudaStreamSynchronize(s));
  int flag = 0;
  RBF_TRY(read_dev_flag(c, s, &flag));
  if (flag & DEV_TIMEOUT) return fail(RBF_ETIMEOUT, "triangular solve wait timed out");
  return RBF_OK;
}
