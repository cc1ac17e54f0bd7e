// Adaptive center selection (Sec. III-A).
//
// The paper counts, with a k-d tree, the points within r_kd of every
// candidate of a mesh over the region of interest and keeps the candidates
// whose count exceeds a threshold.  Here the points are binned into the
// cells of the candidate mesh itself (a counting sort; points beyond the
// mesh are clamped into its border cells) and every candidate counts the
// points of the cells that meet its disc, with the float32 test
// d2 < r_kd^2.  Accepted candidates keep ascending row-major order.
#include <math.h>

#include "common.cuh"

namespace rbf {

__global__ void k_pt_cells(const float* __restrict__ pts, int64_t n, Grid g, int32_t* __restrict__ pcell,
                           int32_t* __restrict__ cnt, int* __restrict__ status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x = pts[3 * i], y = pts[3 * i + 1];
  if (!(isfinite(x) && isfinite(y) && isfinite(pts[3 * i + 2]))) {
    atomicOr(status, DEV_BAD_INDEX);
    pcell[i] = -1;
    return;
  }
  float fx = floorf((x - g.x0) * g.inv_cs), fy = floorf((y - g.y0) * g.inv_cs);
  fx = fminf(fmaxf(fx, 0.f), (float)(g.nx - 1));
  fy = fminf(fmaxf(fy, 0.f), (float)(g.ny - 1));
  int cc = (int)fy * g.nx + (int)fx;
  pcell[i] = cc;
  atomicAdd(&cnt[cc], 1);
}

__global__ void k_pt_fill(const int32_t* __restrict__ pcell, int64_t n, const int32_t* __restrict__ start,
                          int32_t* __restrict__ fill, float2* __restrict__ binned,
                          const float* __restrict__ pts) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int cc = pcell[i];
  if (cc < 0) return;
  int p = start[cc] + atomicAdd(&fill[cc], 1);
  binned[p] = make_float2(pts[3 * i], pts[3 * i + 1]);
}

// candidate (i, j) at (x0 + (i + 0.5) h, y0 + (j + 0.5) h): one FP64 multiply, one FP64 add
__device__ __forceinline__ double cand_coord(double x0, int i, double h) {
  return __dadd_rn(x0, __dmul_rn((double)i + 0.5, h));
}

__global__ void __launch_bounds__(256) k_count_cands(double x0, double y0, double h, Grid g, float r2, float rc,
                                                     const int32_t* __restrict__ start,
                                                     const float2* __restrict__ binned,
                                                     int32_t* __restrict__ counts) {
  int64_t cidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cidx >= (int64_t)g.nx * g.ny) return;
  int i = (int)(cidx % g.nx), j = (int)(cidx / g.nx);
  float cx = (float)cand_coord(x0, i, h), cy = (float)cand_coord(y0, j, h);
  int R = (int)ceilf(rc) + 1;
  int jlo = max(j - R, 0), jhi = min(j + R, g.ny - 1);
  int ilo = max(i - R, 0), ihi = min(i + R, g.nx - 1);
  int c = 0;
  for (int cj = jlo; cj <= jhi; ++cj) {
    int a = start[cj * g.nx + ilo], b = start[cj * g.nx + ihi + 1];
    for (int k = a; k < b; ++k) {
      float2 p = binned[k];
      if (d2_rn(p.x, p.y, cx, cy) < r2) ++c;
    }
  }
  counts[cidx] = c;
}

__global__ void k_accept(const int32_t* __restrict__ counts, int64_t nc, int min_count, int32_t* __restrict__ acc) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nc) acc[k] = counts[k] >= min_count ? 1 : 0;
}

__global__ void k_emit(const int32_t* __restrict__ acc, const int32_t* __restrict__ pos, int64_t nc, int nx,
                       double x0, double y0, double h, double* __restrict__ out) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nc || !acc[k]) return;
  int i = (int)(k % nx), j = (int)(k / nx);
  int64_t p = pos[k];
  out[2 * p] = cand_coord(x0, i, h);
  out[2 * p + 1] = cand_coord(y0, j, h);
}

}  // namespace rbf

using namespace rbf;

extern "C" rbf_status rbf_build_centers(rbf_ctx* cx, const float* pts, int64_t n, int32_t* counts,
                                        int64_t* M_out, void* stream) {
  RBF_TRY(check_ctx(cx, false));
  Ctx* c = C(cx);
  const rbf_config& cfg = c->cfg;
  if (!M_out) return fail(RBF_EINVAL, "null M_out");
  if (n < 0) return fail(RBF_EINVAL, "negative n");
  if (n > 0 && !pts) return fail(RBF_EINVAL, "null points");
  if (!(cfg.mesh_h > 0) || cfg.mesh_nx <= 0 || cfg.mesh_ny <= 0 || !(cfg.r_kd > 0))
    return fail(RBF_EINVAL, "candidate mesh and r_kd must be positive");
  int64_t nc = (int64_t)cfg.mesh_nx * cfg.mesh_ny;
  if (nc > ((int64_t)1 << 30)) return fail(RBF_EINVAL, "candidate mesh too large");
  cudaStream_t s = (cudaStream_t)stream;
  Grid g;
  g.x0 = (float)cfg.mesh_x0;
  g.y0 = (float)cfg.mesh_y0;
  g.cs = (float)cfg.mesh_h;
  g.inv_cs = (float)(1.0 / cfg.mesh_h);
  g.nx = cfg.mesh_nx;
  g.ny = cfg.mesh_ny;
  Buf& pcell = c->scratch(0);
  Buf& cnt = c->scratch(1);
  Buf& start = c->scratch(2);
  Buf& binned = c->scratch(3);
  Buf& cc = c->scratch(4);
  Buf& acc = c->scratch(5);
  Buf& pos = c->scratch(6);
  Buf& outc = c->scratch(7);
  RBF_TRY(pcell.ensure((size_t)(n + 1) * sizeof(int32_t)));
  RBF_TRY(cnt.ensure((size_t)(nc + 1) * sizeof(int32_t)));
  RBF_TRY(start.ensure((size_t)(nc + 1) * sizeof(int32_t)));
  RBF_TRY(binned.ensure((size_t)(n + 1) * sizeof(float2)));
  RBF_TRY(cc.ensure((size_t)(nc + 1) * sizeof(int32_t)));
  RBF_TRY(acc.ensure((size_t)(nc + 1) * sizeof(int32_t)));
  RBF_TRY(pos.ensure((size_t)(nc + 1) * sizeof(int32_t)));
  RBF_CUDA(cudaMemsetAsync(cnt.p, 0, (size_t)(nc + 1) * sizeof(int32_t), s));
  unsigned nbp = (unsigned)((n + 255) / 256), nbc = (unsigned)((nc + 255) / 256);
  if (n > 0) {
    { k_pt_cells<<<nbp, 256, 0, s>>>(pts, n, g, pcell.as<int32_t>(), cnt.as<int32_t>(), c->dflag.as<int>()); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }
  RBF_TRY(scan_i32(c, cnt.as<int32_t>(), start.as<int32_t>(), nc, s, 48));
  RBF_CUDA(cudaMemsetAsync(cnt.p, 0, (size_t)(nc + 1) * sizeof(int32_t), s));
  if (n > 0) {
    { k_pt_fill<<<nbp, 256, 0, s>>>(pcell.as<int32_t>(), n, start.as<int32_t>(), cnt.as<int32_t>(),
                                  binned.as<float2>(), pts); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }
  float r32 = (float)cfg.r_kd;
  float r2 = r32 * r32;
  float rc = (float)(cfg.r_kd / cfg.mesh_h);
  int32_t* cnt_out = counts ? counts : cc.as<int32_t>();
  { k_count_cands<<<nbc, 256, 0, s>>>(cfg.mesh_x0, cfg.mesh_y0, cfg.mesh_h, g, r2, rc, start.as<int32_t>(),
                                    binned.as<float2>(), cnt_out); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  { k_accept<<<nbc, 256, 0, s>>>(cnt_out, nc, cfg.min_count, acc.as<int32_t>()); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  RBF_TRY(scan_i32(c, acc.as<int32_t>(), pos.as<int32_t>(), nc, s, 48));
  int32_t* h32 = (int32_t*)c->host_small;
  RBF_CUDA(cudaMemcpyAsync(h32, pos.as<int32_t>() + nc, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  int flag = 0;
  RBF_TRY(read_dev_flag(c, s, &flag));
  if (flag & DEV_BAD_INDEX) return fail(RBF_EINVAL, "a point has a non-finite coordinate");
  int64_t M = h32[0];
  *M_out = M;
  if (M == 0) {
    c->M = 0;
    RBF_TRY(reset_update_state(c));
    return RBF_OK;
  }
  RBF_TRY(outc.ensure((size_t)M * 2 * sizeof(double)));
  { k_emit<<<nbc, 256, 0, s>>>(acc.as<int32_t>(), pos.as<int32_t>(), nc, cfg.mesh_nx, cfg.mesh_x0, cfg.mesh_y0,
                             cfg.mesh_h, outc.as<double>()); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  // install_centers copies from outc; it uses scratch slots 0-1 and 48+ only
  // after the copy, so outc (slot 7) stays valid.
  return install_centers(c, outc.as<double>(), M, s);
}
