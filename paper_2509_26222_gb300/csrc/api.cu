// Context life cycle, error reporting, scans, the center hash grid and the
// small C-ABI getters/setters of librbfgb.so.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "common.cuh"

namespace rbf {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

rbf_status fail(rbf_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

rbf_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  rbf_status st = (e == cudaErrorMemoryAllocation) ? RBF_ENOMEM : RBF_ECUDA;
  return fail(st, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

rbf_status Buf::ensure(size_t nbytes) {
  if (nbytes <= bytes && p) return RBF_OK;
  if (p) {
    cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  // grow to the next power of two (25% slack above 1 GiB) so that sizes that
  // creep up frame by frame do not reallocate -- and synchronize -- each call
  size_t want = 256;
  if (nbytes > ((size_t)1 << 30)) {
    want = (nbytes + nbytes / 4 + 255) & ~(size_t)255;
  } else {
    while (want < nbytes) want <<= 1;
  }
  cudaError_t e = cudaMalloc(&p, want);
  if (e != cudaSuccess) {
    p = nullptr;
    return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
  }
  bytes = want;
  return RBF_OK;
}

void Buf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

rbf_status check_ctx(rbf_ctx* c, bool need_centers) {
  if (!c) return fail(RBF_EINVAL, "null context");
  Ctx* x = C(c);
  int dev = -1;
  RBF_CUDA(cudaGetDevice(&dev));
  if (dev != x->device)
    return fail(RBF_ESTATE, "context lives on device %d but device %d is current", x->device, dev);
  if (need_centers && x->M <= 0) return fail(RBF_ESTATE, "no centers installed");
  return RBF_OK;
}

double eval_radius(const rbf_config& cfg) {
  return cfg.kernel == RBF_KERNEL_WENDLAND ? cfg.rho : cfg.cutoff_mult * cfg.sigma;
}

double assembly_radius(const rbf_config& cfg, double noise) {
  if (cfg.kernel == RBF_KERNEL_WENDLAND) return cfg.rho;
  return cfg.cutoff_mult * sqrt(cfg.sigma * cfg.sigma + noise * noise);
}

rbf_status read_dev_flag(Ctx* c, cudaStream_t s, int* flag) {
  // the pinned word of a top-level context (sub-contexts of a batch have none)
  int local = 0;
  int32_t* hp = c->host_small ? (int32_t*)c->host_small + 20 : &local;
  RBF_CUDA(cudaMemcpyAsync(hp, c->dflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  RBF_CUDA(cudaStreamSynchronize(s));
  const int h = *hp;
  *flag = h;
  if (h) RBF_CUDA(cudaMemsetAsync(c->dflag.p, 0, sizeof(int), s));
  return RBF_OK;
}

// ---------------------------------------------------------------------------
// Exclusive scans (block-local scan, recursive scan of block totals, add)
// ---------------------------------------------------------------------------
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_PER_THREAD = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER_THREAD;

template <class Tin, class Tout>
__global__ void k_scan_tiles(const Tin* __restrict__ in, Tout* __restrict__ out, int64_t n,
                             Tout* __restrict__ tile_sums) {
  __shared__ Tout warp_tot[SCAN_THREADS / 32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_PER_THREAD;
  Tout v[SCAN_PER_THREAD];
  Tout sum = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    int64_t i = base + k;
    v[k] = (i < n) ? (Tout)in[i] : (Tout)0;
    sum += v[k];
  }
  // inclusive warp scan of the thread sums
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  Tout inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    Tout y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    Tout t = (lane < SCAN_THREADS / 32) ? warp_tot[lane] : (Tout)0;
    Tout ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      Tout y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < SCAN_THREADS / 32) warp_tot[lane] = ti - t;  // exclusive
    if (lane == SCAN_THREADS / 32 - 1) tile_sums[blockIdx.x] = ti;
  }
  __syncthreads();
  Tout run = warp_tot[wid] + inc - sum;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    int64_t i = base + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
}

template <class T>
__global__ void k_scan_add(T* __restrict__ out, int64_t n, const T* __restrict__ offs) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += offs[i / SCAN_TILE];
}

template <class Tin, class Tout>
__global__ void k_scan_total(const Tin* in, Tout* out, int64_t n) {
  if (threadIdx.x == 0 && blockIdx.x == 0) out[n] = (n > 0) ? out[n - 1] + (Tout)in[n - 1] : (Tout)0;
}

// The whole scan in one CTA of 1024 threads for short inputs: chunks of
// 1024 x 8 elements in turn, each scanned in the block and offset by the
// running total of the chunks before it; out[n] = the total.
constexpr int SCAN1_THREADS = 1024;
constexpr int64_t SCAN1_MAX = 32 * SCAN1_THREADS * SCAN_PER_THREAD;
template <class Tin, class Tout>
__global__ void __launch_bounds__(SCAN1_THREADS) k_scan_one(const Tin* __restrict__ in, Tout* __restrict__ out,
                                                             int64_t n) {
  __shared__ Tout warp_tot[SCAN1_THREADS / 32];
  __shared__ Tout carry_s;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int64_t c0 = 0; c0 < n; c0 += (int64_t)SCAN1_THREADS * SCAN_PER_THREAD) {
    const int64_t base = c0 + (int64_t)threadIdx.x * SCAN_PER_THREAD;
    const Tout carry = carry_s;  // read before warp 0 rewrites it (after the next barrier)
    Tout v[SCAN_PER_THREAD];
    Tout sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
      const int64_t i = base + k;
      v[k] = (i < n) ? (Tout)in[i] : (Tout)0;
      sum += v[k];
    }
    Tout inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const Tout y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      const Tout t = warp_tot[lane];
      Tout ti = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const Tout y = __shfl_up_sync(0xffffffffu, ti, o);
        if (lane >= o) ti += y;
      }
      warp_tot[lane] = ti - t;  // exclusive
      if (lane == 31) carry_s = carry + ti;
    }
    __syncthreads();
    Tout run = carry + warp_tot[wid] + inc - sum;
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
      const int64_t i = base + k;
      if (i < n) out[i] = run;
      run += v[k];
    }
    __syncthreads();  // warp_tot and carry_s are rewritten by the next chunk
  }
  if (threadIdx.x == 0) out[n] = carry_s;
}

template <class Tin, class Tout>
static rbf_status scan_impl(Ctx* c, const Tin* in, Tout* out, int64_t n, cudaStream_t s,
                            int slot) {
  if (n <= 0) {
    { k_scan_total<Tin, Tout><<<1, 1, 0, s>>>(in, out, 0); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    return RBF_OK;
  }
  if (n <= SCAN1_MAX) {
    { k_scan_one<Tin, Tout><<<1, SCAN1_THREADS, 0, s>>>(in, out, n); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    return RBF_OK;
  }
  int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  Buf& sums = c->scratch(slot);
  RBF_TRY(sums.ensure((size_t)(tiles + 1) * sizeof(Tout)));
  { k_scan_tiles<Tin, Tout><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, sums.as<Tout>()); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  if (tiles > 1) {
    Buf& offs = c->scratch(slot + 1);
    RBF_TRY(offs.ensure((size_t)(tiles + 1) * sizeof(Tout)));
    RBF_TRY((scan_impl<Tout, Tout>(c, sums.as<Tout>(), offs.as<Tout>(), tiles, s, slot + 2)));
    { k_scan_add<Tout><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, offs.as<Tout>()); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }
  { k_scan_total<Tin, Tout><<<1, 1, 0, s>>>(in, out, n); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  return RBF_OK;
}

rbf_status scan_i32_to_i64(Ctx* c, const int32_t* in, int64_t* out, int64_t n, cudaStream_t s,
                           int slot) {
  return scan_impl<int32_t, int64_t>(c, in, out, n, s, slot);
}

rbf_status scan_i32(Ctx* c, const int32_t* in, int32_t* out, int64_t n, cudaStream_t s,
                    int slot) {
  return scan_impl<int32_t, int32_t>(c, in, out, n, s, slot);
}

// ---------------------------------------------------------------------------
// Center hash grid: counting sort of the centers by cell, ids ascending
// within each cell, and a float32 (x, y, w) copy in slot order.
// ---------------------------------------------------------------------------
__global__ void k_center_cells(const double* __restrict__ c64, int64_t M, Grid g,
                               int32_t* __restrict__ cell, int32_t* __restrict__ count) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  float x = (float)c64[2 * j], y = (float)c64[2 * j + 1];
  int ix = (int)floorf((x - g.x0) * g.inv_cs);
  int iy = (int)floorf((y - g.y0) * g.inv_cs);
  ix = min(max(ix, 0), g.nx - 1);
  iy = min(max(iy, 0), g.ny - 1);
  int cc = iy * g.nx + ix;
  cell[j] = cc;
  atomicAdd(&count[cc], 1);
}

__global__ void k_center_fill(const int32_t* __restrict__ cell, int64_t M,
                              const int32_t* __restrict__ start, int32_t* __restrict__ fill,
                              int32_t* __restrict__ sorted_id) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  int cc = cell[j];
  int pos = start[cc] + atomicAdd(&fill[cc], 1);
  sorted_id[pos] = (int32_t)j;
}

// ids ascending inside each cell (cells hold a handful of centers)
__global__ void k_sort_cells(const int32_t* __restrict__ start, int ncell, int32_t* __restrict__ ids) {
  int cidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (cidx >= ncell) return;
  int a = start[cidx], b = start[cidx + 1];
  for (int i = a + 1; i < b; ++i) {
    int v = ids[i];
    int k = i - 1;
    while (k >= a && ids[k] > v) {
      ids[k + 1] = ids[k];
      --k;
    }
    ids[k + 1] = v;
  }
}

__global__ void k_sorted_xyw(const double* __restrict__ c64, const double* __restrict__ w,
                             const int32_t* __restrict__ sorted_id, int64_t M,
                             float4* __restrict__ xyw) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  int j = sorted_id[s];
  xyw[s] = make_float4((float)c64[2 * j], (float)c64[2 * j + 1], (float)w[j], 0.f);
}

__global__ void k_lattice_w(const double* __restrict__ c64, const double* __restrict__ w,
                            int64_t M, double x0, double y0, double inv_h, int nx, int ny,
                            float* __restrict__ wl) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  int ix = (int)floor((c64[2 * j] - x0) * inv_h);
  int iy = (int)floor((c64[2 * j + 1] - y0) * inv_h);
  if (ix >= 0 && ix < nx && iy >= 0 && iy < ny) wl[(int64_t)iy * nx + ix] = (float)w[j];
}

// W2[j][i] = (Wpad[j][i], Wpad[j][i + 1]) with Wpad = W padded by pad zeros
__global__ void k_build_w2(const float* __restrict__ W, int nx, int ny, int pad, int pitch, int rows,
                           float2* __restrict__ W2) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)pitch * rows) return;
  int j = (int)(e / pitch) - pad, i = (int)(e % pitch) - pad;
  float a = (j >= 0 && j < ny && i >= 0 && i < nx) ? W[(int64_t)j * nx + i] : 0.f;
  float b = (j >= 0 && j < ny && i + 1 >= 0 && i + 1 < nx) ? W[(int64_t)j * nx + i + 1] : 0.f;
  W2[e] = make_float2(a, b);
}

rbf_status refresh_center_weights(Ctx* c, cudaStream_t s) {
  int64_t M = c->M;
  if (M <= 0) return RBF_OK;
  unsigned nb = (unsigned)((M + 255) / 256);
  { k_sorted_xyw<<<nb, 256, 0, s>>>(c->c64.as<double>(), c->w.as<double>(),
                                  c->sorted_id.as<int32_t>(), M, c->sorted_xyw.as<float4>()); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  if (c->lat.on) {
    size_t cells = (size_t)c->lat.nx * c->lat.ny;
    RBF_CUDA(cudaMemsetAsync(c->wlat.p, 0, cells * sizeof(float), s));
    { k_lattice_w<<<nb, 256, 0, s>>>(c->c64.as<double>(), c->w.as<double>(), M, c->lat.x0,
                                   c->lat.y0, 1.0 / c->lat.h, c->lat.nx, c->lat.ny,
                                   c->wlat.as<float>()); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    if (c->lat_rc > 0) {
      int rc = c->lat_rc, pitch = c->lat.nx + 4 * rc, rows = c->lat.ny + 4 * rc;
      int64_t tot = (int64_t)pitch * rows;
      { k_build_w2<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(c->wlat.as<float>(), c->lat.nx, c->lat.ny, 2 * rc,
                                                               pitch, rows, c->wlat2.as<float2>()); ::rbf::note_launch(); }
      RBF_CUDA(cudaGetLastError());
    }
  }
  return RBF_OK;
}

// Square lattice detection: every center at (x0 + (i + 0.5) h, y0 + (j + 0.5) h).
static Lattice detect_lattice(const std::vector<double>& c) {
  Lattice L;
  size_t M = c.size() / 2;
  if (M < 4) return L;
  std::vector<double> xs(M), ys(M);
  for (size_t j = 0; j < M; ++j) {
    xs[j] = c[2 * j];
    ys[j] = c[2 * j + 1];
  }
  auto uniq = [](std::vector<double> v) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    return v;
  };
  std::vector<double> ux = uniq(xs), uy = uniq(ys);
  if (ux.size() < 2 || uy.size() < 2) return L;
  double hx = 1e300, hy = 1e300;
  for (size_t k = 1; k < ux.size(); ++k) hx = std::min(hx, ux[k] - ux[k - 1]);
  for (size_t k = 1; k < uy.size(); ++k) hy = std::min(hy, uy[k] - uy[k - 1]);
  if (!(hx > 0) || fabs(hx - hy) > 1e-9 * hx) return L;
  double h = hx;
  double xmin = ux.front(), ymin = uy.front();
  for (size_t j = 0; j < M; ++j) {
    double fx = (xs[j] - xmin) / h, fy = (ys[j] - ymin) / h;
    if (fabs(fx - nearbyint(fx)) > 1e-6 || fabs(fy - nearbyint(fy)) > 1e-6) return L;
  }
  L.on = true;
  L.h = h;
  L.x0 = xmin - 0.5 * h;
  L.y0 = ymin - 0.5 * h;
  L.nx = (int)nearbyint((ux.back() - xmin) / h) + 1;
  L.ny = (int)nearbyint((uy.back() - ymin) / h) + 1;
  if ((double)L.nx * L.ny > 64.0 * 1024 * 1024) L.on = false;  // too sparse to densify
  return L;
}

rbf_status build_center_grid(Ctx* c, cudaStream_t s) {
  int64_t M = c->M;
  std::vector<double> hc((size_t)M * 2);
  RBF_CUDA(cudaMemcpyAsync(hc.data(), c->c64.p, hc.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, s));
  RBF_CUDA(cudaStreamSynchronize(s));
  double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
  for (int64_t j = 0; j < M; ++j) {
    double x = hc[2 * j], y = hc[2 * j + 1];
    if (!std::isfinite(x) || !std::isfinite(y))
      return fail(RBF_EINVAL, "center %lld is not finite", (long long)j);
    xmin = std::min(xmin, x);
    xmax = std::max(xmax, x);
    ymin = std::min(ymin, y);
    ymax = std::max(ymax, y);
  }
  c->lat = detect_lattice(hc);
  double r = eval_radius(c->cfg);
  double cs;
  Grid g;
  if (c->lat.on && c->lat.h <= r) {
    cs = c->lat.h;
    g.x0 = (float)c->lat.x0;
    g.y0 = (float)c->lat.y0;
    g.nx = c->lat.nx;
    g.ny = c->lat.ny;
  } else {
    double area = std::max((xmax - xmin) * (ymax - ymin), 1e-12);
    cs = sqrt(1.5 * area / (double)M);
    cs = std::min(std::max(cs, r / 8.0), r);
    g.x0 = (float)(xmin - 0.5 * cs);
    g.y0 = (float)(ymin - 0.5 * cs);
    double nxd = floor((xmax - (double)g.x0) / cs) + 1, nyd = floor((ymax - (double)g.y0) / cs) + 1;
    if (nxd * nyd > 64.0 * 1024 * 1024) {
      double scale = sqrt(nxd * nyd / (64.0 * 1024 * 1024));
      cs *= scale;
      nxd = floor((xmax - (double)g.x0) / cs) + 1;
      nyd = floor((ymax - (double)g.y0) / cs) + 1;
    }
    g.nx = (int)nxd;
    g.ny = (int)nyd;
  }
  g.cs = (float)cs;
  g.inv_cs = (float)(1.0 / cs);
  c->grid = g;
  int ncell = g.nx * g.ny;
  RBF_TRY(c->cell_start.ensure((size_t)(ncell + 1) * sizeof(int32_t)));
  RBF_TRY(c->sorted_id.ensure((size_t)M * sizeof(int32_t)));
  RBF_TRY(c->sorted_xyw.ensure((size_t)M * sizeof(float4)));
  Buf& cell = c->scratch(0);
  Buf& cnt = c->scratch(1);
  RBF_TRY(cell.ensure((size_t)M * sizeof(int32_t)));
  RBF_TRY(cnt.ensure((size_t)(ncell + 1) * sizeof(int32_t)));
  RBF_CUDA(cudaMemsetAsync(cnt.p, 0, (size_t)(ncell + 1) * sizeof(int32_t), s));
  unsigned nb = (unsigned)((M + 255) / 256);
  { k_center_cells<<<nb, 256, 0, s>>>(c->c64.as<double>(), M, g, cell.as<int32_t>(),
                                    cnt.as<int32_t>()); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  RBF_TRY(scan_i32(c, cnt.as<int32_t>(), c->cell_start.as<int32_t>(), ncell, s, 48));
  RBF_CUDA(cudaMemsetAsync(cnt.p, 0, (size_t)(ncell + 1) * sizeof(int32_t), s));
  { k_center_fill<<<nb, 256, 0, s>>>(cell.as<int32_t>(), M, c->cell_start.as<int32_t>(),
                                   cnt.as<int32_t>(), c->sorted_id.as<int32_t>()); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  { k_sort_cells<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(c->cell_start.as<int32_t>(), ncell,
                                                               c->sorted_id.as<int32_t>()); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  c->lat_rc = 0;
  if (c->lat.on && c->cfg.kernel == RBF_KERNEL_WENDLAND) {
    int rc = (int)ceil(c->cfg.rho / c->lat.h - 1e-6);
    if (rc >= 1 && rc <= 4) c->lat_rc = rc;
  }
  if (c->lat.on) {
    RBF_TRY(c->wlat.ensure((size_t)c->lat.nx * c->lat.ny * sizeof(float)));
    if (c->lat_rc > 0)
      RBF_TRY(c->wlat2.ensure((size_t)(c->lat.nx + 4 * c->lat_rc) * (c->lat.ny + 4 * c->lat_rc) * sizeof(float2)));
    // node coordinates exactly as the float32 copies of the float64 centers
    std::vector<float> xs((size_t)c->lat.nx), ys((size_t)c->lat.ny);
    for (int i = 0; i < c->lat.nx; ++i) xs[i] = (float)(c->lat.x0 + ((double)i + 0.5) * c->lat.h);
    for (int j = 0; j < c->lat.ny; ++j) ys[j] = (float)(c->lat.y0 + ((double)j + 0.5) * c->lat.h);
    // the lattice origin comes from a center, so take the exact coordinates of
    // the centers themselves where a row or column holds one
    for (int64_t k = 0; k < M; ++k) {
      int ix = (int)floor((hc[2 * k] - c->lat.x0) / c->lat.h);
      int iy = (int)floor((hc[2 * k + 1] - c->lat.y0) / c->lat.h);
      if (ix >= 0 && ix < c->lat.nx) xs[ix] = (float)hc[2 * k];
      if (iy >= 0 && iy < c->lat.ny) ys[iy] = (float)hc[2 * k + 1];
    }
    if (c->lat_rc > 0) {
      // float-float node coordinates over the window range of the fixed-window
      // kernel: the query's offset from its node is then exact to float32
      // rounding of the offset itself, not of the coordinate
      const int rc = c->lat_rc;
      auto tab = [&](int n, double o, int axis) {
        std::vector<float2> t((size_t)(n + 2 * rc + 1));
        for (int i = -(rc + 1); i < n + rc; ++i) {
          double v = o + ((double)i + 0.5) * c->lat.h;
          float hi = (float)v;
          t[(size_t)(i + rc + 1)] = make_float2(hi, (float)(v - (double)hi));
        }
        for (int64_t k = 0; k < M; ++k) {
          double v = hc[2 * k + axis];
          int i = (int)floor((v - o) / c->lat.h);
          if (i >= 0 && i < n) {
            float hi = (float)v;
            t[(size_t)(i + rc + 1)] = make_float2(hi, (float)(v - (double)hi));
          }
        }
        return t;
      };
      std::vector<float2> xt = tab(c->lat.nx, c->lat.x0, 0), yt = tab(c->lat.ny, c->lat.y0, 1);
      RBF_TRY(c->lat_xhl.ensure(xt.size() * sizeof(float2)));
      RBF_TRY(c->lat_yhl.ensure(yt.size() * sizeof(float2)));
      RBF_CUDA(cudaMemcpyAsync(c->lat_xhl.p, xt.data(), xt.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
      RBF_CUDA(cudaMemcpyAsync(c->lat_yhl.p, yt.data(), yt.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
      RBF_CUDA(cudaStreamSynchronize(s));
    }
    RBF_TRY(c->lat_xs.ensure(xs.size() * sizeof(float)));
    RBF_TRY(c->lat_ys.ensure(ys.size() * sizeof(float)));
    RBF_CUDA(cudaMemcpyAsync(c->lat_xs.p, xs.data(), xs.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    RBF_CUDA(cudaMemcpyAsync(c->lat_ys.p, ys.data(), ys.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    RBF_CUDA(cudaStreamSynchronize(s));
  }
  return refresh_center_weights(c, s);
}

rbf_status reset_update_state(Ctx* c) {
  c->a = 0;
  c->pg_on = false;
  c->arena_used = 0;
  c->zi_valid = false;
  c->bw_lf = BW_DENSE;
  c->Hs.valid = false;
  c->Hs_next.valid = false;
  // the outside covariance store keeps its allocation: it is zeroed and set to
  // the prior when the next departure turns it on
  return RBF_OK;
}

rbf_status install_centers(Ctx* c, const double* cxy, int64_t M, cudaStream_t s) {
  RBF_TRY(c->c64.ensure((size_t)M * 2 * sizeof(double)));
  RBF_CUDA(cudaMemcpyAsync(c->c64.p, cxy, (size_t)M * 2 * sizeof(double),
                           cudaMemcpyDeviceToDevice, s));
  RBF_TRY(c->w.ensure((size_t)M * sizeof(double)));
  RBF_CUDA(cudaMemsetAsync(c->w.p, 0, (size_t)M * sizeof(double), s));
  RBF_TRY(c->A.ensure((size_t)M * sizeof(int32_t)));
  RBF_TRY(c->g2l.ensure((size_t)M * sizeof(int32_t)));
  RBF_CUDA(cudaMemsetAsync(c->g2l.p, 0xff, (size_t)M * sizeof(int32_t), s));
  RBF_TRY(c->departed.ensure((size_t)M * sizeof(int32_t)));
  RBF_CUDA(cudaMemsetAsync(c->departed.p, 0, (size_t)M * sizeof(int32_t), s));
  RBF_TRY(c->blkref.ensure((size_t)M * sizeof(BlkRef)));
  RBF_CUDA(cudaMemsetAsync(c->blkref.p, 0xff, (size_t)M * sizeof(BlkRef), s));  // base = -1: never left
  c->M = M;
  RBF_TRY(reset_update_state(c));
  rbf_status st = build_center_grid(c, s);
  if (st != RBF_OK) {
    c->M = 0;
    return st;
  }
  RBF_CUDA(cudaStreamSynchronize(s));
  return RBF_OK;
}

static cudaEvent_t take_event(Ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

StageTimer::StageTimer(Ctx* c_, int stage_, cudaStream_t s_, double work_)
    : c(c_), stage(stage_), s(s_), work(work_) {
  if (!c->prof) return;
  a = take_event(c);
  if (a) cudaEventRecord(a, s);
}

StageTimer::~StageTimer() {
  if (!a) return;
  cudaEvent_t b = take_event(c);
  if (!b) return;
  cudaEventRecord(b, s);
  c->marks.push_back({stage, a, b, work});
}

static void profile_collect(Ctx* c) {
  for (auto& m : c->marks) {
    float ms = 0.f;
    cudaEventSynchronize(m.b);
    if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
      c->prof_ms[m.stage] += ms;
      c->prof_work[m.stage] += m.work;
      c->prof_count[m.stage] += 1;
    }
    c->ev_pool.push_back(m.a);
    c->ev_pool.push_back(m.b);
  }
  c->marks.clear();
}

}  // namespace rbf

using namespace rbf;

extern "C" rbf_status rbf_launch_count(int64_t* n) {
  if (!n) return fail(RBF_EINVAL, "null output");
  *n = (int64_t)g_launches.load();
  return RBF_OK;
}

extern "C" rbf_status rbf_profile_enable(rbf_ctx* cx, int on) {
  RBF_TRY(check_ctx(cx, false));
  C(cx)->prof = on != 0;
  return RBF_OK;
}

extern "C" rbf_status rbf_profile_read(rbf_ctx* cx, double* ms, double* work, int64_t* count, int reset) {
  RBF_TRY(check_ctx(cx, false));
  Ctx* c = C(cx);
  profile_collect(c);
  for (int k = 0; k < RBF_NSTAGE; ++k) {
    if (ms) ms[k] = c->prof_ms[k];
    if (work) work[k] = c->prof_work[k];
    if (count) count[k] = c->prof_count[k];
    if (reset) {
      c->prof_ms[k] = 0.0;
      c->prof_work[k] = 0.0;
      c->prof_count[k] = 0;
    }
  }
  return RBF_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" const char* rbf_last_error(void) { return g_last_error.c_str(); }

extern "C" rbf_status rbf_create(const rbf_config* cfg, rbf_ctx** out) {
  g_last_error.clear();
  if (!cfg || !out) return fail(RBF_EINVAL, "null argument");
  *out = nullptr;
  if (cfg->kernel != RBF_KERNEL_WENDLAND && cfg->kernel != RBF_KERNEL_GAUSSIAN)
    return fail(RBF_EINVAL, "unknown kernel %d", cfg->kernel);
  if (cfg->update_precision != RBF_UPDATE_FP64 && cfg->update_precision != RBF_UPDATE_MIXED)
    return fail(RBF_EINVAL, "unknown update precision %d", cfg->update_precision);
  if (cfg->loss != RBF_LOSS_HUBER && cfg->loss != RBF_LOSS_L2)
    return fail(RBF_EINVAL, "unknown loss %d", cfg->loss);
  if (cfg->kernel == RBF_KERNEL_WENDLAND && !(cfg->rho > 0))
    return fail(RBF_EINVAL, "rho must be > 0");
  if (cfg->kernel == RBF_KERNEL_GAUSSIAN && !(cfg->sigma > 0 && cfg->cutoff_mult > 0))
    return fail(RBF_EINVAL, "sigma and cutoff_mult must be > 0");
  if (!(cfg->lambda > 0)) return fail(RBF_EINVAL, "lambda must be > 0");
  if (cfg->loss == RBF_LOSS_HUBER && !(cfg->huber_delta > 0))
    return fail(RBF_EINVAL, "huber_delta must be > 0");
  if (cfg->refine_sweeps < 0 || cfg->refine_sweeps > 16)
    return fail(RBF_EINVAL, "refine_sweeps must be in [0, 16]");
  if (cfg->exact != 0 && cfg->exact != 1) return fail(RBF_EINVAL, "exact must be 0 or 1");
  if (cfg->reserved1 != 0) return fail(RBF_EINVAL, "reserved1 must be 0");
  rbf_ctx* c = new (std::nothrow) rbf_ctx();
  if (!c) return fail(RBF_ENOMEM, "host allocation failed");
  Ctx* x = C(c);
  x->cfg = *cfg;
  if (cfg->refine_sweeps > 0) x->refine_sweeps = x->refine_sweeps_cov = cfg->refine_sweeps;
  if (cfg->inverse_max != 0) x->inv_max = cfg->inverse_max < 0 ? -1 : cfg->inverse_max;
  cudaError_t e = cudaGetDevice(&x->device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__);
  }
  rbf_status st = x->dflag.ensure(16 * sizeof(int));
  if (st == RBF_OK) {
    e = cudaMemset(x->dflag.p, 0, 16 * sizeof(int));
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMemset", __FILE__, __LINE__);
  }
  if (st == RBF_OK) {
    e = cudaMallocHost((void**)&x->host_small, 64 * sizeof(int64_t));
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMallocHost", __FILE__, __LINE__);
  }
  if (st != RBF_OK) {
    x->dflag.release();
    delete c;
    return st;
  }
  noalloc_forget(x->device);
  *out = c;
  return RBF_OK;
}

extern "C" rbf_status rbf_test_hook(rbf_ctx* c, int32_t hook, double value) {
  RBF_TRY(check_ctx(c, false));
  Ctx* x = C(c);
  switch (hook) {
    case RBF_HOOK_DIAG_SHIFT:
      if (!isfinite(value)) return fail(RBF_EINVAL, "diagonal shift must be finite");
      x->diag_shift = value;
      return RBF_OK;
    case RBF_HOOK_WAIT_LIMIT:
      if (!(value >= 0 && value <= 1e12)) return fail(RBF_EINVAL, "wait limit must be in [0, 1e12]");
      x->spin_limit = (long long)value;
      return RBF_OK;
    case RBF_HOOK_FACTOR_CHAIN:
      if (value != 0.0 && value != 1.0) return fail(RBF_EINVAL, "factor-chain takes 0 or 1");
      x->df_ok = value == 0.0;
      return RBF_OK;
    case RBF_HOOK_WAIT_NEVER:
      if (value != 0.0 && value != 1.0) return fail(RBF_EINVAL, "wait-never takes 0 or 1");
      x->wait_xor = value != 0.0 ? 0x40000000 : 0;
      return RBF_OK;
    default:
      return fail(RBF_EINVAL, "unknown hook %d", hook);
  }
}

extern "C" rbf_status rbf_destroy(rbf_ctx* c) {
  if (!c) return RBF_OK;
  Ctx* x = C(c);
  cudaDeviceSynchronize();
  batch_destroy(x);
  Buf* bufs[] = {&x->c64, &x->w, &x->cell_start, &x->sorted_id, &x->sorted_xyw, &x->wlat, &x->lat_xs, &x->lat_ys, &x->wlat2, &x->lat_xhl, &x->lat_yhl,
                 &x->A, &x->g2l, &x->H, &x->L, &x->Lf, &x->Zd, &x->Zi, &x->Hs.rp, &x->Hs.col, &x->Hs.val, &x->Hs_next.rp, &x->Hs_next.col, &x->Hs_next.val, &x->blkref, &x->arena, &x->departed, &x->dflag, &x->sync_flags, &x->df_flags};
  for (Buf* b : bufs) b->release();
  for (Buf& b : x->ws) b.release();
  for (auto& st : x->bs)
    if (st) cudaStreamDestroy(st);
  for (auto& ev : x->bev)
    if (ev) cudaEventDestroy(ev);
  if (x->la_stream) cudaStreamDestroy(x->la_stream);
  for (auto& ev : x->la_ev)
    if (ev) cudaEventDestroy(ev);
  if (x->host_small) cudaFreeHost(x->host_small);
  for (auto& m : x->marks) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  for (cudaEvent_t e : x->ev_pool) cudaEventDestroy(e);
  delete c;
  return RBF_OK;
}

extern "C" rbf_status rbf_set_centers(rbf_ctx* c, const double* cxy, int64_t M, void* stream) {
  RBF_TRY(check_ctx(c, false));
  if (M <= 0 || !cxy) return fail(RBF_EINVAL, "need M > 0 centers and a non-null pointer");
  if (M > (int64_t)1 << 30) return fail(RBF_EINVAL, "too many centers");
  return install_centers(C(c), cxy, M, (cudaStream_t)stream);
}

extern "C" rbf_status rbf_num_centers(rbf_ctx* c, int64_t* M_out) {
  RBF_TRY(check_ctx(c, false));
  if (!M_out) return fail(RBF_EINVAL, "null M_out");
  *M_out = C(c)->M;
  return RBF_OK;
}

extern "C" rbf_status rbf_get_centers(rbf_ctx* c, double* cxy, void* stream) {
  RBF_TRY(check_ctx(c, true));
  if (!cxy) return fail(RBF_EINVAL, "null output");
  Ctx* x = C(c);
  RBF_CUDA(cudaMemcpyAsync(cxy, x->c64.p, (size_t)x->M * 2 * sizeof(double),
                           cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return RBF_OK;
}

extern "C" rbf_status rbf_get_weights(rbf_ctx* c, double* w, void* stream) {
  RBF_TRY(check_ctx(c, true));
  if (!w) return fail(RBF_EINVAL, "null output");
  Ctx* x = C(c);
  RBF_CUDA(cudaMemcpyAsync(w, x->w.p, (size_t)x->M * sizeof(double), cudaMemcpyDeviceToDevice,
                           (cudaStream_t)stream));
  return RBF_OK;
}

extern "C" rbf_status rbf_set_weights(rbf_ctx* c, const double* w, void* stream) {
  RBF_TRY(check_ctx(c, true));
  if (!w) return fail(RBF_EINVAL, "null input");
  Ctx* x = C(c);
  cudaStream_t s = (cudaStream_t)stream;
  RBF_CUDA(cudaMemcpyAsync(x->w.p, w, (size_t)x->M * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return refresh_center_weights(x, s);
}
