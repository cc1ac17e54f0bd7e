// Batched terrain patches: many independent terrains, each updated once from
// the prior (Sec. III-C; equal to batch ridge of Sec. III-B) and evaluated
// (Eq. RBF_fml), in one call.
//
// Every patch's pipeline has sizes bounded by its M, n and Q, so it needs no
// host synchronization: every point finds its neighbour nodes in the patch
// lattice and adds its products to m~ m~^T and m~ z by exact (order-independent)
// integer accumulation, the M x M information matrix lambda I + m~ m~^T is
// factored within its band (FP64, or the mixed-precision tensor-core path)
// and solved, and the queries are evaluated over the lattice window.  Patches are spread over internal streams, each
// with its own workspace context; the first call for a batch shape runs
// eagerly (sizing every buffer), later calls with the same descriptors replay
// a CUDA graph recorded from the same enqueue sequence.
//
// A tiny autotuner picks, per power-of-two bucket of M, the faster of the two
// factorization paths (timed once on a synthetic SPD matrix of that size).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace rbf {

struct PatchGeom {
  double x0, y0, h;
  int nx, rows;
  int64_t M, n, Q;
  int rca, rce;      // support radii in nodes (assembly, evaluation)
  float r2a, r2e;    // float32 squared radii
  double inv_rho, g_scale, g_inv2s2;  // regression-row parameters
  float e_inv_rho, e_inv2s2, e_gscale;
  int kernel;
};

__device__ __forceinline__ double node_coord(double x0, int i, double h) {
  return __dadd_rn(x0, __dmul_rn((double)i + 0.5, h));
}

// One warp per point: its neighbour nodes (the float32 rule at the assembly
// radius over the 2 rca x 2 rca node window), their regression entries, and
// the exact integer accumulation of every product m_{i,l1} m_{i,l2} (lower
// triangle) and m_{i,l} z_i (the accumulation of the main update path).
// Non-finite points set DEV_BAD_INDEX and are skipped.
constexpr int BP_MAXK = 128;  // window nodes per point kept in shared memory
__global__ void __launch_bounds__(256) k_bp_gram(PatchGeom G, const float* __restrict__ pts, double gscale,
                                                 unsigned long long* __restrict__ Gacc,
                                                 unsigned long long* __restrict__ Uacc, int* __restrict__ status) {
  __shared__ int32_t sid[8][BP_MAXK];
  __shared__ double sm[8][BP_MAXK];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (p >= G.n) return;
  const float px = pts[3 * p], py = pts[3 * p + 1], pz = pts[3 * p + 2];
  if (!(isfinite(px) && isfinite(py) && isfinite(pz))) {
    if (lane == 0) atomicOr(status, DEV_BAD_INDEX);
    return;
  }
  const int W = 2 * G.rca;
  const double pu = ((double)px - G.x0) / G.h - 0.5, pv = ((double)py - G.y0) / G.h - 0.5;
  const int ib = (int)floor(fmin(fmax(pu, -2.0 * W), (double)G.nx + 2.0 * W)) - G.rca + 1;
  const int jb = (int)floor(fmin(fmax(pv, -2.0 * W), (double)G.rows + 2.0 * W)) - G.rca + 1;
  int K = 0;
  for (int t0 = 0; t0 < W * W; t0 += 32) {
    int t = t0 + lane;
    bool in = false;
    int64_t id = 0;
    double m = 0.0;
    if (t < W * W) {
      int i2 = ib + t % W, j2 = jb + t / W;
      if (i2 >= 0 && i2 < G.nx && j2 >= 0 && j2 < G.rows) {
        id = (int64_t)j2 * G.nx + i2;
        if (id < G.M) {
          double cx = node_coord(G.x0, i2, G.h), cy = node_coord(G.y0, j2, G.h);
          if (d2_rn(px, py, (float)cx, (float)cy) < G.r2a) {
            double ex = (double)px - cx, ey = (double)py - cy;
            m = row_value(G.kernel, ex * ex + ey * ey, G.inv_rho, G.g_scale, G.g_inv2s2);
            in = true;
          }
        }
      }
    }
    unsigned mask = __ballot_sync(0xffffffffu, in);
    int pos = K + __popc(mask & ((1u << lane) - 1u));
    if (in && pos < BP_MAXK) {
      sid[wid][pos] = (int32_t)id;
      sm[wid][pos] = m;
    }
    K += __popc(mask);
  }
  if (K > BP_MAXK) {
    if (lane == 0) atomicOr(status, DEV_BAD_INDEX);
    return;
  }
  __syncwarp();
  for (int t = lane; t < K; t += 32) add_u128(Uacc + 2 * (int64_t)sid[wid][t], sm[wid][t] * (double)pz);
  for (int t1 = 0; t1 < K; ++t1) {
    const int64_t l1 = sid[wid][t1];
    const double m1 = sm[wid][t1];
    for (int t2 = lane; t2 <= t1; t2 += 32) {
      int64_t l2 = sid[wid][t2];
      int64_t hi = l1 > l2 ? l1 : l2, lo = l1 > l2 ? l2 : l1;
      atomicAdd(Gacc + hi * G.M + lo, (unsigned long long)__double2ll_rn(m1 * sm[wid][t2] * gscale));
    }
  }
}

// H = lambda I + (accumulated m~ m~^T), both triangles; u = m~ z
__global__ void k_bp_merge(int64_t M, double inv_gscale, double lam, const unsigned long long* __restrict__ Gacc,
                           const unsigned long long* __restrict__ Uacc, double* __restrict__ H,
                           double* __restrict__ u) {
  const int64_t l1 = blockIdx.y;
  for (int64_t l2 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l2 <= l1; l2 += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long q = Gacc[l1 * M + l2];
    if (q == 0ull && l2 != l1) continue;
    double v = (double)(long long)q * inv_gscale;
    if (l2 == l1) v += lam;
    H[l1 * M + l2] = v;
    if (l2 != l1) H[l2 * M + l1] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0)
    u[l1] = (double)(long long)Uacc[2 * l1 + 1] + ldexp((double)Uacc[2 * l1], -64);
}

__global__ void k_bp_eval(PatchGeom G, const double* __restrict__ w, const float2* __restrict__ q,
                          float* __restrict__ h, float2* __restrict__ grad) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= G.Q) return;
  float2 p = q[k];
  float ah = 0.f, ax = 0.f, ay = 0.f;
  if (isfinite(p.x) && isfinite(p.y)) {
    double pu = ((double)p.x - G.x0) / G.h - 0.5, pv = ((double)p.y - G.y0) / G.h - 0.5;
    pu = fmin(fmax(pu, -4.0 * G.rce - 4.0), (double)G.nx + 4.0 * G.rce);
    pv = fmin(fmax(pv, -4.0 * G.rce - 4.0), (double)G.rows + 4.0 * G.rce);
    int ib = (int)floor(pu) - G.rce + 1, jb = (int)floor(pv) - G.rce + 1;
    for (int dj = 0; dj < 2 * G.rce; ++dj) {
      int j = jb + dj;
      if (j < 0 || j >= G.rows) continue;
      float cy = (float)node_coord(G.y0, j, G.h);
      float dy = p.y - cy;
      for (int di = 0; di < 2 * G.rce; ++di) {
        int i = ib + di;
        if (i < 0 || i >= G.nx) continue;
        int64_t id = (int64_t)j * G.nx + i;
        if (id >= G.M) continue;
        float cx = (float)node_coord(G.x0, i, G.h);
        float dx = p.x - cx;
        float d2 = fmaf(dx, dx, dy * dy);
        if (!(d2 < G.r2e)) continue;
        float wf = (float)w[id];
        if (G.kernel == RBF_KERNEL_WENDLAND) {
          float s = sqrtf(d2) * G.e_inv_rho;
          float t = fmaxf(1.f - s, 0.f);
          float cw = wf * t * t * t;
          ah = fmaf(cw, t * fmaf(4.f, s, 1.f), ah);
          ax = fmaf(cw, dx, ax);
          ay = fmaf(cw, dy, ay);
        } else {
          float e = wf * __expf(-d2 * G.e_inv2s2);
          ah += e;
          ax = fmaf(e, dx, ax);
          ay = fmaf(e, dy, ay);
        }
      }
    }
  } else {
    ah = ax = ay = __int_as_float(0x7fc00000);
  }
  h[k] = ah;
  if (grad) grad[k] = make_float2(ax * G.e_gscale, ay * G.e_gscale);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct BatchState {
  void* persistent = nullptr;  // state of the mixed-precision path (bqueue.cu)
  std::vector<Ctx*> sub;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  // autotuned choice per log2(M) bucket: 0 unknown, 1 FP64, 2 mixed
  int choice[32] = {0};
  struct Graph {
    std::vector<unsigned char> key;
    cudaGraphExec_t exec = nullptr;
  };
  std::vector<Graph> graphs;
  std::vector<std::vector<unsigned char>> seen;  // shapes run eagerly once
  cudaStream_t cap_stream = nullptr;              // root of graph capture
};

static PatchGeom make_geom(const rbf_config& cfg, const rbf_patch& p) {
  PatchGeom G;
  G.x0 = p.x0;
  G.y0 = p.y0;
  G.h = p.spacing;
  G.nx = p.nx;
  G.rows = (int)((p.M + p.nx - 1) / p.nx);
  G.M = p.M;
  G.n = p.n;
  G.Q = p.Q;
  G.kernel = cfg.kernel;
  double ra = assembly_radius(cfg, 0.0), re = eval_radius(cfg);
  G.rca = (int)ceil(ra / p.spacing - 1e-9);
  G.rce = (int)ceil(re / p.spacing - 1e-9);
  float ra32 = (float)ra, re32 = (float)re;
  G.r2a = ra32 * ra32;
  G.r2e = re32 * re32;
  G.inv_rho = 1.0 / cfg.rho;
  double st2 = cfg.sigma * cfg.sigma;
  G.g_scale = 1.0;
  G.g_inv2s2 = 1.0 / (2.0 * st2);
  G.e_inv_rho = (float)(1.0 / cfg.rho);
  G.e_inv2s2 = (float)(1.0 / (2.0 * cfg.sigma * cfg.sigma));
  G.e_gscale = cfg.kernel == RBF_KERNEL_WENDLAND ? (float)(-20.0 / (cfg.rho * cfg.rho))
                                                 : (float)(-1.0 / (cfg.sigma * cfg.sigma));
  return G;
}

static inline unsigned nb256(int64_t n) { return (unsigned)((n + 255) / 256); }

// half-bandwidth of m~ m~^T for a patch (row-major node ids)
static int64_t patch_bandwidth(const PatchGeom& G) {
  int64_t bw = 2 * (int64_t)G.rca * ((int64_t)G.nx + 1);
  return bw < G.M ? bw : BW_DENSE;
}

// Enqueue one patch on stream s with the workspace of sub-context sc.
static rbf_status run_patch(Ctx* sc, const rbf_config& cfg, const rbf_patch& P, bool mixed, cudaStream_t s) {
  PatchGeom G = make_geom(cfg, P);
  const int64_t M = G.M, n = G.n;
  Buf& Gacc = sc->scratch(0);
  Buf& Uacc = sc->scratch(1);
  Buf& H = sc->scratch(4);
  Buf& L = sc->scratch(5);
  Buf& u = sc->scratch(6);
  Buf& Wf = sc->scratch(7);
  Buf& Zd = sc->scratch(8);
  if (M > 65535) return fail(RBF_EINVAL, "batch: a patch has more than 65535 centers");
  RBF_TRY(Gacc.ensure((size_t)M * M * sizeof(unsigned long long)));
  RBF_TRY(Uacc.ensure((size_t)2 * M * sizeof(unsigned long long)));
  RBF_TRY(H.ensure((size_t)M * M * sizeof(double)));
  RBF_TRY(u.ensure((size_t)M * sizeof(double)));
  const int64_t ldw = (M + 3) & ~(int64_t)3;
  if (mixed) {
    RBF_TRY(Wf.ensure((size_t)M * ldw * sizeof(float)));
    RBF_TRY(Zd.ensure((size_t)((M + 63) / 64) * 64 * 64 * sizeof(float)));
  } else {
    RBF_TRY(L.ensure((size_t)M * M * sizeof(double)));
  }
  if (4 * G.rca * G.rca > 128) return fail(RBF_EINVAL, "batch: support radius too large for the lattice spacing");
  // the sync-free solves of this workspace start from cleared flags
  if (sc->sync_flags.p) RBF_CUDA(cudaMemsetAsync(sc->sync_flags.p, 0, sc->sync_flags.bytes, s));
  // lambda I + m~ m~^T and m~ z by exact integer accumulation over the points
  RBF_CUDA(cudaMemsetAsync(Gacc.p, 0, (size_t)M * M * sizeof(unsigned long long), s));
  RBF_CUDA(cudaMemsetAsync(Uacc.p, 0, (size_t)2 * M * sizeof(unsigned long long), s));
  RBF_CUDA(cudaMemsetAsync(H.p, 0, (size_t)M * M * sizeof(double), s));
  const double gscale = ldexp(1.0, 62 - (int)ceil(log2((double)n + 1.0)));
  if (n > 0) {
    { k_bp_gram<<<nb256(n * 32), 256, 0, s>>>(G, P.pts, gscale, Gacc.as<unsigned long long>(),
                                             Uacc.as<unsigned long long>(), sc->dflag.as<int>()); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }
  {
    dim3 mg((unsigned)((M + 255) / 256 < 8 ? (M + 255) / 256 : 8), (unsigned)M);
    { k_bp_merge<<<mg, 256, 0, s>>>(M, 1.0 / gscale, cfg.lambda, Gacc.as<unsigned long long>(),
                                    Uacc.as<unsigned long long>(), H.as<double>(), u.as<double>()); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }
  // the update from the prior has the band structure of m~ m~^T: centers
  // coupled through a point are at most 2 rca nodes apart in each direction
  const int64_t bw = patch_bandwidth(G);
  if (mixed) {
    RBF_TRY(potrf_mixed(sc, H.as<double>(), M, M, Wf.as<float>(), ldw, Zd.as<float>(), s, bw));
    RBF_TRY(mixed_solve(sc, H.as<double>(), M, nullptr, Wf.as<float>(), ldw, Zd.as<float>(), nullptr, M, u.as<double>(), 1,
                        sc->refine_sweeps, s, bw));
  } else {
    RBF_CUDA(cudaMemcpyAsync(L.p, H.p, (size_t)M * M * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RBF_TRY(potrf_lower(sc, L.as<double>(), M, M, M, false, s, bw));
    RBF_TRY(chol_solve(sc, H.as<double>(), L.as<double>(), M, M, u.as<double>(), false, s, bw));
  }
  RBF_CUDA(cudaMemcpyAsync(P.w, u.p, (size_t)M * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (G.Q > 0) {
    { k_bp_eval<<<nb256(G.Q), 256, 0, s>>>(G, P.w, (const float2*)P.q, P.h, (float2*)P.grad); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }
  return RBF_OK;
}

static Ctx* new_sub(const Ctx* parent) {
  Ctx* sc = new (std::nothrow) Ctx();
  if (!sc) return nullptr;
  sc->cfg = parent->cfg;
  sc->device = parent->device;
  sc->refine_sweeps = parent->refine_sweeps;
  sc->refine_sweeps_cov = parent->refine_sweeps_cov;
  sc->la_ok = false;  // the same kernel sequence eagerly and in the captured graph
  if (sc->dflag.ensure(16 * sizeof(int)) != RBF_OK || cudaMemset(sc->dflag.p, 0, 16 * sizeof(int)) != cudaSuccess) {
    delete sc;
    return nullptr;
  }
  return sc;
}

static void free_sub(Ctx* sc) {
  if (!sc) return;
  for (Buf& b : sc->ws) b.release();
  sc->dflag.release();
  sc->sync_flags.release();
  delete sc;
}

void batch_destroy(Ctx* c) {
  BatchState* B = reinterpret_cast<BatchState*>(c->batch);
  if (!B) return;
  for (auto& g : B->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (cudaEvent_t e : B->events) cudaEventDestroy(e);
  for (cudaStream_t s : B->streams) cudaStreamDestroy(s);
  if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
  for (Ctx* sc : B->sub) free_sub(sc);
  bq_destroy(B->persistent);
  delete B;
  c->batch = nullptr;
}

// Time FP64 and mixed factorization + solve on a synthetic SPD matrix of size m.
static rbf_status autotune(Ctx* sc, int64_t m, int64_t bw, cudaStream_t s, int* pick) {
  Buf H, L, Wf, Zd, u;
  RBF_TRY(H.ensure((size_t)m * m * sizeof(double)));
  RBF_TRY(L.ensure((size_t)m * m * sizeof(double)));
  int64_t ldw = (m + 3) & ~(int64_t)3;
  RBF_TRY(Wf.ensure((size_t)m * ldw * sizeof(float)));
  RBF_TRY(Zd.ensure((size_t)((m + 63) / 64) * 64 * 64 * sizeof(float)));
  RBF_TRY(u.ensure((size_t)m * sizeof(double)));
  std::vector<double> h((size_t)m * m, 0.0), uh((size_t)m, 1.0);
  for (int64_t i = 0; i < m; ++i) {
    h[i * m + i] = 4.0;
    if (i + 1 < m) h[i * m + i + 1] = h[(i + 1) * m + i] = -1.0;
  }
  RBF_CUDA(cudaMemcpyAsync(H.p, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  cudaEvent_t e0, e1;
  RBF_CUDA(cudaEventCreate(&e0));
  RBF_CUDA(cudaEventCreate(&e1));
  float t[2] = {0.f, 0.f};
  for (int path = 0; path < 2; ++path) {
    for (int rep = 0; rep < 2; ++rep) {
      RBF_CUDA(cudaMemcpyAsync(u.p, uh.data(), uh.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      RBF_CUDA(cudaEventRecord(e0, s));
      if (path == 0) {
        RBF_CUDA(cudaMemcpyAsync(L.p, H.p, (size_t)m * m * sizeof(double), cudaMemcpyDeviceToDevice, s));
        RBF_TRY(potrf_lower(sc, L.as<double>(), m, m, m, false, s, bw));
        RBF_TRY(chol_solve(sc, H.as<double>(), L.as<double>(), m, m, u.as<double>(), false, s, bw));
      } else {
        RBF_TRY(potrf_mixed(sc, H.as<double>(), m, m, Wf.as<float>(), ldw, Zd.as<float>(), s, bw));
        RBF_TRY(mixed_solve(sc, H.as<double>(), m, nullptr, Wf.as<float>(), ldw, Zd.as<float>(), nullptr, m, u.as<double>(), 1,
                            sc->refine_sweeps, s, bw));
      }
      RBF_CUDA(cudaEventRecord(e1, s));
      RBF_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      RBF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      t[path] = ms;  // second repetition counts
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  H.release();
  L.release();
  Wf.release();
  Zd.release();
  u.release();
  *pick = t[1] < t[0] ? 2 : 1;
  return RBF_OK;
}

static int bucket_of(int64_t M) {
  int b = 0;
  while ((int64_t(1) << (b + 1)) <= M && b < 30) ++b;
  return b;
}

}  // namespace rbf

using namespace rbf;

extern "C" rbf_status rbf_batch_update_eval(rbf_ctx* cx, const rbf_patch* patches, int32_t npatch, void* stream) {
  RBF_TRY(check_ctx(cx, false));
  if (npatch < 0) return fail(RBF_EINVAL, "negative npatch");
  if (npatch == 0) return RBF_OK;
  if (!patches) return fail(RBF_EINVAL, "null patches");
  Ctx* c = C(cx);
  for (int32_t k = 0; k < npatch; ++k) {
    const rbf_patch& p = patches[k];
    if (!(p.spacing > 0) || p.nx <= 0 || p.M <= 0 || p.n < 0 || p.Q < 0 || !p.w || (p.n > 0 && !p.pts) ||
        (p.Q > 0 && (!p.q || !p.h)) || !isfinite(p.x0) || !isfinite(p.y0))
      return fail(RBF_EINVAL, "patch %d: bad descriptor", k);
    if (p.M > 16384) return fail(RBF_EINVAL, "patch %d: M > 16384", k);
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (!c->batch) {
    BatchState* B = new (std::nothrow) BatchState();
    if (!B) return fail(RBF_ENOMEM, "host allocation failed");
    c->batch = B;
    const int S = 8;
    for (int k = 0; k < S; ++k) {
      Ctx* sc = new_sub(c);
      cudaStream_t st = nullptr;
      cudaEvent_t ev = nullptr;
      if (!sc || cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        free_sub(sc);
        batch_destroy(c);
        return fail(RBF_ENOMEM, "batch: could not create streams");
      }
      B->sub.push_back(sc);
      B->streams.push_back(st);
      B->events.push_back(ev);
    }
    cudaEvent_t fork = nullptr;
    RBF_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    B->events.push_back(fork);
    RBF_CUDA(cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking));
  }
  BatchState* B = reinterpret_cast<BatchState*>(c->batch);
  const int S = (int)B->sub.size();
  const bool allow_mixed = c->cfg.update_precision == RBF_UPDATE_MIXED;
  if (allow_mixed && c->df_ok) {
    // the persistent launches (bqueue.cu) serve the mixed-precision batch
    bool handled = false;
    RBF_TRY(bq_run(c, &B->persistent, patches, npatch, s, &handled));
    if (handled) {
      RBF_CUDA(cudaStreamSynchronize(s));
      int f = 0;
      RBF_TRY(read_dev_flag(c, s, &f));
      if (f & DEV_BAD_INDEX) return fail(RBF_EINVAL, "a patch has a non-finite point");
      if (f & DEV_NOT_SPD) return fail(RBF_ENOTSPD, "a patch's information matrix is not SPD");
      if (f & DEV_TIMEOUT) return fail(RBF_ETIMEOUT, "a bounded wait timed out");
      return RBF_OK;
    }
  }
  // factorization path per patch (autotuned per size bucket)
  std::vector<char> mixed((size_t)npatch, 0);
  for (int32_t k = 0; k < npatch; ++k) {
    if (!allow_mixed) continue;
    int b = bucket_of(patches[k].M);
    if (!B->choice[b]) {
      int pick = 1;
      RBF_TRY(autotune(B->sub[0], patches[k].M, patch_bandwidth(make_geom(c->cfg, patches[k])), s, &pick));
      B->choice[b] = pick;
    }
    mixed[k] = B->choice[b] == 2;
  }
  // greedy assignment, largest first
  std::vector<int32_t> idx((size_t)npatch);
  for (int32_t k = 0; k < npatch; ++k) idx[k] = k;
  auto cost = [&](int32_t k) {
    double m = (double)patches[k].M;
    return m * m * m + 50.0 * (double)patches[k].n * 64.0;
  };
  std::sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return cost(a) > cost(b); });
  std::vector<double> load((size_t)S, 0.0);
  std::vector<std::vector<int32_t>> plan((size_t)S);
  for (int32_t k : idx) {
    int best = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    plan[best].push_back(k);
    load[best] += cost(k);
  }
  // graph cache key: descriptors + path choices
  std::vector<unsigned char> key((size_t)npatch * sizeof(rbf_patch) + (size_t)npatch);
  memcpy(key.data(), patches, (size_t)npatch * sizeof(rbf_patch));
  memcpy(key.data() + (size_t)npatch * sizeof(rbf_patch), mixed.data(), (size_t)npatch);
  cudaEvent_t fork = B->events.back();
  // fork from `root`, run every stream's patches, join back into `root`
  auto enqueue = [&](cudaStream_t root) -> rbf_status {
    RBF_CUDA(cudaEventRecord(fork, root));
    for (int k = 0; k < S; ++k) {
      if (plan[k].empty()) continue;
      RBF_CUDA(cudaStreamWaitEvent(B->streams[k], fork, 0));
      for (int32_t pid : plan[k]) RBF_TRY(run_patch(B->sub[k], c->cfg, patches[pid], mixed[pid] != 0, B->streams[k]));
      RBF_CUDA(cudaEventRecord(B->events[k], B->streams[k]));
      RBF_CUDA(cudaStreamWaitEvent(root, B->events[k], 0));
    }
    return RBF_OK;
  };
  for (Ctx* sc : B->sub) sc->prof = false;
  bool seen = false;
  for (auto& v : B->seen)
    if (v == key) seen = true;
  cudaGraphExec_t exec = nullptr;
  for (auto& g : B->graphs)
    if (g.key == key) exec = g.exec;
  if (exec) {
    RBF_CUDA(cudaGraphLaunch(exec, s));
    ::rbf::note_launch();
  } else if (!seen) {
    RBF_TRY(enqueue(s));  // eager: sizes every workspace
    if (B->seen.size() >= 8) B->seen.erase(B->seen.begin());
    B->seen.push_back(key);
  } else {
    // record on an internal stream (the caller's may be the legacy stream,
    // which cannot be captured); the graph is then launched on the caller's
    cudaStream_t cs = B->cap_stream;
    RBF_CUDA(cudaStreamSynchronize(s));
    cudaGraph_t graph = nullptr;
    RBF_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    rbf_status st = enqueue(cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (st != RBF_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture", __FILE__, __LINE__);
    cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) return cuda_fail(e3, "cudaGraphInstantiate", __FILE__, __LINE__);
    if (B->graphs.size() >= 4) {
      cudaGraphExecDestroy(B->graphs.front().exec);
      B->graphs.erase(B->graphs.begin());
    }
    B->graphs.push_back({key, exec});
    RBF_CUDA(cudaGraphLaunch(exec, s));
    ::rbf::note_launch();
  }
  RBF_CUDA(cudaStreamSynchronize(s));
  int flags = 0;
  for (Ctx* sc : B->sub) {
    int f = 0;
    RBF_TRY(read_dev_flag(sc, s, &f));
    flags |= f;
  }
  if (flags & DEV_BAD_INDEX) return fail(RBF_EINVAL, "a patch has a non-finite point");
  if (flags & DEV_NOT_SPD) return fail(RBF_ENOTSPD, "a patch's information matrix is not SPD");
  if (flags & DEV_TIMEOUT) return fail(RBF_ETIMEOUT, "a bounded wait timed out");
  return RBF_OK;
}
