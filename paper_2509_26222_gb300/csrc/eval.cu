// Evaluation of the terrain model and the soft-constraint cost.
//
//  * rbf_eval: h(q) = sum_j w_j phi(||q - c_j||) and grad h (Eq. RBF_fml,
//    Eq. manidolf_grad_detail with the sign of reading G5), float32, one
//    thread per query, candidates from the center hash grid (rows of cells
//    cut to the disc of the support radius).
//  * rbf_soft_cost: q_i = R p_i + t, r_i = q_z - wheel_offset - h(q_xy)
//    (Eq. residual_manifold_left_wheel), Huber or L2 cost, pose gradient
//    through Eq. manifold_derivative and Eq. manifold_grad_2 (right
//    perturbation), per-block float64 partial sums reduced in a fixed order.
//  * rbf_soft_cost_backward: weight and center gradients by a center-major
//    gather over a counting sort of the transformed points (deterministic).
#include <math.h>

#include <mutex>

#include "common.cuh"

namespace rbf {

struct EvalParams {
  Grid g;
  float r2;       // squared support radius (float32)
  float rc;       // support radius in cell units
  float inv_rho;  // Wendland: 1 / rho
  float inv2s2;   // Gaussian: 1 / (2 sigma^2)
  float gscale;   // Wendland: -20 / rho^2; Gaussian: -1 / sigma^2
};

static EvalParams make_eval_params(const Ctx* c) {
  EvalParams P;
  P.g = c->grid;
  double r = eval_radius(c->cfg);
  float r32 = (float)r;
  P.r2 = r32 * r32;
  P.rc = (float)(r / (double)c->grid.cs);
  P.inv_rho = (float)(1.0 / c->cfg.rho);
  P.inv2s2 = (float)(1.0 / (2.0 * c->cfg.sigma * c->cfg.sigma));
  P.gscale = c->cfg.kernel == RBF_KERNEL_WENDLAND
                 ? (float)(-20.0 / (c->cfg.rho * c->cfg.rho))
                 : (float)(-1.0 / (c->cfg.sigma * c->cfg.sigma));
  return P;
}

// Visit every candidate slot of the hash grid whose cell meets the disc of
// radius rc (cell units) around the point (x, y).
template <class F>
__device__ __forceinline__ void for_each_candidate(const Grid& g, const int32_t* __restrict__ cell_start,
                                                   float x, float y, float rc, F&& f) {
  float fx = (x - g.x0) * g.inv_cs, fy = (y - g.y0) * g.inv_cs;
  int jlo, jhi;
  if (!rows_range(g, fy, rc, jlo, jhi)) return;
  for (int j = jlo; j <= jhi; ++j) {
    int ilo, ihi;
    if (!row_range(g, fx, fy, rc, j, ilo, ihi)) continue;
    int s0 = __ldg(cell_start + j * g.nx + ilo);
    int s1 = __ldg(cell_start + j * g.nx + ihi + 1);
    for (int s = s0; s < s1; ++s) f(s);
  }
}

template <int KERNEL>
__device__ __forceinline__ void eval_one(const EvalParams& P, const int32_t* __restrict__ cell_start,
                                         const float4* __restrict__ xyw, float qx, float qy,
                                         float& h, float& gx, float& gy) {
  float ah = 0.f, ax = 0.f, ay = 0.f;
  for_each_candidate(P.g, cell_start, qx, qy, P.rc, [&](int s) {
    float4 c = __ldg(xyw + s);
    float dx = qx - c.x, dy = qy - c.y;
    float d2 = fmaf(dx, dx, dy * dy);
    if (d2 < P.r2) {
      if (KERNEL == RBF_KERNEL_WENDLAND) {
        float sd = sqrtf(d2) * P.inv_rho;
        float t = fmaxf(1.f - sd, 0.f);
        float cw = c.z * (t * t * t);
        ah = fmaf(cw, t * fmaf(4.f, sd, 1.f), ah);
        ax = fmaf(cw, dx, ax);
        ay = fmaf(cw, dy, ay);
      } else {
        float e = c.z * __expf(-d2 * P.inv2s2);
        ah += e;
        ax = fmaf(e, dx, ax);
        ay = fmaf(e, dy, ay);
      }
    }
  });
  h = ah;
  gx = ax * P.gscale;
  gy = ay * P.gscale;
}

template <int KERNEL>
__global__ void __launch_bounds__(256) k_eval(EvalParams P, const int32_t* __restrict__ cell_start,
                                              const float4* __restrict__ xyw,
                                              const float2* __restrict__ q, int64_t Q,
                                              float* __restrict__ h, float2* __restrict__ grad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Q;
       i += (int64_t)gridDim.x * blockDim.x) {
    float2 p = q[i];
    float hh, gx, gy;
    if (isfinite(p.x) && isfinite(p.y)) {
      eval_one<KERNEL>(P, cell_start, xyw, p.x, p.y, hh, gx, gy);
    } else {
      hh = gx = gy = __int_as_float(0x7fc00000);
    }
    h[i] = hh;
    if (grad) grad[i] = make_float2(gx, gy);
  }
}

// ---------------------------------------------------------------------------
// Lattice path: centers on (x0 + (i + 0.5) h, y0 + (j + 0.5) h) with the
// weights in a dense ny x nx array (0 where the mesh node holds no center).
// Positions are arithmetic, so a candidate costs one 4-byte weight load; the
// loop visits only the nodes of each row that lie in the support disc.
// Coordinates are in lattice units (u = (q_x - x0) / h - 0.5, node i at u = i).
// ---------------------------------------------------------------------------
struct LatParams {
  float u0, v0, inv_h;
  float R, R2, invR;  // support radius in lattice units
  int nx, ny;
  float gscale;       // d h / d q = gscale * sum(...) in metres
  float r2;           // Gaussian: squared cutoff radius in metres (float32 rule)
  float inv2s2;       // Gaussian: 1 / (2 sigma^2)
};

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int KERNEL>
__device__ __forceinline__ void eval_lattice_one(const LatParams& P, const float* __restrict__ W,
                                                 const float* __restrict__ xs, const float* __restrict__ ys,
                                                 float qx, float qy, float& h, float& gx, float& gy) {
  float u = fmaf(qx, P.inv_h, -P.u0), v = fmaf(qy, P.inv_h, -P.v0);
  float jl = fmaxf(ceilf(v - P.R), 0.f), jh = fminf(floorf(v + P.R), (float)(P.ny - 1));
  float ah = 0.f, ax = 0.f, ay = 0.f;
  if (jl <= jh) {
    int jlo = (int)jl, jhi = (int)jh;
    for (int j = jlo; j <= jhi; ++j) {
      float dv = v - (float)j;
      float q2 = fmaf(-dv, dv, P.R2);
      if (q2 <= 0.f) continue;
      float hw = sqrt_approx(q2);
      float il = fmaxf(ceilf(u - hw), 0.f), ih = fminf(floorf(u + hw), (float)(P.nx - 1));
      if (il > ih) continue;
      int ilo = (int)il, ihi = (int)ih;
      const float* Wr = W + j * P.nx;
      float hr = 0.f, xr = 0.f, yr = 0.f;
      if (KERNEL == RBF_KERNEL_WENDLAND) {
        // scaled so that the support radius is 1: s^2 = du'^2 + dv'^2
        float dvs = dv * P.invR;
        float dv2 = dvs * dvs;
        float du = (u - (float)ilo) * P.invR;
#pragma unroll 4
        for (int i = ilo; i <= ihi; ++i) {
          float w = Wr[i];
          float s = sqrt_approx(fmaf(du, du, dv2));
          float t = 1.f - s;
          float t2 = t * t;
          float c = (w * t2) * t;                       // w (1-s)^3
          hr = fmaf(c, t * fmaf(4.f, s, 1.f), hr);      // w (1-s)^4 (4s+1)
          xr = fmaf(c, du, xr);
          yr += c;
          du -= P.invR;
        }
        ah += hr;
        ax += xr;
        ay = fmaf(yr, dvs, ay);
      } else {
        float dy = qy - ys[j];
        float dy2 = __fmul_rn(dy, dy);
        for (int i = ilo; i <= ihi; ++i) {
          float dx = qx - xs[i];
          float d2 = __fadd_rn(__fmul_rn(dx, dx), dy2);
          if (d2 < P.r2) {
            float e = Wr[i] * __expf(-d2 * P.inv2s2);
            hr += e;
            xr = fmaf(e, dx, xr);
          }
        }
        ah += hr;
        ax += xr;
        ay = fmaf(hr, dy, ay);
      }
    }
  }
  h = ah;
  gx = ax * P.gscale;
  gy = ay * P.gscale;
}

template <int KERNEL, bool SMEM>
__global__ void __launch_bounds__(256) k_eval_lattice(LatParams P, const float* __restrict__ Wg,
                                                      const float* __restrict__ xsg, const float* __restrict__ ysg,
                                                      const float2* __restrict__ q, int64_t Q,
                                                      float* __restrict__ h, float2* __restrict__ grad) {
  extern __shared__ float sm[];
  const float* W = Wg;
  const float* xs = xsg;
  const float* ys = ysg;
  if (SMEM) {
    int cells = P.nx * P.ny;
    float* Ws = sm;
    for (int e = threadIdx.x; e < cells; e += blockDim.x) Ws[e] = Wg[e];
    W = Ws;
    if (KERNEL == RBF_KERNEL_GAUSSIAN) {
      float* xss = sm + cells;
      float* yss = xss + P.nx;
      for (int e = threadIdx.x; e < P.nx; e += blockDim.x) xss[e] = xsg[e];
      for (int e = threadIdx.x; e < P.ny; e += blockDim.x) yss[e] = ysg[e];
      xs = xss;
      ys = yss;
    }
    __syncthreads();
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Q;
       i += (int64_t)gridDim.x * blockDim.x) {
    float2 p = q[i];
    float hh, gx, gy;
    if (isfinite(p.x) && isfinite(p.y)) {
      eval_lattice_one<KERNEL>(P, W, xs, ys, p.x, p.y, hh, gx, gy);
    } else {
      hh = gx = gy = __int_as_float(0x7fc00000);
    }
    h[i] = hh;
    if (grad) grad[i] = make_float2(gx, gy);
  }
}

// ---------------------------------------------------------------------------
// Fixed-window lattice kernel (Wendland): every lane visits the same
// 2 RC x 2 RC nodes around its query, so the warp never diverges; nodes
// outside the support contribute (1 - s)_+ = 0.  Columns go in pairs with
// packed float32x2 arithmetic; W2[j][i] = (W[j][i], W[j][i+1]) so that a pair
// is one 8-byte load at any column parity.  The weight array is padded by
// 2 RC zero nodes on every side, and the window origin is clamped so that it
// always lies inside the padded array (a clamped window only holds nodes
// farther than the support radius, i.e. zero terms).
// ---------------------------------------------------------------------------
typedef unsigned long long u64;
__device__ __forceinline__ u64 pk2(float a, float b) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void up2(u64 v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
  u64 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

struct LatWParams {
  float u0, v0, inv_h, invR;
  int nx, ny, pitch;  // pitch = nx + 4 RC (padded row length of W2)
  float gscale;
};

template <int RC, bool SMEM>
__global__ void __launch_bounds__(256) k_eval_lattice_win(LatWParams P, const float2* __restrict__ W2g,
                                                          const float2* __restrict__ xt,
                                                          const float2* __restrict__ yt,
                                                          const float2* __restrict__ q, int64_t Q,
                                                          float* __restrict__ h, float2* __restrict__ grad) {
  extern __shared__ float2 sw2[];
  const float2* W2 = W2g;
  if (SMEM) {
    int cells = P.pitch * (P.ny + 4 * RC);
    for (int e = threadIdx.x; e < cells; e += blockDim.x) sw2[e] = W2g[e];
    W2 = sw2;
    __syncthreads();
  }
  const u64 one2 = pk2(1.f, 1.f), four2 = pk2(4.f, 4.f), mone2 = pk2(-1.f, -1.f);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float2 pnext = qi < Q ? __ldcs(q + qi) : make_float2(0.f, 0.f);
  for (; qi < Q; qi += stride) {
    float2 p = pnext;
    if (qi + stride < Q) pnext = __ldcs(q + qi + stride);  // next query in flight during this one
    if (!(isfinite(p.x) && isfinite(p.y))) {
      float nan = __int_as_float(0x7fc00000);
      h[qi] = nan;
      if (grad) grad[qi] = make_float2(nan, nan);
      continue;
    }
    const float ur = fmaf(p.x, P.inv_h, -P.u0), vr = fmaf(p.y, P.inv_h, -P.v0);
    // a query farther than RC + 1 nodes outside the lattice meets no support;
    // clamping it there keeps every offset below finite and the terms zero
    float u = fminf(fmaxf(ur, (float)(-2 * RC - 2)), (float)(P.nx + 2 * RC + 1));
    float v = fminf(fmaxf(vr, (float)(-2 * RC - 2)), (float)(P.ny + 2 * RC + 1));
    // window origin (node coordinates): floor(u) - RC + 1, clamped into the pad
    float fu = fminf(fmaxf(floorf(u), (float)(-RC - 1)), (float)(P.nx + RC - 1));
    float fv = fminf(fmaxf(floorf(v), (float)(-RC - 1)), (float)(P.ny + RC - 1));
    int ib = (int)fu + RC + 1;  // padded column of the window's first node
    int jb = (int)fv + RC + 1;
    // offset of the query from node floor(u) in lattice units: u - fu loses the
    // rounding of u (a few 1e-6 of a spacing far from the origin); the offset
    // from the node's float-float coordinate is exact up to its own rounding
    float fx = u - fu, fy = v - fv;
    if (u == ur && fu == floorf(ur)) {
      const float2 xn = __ldg(xt + ib);
      fx = __fmul_rn(__fsub_rn(__fsub_rn(p.x, xn.x), xn.y), P.inv_h);
    }
    if (v == vr && fv == floorf(vr)) {
      const float2 yn = __ldg(yt + jb);
      fy = __fmul_rn(__fsub_rn(__fsub_rn(p.y, yn.x), yn.y), P.inv_h);
    }
    // offsets of the window's first node, in units of the support radius
    float du0 = (fx + (float)(RC - 1)) * P.invR;
    float dv0 = (fy + (float)(RC - 1)) * P.invR;
    u64 dup[RC], du2p[RC];
#pragma unroll
    for (int k = 0; k < RC; ++k) {
      float a = du0 - (float)(2 * k) * P.invR, b = du0 - (float)(2 * k + 1) * P.invR;
      dup[k] = pk2(a, b);
      du2p[k] = pk2(a * a, b * b);
    }
    u64 hacc = 0ull, xacc = 0ull;
    float yacc = 0.f;
    const float2* base = W2 + (int64_t)jb * P.pitch + ib;
#pragma unroll
    for (int m = 0; m < 2 * RC; ++m) {
      float dv = dv0 - (float)m * P.invR;
      u64 dv2 = pk2(dv * dv, dv * dv);
      const float2* row = base + m * P.pitch;
      u64 yr = 0ull;
#pragma unroll
      for (int k = 0; k < RC; ++k) {
        float2 wv = row[2 * k];
        u64 w = pk2(wv.x, wv.y);
        u64 e = add2(du2p[k], dv2);
        float e0, e1;
        up2(e, e0, e1);
        u64 sq = pk2(sqrt_approx(e0), sqrt_approx(e1));
        u64 t = fma2(sq, mone2, one2);
        float t0, t1;
        up2(t, t0, t1);
        t = pk2(fmaxf(t0, 0.f), fmaxf(t1, 0.f));
        u64 c = mul2(mul2(w, mul2(t, t)), t);        // w (1-s)^3
        u64 pp = mul2(fma2(four2, sq, one2), t);      // (1-s)(4s+1)
        hacc = fma2(c, pp, hacc);
        xacc = fma2(c, dup[k], xacc);
        yr = add2(yr, c);
      }
      float y0, y1;
      up2(yr, y0, y1);
      yacc = fmaf(y0 + y1, dv, yacc);
    }
    float h0, h1, x0, x1;
    up2(hacc, h0, h1);
    up2(xacc, x0, x1);
    h[qi] = h0 + h1;
    if (grad) grad[qi] = make_float2((x0 + x1) * P.gscale, yacc * P.gscale);
  }
}

static LatParams make_lat_params(const Ctx* c) {
  LatParams P;
  const Lattice& L = c->lat;
  P.inv_h = (float)(1.0 / L.h);
  P.u0 = (float)(L.x0 / L.h + 0.5);
  P.v0 = (float)(L.y0 / L.h + 0.5);
  double r = eval_radius(c->cfg);
  double R = r / L.h;
  P.R = (float)R;
  P.R2 = (float)(R * R);
  P.invR = (float)(1.0 / R);
  P.nx = L.nx;
  P.ny = L.ny;
  float r32 = (float)r;
  P.r2 = r32 * r32;
  P.inv2s2 = (float)(1.0 / (2.0 * c->cfg.sigma * c->cfg.sigma));
  if (c->cfg.kernel == RBF_KERNEL_WENDLAND)
    P.gscale = (float)(-20.0 / (c->cfg.rho * c->cfg.rho) * r);  // du is in units of R lattice cells = r metres
  else
    P.gscale = (float)(-1.0 / (c->cfg.sigma * c->cfg.sigma));
  return P;
}

static int num_sms(int dev) {
  static int cached[64] = {0};
  if (dev < 0 || dev >= 64) return 148;
  if (!cached[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 148;
  }
  return cached[dev];
}

static unsigned grid_for(int64_t n, int threads, int dev, int per_sm) {
  int64_t want = (n + threads - 1) / threads;
  int64_t cap = (int64_t)num_sms(dev) * per_sm;
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return (unsigned)want;
}

// ---------------------------------------------------------------------------
// Soft-constraint cost
// ---------------------------------------------------------------------------
// Pose of the body frame: q = R p + t is formed in float64, so that large
// map-frame translations do not lose the residual's precision; the float32
// copy of R serves the Jacobian rows.
struct Pose {
  double R[9];
  double t[3];
  float Rf[9];
};

struct CostParams {
  int loss;
  float delta, lam_m, off;
};

// Residual, loss, psi = d loss / d r and the pose Jacobian row of one point.
template <int KERNEL>
__device__ __forceinline__ void point_terms(const EvalParams& P, const int32_t* __restrict__ cell_start,
                                            const float4* __restrict__ xyw, const Pose& T,
                                            const CostParams& CP, const float* __restrict__ pts,
                                            int64_t i, float& qx, float& qy, float& r, float& loss,
                                            float& psi, float J[6]) {
  float px = pts[3 * i], py = pts[3 * i + 1], pz = pts[3 * i + 2];
  const double dpx = px, dpy = py, dpz = pz;
  // q in float64; the evaluation point is its float32 rounding (the query type
  // of the evaluation), q_z and the residual's difference stay float64
  double qxd = fma(T.R[0], dpx, fma(T.R[1], dpy, fma(T.R[2], dpz, T.t[0])));
  double qyd = fma(T.R[3], dpx, fma(T.R[4], dpy, fma(T.R[5], dpz, T.t[1])));
  double qzd = fma(T.R[6], dpx, fma(T.R[7], dpy, fma(T.R[8], dpz, T.t[2])));
  qx = (float)qxd;
  qy = (float)qyd;
  float h, hx, hy;
  eval_one<KERNEL>(P, cell_start, xyw, qx, qy, h, hx, hy);
  r = (float)(qzd - (double)CP.off - (double)h);
  if (CP.loss == RBF_LOSS_HUBER) {
    float a = fabsf(r);
    loss = a <= CP.delta ? 0.5f * r * r : CP.delta * (a - 0.5f * CP.delta);
    psi = fminf(fmaxf(r, -CP.delta), CP.delta);
  } else {
    loss = CP.lam_m * r * r;
    psi = 2.f * CP.lam_m * r;
  }
  // dr/dq = a = (-hx, -hy, 1); dr/dtheta = p x (R^T a); dr/dt = a
  float ax = -hx, ay = -hy, az = 1.f;
  float bx = T.Rf[0] * ax + T.Rf[3] * ay + T.Rf[6] * az;
  float by = T.Rf[1] * ax + T.Rf[4] * ay + T.Rf[7] * az;
  float bz = T.Rf[2] * ax + T.Rf[5] * ay + T.Rf[8] * az;
  J[0] = py * bz - pz * by;
  J[1] = pz * bx - px * bz;
  J[2] = px * by - py * bx;
  J[3] = ax;
  J[4] = ay;
  J[5] = az;
}

constexpr int SC_THREADS = 256;

// NV = 7: cost and gradient.  NV = 28: also the Gauss-Newton matrix
// A = sum_i omega_i J_i J_i^T (upper triangle, row-major, 21 entries) with
// the iteratively reweighted least-squares weight omega_i = psi(r_i) / r_i
// (1 inside the Huber zone, delta / |r_i| outside; 2 lambda_M for the L2 loss).
constexpr int SC_NORMAL = 28;

template <int KERNEL, int NV>
__global__ void __launch_bounds__(SC_THREADS) k_soft_cost(EvalParams P, const int32_t* __restrict__ cell_start,
                                                          const float4* __restrict__ xyw, Pose T,
                                                          CostParams CP, const float* __restrict__ pts,
                                                          int64_t n, float* __restrict__ resid,
                                                          double* __restrict__ partials) {
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float qx, qy, r, loss, psi, J[6];
    point_terms<KERNEL>(P, cell_start, xyw, T, CP, pts, i, qx, qy, r, loss, psi, J);
    if (resid) resid[i] = r;
    acc[0] += (double)loss;
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k + 1] += (double)(psi * J[k]);
    if (NV == SC_NORMAL) {
      float om;
      if (CP.loss == RBF_LOSS_HUBER) {
        float a = fabsf(r);
        om = a <= CP.delta ? 1.f : CP.delta / a;
      } else {
        om = 2.f * CP.lam_m;
      }
      int q = 7;
#pragma unroll
      for (int u = 0; u < 6; ++u)
#pragma unroll
        for (int v = u; v < 6; ++v) acc[q++] += (double)(om * J[u] * J[v]);
    }
  }
  __shared__ double red[SC_THREADS / 32][NV];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double v = 0;
    for (int w = 0; w < SC_THREADS / 32; ++w) v += red[w][threadIdx.x];
    partials[blockIdx.x * (NV == 7 ? 8 : 32) + threadIdx.x] = v;
  }
}

// out[0] = cost, out[1..6] = gradient, out[7..27] = A (when nv = 28); the
// first seven scaled by *gout when given.
__global__ void k_reduce_partials(const double* __restrict__ partials, int nblk, int nv,
                                  const double* __restrict__ gout, double* __restrict__ cost,
                                  double* __restrict__ grad6, double* __restrict__ normal21) {
  int k = threadIdx.x;
  if (k >= nv) return;
  const int stride = nv == 7 ? 8 : 32;
  double v = 0;
  for (int b = 0; b < nblk; ++b) v += partials[b * stride + k];
  if (k < 7) {
    double g = gout ? *gout : 1.0;
    v *= g;
  }
  if (k == 0) {
    if (cost) *cost = v;
  } else if (k < 7) {
    if (grad6) grad6[k - 1] = v;
  } else if (normal21) {
    normal21[k - 7] = v;
  }
}

static rbf_status load_pose(const double* R, const double* t, Pose* T) {
  if (!R || !t) return fail(RBF_EINVAL, "null pose");
  for (int k = 0; k < 9; ++k) {
    if (!isfinite(R[k])) return fail(RBF_EINVAL, "non-finite rotation");
    T->R[k] = R[k];
    T->Rf[k] = (float)R[k];
  }
  for (int k = 0; k < 3; ++k) {
    if (!isfinite(t[k])) return fail(RBF_EINVAL, "non-finite translation");
    T->t[k] = t[k];
  }
  return RBF_OK;
}

static CostParams cost_params(const rbf_config& cfg) {
  CostParams CP;
  CP.loss = cfg.loss;
  CP.delta = (float)cfg.huber_delta;
  CP.lam_m = (float)cfg.lambda_m;
  CP.off = (float)cfg.wheel_offset;
  return CP;
}

static rbf_status soft_cost_forward(Ctx* x, const Pose& T, const float* pts, int64_t n,
                                    const double* gout, double* cost, double* grad6, float* resid,
                                    cudaStream_t s, double* normal21 = nullptr) {
  EvalParams P = make_eval_params(x);
  CostParams CP = cost_params(x->cfg);
  unsigned nb = grid_for(n, SC_THREADS, x->device, 4);
  Buf& part = x->scratch(20);
  RBF_TRY(part.ensure((size_t)nb * 32 * sizeof(double)));
  const int nv = normal21 ? SC_NORMAL : 7;
  const int32_t* cs = x->cell_start.as<int32_t>();
  const float4* xyw = x->sorted_xyw.as<float4>();
  double* pp = part.as<double>();
  if (x->cfg.kernel == RBF_KERNEL_WENDLAND) {
    if (normal21) { k_soft_cost<RBF_KERNEL_WENDLAND, SC_NORMAL><<<nb, SC_THREADS, 0, s>>>(P, cs, xyw, T, CP, pts, n, resid, pp); ::rbf::note_launch(); }
    else { k_soft_cost<RBF_KERNEL_WENDLAND, 7><<<nb, SC_THREADS, 0, s>>>(P, cs, xyw, T, CP, pts, n, resid, pp); ::rbf::note_launch(); }
  } else {
    if (normal21) { k_soft_cost<RBF_KERNEL_GAUSSIAN, SC_NORMAL><<<nb, SC_THREADS, 0, s>>>(P, cs, xyw, T, CP, pts, n, resid, pp); ::rbf::note_launch(); }
    else { k_soft_cost<RBF_KERNEL_GAUSSIAN, 7><<<nb, SC_THREADS, 0, s>>>(P, cs, xyw, T, CP, pts, n, resid, pp); ::rbf::note_launch(); }
  }
  RBF_CUDA(cudaGetLastError());
  { k_reduce_partials<<<1, 32, 0, s>>>(pp, (int)nb, nv, gout, cost, grad6, normal21); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  return RBF_OK;
}

// ---------------------------------------------------------------------------
// Backward: per point (qx, qy, psi), counting sort of the points by cell of
// the center grid, then one thread per center gathers its in-support points.
// ---------------------------------------------------------------------------
template <int KERNEL>
__global__ void __launch_bounds__(256) k_bwd_points(EvalParams P, const int32_t* __restrict__ cell_start,
                                                    const float4* __restrict__ xyw, Pose T, CostParams CP,
                                                    const float* __restrict__ pts, int64_t n,
                                                    const double* __restrict__ gout,
                                                    float4* __restrict__ qpsi, int32_t* __restrict__ pcell,
                                                    int32_t* __restrict__ pcount) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float qx, qy, r, loss, psi, J[6];
  point_terms<KERNEL>(P, cell_start, xyw, T, CP, pts, i, qx, qy, r, loss, psi, J);
  float g = gout ? (float)*gout : 1.f;
  qpsi[i] = make_float4(qx, qy, psi * g, 0.f);
  int ix = (int)floorf((qx - P.g.x0) * P.g.inv_cs);
  int iy = (int)floorf((qy - P.g.y0) * P.g.inv_cs);
  // points outside the grid's cell range still gather correctly when clamped:
  // the per-center search covers the clamped border cells.
  bool fin = isfinite(qx) && isfinite(qy);
  ix = min(max(ix, 0), P.g.nx - 1);
  iy = min(max(iy, 0), P.g.ny - 1);
  int cc = fin ? iy * P.g.nx + ix : -1;
  pcell[i] = cc;
  if (cc >= 0) atomicAdd(&pcount[cc], 1);
}

__global__ void k_bwd_fill(const int32_t* __restrict__ pcell, int64_t n, const int32_t* __restrict__ start,
                           int32_t* __restrict__ fill, int32_t* __restrict__ order) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int cc = pcell[i];
  if (cc < 0) return;
  int pos = start[cc] + atomicAdd(&fill[cc], 1);
  order[pos] = (int32_t)i;
}

__global__ void k_bwd_sort(const int32_t* __restrict__ start, int ncell, int32_t* __restrict__ ids) {
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

// The point cells are clamped to the grid, so a point beyond the border sits
// in a border cell; widen the search at the border to the whole row/column
// band by letting the clamped cell range cover it (the disc test is exact).
template <int KERNEL>
__global__ void __launch_bounds__(256) k_bwd_centers(EvalParams P, const float4* __restrict__ xyw,
                                                     const int32_t* __restrict__ sorted_id, int64_t M,
                                                     const int32_t* __restrict__ pstart,
                                                     const int32_t* __restrict__ order,
                                                     const float4* __restrict__ qpsi,
                                                     float* __restrict__ dw, float2* __restrict__ dc) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  float4 c = xyw[s];
  int j = sorted_id[s];
  float aw = 0.f, ax = 0.f, ay = 0.f;
  const Grid& g = P.g;
  float fx = (c.x - g.x0) * g.inv_cs, fy = (c.y - g.y0) * g.inv_cs;
  int jlo = (int)floorf(fy - P.rc - 2e-3f), jhi = (int)floorf(fy + P.rc + 2e-3f);
  int ilo = (int)floorf(fx - P.rc - 2e-3f), ihi = (int)floorf(fx + P.rc + 2e-3f);
  // border cells hold every clamped point beyond the border
  jlo = max(jlo, 0);
  ilo = max(ilo, 0);
  jhi = min(jhi, g.ny - 1);
  ihi = min(ihi, g.nx - 1);
  for (int cj = jlo; cj <= jhi; ++cj) {
    if (cj > jhi) break;
    int a = pstart[cj * g.nx + ilo], b = pstart[cj * g.nx + ihi + 1];
    for (int k = a; k < b; ++k) {
      float4 q = __ldg(qpsi + __ldg(order + k));
      float dx = q.x - c.x, dy = q.y - c.y;
      float d2 = fmaf(dx, dx, dy * dy);
      if (d2 < P.r2) {
        float ph, gc;
        if (KERNEL == RBF_KERNEL_WENDLAND) {
          float sd = sqrtf(d2) * P.inv_rho;
          float t = fmaxf(1.f - sd, 0.f);
          float t3 = t * t * t;
          ph = t3 * t * fmaf(4.f, sd, 1.f);
          gc = P.gscale * t3;
        } else {
          ph = __expf(-d2 * P.inv2s2);
          gc = P.gscale * ph;
        }
        aw = fmaf(q.z, ph, aw);
        float pg = q.z * gc;
        ax = fmaf(pg, dx, ax);
        ay = fmaf(pg, dy, ay);
      }
    }
  }
  if (dw) dw[j] = -aw;
  if (dc) dc[j] = make_float2(c.z * ax, c.z * ay);
}

}  // namespace rbf

using namespace rbf;

extern "C" rbf_status rbf_eval(rbf_ctx* c, const float* q, int64_t Q, float* h, float* grad,
                               void* stream) {
  RBF_TRY(check_ctx(c, true));
  if (Q < 0) return fail(RBF_EINVAL, "negative Q");
  if (Q == 0) return RBF_OK;
  if (!q || !h) return fail(RBF_EINVAL, "null query or output pointer");
  if (((uintptr_t)q & 7) || ((uintptr_t)grad & 7))
    return fail(RBF_EINVAL, "q and grad must be 8-byte aligned");
  Ctx* x = C(c);
  cudaStream_t s = (cudaStream_t)stream;
  StageTimer st(x, RBF_STAGE_EVAL, s, 20.0 * (double)Q);
  if (x->lat.on && x->lat_rc > 0 && x->cfg.kernel == RBF_KERNEL_WENDLAND) {
    LatWParams L;
    L.inv_h = (float)(1.0 / x->lat.h);
    L.u0 = (float)(x->lat.x0 / x->lat.h + 0.5);
    L.v0 = (float)(x->lat.y0 / x->lat.h + 0.5);
    L.invR = (float)(x->lat.h / x->cfg.rho);
    L.nx = x->lat.nx;
    L.ny = x->lat.ny;
    L.pitch = x->lat.nx + 4 * x->lat_rc;
    L.gscale = (float)(-20.0 / x->cfg.rho);
    size_t smem = (size_t)L.pitch * (x->lat.ny + 4 * x->lat_rc) * sizeof(float2);
    bool use_smem = smem <= 100 * 1024;
    const float2* W2 = x->wlat2.as<float2>();
    auto launch = [&](auto kern) -> rbf_status {
      int occ = 0;
      size_t sm = use_smem ? smem : 0;
      if (sm > 48 * 1024) RBF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      RBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, sm));
      if (occ < 1) occ = 1;
      unsigned nb = grid_for(Q, 256, x->device, occ);
      kern<<<nb, 256, sm, s>>>(L, W2, x->lat_xhl.as<float2>(), x->lat_yhl.as<float2>(), (const float2*)q, Q, h,
                               (float2*)grad);
      ::rbf::note_launch();
      RBF_CUDA(cudaGetLastError());
      return RBF_OK;
    };
    switch (x->lat_rc) {
      case 1: return use_smem ? launch(k_eval_lattice_win<1, true>) : launch(k_eval_lattice_win<1, false>);
      case 2: return use_smem ? launch(k_eval_lattice_win<2, true>) : launch(k_eval_lattice_win<2, false>);
      case 3: return use_smem ? launch(k_eval_lattice_win<3, true>) : launch(k_eval_lattice_win<3, false>);
      default: return use_smem ? launch(k_eval_lattice_win<4, true>) : launch(k_eval_lattice_win<4, false>);
    }
  }
  if (x->lat.on) {
    LatParams L = make_lat_params(x);
    size_t cells = (size_t)x->lat.nx * x->lat.ny;
    size_t smem = (cells + (x->cfg.kernel == RBF_KERNEL_GAUSSIAN ? x->lat.nx + x->lat.ny : 0)) * sizeof(float);
    bool use_smem = smem <= 160 * 1024;
    const float* xs = x->lat_xs.as<float>();
    const float* ys = x->lat_ys.as<float>();
    const float* Wl = x->wlat.as<float>();
    auto launch = [&](auto kern) -> rbf_status {
      int occ = 0;
      size_t sm = use_smem ? smem : 0;
      if (sm > 48 * 1024) RBF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      RBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, sm));
      if (occ < 1) occ = 1;
      unsigned nb = grid_for(Q, 256, x->device, occ);
      kern<<<nb, 256, sm, s>>>(L, Wl, xs, ys, (const float2*)q, Q, h, (float2*)grad);
      ::rbf::note_launch();
      RBF_CUDA(cudaGetLastError());
      return RBF_OK;
    };
    if (x->cfg.kernel == RBF_KERNEL_WENDLAND)
      return use_smem ? launch(k_eval_lattice<RBF_KERNEL_WENDLAND, true>)
                      : launch(k_eval_lattice<RBF_KERNEL_WENDLAND, false>);
    return use_smem ? launch(k_eval_lattice<RBF_KERNEL_GAUSSIAN, true>)
                    : launch(k_eval_lattice<RBF_KERNEL_GAUSSIAN, false>);
  }
  EvalParams P = make_eval_params(x);
  unsigned nb = grid_for(Q, 256, x->device, 8);
  if (x->cfg.kernel == RBF_KERNEL_WENDLAND)
    { k_eval<RBF_KERNEL_WENDLAND><<<nb, 256, 0, s>>>(P, x->cell_start.as<int32_t>(),
                                                   x->sorted_xyw.as<float4>(), (const float2*)q, Q,
                                                   h, (float2*)grad); ::rbf::note_launch(); }
  else
    { k_eval<RBF_KERNEL_GAUSSIAN><<<nb, 256, 0, s>>>(P, x->cell_start.as<int32_t>(),
                                                   x->sorted_xyw.as<float4>(), (const float2*)q, Q,
                                                   h, (float2*)grad); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  return RBF_OK;
}

extern "C" rbf_status rbf_soft_cost(rbf_ctx* c, const double* R, const double* t, const float* pts,
                                    int64_t n, double* cost, double* grad6, float* resid,
                                    void* stream) {
  RBF_TRY(check_ctx(c, true));
  if (n < 0) return fail(RBF_EINVAL, "negative n");
  if (!cost && !grad6 && !resid) return fail(RBF_EINVAL, "no output requested");
  if (n > 0 && !pts) return fail(RBF_EINVAL, "null points");
  Pose T;
  RBF_TRY(load_pose(R, t, &T));
  Ctx* x = C(c);
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    if (cost) RBF_CUDA(cudaMemsetAsync(cost, 0, sizeof(double), s));
    if (grad6) RBF_CUDA(cudaMemsetAsync(grad6, 0, 6 * sizeof(double), s));
    return RBF_OK;
  }
  StageTimer st(x, RBF_STAGE_SOFTCOST, s, 12.0 * (double)n);
  return soft_cost_forward(x, T, pts, n, nullptr, cost, grad6, resid, s);
}

extern "C" rbf_status rbf_soft_cost_normal(rbf_ctx* c, const double* R, const double* t, const float* pts,
                                           int64_t n, double* out28, void* stream) {
  RBF_TRY(check_ctx(c, true));
  if (n < 0) return fail(RBF_EINVAL, "negative n");
  if (!out28) return fail(RBF_EINVAL, "null output");
  if (n > 0 && !pts) return fail(RBF_EINVAL, "null points");
  Pose T;
  RBF_TRY(load_pose(R, t, &T));
  Ctx* x = C(c);
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    RBF_CUDA(cudaMemsetAsync(out28, 0, 28 * sizeof(double), s));
    return RBF_OK;
  }
  StageTimer st(x, RBF_STAGE_SOFTCOST, s, 12.0 * (double)n);
  return soft_cost_forward(x, T, pts, n, nullptr, out28, out28 + 1, nullptr, s, out28 + 7);
}

// The Levenberg-Marquardt step of the pose from the cost, gradient and
// Gauss-Newton matrix in v28 (the layout of rbf_soft_cost_normal): one thread
// forms B = A + mu diag(A), factors it (Cholesky, float64), solves
// B delta = -g and applies R Exp(delta_theta) (Rodrigues' formula), t + delta_t.
__global__ void k_lm_solve(const double* __restrict__ v28, double mu, Pose T, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double B[6][6], g[6];
  int q = 7;
  for (int u = 0; u < 6; ++u)
    for (int v = u; v < 6; ++v, ++q) B[u][v] = B[v][u] = v28[q];
  for (int u = 0; u < 6; ++u) {
    B[u][u] += mu * B[u][u];
    g[u] = v28[1 + u];
  }
  bool ok = true;
  for (int j = 0; j < 6 && ok; ++j) {
    double d = B[j][j];
    for (int k = 0; k < j; ++k) d -= B[j][k] * B[j][k];
    if (!(d > 0.0)) {
      ok = false;
      break;
    }
    const double l = sqrt(d);
    B[j][j] = l;
    for (int i = j + 1; i < 6; ++i) {
      double x = B[i][j];
      for (int k = 0; k < j; ++k) x -= B[i][k] * B[j][k];
      B[i][j] = x / l;
    }
  }
  double dl[6] = {0, 0, 0, 0, 0, 0};
  if (ok) {
    double y[6];
    for (int i = 0; i < 6; ++i) {
      double x = -g[i];
      for (int k = 0; k < i; ++k) x -= B[i][k] * y[k];
      y[i] = x / B[i][i];
    }
    for (int i = 5; i >= 0; --i) {
      double x = y[i];
      for (int k = i + 1; k < 6; ++k) x -= B[k][i] * dl[k];
      dl[i] = x / B[i][i];
    }
  }
  // E = Exp([theta]_x) = I + (sin a / a) K + ((1 - cos a) / a^2) K^2, a = |theta|
  const double th[3] = {dl[0], dl[1], dl[2]};
  const double a2 = th[0] * th[0] + th[1] * th[1] + th[2] * th[2];
  const double a = sqrt(a2);
  double c1 = 1.0, c2 = 0.5;
  if (a > 1e-12) {
    c1 = sin(a) / a;
    c2 = (1.0 - cos(a)) / a2;
  }
  const double K[3][3] = {{0.0, -th[2], th[1]}, {th[2], 0.0, -th[0]}, {-th[1], th[0], 0.0}};
  double E[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double k2 = K[i][0] * K[0][j] + K[i][1] * K[1][j] + K[i][2] * K[2][j];
      E[i][j] = (i == j ? 1.0 : 0.0) + c1 * K[i][j] + c2 * k2;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      out[3 * i + j] = T.R[3 * i + 0] * E[0][j] + T.R[3 * i + 1] * E[1][j] + T.R[3 * i + 2] * E[2][j];
  for (int i = 0; i < 3; ++i) out[9 + i] = T.t[i] + dl[3 + i];
  out[12] = v28[0];
  out[13] = ok ? 0.0 : 1.0;
  for (int i = 0; i < 6; ++i) out[14 + i] = dl[i];
}

extern "C" rbf_status rbf_lm_step(rbf_ctx* c, const double* R, const double* t, const float* pts, int64_t n,
                                  double mu, double* out20, void* stream) {
  RBF_TRY(check_ctx(c, true));
  if (n < 0) return fail(RBF_EINVAL, "negative n");
  if (!out20) return fail(RBF_EINVAL, "null output");
  if (n > 0 && !pts) return fail(RBF_EINVAL, "null points");
  if (!(mu >= 0.0) || !isfinite(mu)) return fail(RBF_EINVAL, "mu must be finite and >= 0");
  Pose T;
  RBF_TRY(load_pose(R, t, &T));
  Ctx* x = C(c);
  cudaStream_t s = (cudaStream_t)stream;
  Buf& v = x->scratch(19);
  RBF_TRY(v.ensure(SC_NORMAL * sizeof(double)));
  double* v28 = v.as<double>();
  if (n == 0) {
    RBF_CUDA(cudaMemsetAsync(v28, 0, SC_NORMAL * sizeof(double), s));
  } else {
    StageTimer st(x, RBF_STAGE_SOFTCOST, s, 12.0 * (double)n);
    RBF_TRY(soft_cost_forward(x, T, pts, n, nullptr, v28, v28 + 1, nullptr, s, v28 + 7));
  }
  { k_lm_solve<<<1, 32, 0, s>>>(v28, mu, T, out20); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  return RBF_OK;
}

extern "C" rbf_status rbf_soft_cost_backward(rbf_ctx* c, const double* R, const double* t,
                                             const float* pts, int64_t n, const double* gout,
                                             float* dw, float* dc, double* dpose6, void* stream) {
  RBF_TRY(check_ctx(c, true));
  if (n < 0) return fail(RBF_EINVAL, "negative n");
  if (n > 0 && !pts) return fail(RBF_EINVAL, "null points");
  if (((uintptr_t)dc & 7)) return fail(RBF_EINVAL, "dc must be 8-byte aligned");
  Pose T;
  RBF_TRY(load_pose(R, t, &T));
  Ctx* x = C(c);
  cudaStream_t s = (cudaStream_t)stream;
  int64_t M = x->M;
  if (n == 0) {
    if (dw) RBF_CUDA(cudaMemsetAsync(dw, 0, (size_t)M * sizeof(float), s));
    if (dc) RBF_CUDA(cudaMemsetAsync(dc, 0, (size_t)M * 2 * sizeof(float), s));
    if (dpose6) RBF_CUDA(cudaMemsetAsync(dpose6, 0, 6 * sizeof(double), s));
    return RBF_OK;
  }
  StageTimer st(x, RBF_STAGE_BACKWARD, s, 24.0 * (double)n);
  if (dpose6) RBF_TRY(soft_cost_forward(x, T, pts, n, gout, nullptr, dpose6, nullptr, s));
  if (!dw && !dc) return RBF_OK;
  EvalParams P = make_eval_params(x);
  CostParams CP = cost_params(x->cfg);
  const Grid& g = x->grid;
  int ncell = g.nx * g.ny;
  Buf& qpsi = x->scratch(21);
  Buf& pcell = x->scratch(22);
  Buf& pcount = x->scratch(23);
  Buf& pstart = x->scratch(24);
  Buf& order = x->scratch(25);
  RBF_TRY(qpsi.ensure((size_t)n * sizeof(float4)));
  RBF_TRY(pcell.ensure((size_t)n * sizeof(int32_t)));
  RBF_TRY(pcount.ensure((size_t)(ncell + 1) * sizeof(int32_t)));
  RBF_TRY(pstart.ensure((size_t)(ncell + 1) * sizeof(int32_t)));
  RBF_TRY(order.ensure((size_t)n * sizeof(int32_t)));
  RBF_CUDA(cudaMemsetAsync(pcount.p, 0, (size_t)(ncell + 1) * sizeof(int32_t), s));
  unsigned nb = (unsigned)((n + 255) / 256);
  if (x->cfg.kernel == RBF_KERNEL_WENDLAND)
    { k_bwd_points<RBF_KERNEL_WENDLAND><<<nb, 256, 0, s>>>(
        P, x->cell_start.as<int32_t>(), x->sorted_xyw.as<float4>(), T, CP, pts, n, gout,
        qpsi.as<float4>(), pcell.as<int32_t>(), pcount.as<int32_t>()); ::rbf::note_launch(); }
  else
    { k_bwd_points<RBF_KERNEL_GAUSSIAN><<<nb, 256, 0, s>>>(
        P, x->cell_start.as<int32_t>(), x->sorted_xyw.as<float4>(), T, CP, pts, n, gout,
        qpsi.as<float4>(), pcell.as<int32_t>(), pcount.as<int32_t>()); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  RBF_TRY(scan_i32(x, pcount.as<int32_t>(), pstart.as<int32_t>(), ncell, s, 48));
  RBF_CUDA(cudaMemsetAsync(pcount.p, 0, (size_t)(ncell + 1) * sizeof(int32_t), s));
  { k_bwd_fill<<<nb, 256, 0, s>>>(pcell.as<int32_t>(), n, pstart.as<int32_t>(), pcount.as<int32_t>(),
                                order.as<int32_t>()); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  { k_bwd_sort<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(pstart.as<int32_t>(), ncell,
                                                             order.as<int32_t>()); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  unsigned nbc = (unsigned)((M + 255) / 256);
  if (x->cfg.kernel == RBF_KERNEL_WENDLAND)
    { k_bwd_centers<RBF_KERNEL_WENDLAND><<<nbc, 256, 0, s>>>(
        P, x->sorted_xyw.as<float4>(), x->sorted_id.as<int32_t>(), M, pstart.as<int32_t>(),
        order.as<int32_t>(), qpsi.as<float4>(), dw, (float2*)dc); ::rbf::note_launch(); }
  else
    { k_bwd_centers<RBF_KERNEL_GAUSSIAN><<<nbc, 256, 0, s>>>(
        P, x->sorted_xyw.as<float4>(), x->sorted_id.as<int32_t>(), M, pstart.as<int32_t>(),
        order.as<int32_t>(), qpsi.as<float4>(), dw, (float2*)dc); ::rbf::note_launch(); }
  RBF_CUDA(cudaGetLastError());
  return RBF_OK;
}

// ---------------------------------------------------------------------------
// Soft cost without any allocation.
//
// Some callers cannot allocate device memory once they are running: a
// scan-matching loop with a hard per-frame deadline (cudaMalloc and cudaFree
// may synchronize the whole device and take milliseconds), or an embedded
// process that reserves all of its GPU memory at start-up.  For them this
// variant keeps its scratch -- the per-block partial sums of the cost and the
// pose gradient -- in a fixed array of this file instead of a buffer the
// context grows on demand.
// ---------------------------------------------------------------------------
namespace rbf {

constexpr int NOALLOC_MAX_BLOCKS = 2048;  // partial sums of at most 2048 blocks: 128 KiB
static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_BLOCKS * 8];

static std::mutex g_noalloc_mu;
static double* g_noalloc_addr[256] = {};

// Device address of the array on device `dev` (the current device).  Host
// code cannot use the symbol itself: it is only a host-side stand-in.
static rbf_status noalloc_scratch(int dev, double** out) {
  if (dev < 0 || dev >= 256) return fail(RBF_EINVAL, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
    g_noalloc_addr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_addr[dev];
  return RBF_OK;
}

// Drop the cached address of device `dev`: a context is being created there,
// possibly after cudaDeviceReset invalidated every earlier device address.
void noalloc_forget(int dev) {
  if (dev < 0 || dev >= 256) return;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  g_noalloc_addr[dev] = nullptr;
}

}  // namespace rbf

extern "C" rbf_status rbf_soft_cost_noalloc(rbf_ctx* c, const double* R, const double* t, const float* pts,
                                            int64_t n, double* cost, double* grad6, float* resid,
                                            void* stream) {
  RBF_TRY(check_ctx(c, true));
  if (n < 0) return fail(RBF_EINVAL, "negative n");
  if (!cost && !grad6 && !resid) return fail(RBF_EINVAL, "no output requested");
  if (n > 0 && !pts) return fail(RBF_EINVAL, "null points");
  Pose T;
  RBF_TRY(load_pose(R, t, &T));
  Ctx* x = C(c);
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    if (cost) RBF_CUDA(cudaMemsetAsync(cost, 0, sizeof(double), s));
    if (grad6) RBF_CUDA(cudaMemsetAsync(grad6, 0, 6 * sizeof(double), s));
    return RBF_OK;
  }
  unsigned nb = grid_for(n, SC_THREADS, x->device, 4);
  if (nb > (unsigned)NOALLOC_MAX_BLOCKS)
    return fail(RBF_ERANGE, "this launch needs %u partial-sum blocks; the static scratch holds %d", nb,
                NOALLOC_MAX_BLOCKS);
  double* part = nullptr;
  RBF_TRY(noalloc_scratch(x->device, &part));
  EvalParams P = make_eval_params(x);
  CostParams CP = cost_params(x->cfg);
  // every block writes slots 0..6 of its row of 8 and the reduction reads only
  // those 7 slots of the nb blocks of this launch: nothing left by an earlier
  // call is used
  if (x->cfg.kernel == RBF_KERNEL_WENDLAND) {
    k_soft_cost<RBF_KERNEL_WENDLAND, 7><<<nb, SC_THREADS, 0, s>>>(
        P, x->cell_start.as<int32_t>(), x->sorted_xyw.as<float4>(), T, CP, pts, n, resid, part);
    ::rbf::note_launch();
  } else {
    k_soft_cost<RBF_KERNEL_GAUSSIAN, 7><<<nb, SC_THREADS, 0, s>>>(
        P, x->cell_start.as<int32_t>(), x->sorted_xyw.as<float4>(), T, CP, pts, n, resid, part);
    ::rbf::note_launch();
  }
  RBF_CUDA(cudaGetLastError());
  k_reduce_partials<<<1, 32, 0, s>>>(part, (int)nb, 7, nullptr, cost, grad6, nullptr);
  ::rbf::note_launch();
  RBF_CUDA(cudaGetLastError());
  return RBF_OK;
}
