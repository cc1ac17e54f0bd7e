// Batched terrain patches in persistent launches: the mixed-precision path of
// rbf_batch_update_eval.
//
// Every patch is its own terrain, updated once from the prior (Sec. III-C;
// from the prior this is the ridge estimate of Sec. III-B) and evaluated at
// its queries (Eq. RBF_fml).  All patches of a batch go through the same
// short sequence of launches, each over all patches at once, and the
// sequence is recorded into one CUDA graph per batch shape:
//
//  1. binning   the points of every patch are counted and sorted into
//               chunks of ch x ch lattice nodes (three launches);
//  2. Gram      persistent CTAs pull chunks from a counter; a CTA adds the
//               products m_{i,a} m_{i,b} and m_{i,a} z_i of the chunk's
//               points exactly (fixed-point integers, as the main update)
//               into a window of the band in shared memory, then flushes
//               the nonzero sums to the patch's band tiles with one global
//               atomic each;
//  3. merge     H' = lambda I + m~ m~^T per band tile (float64, in place) and
//               its float32 copy; u = m~ z;
//  4. factor    one cooperative launch factors every patch's band in float32
//               by 64 x 64 tiles; the tiles of all patches are owned
//               round-robin by the CTAs, each CTA runs a task list planned
//               on the host once per batch shape (updates, panel products,
//               diagonal factorizations and inverses, in an order every CTA
//               agrees on) and waits on per-tile ready flags with bounded
//               spins;
//  5. solve     refinement sweeps: persistent CTAs pull patches and solve
//               with the float32 factor by block substitution within the
//               band; a residual launch forms r = u - H' x in float64 over
//               every band tile (per-tile products, then a fixed-order sum
//               per row, so every run gives the same bits);
//  6. eval      h and grad h at every patch's queries (lattice window).
//
// A small autotuner picks, per power-of-two bucket of M, the chunk edge of
// the Gram (4 or 8 nodes) and the CTA size of the evaluation (128, 256 or
// 512 threads), by timing each option on the bucket's own patches during the
// first call of a batch shape.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "tiles.cuh"

namespace rbf {

// One patch, in plan order (largest M first).
struct BqPatch {
  double x0, y0, h;
  const float* pts;
  const float* q;
  double* w;
  float* hq;
  float2* gq;
  long long n, Q, M;
  long long pt0;     // first point in the batch numbering
  long long q0;      // first query
  long long tile0;   // first band tile
  long long vec0;    // first entry of the batch vectors (nb * 64 per patch)
  long long zd0;     // first diagonal-block inverse
  long long chunk0;  // first point chunk
  double gscale;     // fixed-point scale of the exact Gram sums (2^gs units per 1)
  int nx, rows, nb, bwb;
  int ch, cx, cy, ntile;
  int gs, pad;
  double inv_h;      // 1 / h
};

struct BqGeom {
  int kernel, rca, rce;
  float r2a, r2e;
  double inv_rho, g_scale, g_inv2s2, lambda;
  float e_inv_rho, e_inv2s2, e_gscale;
};

__device__ __forceinline__ double bq_node(double x0, int i, double h) {
  return __dadd_rn(x0, __dmul_rn((double)i + 0.5, h));
}

// largest p with start(p) <= g (starts ascending, start(0) <= g)
template <class F>
__device__ __forceinline__ int bq_find(int np, long long g, F start) {
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (start(mid) <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// lattice cell of a point (node floor(u), clamped to the lattice)
__device__ __forceinline__ void bq_cell(const BqPatch& p, float px, float py, int& ix, int& iy, double& pu,
                                        double& pv) {
  pu = ((double)px - p.x0) * p.inv_h - 0.5;
  pv = ((double)py - p.y0) * p.inv_h - 0.5;
  pu = fmin(fmax(pu, -1.0), (double)p.nx);
  pv = fmin(fmax(pv, -1.0), (double)p.rows);
  ix = (int)floor(pu);
  iy = (int)floor(pv);
}

// 1. binning --------------------------------------------------------------
__global__ void k_bq_count(const BqPatch* __restrict__ P, int np, long long npts, int32_t* __restrict__ pchunk,
                           int32_t* __restrict__ count, int* __restrict__ status) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= npts) return;
  const int p = bq_find(np, g, [&](int k) { return P[k].pt0; });
  const BqPatch& B = P[p];
  const long long i = g - B.pt0;
  const float px = B.pts[3 * i], py = B.pts[3 * i + 1], pz = B.pts[3 * i + 2];
  if (!(isfinite(px) && isfinite(py) && isfinite(pz))) {
    atomicOr(status, DEV_BAD_INDEX);
    pchunk[g] = -1;
    return;
  }
  int ix, iy;
  double pu, pv;
  bq_cell(B, px, py, ix, iy, pu, pv);
  ix = min(max(ix, 0), B.nx - 1);
  iy = min(max(iy, 0), B.rows - 1);
  const int c = (int)(B.chunk0 + (long long)(iy / B.ch) * B.cx + ix / B.ch);
  pchunk[g] = c;
  atomicAdd(count + c, 1);
}

__global__ void k_bq_fill(long long npts, const int32_t* __restrict__ pchunk, const int32_t* __restrict__ start,
                          int32_t* __restrict__ fill, int32_t* __restrict__ order) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= npts) return;
  const int c = pchunk[g];
  if (c < 0) return;
  order[start[c] + atomicAdd(fill + c, 1)] = (int32_t)g;
}

// 2. Gram -------------------------------------------------------------------
// window of a chunk: nodes chunk origin - rca + 1 .. chunk end - 1 + rca per
// axis (W = ch + 2 rca - 1); two neighbours of one point are at most
// 2 rca - 1 nodes apart per axis, so their window-local indices differ by at
// most BW = (2 rca - 1)(W + 1): the sums are kept as a band of the window
constexpr int BQ_MAXK = 64;    // in-support window nodes of one point kept in shared memory
constexpr int BQ_SLICE = 512;  // points of one Gram work item (a chunk with more is split)

// work items of every chunk: ceil(count / BQ_SLICE)
__global__ void k_bq_items(long long nchunks, const int32_t* __restrict__ count, int32_t* __restrict__ items) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nchunks) items[c] = (count[c] + BQ_SLICE - 1) / BQ_SLICE;
}

__device__ __forceinline__ int bq_window(int ch, int rca) { return ch + 2 * rca - 1; }
__device__ __forceinline__ int bq_band(int ch, int rca) { return (2 * rca - 1) * (bq_window(ch, rca) + 1); }

// a 128-bit value (lo, hi) added to a 128-bit accumulator
__device__ __forceinline__ void bq_add_u128_words(unsigned long long* U, unsigned long long lo, unsigned long long hi) {
  const unsigned long long old = atomicAdd(U, lo);
  const unsigned long long h = hi + ((old + lo < old) ? 1ull : 0ull);
  if (h != 0ull) atomicAdd(U + 1, h);
}

// Shared memory of the Gram: the band of the window as pairs of 32-bit words
// (low, high) -- a 64-bit sum kept as two halves so that every update is a
// native 32-bit shared-memory atomic (the carry of the low half goes to the
// high half) -- then one private 128-bit accumulator of u per warp and window
// node, updated without atomics (a point's window nodes are distinct).
__device__ __forceinline__ void bq_add_split(unsigned* G2, unsigned long long v) {
  const unsigned lo = (unsigned)v, hi = (unsigned)(v >> 32);
  const unsigned old = atomicAdd(G2, lo);
  const unsigned h = hi + ((old + lo < old) ? 1u : 0u);
  if (h) atomicAdd(G2 + 1, h);
}

__global__ void __launch_bounds__(256) k_bq_gram(const BqPatch* __restrict__ P, int np, BqGeom G,
                                                 const int32_t* __restrict__ cstart, const int32_t* __restrict__ order,
                                                 const int32_t* __restrict__ istart, long long cbeg, long long cend,
                                                 int* __restrict__ counter, unsigned long long* __restrict__ Gt,
                                                 unsigned long long* __restrict__ Ut) {
  extern __shared__ unsigned long long sg[];
  __shared__ int32_t sid[8][BQ_MAXK];
  __shared__ double smv[8][BQ_MAXK];
  __shared__ unsigned long long smq[8][BQ_MAXK];
  __shared__ FF nodex[64], nodey[64];  // window node coordinates (float-float), W <= 64
  __shared__ long long cur;
  const FF inv_rho = ff_of(G.inv_rho);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int rca = G.rca, R2 = 2 * rca;
  const long long ibeg = istart[cbeg], iend = istart[cend];
  for (;;) {
    if (tid == 0) cur = ibeg + atomicAdd(counter, 1);
    __syncthreads();
    const long long item = cur;
    if (item >= iend) return;
    // chunk of the item: the last c in [cbeg, cend) with istart[c] <= item
    long long clo = cbeg, chi = cend - 1;
    while (clo < chi) {
      const long long mid = (clo + chi + 1) >> 1;
      if (istart[mid] <= item) clo = mid;
      else chi = mid - 1;
    }
    const long long c = clo;
    const int p = bq_find(np, c, [&](int k) { return P[k].chunk0; });
    const BqPatch& B = P[p];
    const int lc = (int)(c - B.chunk0), bx = lc % B.cx, by = lc / B.cx;
    const int W = bq_window(B.ch, rca), BW = bq_band(B.ch, rca);
    const int wx0 = bx * B.ch - rca + 1, wy0 = by * B.ch - rca + 1;
    const int nG = W * W * (BW + 1);
    unsigned* sG = reinterpret_cast<unsigned*>(sg);        // nG pairs of words
    unsigned long long* sU = sg + nG + (long long)wid * 2 * W * W;  // this warp's u sums
    for (int e = tid; e < nG + 16 * W * W; e += blockDim.x) sg[e] = 0ull;
    if (tid < W) {
      nodex[tid] = ff_of(bq_node(B.x0, wx0 + tid, B.h));
      nodey[tid] = ff_of(bq_node(B.y0, wy0 + tid, B.h));
    }
    __syncthreads();
    const int a0 = cstart[c] + (int)(item - istart[c]) * BQ_SLICE;
    const int a1 = a0 + BQ_SLICE < cstart[c + 1] ? a0 + BQ_SLICE : cstart[c + 1];
    for (int a = a0 + wid; a < a1; a += 8) {
      const long long g = order[a];
      const long long i = g - B.pt0;
      const float px = B.pts[3 * i], py = B.pts[3 * i + 1], pz = B.pts[3 * i + 2];
      int ix, iy;
      double pu, pv;
      bq_cell(B, px, py, ix, iy, pu, pv);
      const int ib = ix - rca + 1, jb = iy - rca + 1;
      int K = 0;
      for (int t0 = 0; t0 < R2 * R2; t0 += 32) {
        const int t = t0 + lane;
        bool in = false;
        int li = 0;
        double m = 0.0;
        unsigned long long mq = 0ull;
        if (t < R2 * R2) {
          const int i2 = ib + t % R2, j2 = jb + t / R2;
          if (i2 >= 0 && i2 < B.nx && j2 >= 0 && j2 < B.rows && (long long)j2 * B.nx + i2 < B.M) {
            const FF cx = nodex[i2 - wx0], cy = nodey[j2 - wy0];
            if (d2_rn(px, py, cx.hi, cy.hi) < G.r2a) {  // cx.hi is the float32 rounding of the node
              li = (j2 - wy0) * W + (i2 - wx0);
              in = true;
              if (G.kernel == RBF_KERNEL_WENDLAND) {
                // m = (1 - s)^4 (4 s + 1), s = |p - c| / rho, in float-float
                const FF dx = ff_two_sum(__fsub_rn(px, cx.hi), -cx.lo);  // px - cx.hi is exact
                const FF dy = ff_two_sum(__fsub_rn(py, cy.hi), -cy.lo);
                const FF sr = ff_mul(ff_sqrt(ff_add(ff_mul(dx, dx), ff_mul(dy, dy))), inv_rho);
                const FF t = ff_add({1.f, 0.f}, {-sr.hi, -sr.lo});
                const FF t2 = ff_mul(t, t);
                const FF mm = ff_mul(ff_mul(t2, t2), ff_add({4.f * sr.hi, 4.f * sr.lo}, {1.f, 0.f}));
                m = (double)mm.hi + (double)mm.lo;
                mq = __float2ull_rn(ldexpf(mm.hi, 52)) + (unsigned long long)__float2ll_rn(ldexpf(mm.lo, 52));
              } else {
                const double ex = (double)px - ((double)cx.hi + (double)cx.lo);
                const double ey = (double)py - ((double)cy.hi + (double)cy.lo);
                m = row_value(G.kernel, ex * ex + ey * ey, G.inv_rho, G.g_scale, G.g_inv2s2);
                mq = __double2ull_rn(ldexp(m, 52));
              }
            }
          }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, in);
        const int pos = K + __popc(mask & ((1u << lane) - 1u));
        if (in && pos < BQ_MAXK) {
          sid[wid][pos] = li;
          smv[wid][pos] = m;
          smq[wid][pos] = mq;  // m in [0, 1] with 2^52 units per 1
        }
        K += __popc(mask);
      }
      K = K < BQ_MAXK ? K : BQ_MAXK;
      __syncwarp();
      // m z into this warp's private 128-bit sums (2^64 units per 1): the
      // lanes hold distinct nodes, and the warp's points come one at a time
      for (int t = lane; t < K; t += 32) {
        const double xz = smv[wid][t] * (double)pz;
        const double hi = floor(xz);
        const unsigned long long lo = __double2ull_rz(ldexp(xz - hi, 64));
        unsigned long long* u2 = sU + 2 * sid[wid][t];
        const unsigned long long o = u2[0];
        u2[0] = o + lo;
        u2[1] += (unsigned long long)((long long)hi + ((o + lo < o) ? 1ll : 0ll));
      }
      // products m_a m_b in integer arithmetic: the exact 106-bit product of
      // the 52-bit fixed-point values, rounded to 2^gs units per 1
      const int sh = 104 - B.gs;
      for (int t1 = 0; t1 < K; ++t1) {
        const int l1 = sid[wid][t1];
        const unsigned long long q1 = smq[wid][t1];
        for (int t2 = lane; t2 <= t1; t2 += 32) {
          const int l2 = sid[wid][t2];
          const unsigned long long q2 = smq[wid][t2];
          const unsigned long long phi = __umul64hi(q1, q2), plo = q1 * q2;
          const unsigned long long v = ((phi << (64 - sh)) | (plo >> sh)) + ((plo >> (sh - 1)) & 1ull);
          const int hi = l1 > l2 ? l1 : l2, lo = l1 > l2 ? l2 : l1;
          bq_add_split(sG + 2 * ((long long)hi * (BW + 1) + (hi - lo)), v);
        }
      }
      __syncwarp();
    }
    __syncthreads();
    // flush the nonzero window sums to the patch's band tiles
    for (int e = tid; e < nG; e += blockDim.x) {
      const unsigned long long v = (unsigned long long)sG[2 * e] | ((unsigned long long)sG[2 * e + 1] << 32);
      if (v == 0ull) continue;
      const int hi = e / (BW + 1), lo = hi - e % (BW + 1);
      const long long g1 = (long long)(wy0 + hi / W) * B.nx + (wx0 + hi % W);
      const long long g2 = (long long)(wy0 + lo / W) * B.nx + (wx0 + lo % W);
      const long long ga = g1 > g2 ? g1 : g2, gb = g1 > g2 ? g2 : g1;
      const int ti = (int)(ga >> 6), tl = (int)(gb >> 6);
      const long long t = B.tile0 + df_colstart(tl, B.nb, B.bwb) + (ti - tl);
      atomicAdd(Gt + t * 4096 + (ga & 63) * 64 + (gb & 63), v);
    }
    // the eight warps' u sums, added exactly, then to the patch's vector
    for (int li = tid; li < W * W; li += blockDim.x) {
      unsigned long long lo = 0ull, hi = 0ull;
      for (int w = 0; w < 8; ++w) {
        const unsigned long long* u2 = sg + nG + (long long)w * 2 * W * W + 2 * li;
        const unsigned long long o = lo;
        lo += u2[0];
        hi += u2[1] + ((lo < o) ? 1ull : 0ull);
      }
      if (lo == 0ull && hi == 0ull) continue;
      const long long gid = (long long)(wy0 + li / W) * B.nx + (wx0 + li % W);
      bq_add_u128_words(Ut + 2 * (B.vec0 + gid), lo, hi);
    }
    __syncthreads();
  }
}

// 3. merge: tile t of H' = lambda I + G (float64, in place of the integer
// sums; both triangles of a diagonal tile), its float32 copy, and u
__global__ void __launch_bounds__(256) k_bq_merge(const BqPatch* __restrict__ P, int np, double lambda,
                                                  unsigned long long* __restrict__ Gt, float* __restrict__ Wt,
                                                  const unsigned long long* __restrict__ Ut, double* __restrict__ u) {
  __shared__ long long sv[64 * 64];
  const long long t = blockIdx.x;
  const int p = bq_find(np, t, [&](int k) { return P[k].tile0; });
  const BqPatch& B = P[p];
  const int lt = (int)(t - B.tile0);
  int l = 0;
  while (df_colstart(l + 1, B.nb, B.bwb) <= lt) ++l;
  const int i = l + (lt - df_colstart(l, B.nb, B.bwb));
  const int ri = (int)min((long long)64, B.M - (long long)i * 64), rl = (int)min((long long)64, B.M - (long long)l * 64);
  unsigned long long* gt = Gt + t * 4096;
  for (int e = threadIdx.x; e < 4096; e += blockDim.x) sv[e] = (long long)gt[e];
  __syncthreads();
  double* ht = reinterpret_cast<double*>(gt);
  float* wt = Wt + t * 4096;
  const double inv = 1.0 / B.gscale;
  for (int e = threadIdx.x; e < 4096; e += blockDim.x) {
    const int r = e >> 6, cc = e & 63;
    double x = 0.0;
    if (r < ri && cc < rl) {
      if (i == l) {
        x = (double)(cc <= r ? sv[e] : sv[cc * 64 + r]) * inv;
        if (r == cc) x += lambda;
      } else {
        x = (double)sv[e] * inv;
      }
    }
    ht[e] = x;
    wt[e] = (float)x;
  }
  if (i == l && threadIdx.x < 64) {
    const int r = threadIdx.x;
    const long long v = B.vec0 + (long long)i * 64 + r;
    u[v] = r < ri ? (double)(long long)Ut[2 * v + 1] + ldexp((double)Ut[2 * v], -64) : 0.0;
  }
}

// 4. factor -----------------------------------------------------------------
// task: x = kind | patch << 2 (kind 0: update U(i, l; k), 1: panel P(i, l),
// 2: diagonal D(l)), y = i, z = l, w = k
struct BqFactorParams {
  const BqPatch* P;
  float* Wt;
  float* Zd;
  const int4* tasks;
  const int32_t* toff;  // tasks of CTA b: [toff[b], toff[b + 1])
  int* flags;           // ntiles ready flags, then the abort word
  int ntiles, epoch;
  int* status;
  long long spin;
};

__device__ __forceinline__ bool bq_wait2(const BqFactorParams& F, unsigned* seen, long long a, long long b,
                                         int* bail) {
  const int tid = threadIdx.x;
  if (tid == 0 || tid == 32) {
    const long long idx = tid == 0 ? a : b;
    if (idx >= 0 && !(seen[idx >> 5] & (1u << (idx & 31)))) {
      long long it = 0;
      bool ok = true;
      while (ld_acq(F.flags + idx) != F.epoch) {
        if (ld_acq(F.flags + F.ntiles) == F.epoch) {
          ok = false;
          break;
        }
        if (++it > F.spin) {
          atomicOr(F.status, DEV_TIMEOUT);
          st_rel(F.flags + F.ntiles, F.epoch);
          ok = false;
          break;
        }
        __nanosleep(32);
      }
      if (ok) atomicOr(seen + (idx >> 5), 1u << (idx & 31));
      else *bail = 1;
    }
  }
  __syncthreads();
  return *bail == 0;
}

constexpr int BQ_R0 = 2 * MB * MXS_LD + 32 * 33 + MB + 64;  // floats: diagonal factorization (>= two staged tiles)

__global__ void __launch_bounds__(TL_THREADS) k_bq_factor(BqFactorParams F) {
  extern __shared__ float fs[];
  __shared__ int bail;
  float* As = fs;
  float* Bs = fs + 64 * 64;
  unsigned* seen = reinterpret_cast<unsigned*>(fs + BQ_R0);
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  for (int e = tid; e < (F.ntiles + 31) / 32; e += TL_THREADS) seen[e] = 0u;
  if (tid == 0) bail = 0;
  __syncthreads();
  const int t0 = F.toff[blockIdx.x], t1 = F.toff[blockIdx.x + 1];
  for (int ti = t0; ti < t1; ++ti) {
    const int4 T = F.tasks[ti];
    const int kind = T.x & 3, p = T.x >> 2, i = T.y, l = T.z, k = T.w;
    const BqPatch& B = F.P[p];
    auto rows_of = [&](int b) { return (int)min((long long)64, B.M - (long long)b * 64); };
    auto gtile = [&](int r, int cidx) { return B.tile0 + df_colstart(cidx, B.nb, B.bwb) + (r - cidx); };
    if (kind == 0) {
      if (!bq_wait2(F, seen, gtile(i, k), i != l ? gtile(l, k) : -1, &bail)) return;
      const int ri = rows_of(i), rl = rows_of(l), ck = rows_of(k);
      df_stage(As, F.Wt + gtile(i, k) * 4096, 64, ri, ck);
      if (i != l) df_stage(Bs, F.Wt + gtile(l, k) * 4096, 64, rl, ck);
      __syncthreads();
      float acc[4][4] = {};
      df_mma(acc, As, i != l ? Bs : As, ty, tx);
      float* dst = F.Wt + gtile(i, l) * 4096;
#pragma unroll
      for (int uu = 0; uu < 4; ++uu) {
        const int r = ty * 4 + uu;
        float4* q4 = reinterpret_cast<float4*>(dst + r * 64 + tx * 4);
        float4 v = __ldcg(q4);
        v.x -= acc[uu][0];
        v.y -= acc[uu][1];
        v.z -= acc[uu][2];
        v.w -= acc[uu][3];
        __stcg(q4, v);
      }
      __syncthreads();
    } else if (kind == 1) {
      if (!bq_wait2(F, seen, gtile(l, l), -1, &bail)) return;
      const long long me = gtile(i, l);
      df_stage(As, F.Wt + me * 4096, 64, 64, 64);
      df_stage(Bs, F.Zd + (B.zd0 + l) * 4096, 64, 64, 64);
      __syncthreads();
      float acc[4][4] = {};
      df_mma(acc, As, Bs, ty, tx);
      float* dst = F.Wt + me * 4096;
      const int ri = rows_of(i);
#pragma unroll
      for (int uu = 0; uu < 4; ++uu) {
        const int r = ty * 4 + uu;
        float4 v = make_float4(acc[uu][0], acc[uu][1], acc[uu][2], acc[uu][3]);
        if (r >= ri) v = make_float4(0.f, 0.f, 0.f, 0.f);
        __stcg(reinterpret_cast<float4*>(dst + r * 64 + tx * 4), v);
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_rel(F.flags + me, F.epoch);
      }
    } else {
      float* Tm = fs;
      float* Z = Tm + MB * MXS_LD;
      float* Y = Z + MB * MXS_LD;
      float* rd = Y + 32 * 33;
      float* col = rd + MB;
      const long long me = gtile(l, l);
      const float* src = F.Wt + me * 4096;
      const int kb = rows_of(l);
      for (int e = tid; e < MB * MB; e += TL_THREADS) {
        const int r = e >> 6, cc = e & 63;
        float v = (r < kb && cc <= r) ? __ldcg(src + e) : 0.f;
        if (r >= kb && r == cc) v = 1.f;  // identity beyond a ragged last block
        Tm[r * MXS_LD + cc] = v;
        Z[r * MXS_LD + cc] = 0.f;
      }
      __syncthreads();
      tile_chol_inv(Tm, Z, Y, rd, col, F.status);
      float* zd = F.Zd + (B.zd0 + l) * 4096;
      float* dst = F.Wt + me * 4096;
      for (int e = tid; e < MB * MB; e += TL_THREADS) {
        const int r = e >> 6, cc = e & 63;
        __stcg(zd + e, Z[r * MXS_LD + cc]);
        __stcg(dst + e, (r < kb && cc <= r) ? Tm[r * MXS_LD + cc] : 0.f);
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_rel(F.flags + me, F.epoch);
      }
    }
  }
}

// 5. solve ------------------------------------------------------------------
// Row `row` (= tid / 4) of a 64 x 64 row-major tile (or of its transpose),
// columns 16 (tid % 4) .. + 15, loaded to registers.
__device__ __forceinline__ void bq_load16(const float* __restrict__ A, bool transpose, float (&v)[16]) {
  const int tid = threadIdx.x, row = tid >> 2, part = tid & 3;
  if (!transpose) {
    const float4* p = reinterpret_cast<const float4*>(A + row * 64 + part * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 t = __ldcg(p + q);
      v[4 * q] = t.x;
      v[4 * q + 1] = t.y;
      v[4 * q + 2] = t.z;
      v[4 * q + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __ldcg(A + (part * 16 + c) * 64 + row);
  }
}

__device__ __forceinline__ float bq_dot16(const float (&v)[16], const float* x) {
  const int part = threadIdx.x & 3;
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 16; ++c) s = fmaf(v[c], x[part * 16 + c], s);
  return s;
}

__device__ __forceinline__ float bq_quad_sum(float s) {
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  return s;
}

constexpr int BQ_SOLVE_GROUP = 4;  // band tiles of one block row applied per pass

// persistent: CTAs pull patches; solve H' c = r with the float32 factor
// (forward then backward block substitution within the band), then x += c.
// The band tiles of a block row are applied in passes of BQ_SOLVE_GROUP, their
// loads in flight together.
__global__ void __launch_bounds__(256) k_bq_solve(const BqPatch* __restrict__ P, int np, const float* __restrict__ Wt,
                                                  const float* __restrict__ Zd, const double* __restrict__ r,
                                                  float* __restrict__ f, double* __restrict__ x, int* __restrict__ counter) {
  __shared__ float acc[64], vk[BQ_SOLVE_GROUP][64];
  __shared__ int cur;
  const int tid = threadIdx.x, row = tid >> 2, part = tid & 3;
  for (;;) {
    if (tid == 0) cur = atomicAdd(counter, 1);
    __syncthreads();
    const int p = cur;
    if (p >= np) return;
    const BqPatch& B = P[p];
    auto gtile = [&](int rr, int cidx) { return B.tile0 + df_colstart(cidx, B.nb, B.bwb) + (rr - cidx); };
    float* fv = f + B.vec0;
    const double* rv = r + B.vec0;
    // forward: y_b = Z_bb (r_b - sum_k L_bk y_k)
    for (int b = 0; b < B.nb; ++b) {
      if (tid < 64) acc[tid] = (float)rv[b * 64 + tid];
      __syncthreads();
      const int k0 = b - B.bwb > 0 ? b - B.bwb : 0;
      float s = 0.f;
      for (int kg = k0; kg < b; kg += BQ_SOLVE_GROUP) {
        const int ng = b - kg < BQ_SOLVE_GROUP ? b - kg : BQ_SOLVE_GROUP;
        for (int e = tid; e < ng * 64; e += 256) vk[e >> 6][e & 63] = fv[(kg + (e >> 6)) * 64 + (e & 63)];
        __syncthreads();
        float v[BQ_SOLVE_GROUP][16];
#pragma unroll
        for (int j = 0; j < BQ_SOLVE_GROUP; ++j)
          if (j < ng) bq_load16(Wt + gtile(b, kg + j) * 4096, false, v[j]);
#pragma unroll
        for (int j = 0; j < BQ_SOLVE_GROUP; ++j)
          if (j < ng) s += bq_dot16(v[j], vk[j]);
        __syncthreads();
      }
      s = bq_quad_sum(s);
      if (part == 0) acc[row] -= s;
      __syncthreads();
      float zv[16];
      bq_load16(Zd + (B.zd0 + b) * 4096, false, zv);
      const float y = bq_quad_sum(bq_dot16(zv, acc));
      if (part == 0) fv[b * 64 + row] = y;
      __syncthreads();
    }
    // backward: c_b = Z_bb^T (y_b - sum_k L_kb^T c_k)
    for (int b = B.nb - 1; b >= 0; --b) {
      if (tid < 64) acc[tid] = fv[b * 64 + tid];
      __syncthreads();
      const int k1 = b + B.bwb < B.nb - 1 ? b + B.bwb : B.nb - 1;
      float s = 0.f;
      for (int kg = b + 1; kg <= k1; kg += BQ_SOLVE_GROUP) {
        const int ng = k1 + 1 - kg < BQ_SOLVE_GROUP ? k1 + 1 - kg : BQ_SOLVE_GROUP;
        for (int e = tid; e < ng * 64; e += 256) vk[e >> 6][e & 63] = fv[(kg + (e >> 6)) * 64 + (e & 63)];
        __syncthreads();
        float v[BQ_SOLVE_GROUP][16];
#pragma unroll
        for (int j = 0; j < BQ_SOLVE_GROUP; ++j)
          if (j < ng) bq_load16(Wt + gtile(kg + j, b) * 4096, true, v[j]);
#pragma unroll
        for (int j = 0; j < BQ_SOLVE_GROUP; ++j)
          if (j < ng) s += bq_dot16(v[j], vk[j]);
        __syncthreads();
      }
      s = bq_quad_sum(s);
      if (part == 0) acc[row] -= s;
      __syncthreads();
      float zv[16];
      bq_load16(Zd + (B.zd0 + b) * 4096, true, zv);
      const float cb = bq_quad_sum(bq_dot16(zv, acc));
      if (part == 0) {
        fv[b * 64 + row] = cb;
        if ((long long)b * 64 + row < B.M) x[B.vec0 + b * 64 + row] += (double)cb;
      }
      __syncthreads();
    }
  }
}

// residual, step 1: per band tile (i, l) the products H_il x_l (rows of
// block i) and, below the diagonal, H_il^T x_i (rows of block l)
__global__ void __launch_bounds__(256) k_bq_tile_products(const BqPatch* __restrict__ P, int np,
                                                          const double* __restrict__ Ht, const double* __restrict__ x,
                                                          double* __restrict__ part) {
  __shared__ double xs[2][64];
  __shared__ double red[4][64];
  const long long t = blockIdx.x;
  const int p = bq_find(np, t, [&](int k) { return P[k].tile0; });
  const BqPatch& B = P[p];
  const int lt = (int)(t - B.tile0);
  int l = 0;
  while (df_colstart(l + 1, B.nb, B.bwb) <= lt) ++l;
  const int i = l + (lt - df_colstart(l, B.nb, B.bwb));
  const int tid = threadIdx.x;
  if (tid < 64) xs[0][tid] = x[B.vec0 + (long long)l * 64 + tid];
  else if (tid < 128) xs[1][tid - 64] = x[B.vec0 + (long long)i * 64 + tid - 64];
  __syncthreads();
  const double* h = Ht + t * 4096;
  // H x_l: thread (rr = tid & 63, q = tid >> 6) sums 16 columns; H^T x_i likewise over rows
  const int rr = tid & 63, q = tid >> 6;
  double s = 0.0;
#pragma unroll 4
  for (int c = q * 16; c < q * 16 + 16; ++c) s = fma(h[rr * 64 + c], xs[0][c], s);
  red[q][rr] = s;
  __syncthreads();
  if (tid < 64) part[t * 128 + tid] = (red[0][tid] + red[1][tid]) + (red[2][tid] + red[3][tid]);
  __syncthreads();
  if (i != l) {
    double s2 = 0.0;
#pragma unroll 4
    for (int rw = q * 16; rw < q * 16 + 16; ++rw) s2 = fma(h[rw * 64 + rr], xs[1][rw], s2);
    red[q][rr] = s2;
    __syncthreads();
    if (tid < 64) part[t * 128 + 64 + tid] = (red[0][tid] + red[1][tid]) + (red[2][tid] + red[3][tid]);
  }
}

// residual, step 2: r = u - sum over the band tiles of the row block, in
// ascending order of the tile's column block
__global__ void k_bq_residual(const BqPatch* __restrict__ P, int np, long long nvec, const double* __restrict__ u,
                              const double* __restrict__ part, double* __restrict__ r) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvec) return;
  const int p = bq_find(np, v, [&](int k) { return P[k].vec0; });
  const BqPatch& B = P[p];
  const long long lv = v - B.vec0;
  const int i = (int)(lv >> 6), rr = (int)(lv & 63);
  if (lv >= B.M) {
    r[v] = 0.0;
    return;
  }
  double s = 0.0;
  const int k0 = i - B.bwb > 0 ? i - B.bwb : 0;
  for (int k = k0; k <= i; ++k) s += part[(B.tile0 + df_colstart(k, B.nb, B.bwb) + (i - k)) * 128 + rr];
  const int k1 = i + B.bwb < B.nb - 1 ? i + B.bwb : B.nb - 1;
  for (int k = i + 1; k <= k1; ++k) s += part[(B.tile0 + df_colstart(i, B.nb, B.bwb) + (k - i)) * 128 + 64 + rr];
  r[v] = u[v] - s;
}

__global__ void k_bq_store_w(const BqPatch* __restrict__ P, int np, long long nvec, const double* __restrict__ x) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvec) return;
  const int p = bq_find(np, v, [&](int k) { return P[k].vec0; });
  const BqPatch& B = P[p];
  const long long lv = v - B.vec0;
  if (lv < B.M) B.w[lv] = x[v];
}

// 6. evaluation over the lattice window (grid-stride over the queries of
// patches [p0, p1), numbered from qbeg)
__global__ void k_bq_eval(const BqPatch* __restrict__ P, int np, BqGeom G, long long qbeg, long long qend,
                          const double* __restrict__ x) {
  for (long long g = qbeg + (long long)blockIdx.x * blockDim.x + threadIdx.x; g < qend;
       g += (long long)gridDim.x * blockDim.x) {
    const int p = bq_find(np, g, [&](int k) { return P[k].q0; });
    const BqPatch& B = P[p];
    const long long k = g - B.q0;
    const float2 q = reinterpret_cast<const float2*>(B.q)[k];
    float ah = 0.f, ax = 0.f, ay = 0.f;
    if (isfinite(q.x) && isfinite(q.y)) {
      double pu = ((double)q.x - B.x0) / B.h - 0.5, pv = ((double)q.y - B.y0) / B.h - 0.5;
      pu = fmin(fmax(pu, -4.0 * G.rce - 4.0), (double)B.nx + 4.0 * G.rce);
      pv = fmin(fmax(pv, -4.0 * G.rce - 4.0), (double)B.rows + 4.0 * G.rce);
      const int ib = (int)floor(pu) - G.rce + 1, jb = (int)floor(pv) - G.rce + 1;
      for (int dj = 0; dj < 2 * G.rce; ++dj) {
        const int j = jb + dj;
        if (j < 0 || j >= B.rows) continue;
        const float dy = q.y - (float)bq_node(B.y0, j, B.h);
        for (int di = 0; di < 2 * G.rce; ++di) {
          const int i = ib + di;
          if (i < 0 || i >= B.nx) continue;
          const long long id = (long long)j * B.nx + i;
          if (id >= B.M) continue;
          const float dx = q.x - (float)bq_node(B.x0, i, B.h);
          const float d2 = fmaf(dx, dx, dy * dy);
          if (!(d2 < G.r2e)) continue;
          const float wf = (float)x[B.vec0 + id];
          if (G.kernel == RBF_KERNEL_WENDLAND) {
            const float s = sqrtf(d2) * G.e_inv_rho;
            const float t = fmaxf(1.f - s, 0.f);
            const float cw = wf * t * t * t;
            ah = fmaf(cw, t * fmaf(4.f, s, 1.f), ah);
            ax = fmaf(cw, dx, ax);
            ay = fmaf(cw, dy, ay);
          } else {
            const float e = wf * __expf(-d2 * G.e_inv2s2);
            ah += e;
            ax = fmaf(e, dx, ax);
            ay = fmaf(e, dy, ay);
          }
        }
      }
    } else {
      ah = ax = ay = __int_as_float(0x7fc00000);
    }
    B.hq[k] = ah;
    if (B.gq) B.gq[k] = make_float2(ax * G.e_gscale, ay * G.e_gscale);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static inline unsigned bq_blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Plan and workspace of one batch shape.
struct BqPlan {
  std::vector<unsigned char> key;
  std::vector<int32_t> order;       // plan position -> caller's patch index
  std::vector<BqPatch> patches;
  std::vector<int> bucket_of_pos;
  std::vector<std::pair<int, int>> buckets;  // [pos begin, pos end) per bucket, plan order
  long long npts = 0, nq = 0, ntiles = 0, nvec = 0, nzd = 0, nchunks = 0;
  int grid = 0;
  Buf dpatches, tasks, toff, tiles64, tiles32, zd, U, u, x, r, f, part, pchunk, order_pts, count, start, fill,
      istart, flags, counters;
  cudaGraphExec_t exec = nullptr;
  bool ran_eager = false;
  void release() {
    Buf* b[] = {&dpatches, &tasks, &toff, &tiles64, &tiles32, &zd, &U, &u, &x, &r, &f, &part, &pchunk, &order_pts,
                &count, &start, &fill, &istart, &flags, &counters};
    for (Buf* p : b) p->release();
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
  }
};

struct BqState {
  int ch[32] = {0};      // autotuned Gram chunk edge per log2(M) bucket (0: not yet tuned)
  int threads[32] = {0};  // autotuned evaluation CTA size per bucket
  std::vector<BqPlan*> plans;
  cudaStream_t cap = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

static int bq_bucket(int64_t M) {
  int b = 0;
  while ((int64_t(1) << (b + 1)) <= M && b < 30) ++b;
  return b;
}

static BqGeom bq_geom(const rbf_config& cfg, double spacing) {
  BqGeom G;
  G.kernel = cfg.kernel;
  const double ra = assembly_radius(cfg, 0.0), re = eval_radius(cfg);
  G.rca = (int)ceil(ra / spacing - 1e-9);
  G.rce = (int)ceil(re / spacing - 1e-9);
  const float ra32 = (float)ra, re32 = (float)re;
  G.r2a = ra32 * ra32;
  G.r2e = re32 * re32;
  G.inv_rho = 1.0 / cfg.rho;
  G.g_scale = 1.0;
  G.g_inv2s2 = 1.0 / (2.0 * cfg.sigma * cfg.sigma);
  G.lambda = cfg.lambda;
  G.e_inv_rho = (float)(1.0 / cfg.rho);
  G.e_inv2s2 = (float)(1.0 / (2.0 * cfg.sigma * cfg.sigma));
  G.e_gscale = cfg.kernel == RBF_KERNEL_WENDLAND ? (float)(-20.0 / (cfg.rho * cfg.rho))
                                                 : (float)(-1.0 / (cfg.sigma * cfg.sigma));
  return G;
}

static int64_t bq_colstart(int l, int nb, int bwb) {
  const int64_t full = nb - bwb > 0 ? nb - bwb : 0;
  if (l <= full) return (int64_t)l * (bwb + 1);
  const int64_t m = l - full, s0 = nb - full;
  return full * (bwb + 1) + m * s0 - m * (m - 1) / 2;
}

constexpr long long BQ_SPIN = 1LL << 22;

// chunk layout of every patch for the chosen edges (plan order)
static void bq_chunks(BqPlan& L) {
  long long c0 = 0;
  for (auto& B : L.patches) {
    B.cx = (B.nx + B.ch - 1) / B.ch;
    B.cy = (B.rows + B.ch - 1) / B.ch;
    B.chunk0 = c0;
    c0 += (long long)B.cx * B.cy;
  }
  L.nchunks = c0;
}

// Task lists of the factorization: the tiles of all patches are owned
// round-robin; every CTA runs its tasks in the global order (stage by stage,
// patches interleaved; within a patch and stage: updates of the next block
// column, its diagonal factorization, its panel tiles, the other updates).
static void bq_tasks(const BqPlan& L, int G, std::vector<int4>& tasks, std::vector<int32_t>& toff) {
  std::vector<std::vector<int4>> per((size_t)G);
  int maxnb = 0;
  for (auto& B : L.patches) maxnb = std::max(maxnb, B.nb);
  auto owner = [&](const BqPatch& B, int i, int l) {
    return (int)((B.tile0 + bq_colstart(l, B.nb, B.bwb) + (i - l)) % G);
  };
  for (int s = -1; s < maxnb - 1; ++s) {
    for (size_t pp = 0; pp < L.patches.size(); ++pp) {
      const BqPatch& B = L.patches[pp];
      const int nb = B.nb, bwb = B.bwb, c = s + 1;
      if (c >= nb) continue;
      const int pk = (int)pp << 2;
      const int imax = std::min(nb - 1, c + bwb);
      if (s >= 0)
        for (int i = c; i <= std::min(nb - 1, s + bwb); ++i) per[owner(B, i, c)].push_back(make_int4(pk | 0, i, c, s));
      per[owner(B, c, c)].push_back(make_int4(pk | 2, c, c, 0));
      for (int i = c + 1; i <= imax; ++i) per[owner(B, i, c)].push_back(make_int4(pk | 1, i, c, 0));
      if (s >= 0)
        for (int l = s + 2; l <= std::min(nb - 1, s + bwb); ++l)
          for (int i = l; i <= std::min(nb - 1, s + bwb); ++i) per[owner(B, i, l)].push_back(make_int4(pk | 0, i, l, s));
    }
  }
  toff.assign((size_t)G + 1, 0);
  tasks.clear();
  for (int b = 0; b < G; ++b) {
    toff[b] = (int32_t)tasks.size();
    tasks.insert(tasks.end(), per[b].begin(), per[b].end());
  }
  toff[G] = (int32_t)tasks.size();
}

static size_t bq_gram_smem(int ch, int rca) {
  const int W = ch + 2 * rca - 1, BW = (2 * rca - 1) * (W + 1);
  return (size_t)(W * W * (BW + 1) + 16 * W * W) * sizeof(unsigned long long);
}

void bq_destroy(void* state) {
  BqState* S = reinterpret_cast<BqState*>(state);
  if (!S) return;
  for (BqPlan* L : S->plans) {
    L->release();
    delete L;
  }
  if (S->cap) cudaStreamDestroy(S->cap);
  if (S->e0) cudaEventDestroy(S->e0);
  if (S->e1) cudaEventDestroy(S->e1);
  delete S;
}

// Every launch of one batch on stream s (also what the graph records).
// Gram and evaluation run per size bucket with the bucket's tuned knobs.
static rbf_status bq_enqueue(Ctx* c, BqState* S, BqPlan& L, const BqGeom& G, cudaStream_t s, int sms,
                             int only_bucket = -1, int gram_ch = 0, int eval_threads = 0, bool gram_only = false,
                             bool eval_only = false) {
  const int np = (int)L.patches.size();
  const BqPatch* dP = L.dpatches.as<BqPatch>();
  int* cnt = L.counters.as<int>();
  if (!eval_only) {
    RBF_CUDA(cudaMemsetAsync(L.counters.p, 0, 64 * sizeof(int), s));
    RBF_CUDA(cudaMemsetAsync(L.tiles64.p, 0, (size_t)L.ntiles * 4096 * sizeof(double), s));
    RBF_CUDA(cudaMemsetAsync(L.U.p, 0, (size_t)L.nvec * 2 * sizeof(unsigned long long), s));
    RBF_CUDA(cudaMemsetAsync(L.count.p, 0, (size_t)(L.nchunks + 1) * sizeof(int32_t), s));
    RBF_CUDA(cudaMemsetAsync(L.fill.p, 0, (size_t)(L.nchunks + 1) * sizeof(int32_t), s));
    if (L.npts > 0) {
      { k_bq_count<<<bq_blocks(L.npts), 256, 0, s>>>(dP, np, L.npts, L.pchunk.as<int32_t>(), L.count.as<int32_t>(),
                                                     c->dflag.as<int>()); ::rbf::note_launch(); }
      RBF_CUDA(cudaGetLastError());
    }
    RBF_TRY(scan_i32(c, L.count.as<int32_t>(), L.start.as<int32_t>(), L.nchunks, s, 90));
    if (L.npts > 0) {
      { k_bq_fill<<<bq_blocks(L.npts), 256, 0, s>>>(L.npts, L.pchunk.as<int32_t>(), L.start.as<int32_t>(),
                                                    L.fill.as<int32_t>(), L.order_pts.as<int32_t>()); ::rbf::note_launch(); }
      RBF_CUDA(cudaGetLastError());
    }
    // Gram work items (a chunk with many points is split into slices); the
    // fill counts are reused as the per-chunk item counts
    { k_bq_items<<<bq_blocks(L.nchunks), 256, 0, s>>>(L.nchunks, L.count.as<int32_t>(), L.fill.as<int32_t>()); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    RBF_TRY(scan_i32(c, L.fill.as<int32_t>(), L.istart.as<int32_t>(), L.nchunks, s, 93));
    for (size_t bk = 0; bk < L.buckets.size(); ++bk) {
      if (only_bucket >= 0 && (int)bk != only_bucket) continue;
      const int pb = L.buckets[bk].first, pe = L.buckets[bk].second;
      const long long cb = L.patches[pb].chunk0;
      const long long ce = pe < np ? L.patches[pe].chunk0 : L.nchunks;
      if (ce <= cb) continue;
      const int ch = L.patches[pb].ch;
      const size_t smem = bq_gram_smem(ch, G.rca);
      int occ = 0;
      RBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bq_gram, 256, smem));
      const unsigned grid = (unsigned)((long long)sms * std::max(occ, 1));
      { k_bq_gram<<<grid, 256, smem, s>>>(dP, np, G, L.start.as<int32_t>(), L.order_pts.as<int32_t>(),
                                          L.istart.as<int32_t>(), cb, ce, cnt + 32 + (int)bk,
                                          L.tiles64.as<unsigned long long>(), L.U.as<unsigned long long>()); ::rbf::note_launch(); }
      RBF_CUDA(cudaGetLastError());
    }
    if (gram_only) return RBF_OK;
    { k_bq_merge<<<(unsigned)L.ntiles, 256, 0, s>>>(dP, np, G.lambda, L.tiles64.as<unsigned long long>(),
                                                    L.tiles32.as<float>(), L.U.as<unsigned long long>(),
                                                    L.u.as<double>()); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
    // factorization: one cooperative launch over the task lists
    BqFactorParams F;
    F.P = dP;
    F.Wt = L.tiles32.as<float>();
    F.Zd = L.zd.as<float>();
    F.tasks = L.tasks.as<int4>();
    F.toff = L.toff.as<int32_t>();
    F.flags = L.flags.as<int>();
    F.ntiles = (int)L.ntiles;
    F.status = c->dflag.as<int>();
    F.spin = c->spin_limit > 0 ? c->spin_limit : BQ_SPIN;
    // ready flags start from zero in every run (graph replays included)
    RBF_CUDA(cudaMemsetAsync(L.flags.p, 0, (size_t)(L.ntiles + 1) * sizeof(int), s));
    F.epoch = 1;
    const size_t fsmem = (size_t)BQ_R0 * sizeof(float) + (size_t)((L.ntiles + 31) / 32) * sizeof(unsigned);
    void* args[] = {(void*)&F};
    RBF_CUDA(cooperative_launch((const void*)k_bq_factor, dim3((unsigned)L.grid), dim3(TL_THREADS), args, fsmem, s));
    // refined solves: x = 0; sweeps of (r = u - H x; solve; x += c)
    const int sweeps = std::min(c->refine_sweeps > 0 ? c->refine_sweeps : 3, 16);
    RBF_CUDA(cudaMemsetAsync(L.x.p, 0, (size_t)L.nvec * sizeof(double), s));
    RBF_CUDA(cudaMemcpyAsync(L.r.p, L.u.p, (size_t)L.nvec * sizeof(double), cudaMemcpyDeviceToDevice, s));
    for (int it = 0; it < sweeps; ++it) {
      if (it > 0) {
        { k_bq_tile_products<<<(unsigned)L.ntiles, 256, 0, s>>>(dP, np, reinterpret_cast<const double*>(L.tiles64.p),
                                                                L.x.as<double>(), L.part.as<double>()); ::rbf::note_launch(); }
        RBF_CUDA(cudaGetLastError());
        { k_bq_residual<<<bq_blocks(L.nvec), 256, 0, s>>>(dP, np, L.nvec, L.u.as<double>(), L.part.as<double>(),
                                                          L.r.as<double>()); ::rbf::note_launch(); }
        RBF_CUDA(cudaGetLastError());
      }
      { k_bq_solve<<<(unsigned)std::min(np, 4 * sms), 256, 0, s>>>(dP, np, L.tiles32.as<float>(), L.zd.as<float>(),
                                                               L.r.as<double>(), L.f.as<float>(), L.x.as<double>(),
                                                               cnt + 1 + it); ::rbf::note_launch(); }
      RBF_CUDA(cudaGetLastError());
    }
    { k_bq_store_w<<<bq_blocks(L.nvec), 256, 0, s>>>(dP, np, L.nvec, L.x.as<double>()); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }
  for (size_t bk = 0; bk < L.buckets.size(); ++bk) {
    if (only_bucket >= 0 && (int)bk != only_bucket) continue;
    const int pb = L.buckets[bk].first, pe = L.buckets[bk].second;
    const long long qb = L.patches[pb].q0;
    const long long qe = pe < np ? L.patches[pe].q0 : L.nq;
    if (qe <= qb) continue;
    const int th = eval_threads > 0 ? eval_threads : S->threads[L.bucket_of_pos[pb]];
    const unsigned grid = (unsigned)std::min<long long>((qe - qb + th - 1) / th, (long long)sms * (2048 / th));
    { k_bq_eval<<<grid, th, 0, s>>>(dP, np, G, qb, qe, L.x.as<double>()); ::rbf::note_launch(); }
    RBF_CUDA(cudaGetLastError());
  }
  (void)gram_ch;
  return RBF_OK;
}

// Build the plan of a batch shape: order, offsets, task lists, workspace.
static rbf_status bq_plan(Ctx* c, BqState* S, const rbf_patch* patches, int32_t npatch, BqPlan& L, int sms) {
  const BqGeom G = bq_geom(c->cfg, patches[0].spacing);
  L.order.resize((size_t)npatch);
  for (int32_t k = 0; k < npatch; ++k) L.order[k] = k;
  std::stable_sort(L.order.begin(), L.order.end(), [&](int32_t a, int32_t b) { return patches[a].M > patches[b].M; });
  L.patches.resize((size_t)npatch);
  L.bucket_of_pos.resize((size_t)npatch);
  long long pt = 0, qq = 0, tl = 0, vv = 0, zz = 0;
  for (int32_t pos = 0; pos < npatch; ++pos) {
    const rbf_patch& p = patches[L.order[pos]];
    BqPatch& B = L.patches[pos];
    memset(&B, 0, sizeof(B));
    B.x0 = p.x0;
    B.y0 = p.y0;
    B.h = p.spacing;
    B.pts = p.pts;
    B.q = p.q;
    B.w = p.w;
    B.hq = p.h;
    B.gq = reinterpret_cast<float2*>(p.grad);
    B.n = p.n;
    B.Q = p.Q;
    B.M = p.M;
    B.nx = p.nx;
    B.rows = (int)((p.M + p.nx - 1) / p.nx);
    B.nb = (int)((p.M + 63) / 64);
    // the update from the prior has the band of m~ m~^T: two centers coupled
    // through a point are at most 2 rca - 1 nodes apart per axis
    const int64_t bw = (int64_t)(2 * G.rca - 1) * ((int64_t)p.nx + 1);
    int bwb = B.nb - 1;
    if (bw < p.M) bwb = std::min<int64_t>(bwb, (bw + 63) / 64 + 1);
    B.bwb = bwb;
    B.ntile = (int)bq_colstart(B.nb, B.nb, B.bwb);
    B.pt0 = pt;
    B.q0 = qq;
    B.tile0 = tl;
    B.vec0 = vv;
    B.zd0 = zz;
    // sums of at most n products in [0, 1] with 2^gs units per 1 stay below
    // 2^62; gs >= 46 for the n < 65,536 of one 16-bit point count
    B.gs = 62 - (int)ceil(log2((double)p.n + 1.0));
    if (B.gs > 52) B.gs = 52;
    B.gscale = ldexp(1.0, B.gs);
    B.inv_h = 1.0 / p.spacing;
    const int bk = bq_bucket(p.M);
    L.bucket_of_pos[pos] = bk;
    B.ch = S->ch[bk] > 0 ? S->ch[bk] : 8;
    pt += p.n;
    qq += p.Q;
    tl += B.ntile;
    vv += (long long)B.nb * 64;
    zz += B.nb;
    if (pos == 0 || L.bucket_of_pos[pos - 1] != bk) L.buckets.push_back({pos, pos + 1});
    else L.buckets.back().second = pos + 1;
  }
  L.npts = pt;
  L.nq = qq;
  L.ntiles = tl;
  L.nvec = vv;
  L.nzd = zz;
  bq_chunks(L);
  // cooperative grid: every co-resident CTA (several per SM hide each
  // other's L2 latency; the task lists depend on the grid size)
  {
    const size_t fsmem = (size_t)BQ_R0 * sizeof(float) + (size_t)((L.ntiles + 31) / 32) * sizeof(unsigned);
    int occ = 0;
    RBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bq_factor, TL_THREADS, fsmem));
    occ = std::max(1, std::min(occ, 4));
    L.grid = (int)std::min<long long>((long long)sms * occ, L.ntiles);
  }
  std::vector<int4> tasks;
  std::vector<int32_t> toff;
  bq_tasks(L, L.grid, tasks, toff);
  RBF_TRY(L.dpatches.ensure(L.patches.size() * sizeof(BqPatch)));
  RBF_TRY(L.tasks.ensure(std::max<size_t>(tasks.size(), 1) * sizeof(int4)));
  RBF_TRY(L.toff.ensure(toff.size() * sizeof(int32_t)));
  RBF_TRY(L.tiles64.ensure((size_t)L.ntiles * 4096 * sizeof(double)));
  RBF_TRY(L.tiles32.ensure((size_t)L.ntiles * 4096 * sizeof(float)));
  RBF_TRY(L.zd.ensure((size_t)L.nzd * 4096 * sizeof(float)));
  RBF_TRY(L.U.ensure((size_t)L.nvec * 2 * sizeof(unsigned long long)));
  RBF_TRY(L.u.ensure((size_t)L.nvec * sizeof(double)));
  RBF_TRY(L.x.ensure((size_t)L.nvec * sizeof(double)));
  RBF_TRY(L.r.ensure((size_t)L.nvec * sizeof(double)));
  RBF_TRY(L.f.ensure((size_t)L.nvec * sizeof(float)));
  RBF_TRY(L.part.ensure((size_t)L.ntiles * 128 * sizeof(double)));
  RBF_TRY(L.pchunk.ensure((size_t)std::max<long long>(L.npts, 1) * sizeof(int32_t)));
  RBF_TRY(L.order_pts.ensure((size_t)std::max<long long>(L.npts, 1) * sizeof(int32_t)));
  // the chunk arrays are sized for the finest chunk edge the tuner tries
  long long maxchunks = 0;
  for (auto& B : L.patches) maxchunks += (long long)((B.nx + 3) / 4) * ((B.rows + 3) / 4);
  RBF_TRY(L.count.ensure((size_t)(maxchunks + 1) * sizeof(int32_t)));
  RBF_TRY(L.start.ensure((size_t)(maxchunks + 1) * sizeof(int32_t)));
  RBF_TRY(L.fill.ensure((size_t)(maxchunks + 1) * sizeof(int32_t)));
  RBF_TRY(L.istart.ensure((size_t)(maxchunks + 1) * sizeof(int32_t)));
  RBF_TRY(L.flags.ensure((size_t)(L.ntiles + 1) * sizeof(int)));
  RBF_TRY(L.counters.ensure(64 * sizeof(int)));
  RBF_CUDA(cudaMemcpy(L.tasks.p, tasks.data(), tasks.size() * sizeof(int4), cudaMemcpyHostToDevice));
  RBF_CUDA(cudaMemcpy(L.toff.p, toff.data(), toff.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  RBF_CUDA(cudaMemcpy(L.dpatches.p, L.patches.data(), L.patches.size() * sizeof(BqPatch), cudaMemcpyHostToDevice));
  return RBF_OK;
}

// Time each option of the two knobs on every bucket whose knobs are not tuned
// yet, then keep the faster.  The runs write the plan's workspace only; the
// real run follows.
static rbf_status bq_autotune(Ctx* c, BqState* S, BqPlan& L, const BqGeom& G, cudaStream_t s, int sms) {
  if (!S->e0) {
    RBF_CUDA(cudaEventCreate(&S->e0));
    RBF_CUDA(cudaEventCreate(&S->e1));
  }
  auto timed = [&](auto&& fn, float* ms) -> rbf_status {
    RBF_CUDA(cudaEventRecord(S->e0, s));
    RBF_TRY(fn());
    RBF_CUDA(cudaEventRecord(S->e1, s));
    RBF_CUDA(cudaEventSynchronize(S->e1));
    RBF_CUDA(cudaEventElapsedTime(ms, S->e0, S->e1));
    return RBF_OK;
  };
  const int chs[2] = {4, 8};
  const int ths[3] = {128, 256, 512};
  for (size_t bk = 0; bk < L.buckets.size(); ++bk) {
    const int b = L.bucket_of_pos[L.buckets[bk].first];
    if (!S->ch[b]) {
      float best = 1e30f;
      int pick = 8;
      for (int ch : chs) {
        if (bq_gram_smem(ch, G.rca) > 200 * 1024) continue;
        for (int pos = L.buckets[bk].first; pos < L.buckets[bk].second; ++pos) L.patches[pos].ch = ch;
        bq_chunks(L);
        RBF_CUDA(cudaMemcpyAsync(L.dpatches.p, L.patches.data(), L.patches.size() * sizeof(BqPatch),
                                 cudaMemcpyHostToDevice, s));
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep)
          RBF_TRY(timed([&]() { return bq_enqueue(c, S, L, G, s, sms, (int)bk, ch, 0, true, false); }, &ms));
        if (ms < best) {
          best = ms;
          pick = ch;
        }
      }
      S->ch[b] = pick;
      for (int pos = L.buckets[bk].first; pos < L.buckets[bk].second; ++pos) L.patches[pos].ch = pick;
    }
  }
  bq_chunks(L);
  RBF_CUDA(cudaMemcpyAsync(L.dpatches.p, L.patches.data(), L.patches.size() * sizeof(BqPatch), cudaMemcpyHostToDevice,
                           s));
  for (size_t bk = 0; bk < L.buckets.size(); ++bk) {
    const int b = L.bucket_of_pos[L.buckets[bk].first];
    if (S->threads[b]) continue;
    float best = 1e30f;
    int pick = 256;
    for (int th : ths) {
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep)
        RBF_TRY(timed([&]() { return bq_enqueue(c, S, L, G, s, sms, (int)bk, 0, th, false, true); }, &ms));
      if (ms < best) {
        best = ms;
        pick = th;
      }
    }
    S->threads[b] = pick;
  }
  return RBF_OK;
}

// The mixed-precision batch.  *handled = false when the batch is outside what
// this path serves (the caller then runs the per-patch pipelines).
rbf_status bq_run(Ctx* c, void** state, const rbf_patch* patches, int32_t npatch, cudaStream_t s, bool* handled) {
  *handled = false;
  const double h0 = patches[0].spacing;
  // (fixed-point Gram sums need n < 2^20 points per patch)
  for (int32_t k = 0; k < npatch; ++k)
    if (patches[k].spacing != h0 || patches[k].M > 65535 || patches[k].n >= (1 << 20) || npatch > (1 << 28))
      return RBF_OK;
  const BqGeom G = bq_geom(c->cfg, h0);
  if (G.rca < 1 || (2 * G.rca) * (2 * G.rca) > BQ_MAXK || bq_gram_smem(4, G.rca) > 200 * 1024 ||
      8 + 2 * G.rca - 1 > 64)
    return RBF_OK;
  int sms = 0;
  RBF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
  static bool attr_done[64] = {false};
  if (!attr_done[c->device & 63]) {
    RBF_CUDA(cudaFuncSetAttribute(k_bq_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    RBF_CUDA(cudaFuncSetAttribute(k_bq_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_done[c->device & 63] = true;
  }
  BqState* S = reinterpret_cast<BqState*>(*state);
  if (!S) {
    S = new (std::nothrow) BqState();
    if (!S) return fail(RBF_ENOMEM, "host allocation failed");
    *state = S;
  }
  std::vector<unsigned char> key((size_t)npatch * sizeof(rbf_patch));
  memcpy(key.data(), patches, key.size());
  BqPlan* L = nullptr;
  for (BqPlan* p : S->plans)
    if (p->key == key) L = p;
  // the factorization's task lists must fit the flag bitmap in shared memory
  if (!L) {
    L = new (std::nothrow) BqPlan();
    if (!L) return fail(RBF_ENOMEM, "host allocation failed");
    L->key = key;
    rbf_status st = bq_plan(c, S, patches, npatch, *L, sms);
    if (st == RBF_OK && (size_t)BQ_R0 * sizeof(float) + (size_t)((L->ntiles + 31) / 32) * sizeof(unsigned) > 200 * 1024)
      st = RBF_ERANGE;
    if (st != RBF_OK) {
      L->release();
      delete L;
      if (st == RBF_ERANGE) return RBF_OK;  // too large for this path
      return st;
    }
    if (S->plans.size() >= 4) {
      S->plans.front()->release();
      delete S->plans.front();
      S->plans.erase(S->plans.begin());
    }
    S->plans.push_back(L);
  }
  *handled = true;
  if (L->exec) {
    RBF_CUDA(cudaGraphLaunch(L->exec, s));
    ::rbf::note_launch();
  } else if (!L->ran_eager) {
    RBF_TRY(bq_autotune(c, S, *L, G, s, sms));
    RBF_TRY(bq_enqueue(c, S, *L, G, s, sms));
    L->ran_eager = true;
  } else {
    if (!S->cap) RBF_CUDA(cudaStreamCreateWithFlags(&S->cap, cudaStreamNonBlocking));
    RBF_CUDA(cudaStreamSynchronize(s));
    cudaGraph_t graph = nullptr;
    RBF_CUDA(cudaStreamBeginCapture(S->cap, cudaStreamCaptureModeThreadLocal));
    rbf_status st = bq_enqueue(c, S, *L, G, S->cap, sms);
    cudaError_t e2 = cudaStreamEndCapture(S->cap, &graph);
    if (st != RBF_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture", __FILE__, __LINE__);
    cudaError_t e3 = cudaGraphInstantiate(&L->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) return cuda_fail(e3, "cudaGraphInstantiate", __FILE__, __LINE__);
    RBF_CUDA(cudaGraphLaunch(L->exec, s));
    ::rbf::note_launch();
  }
  return RBF_OK;
}

}  // namespace rbf
