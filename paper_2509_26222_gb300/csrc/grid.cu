// Gaussian terrain and gradient on a regular raster, on the tensor cores.
//
// With the centers on the square lattice c_ij = (x_i, y_j) the Gaussian of
// Eq. RBF_def factorises per axis, exp(-(dx^2 + dy^2) / 2 s^2) = g(dx) g(dy),
// and so does the truncation when the window is taken per axis (|dx| < r and
// |dy| < r, r = cutoff_mult * s).  On a tile of 128 x 128 raster points
// (x_k, y_l) the terrain and its gradient (Eq. RBF_fml, Eq. manidolf_grad_detail
// with the sign of reading G5) are then products of small matrices over a
// window of kw x kw lattice nodes (kw = 32, or 64 for coarse rasters):
//     T1 = W Ex^T,   T2 = W Ex'^T                       (stage 1)
//     H = Ey T1,     Gx = Ey T2,     Gy = Ey' T1        (stage 2)
// with Ex[k][i] = g(x_k - x_i), Ex'[k][i] = -(x_k - x_i) / s^2 g(x_k - x_i), and
// Ey, Ey' likewise.  Both stages run as tcgen05 MMAs (M = 128, K = kw) with
// every float32 operand split into two bfloat16 parts, a = a_hi + a_lo, and the
// three products a_hi b_hi + a_hi b_lo + a_lo b_hi accumulated in float32 in
// tensor memory (relative error about 2^-16 per term).  The stage-1 results
// are read back from tensor memory, split the same way and written to shared
// memory as the K-major B operands of stage 2.
//
// Operand tiles are K-major, one row of kw bfloat16 per matrix row (64-byte
// swizzle for kw = 32, 128-byte for kw = 64), written by the CTA's threads with
// 16-byte shared stores.  Thread 0 issues the MMAs and commits them to an
// mbarrier; every wait is bounded, and a tile whose wait gives up is written
// as NaN.  The outputs leave through 128-byte swizzled 32 x 32 boxes and bulk
// tensor stores (TMA) where the rows are 16-byte pitched, else through per-warp
// transposes and row stores.  One persistent CTA per SM runs through a
// contiguous run of tiles.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>

#include <cmath>
#include <cstring>

#include "common.cuh"
#include "tc_util.cuh"

namespace rbf {
namespace {

constexpr int GT = 128;                 // raster points per tile side (M and N of stage 2)
constexpr int GK = 64;                  // largest window: lattice nodes per side (K of both stages, N of stage 1)
constexpr int BOX = 32 * 128;           // one 32 x 32 float32 output box (128-byte swizzle)
constexpr int NBOXES = 8 * 3;           // three per warp

// Shared-memory map for windows of KW nodes (offsets from the 1024-byte aligned
// base).  Operand rows hold KW bfloat16: 64 bytes with the 64-byte swizzle for
// KW = 32, 128 bytes with the 128-byte swizzle for KW = 64.  With KW = 32 the
// operands (68 KiB), T1^T and T2^T (32 KiB) and the output boxes (96 KiB) have
// their own space: a tile's bulk stores drain during the next tile, and Ex, Ex'
// stay for the next tile of the same raster column.  With KW = 64 (144 KiB of
// operands) stage 2 reuses the stage-1 A tiles for T1^T and T2^T, the boxes
// reuse the operand space and the next tile waits for their reads.
template <int KW>
struct Lay {
  static constexpr int RB = 2 * KW;       // bytes per operand row
  static constexpr int A = 128 * RB;      // 128-row operand tile
  static constexpr int B = KW * RB;       // KW-row weight tile
  static constexpr int EX_HI = 0, EX_LO = A, EXD_HI = 2 * A, EXD_LO = 3 * A;
  static constexpr int W_HI = 4 * A, W_LO = 4 * A + B;
  static constexpr int EY_HI = 4 * A + 2 * B, EY_LO = EY_HI + A, EYD_HI = EY_LO + A, EYD_LO = EYD_HI + A;
  static constexpr int OPS = EYD_LO + A;
  static constexpr bool SEPARATE = KW == 32;
  static constexpr int T1_HI = SEPARATE ? OPS : EX_HI, T1_LO = SEPARATE ? OPS + A : EX_LO;
  static constexpr int T2_HI = SEPARATE ? OPS + 2 * A : EXD_HI, T2_LO = SEPARATE ? OPS + 3 * A : EXD_LO;
  static constexpr int OPS2 = SEPARATE ? OPS + 4 * A : OPS;
  static constexpr int BOXES = SEPARATE ? (OPS2 + 1023) / 1024 * 1024 : 0;
  static constexpr int END = (BOXES + NBOXES * BOX > OPS2) ? BOXES + NBOXES * BOX : OPS2;
  static constexpr int SMEM = END + 1024;  // alignment slack
  static __device__ __forceinline__ uint32_t off(int r, int c) {
    return KW == 32 ? tc::sw64_offset(r, c) : tc::sw128_offset(r, c);
  }
  static __device__ __forceinline__ uint64_t desc(uint32_t saddr) {
    return KW == 32 ? tc::sdesc_sw64(saddr) : tc::sdesc_sw128(saddr);
  }
};
static_assert(Lay<32>::SMEM <= 227 * 1024 && Lay<64>::SMEM <= 227 * 1024, "shared memory per CTA");
static_assert(Lay<32>::W_LO % 512 == 0 && Lay<64>::W_LO % 1024 == 0, "swizzle atoms of the weight tiles");

// tensor-memory columns
constexpr uint32_t TM_D1 = 0, TM_D2 = 64, TM_H = 128, TM_GX = 256, TM_GY = 384, TM_COLS = 512;

// Instruction descriptor, kind::f16: D float32, A = B = bfloat16, both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(GT >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16_n(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accum,
                                           uint32_t idesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %3, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %4, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(accum), "r"(idesc));
}

// D = A B^T over K = KW as the three split products, A and B given as
// (hi, lo) shared-memory tiles.
template <int KW>
__device__ __forceinline__ void mma_split(uint32_t tmem_d, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                          uint32_t b_lo, uint32_t idesc) {
  const uint32_t as[3] = {a_hi, a_hi, a_lo};
  const uint32_t bs[3] = {b_hi, b_lo, b_hi};
  uint32_t accum = 0;
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const uint64_t ad = Lay<KW>::desc(as[p]), bd = Lay<KW>::desc(bs[p]);
#pragma unroll
    for (int kk = 0; kk < KW / 16; ++kk) {
      mma_bf16_n(tmem_d, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), accum, idesc);
      accum = 1;
    }
  }
}

// (hi, lo) bfloat16 parts of two floats, packed as the pair (v0, v1).
__device__ __forceinline__ void split2(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
  float2 hf = __bfloat1622float2(h);
  __nv_bfloat162 l = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
  hi = *reinterpret_cast<uint32_t*>(&h);
  lo = *reinterpret_cast<uint32_t*>(&l);
}

template <int KW>
__device__ __forceinline__ void st_chunk(uint8_t* tile, int row, int chunk, const uint32_t (&v)[4]) {
  *reinterpret_cast<uint4*>(tile + Lay<KW>::off(row, chunk)) = make_uint4(v[0], v[1], v[2], v[3]);
}

struct GridParams {
  double qx0, qy0, dq;  // raster point (k, l) = (qx0 + k dq, qy0 + l dq)
  int64_t nqx, nqy;
  double lx0, ly0, lh;  // lattice node i at lx0 + (i + 1/2) lh
  double r;             // window radius (float64, for the window origins)
  double inv_lh;        // 1 / lh
  int nx, ny;
  float r2;             // fl32(r)^2 rounded to float32 (membership rule)
  float inv2s2, inv_s2; // 1 / (2 s^2), 1 / s^2
  int kw;               // window width in nodes: 32 or 64 (K of both stages, N of stage 1)
};

// First lattice node of the window of a tile whose first raster coordinate
// is q (one node of slack below; the host picks kw so that kw nodes cover the
// tile).
__device__ __forceinline__ int window_origin(double q, double r, double l0, double inv_lh, int n) {
  double t = (q - r - l0) * inv_lh - 0.5;
  if (!(t > -2.0)) t = -2.0;
  if (t > (double)n) t = (double)n;
  int i = (int)floor(t) - 1;
  return i < 0 ? 0 : i;
}

// Rows of g and g' for one raster coordinate q over the kw window nodes in
// shared memory (nodes past the lattice hold NaN, which fails the test;
// raster points outside the raster give zeros).
template <int KW>
__device__ __forceinline__ void axis_rows(uint8_t* smem, int s_hi, int s_lo, int s_dhi, int s_dlo, int row,
                                          bool in, float q, const float* nodes, const GridParams& P,
                                          int c_begin = 0, int c_end = KW / 8) {
#pragma unroll 1
  for (int c = c_begin; c < c_end; ++c) {
    uint32_t hv[4], lv[4], dhv[4], dlv[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float g[2], gd[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float d = __fsub_rn(q, nodes[c * 8 + 2 * e + u]);
        const float d2 = __fmul_rn(d, d);
        g[u] = 0.f;
        gd[u] = 0.f;
        if (in && d2 < P.r2) {
          g[u] = __expf(-d2 * P.inv2s2);
          gd[u] = -(d * P.inv_s2) * g[u];
        }
      }
      split2(g[0], g[1], hv[e], lv[e]);
      split2(gd[0], gd[1], dhv[e], dlv[e]);
    }
    st_chunk<KW>(smem + s_hi, row, c, hv);
    st_chunk<KW>(smem + s_lo, row, c, lv);
    st_chunk<KW>(smem + s_dhi, row, c, dhv);
    st_chunk<KW>(smem + s_dlo, row, c, dlv);
  }
}

// Bounded wait of thread 0 for the MMAs committed to `mbar` (phase `ph`);
// the verdict goes to every thread through shared memory.
__device__ __forceinline__ bool wait_mma(uint64_t* mbar, uint32_t ph, int* done_s) {
  if (threadIdx.x == 0) {
    long long it = 0;
    bool ok;
    while (!(ok = tc::mbar_try_wait(mbar, ph)) && ++it < tc::WAIT_LIMIT) {
    }
    *done_s = ok ? 1 : 0;
  }
  __syncthreads();
  tc::fence_after();
  return *done_s != 0;
}

// Bulk tensor store of a 32 x 32 float32 box (128-byte swizzled in shared
// memory) at element coordinates (x, y) of the map; the hardware clips what
// lies outside the tensor.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(tc::smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

constexpr int GTHREADS = 256;  // 8 warps: two per tensor-memory lane quadrant
constexpr int TP = 33;         // padded row of the per-warp transpose buffers

// Persistent: each CTA takes a contiguous run of tiles in column-major order
// (tile = tx * nty + ty), so that consecutive tiles mostly share a raster
// column and, with KW = 32 and bulk stores, Ex and Ex' are generated once per
// column.  The bulk stores of a tile drain while the next tile is computed.
template <int KW>
__global__ void __launch_bounds__(GTHREADS) k_eval_grid_tc(GridParams P, const float* __restrict__ xs,
                                                           const float* __restrict__ ys,
                                                           const float* __restrict__ W, float* __restrict__ hout,
                                                           float* __restrict__ gout,
                                                           const __grid_constant__ CUtensorMap map_h,
                                                           const __grid_constant__ CUtensorMap map_g, int use_tma,
                                                           int64_t ntx, int64_t ntiles) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int done_s;
  __shared__ int org[2];
  __shared__ float sx[GK], sy[GK];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int quad = warp & 3;  // tensor-memory lanes 32 quad .. 32 quad + 31
  if (warp == 0) tc::tmem_alloc(&tmem_slot, TM_COLS);
  if (t == 0) tc::mbar_init(&mbar, 1);
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t base = tc::smem_u32(sm);
  const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
  const int row = quad * 32 + lane;  // the tile row this thread reads from tensor memory
  const bool want_g = gout != nullptr;
  bool healthy = true;     // false once a wait has given up: no further MMAs are issued
  uint32_t phase = 0;      // parity of the barrier phase the next commit completes
  uint32_t last = 0;       // parity of the last committed phase
  bool any = false;        // something was committed

  using L = Lay<KW>;
  const int64_t nty = ntiles / ntx;
  const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  const int64_t t_begin = (int64_t)blockIdx.x * per;
  const int64_t t_end = (t_begin + per) < ntiles ? (t_begin + per) : ntiles;
  int64_t ex_col = -1;  // raster column of tiles whose Ex, Ex' the operand tiles hold
  for (int64_t tile = t_begin; tile < t_end; ++tile) {
    const int64_t bx = tile / nty, by = tile % nty;
    const int64_t k0 = bx * GT, l0 = by * GT;
    // the transposing stores reuse the operand space, so Ex, Ex' stay only
    // with the bulk stores
    const bool keep_ex = L::SEPARATE && use_tma && bx == ex_col;
    ex_col = (L::SEPARATE && use_tma) ? bx : -1;
    // boxes over the operands: the previous tile's boxes have been read
    if (!L::SEPARATE && use_tma && lane == 0) bulk_wait_read();
    if (t == 0) {
      org[0] = window_origin(P.qx0 + (double)k0 * P.dq, P.r, P.lx0, P.inv_lh, P.nx);
      org[1] = window_origin(P.qy0 + (double)l0 * P.dq, P.r, P.ly0, P.inv_lh, P.ny);
    }
    __syncthreads();
    const int io = org[0], jo = org[1];
    if (t < GK) sx[t] = (io + t < P.nx) ? xs[io + t] : __int_as_float(0x7fc00000);
    else if (t < 2 * GK) sy[t - GK] = (jo + t - GK < P.ny) ? ys[jo + t - GK] : __int_as_float(0x7fc00000);
    {
      // window weights, kw x kw: row j (N of stage 1), nodes i (K); 8 nodes
      // per chunk, kw * kw / 8 chunks over the threads
      constexpr int cpr = KW / 8;  // chunks per row
#pragma unroll 1
      for (int q = t; q < KW * cpr; q += GTHREADS) {
        const int j = q / cpr, c = q % cpr, jg = jo + j;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int ig = io + c * 8 + e;
          v[e] = (jg < P.ny && ig < P.nx) ? W[(int64_t)jg * P.nx + ig] : 0.f;
        }
        uint32_t hv[4], lv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split2(v[2 * e], v[2 * e + 1], hv[e], lv[e]);
        st_chunk<KW>(sm + L::W_HI, j, c, hv);
        st_chunk<KW>(sm + L::W_LO, j, c, lv);
      }
    }
    __syncthreads();
    // operands: threads 0-127 row t of Ex, Ex' (raster column k0 + t); threads
    // 128-255 row t - 128 of Ey, Ey' (raster row l0 + t - 128)
    if (keep_ex) {
      // Ex, Ex' kept: two threads per row of Ey, Ey', half the chunks each
      const int r = t >> 1, cb = (t & 1) * (KW / 16);
      const int64_t l = l0 + r;
      const float qy = (float)__dadd_rn(P.qy0, __dmul_rn((double)l, P.dq));
      axis_rows<KW>(sm, L::EY_HI, L::EY_LO, L::EYD_HI, L::EYD_LO, r, l < P.nqy, qy, sy, P, cb, cb + KW / 16);
    } else if (t < GT) {
      const int64_t k = k0 + t;
      const float qx = (float)__dadd_rn(P.qx0, __dmul_rn((double)k, P.dq));
      axis_rows<KW>(sm, L::EX_HI, L::EX_LO, L::EXD_HI, L::EXD_LO, t, k < P.nqx, qx, sx, P);
    } else {
      const int64_t l = l0 + (t - GT);
      const float qy = (float)__dadd_rn(P.qy0, __dmul_rn((double)l, P.dq));
      axis_rows<KW>(sm, L::EY_HI, L::EY_LO, L::EYD_HI, L::EYD_LO, t - GT, l < P.nqy, qy, sy, P);
    }
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();

    bool ok = healthy;
    if (ok) {
      // stage 1: T1^T = Ex W^T and T2^T = Ex' W^T (rows = raster columns k, columns = window rows j)
      if (t == 0) {
        mma_split<KW>(tmem + TM_D1, base + L::EX_HI, base + L::EX_LO, base + L::W_HI, base + L::W_LO, idesc_bf16(KW));
        mma_split<KW>(tmem + TM_D2, base + L::EXD_HI, base + L::EXD_LO, base + L::W_HI, base + L::W_LO,
                      idesc_bf16(KW));
        tc::mma_commit(&mbar);
      }
      last = phase;
      any = true;
      ok = wait_mma(&mbar, phase, &done_s);
      phase ^= 1u;
    }
    if (ok) {
      // T1^T (warps 0-3) and T2^T (warps 4-7) back from tensor memory, split and
      // stored as the K-major B operands of stage 2 (over the stage-1 A tiles
      // for KW = 64, in their own space for KW = 32)
      const int which = warp >> 2;
      uint8_t* thi = sm + (which ? L::T2_HI : L::T1_HI);
      uint8_t* tlo = sm + (which ? L::T2_LO : L::T1_LO);
#pragma unroll 1
      for (int half = 0; half < KW / 32; ++half) {
        float v[32];
        tc::tmem_ld32(lane_base + (which ? TM_D2 : TM_D1) + (uint32_t)(half * 32), v);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          uint32_t hv[4], lv[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) split2(v[c * 8 + 2 * e], v[c * 8 + 2 * e + 1], hv[e], lv[e]);
          st_chunk<KW>(thi, row, half * 4 + c, hv);
          st_chunk<KW>(tlo, row, half * 4 + c, lv);
        }
      }
      tc::fence_proxy_async();
      tc::fence_before();
      __syncthreads();
      tc::fence_after();
      // stage 2: H = Ey T1, Gx = Ey T2, Gy = Ey' T1 (rows = raster rows l, columns = raster columns k)
      if (t == 0) {
        mma_split<KW>(tmem + TM_H, base + L::EY_HI, base + L::EY_LO, base + L::T1_HI, base + L::T1_LO, idesc_bf16(GT));
        mma_split<KW>(tmem + TM_GX, base + L::EY_HI, base + L::EY_LO, base + L::T2_HI, base + L::T2_LO, idesc_bf16(GT));
        mma_split<KW>(tmem + TM_GY, base + L::EYD_HI, base + L::EYD_LO, base + L::T1_HI, base + L::T1_LO,
                      idesc_bf16(GT));
        tc::mma_commit(&mbar);
      }
      last = phase;
      ok = wait_mma(&mbar, phase, &done_s);
      phase ^= 1u;
    }
    if (!ok) healthy = false;

    // epilogue: warp w takes tile rows 32 (w % 4) .. + 31 and columns
    // 64 (w / 4) .. + 63 in two blocks of 32; the tensor-memory loads are
    // warp-wide (.sync.aligned).  The operand tiles are free once the stage-2
    // MMAs have completed.
    if (use_tma) {
      // rows of the blocks into 128-byte swizzled boxes (row `lane` of a box is
      // this thread's tensor-memory row), then bulk tensor stores by one lane:
      // h, and grad h as two boxes of 16 (d/dx, d/dy) pairs
      uint8_t* bh = sm + L::BOXES + warp * (3 * BOX);
      uint8_t* bg0 = bh + BOX;
      uint8_t* bg1 = bg0 + BOX;
      const int64_t y0 = l0 + quad * 32;
#pragma unroll 1
      for (int b = 0; b < 2; ++b) {
        const int cb = (warp >> 2) * 2 + b;
        const int64_t kb = k0 + cb * 32;
        if (kb >= P.nqx) break;  // uniform over the warp
        uint32_t rh[32], rx[32], ry[32];  // float32 bit patterns
        if (ok) {
          // the three loads in flight together, one wait
          tc::tmem_ld32_nowait(lane_base + TM_H + (uint32_t)(cb * 32), rh);
          if (want_g) {
            tc::tmem_ld32_nowait(lane_base + TM_GX + (uint32_t)(cb * 32), rx);
            tc::tmem_ld32_nowait(lane_base + TM_GY + (uint32_t)(cb * 32), ry);
          }
          tc::tmem_wait_ld(rh);
          if (want_g) {
            tc::tmem_wait_ld(rx);
            tc::tmem_wait_ld(ry);
          }
        } else {
#pragma unroll
          for (int e = 0; e < 32; ++e) rh[e] = rx[e] = ry[e] = 0x7fc00000u;
        }
        if (lane == 0) bulk_wait_read();  // the boxes' previous stores have read them
        __syncwarp();
#pragma unroll
        for (int c = 0; c < 8; ++c)
          *reinterpret_cast<uint4*>(bh + tc::sw128_offset(lane, c)) =
              make_uint4(rh[4 * c], rh[4 * c + 1], rh[4 * c + 2], rh[4 * c + 3]);
        if (want_g) {
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            *reinterpret_cast<uint4*>(bg0 + tc::sw128_offset(lane, c)) =
                make_uint4(rx[2 * c], ry[2 * c], rx[2 * c + 1], ry[2 * c + 1]);
            *reinterpret_cast<uint4*>(bg1 + tc::sw128_offset(lane, c)) =
                make_uint4(rx[16 + 2 * c], ry[16 + 2 * c], rx[17 + 2 * c], ry[17 + 2 * c]);
          }
        }
        tc::fence_proxy_async();
        __syncwarp();
        if (lane == 0 && y0 < P.nqy) {
          tma_store_2d(&map_h, bh, (int)kb, (int)y0);
          if (want_g) {
            tma_store_2d(&map_g, bg0, (int)(2 * kb), (int)y0);
            if (kb + 16 < P.nqx) tma_store_2d(&map_g, bg1, (int)(2 * kb + 32), (int)y0);  // starts inside the tensor
          }
          bulk_commit();
        }
      }
    } else {
      // each block goes through a padded per-warp buffer so that the global
      // stores write whole rows: 128 contiguous bytes of h and 256 of grad h
      float* th = reinterpret_cast<float*>(sm) + warp * (3 * 32 * TP);
      float* tx = th + 32 * TP;
      float* ty = tx + 32 * TP;
#pragma unroll 1
      for (int b = 0; b < 2; ++b) {
        const int cb = (warp >> 2) * 2 + b;
        const int64_t kb = k0 + cb * 32;
        if (kb >= P.nqx) break;  // uniform over the warp
        float vh[32], vx[32], vy[32];
        if (ok) {
          tc::tmem_ld32(lane_base + TM_H + (uint32_t)(cb * 32), vh);
          if (want_g) {
            tc::tmem_ld32(lane_base + TM_GX + (uint32_t)(cb * 32), vx);
            tc::tmem_ld32(lane_base + TM_GY + (uint32_t)(cb * 32), vy);
          }
        } else {
#pragma unroll
          for (int e = 0; e < 32; ++e) vh[e] = vx[e] = vy[e] = __int_as_float(0x7fc00000);
        }
#pragma unroll
        for (int e = 0; e < 32; ++e) th[lane * TP + e] = vh[e];
        if (want_g) {
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            tx[lane * TP + e] = vx[e];
            ty[lane * TP + e] = vy[e];
          }
        }
        __syncwarp();
        const int64_t k = kb + lane;
        const bool kin = k < P.nqx;
#pragma unroll 4
        for (int r = 0; r < 32; ++r) {
          const int64_t l = l0 + quad * 32 + r;
          if (l >= P.nqy) break;  // uniform over the warp
          if (kin) {
            hout[l * P.nqx + k] = th[r * TP + lane];
            if (want_g)
              *reinterpret_cast<float2*>(gout + 2 * (l * P.nqx + k)) = make_float2(tx[r * TP + lane], ty[r * TP + lane]);
          }
        }
        __syncwarp();
      }
    }
    tc::fence_before();  // tensor-memory loads of this tile before the next tile's MMAs
    __syncthreads();
    tc::fence_after();
  }
  if (use_tma && lane == 0) bulk_wait();  // the stores have completed before the CTA ends
  if (!healthy && any && t == 0) {
    // give the MMAs of the last committed phase one more bounded chance to
    // drain before tensor memory is freed (a commit arrives once every earlier
    // MMA of the thread has completed)
    long long it = 0;
    while (!tc::mbar_try_wait(&mbar, last) && ++it < tc::WAIT_LIMIT) {
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, TM_COLS);
}

}  // namespace

}  // namespace rbf

using namespace rbf;

namespace {
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver (no link against libcuda); looked up
// once, thread-safely (initialisation of a function-local static)
EncodeTiled encode_tiled() {
  static const EncodeTiled fn = []() -> EncodeTiled {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiled>(p);
    return nullptr;
  }();
  return fn;
}
}  // namespace

extern "C" rbf_status rbf_eval_grid(rbf_ctx* cx, double qx0, double qy0, double dq, int64_t nqx, int64_t nqy,
                                    float* h, float* grad, void* stream) {
  RBF_TRY(check_ctx(cx, true));
  if (nqx < 0 || nqy < 0) return fail(RBF_EINVAL, "negative raster size");
  if (!std::isfinite(qx0) || !std::isfinite(qy0) || !std::isfinite(dq) || !(dq > 0.0))
    return fail(RBF_EINVAL, "raster origin and spacing must be finite, spacing > 0");
  if (nqx == 0 || nqy == 0) return RBF_OK;
  if (!h) return fail(RBF_EINVAL, "null h");
  if ((uintptr_t)h % 4 != 0 || (grad && (uintptr_t)grad % 8 != 0))
    return fail(RBF_EINVAL, "h must be 4-byte and grad 8-byte aligned");
  Ctx* c = C(cx);
  if (c->cfg.kernel != RBF_KERNEL_GAUSSIAN)
    return fail(RBF_EINVAL, "the raster evaluation needs the Gaussian kernel (it factorises per axis)");
  if (!c->lat.on) return fail(RBF_EINVAL, "the raster evaluation needs the centers on a square lattice");
  const double r = eval_radius(c->cfg);
  // one tile spans 127 dq + 2 r; with the slack of the window origin it must
  // fit in 64 lattice nodes
  if (127.0 * dq + 2.0 * r > 60.5 * c->lat.h)
    return fail(RBF_ERANGE, "raster spacing %g too coarse for 64-node windows (at most %g); use rbf_eval", dq,
                (60.5 * c->lat.h - 2.0 * r) / 127.0);
  const int64_t tx = (nqx + GT - 1) / GT, ty = (nqy + GT - 1) / GT;
  if (tx > 0x7fffffffLL || ty > 0x7fffffffLL) return fail(RBF_ERANGE, "raster too large");
  if (!std::isfinite(qx0 + (double)(nqx - 1) * dq) || !std::isfinite(qy0 + (double)(nqy - 1) * dq))
    return fail(RBF_EINVAL, "raster coordinates overflow");
  GridParams P;
  P.qx0 = qx0;
  P.qy0 = qy0;
  P.dq = dq;
  P.nqx = nqx;
  P.nqy = nqy;
  P.lx0 = c->lat.x0;
  P.ly0 = c->lat.y0;
  P.lh = c->lat.h;
  P.r = r;
  P.inv_lh = 1.0 / c->lat.h;
  P.nx = c->lat.nx;
  P.ny = c->lat.ny;
  const float r32 = (float)r;
  P.r2 = r32 * r32;
  P.inv2s2 = (float)(1.0 / (2.0 * c->cfg.sigma * c->cfg.sigma));
  P.inv_s2 = (float)(1.0 / (c->cfg.sigma * c->cfg.sigma));
  // windows of 32 nodes where they cover a tile (half the operands and MMAs)
  P.kw = (127.0 * dq + 2.0 * r <= 28.5 * c->lat.h) ? 32 : 64;
  cudaStream_t s = (cudaStream_t)stream;
  static bool attr_set[64] = {false};
  if (!attr_set[c->device & 63]) {
    RBF_CUDA(cudaFuncSetAttribute(k_eval_grid_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay<32>::SMEM));
    RBF_CUDA(cudaFuncSetAttribute(k_eval_grid_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay<64>::SMEM));
    attr_set[c->device & 63] = true;
  }
  // bulk tensor stores need 16-byte aligned outputs and row pitches; other
  // rasters take the transposing stores
  CUtensorMap map_h, map_g;
  memset(&map_h, 0, sizeof(map_h));
  memset(&map_g, 0, sizeof(map_g));
  // (box coordinates are 32-bit: the gradient's x reaches 2 nqx)
  int use_tma = (nqx % 4 == 0) && ((uintptr_t)h % 16 == 0) && (!grad || (uintptr_t)grad % 16 == 0) &&
                2 * nqx + 64 < 0x7fffffffLL && nqy < 0x7fffffffLL;
  if (use_tma) {
    EncodeTiled enc = encode_tiled();
    if (!enc) return fail(RBF_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint32_t box[2] = {32, 32}, estr[2] = {1, 1};
    const cuuint64_t dh[2] = {(cuuint64_t)nqx, (cuuint64_t)nqy}, sh[1] = {(cuuint64_t)nqx * 4};
    CUresult e = enc(&map_h, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h, dh, sh, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (e != CUDA_SUCCESS) return fail(RBF_ECUDA, "tensor map of h: error %d", (int)e);
    if (grad) {
      const cuuint64_t dg[2] = {(cuuint64_t)(2 * nqx), (cuuint64_t)nqy}, sg[1] = {(cuuint64_t)nqx * 8};
      e = enc(&map_g, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, grad, dg, sg, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (e != CUDA_SUCCESS) return fail(RBF_ECUDA, "tensor map of grad: error %d", (int)e);
    }
  }
  // one persistent CTA per SM (the shared memory allows one)
  static int sms[64] = {0};
  if (!sms[c->device & 63]) RBF_CUDA(cudaDeviceGetAttribute(&sms[c->device & 63], cudaDevAttrMultiProcessorCount, c->device));
  const int64_t ntiles = tx * ty;
  const unsigned nblk = (unsigned)(ntiles < sms[c->device & 63] ? ntiles : sms[c->device & 63]);
  StageTimer st(c, RBF_STAGE_EVAL_GRID, s, (grad ? 12.0 : 4.0) * (double)nqx * (double)nqy);
  if (P.kw == 32)
    k_eval_grid_tc<32><<<nblk, GTHREADS, Lay<32>::SMEM, s>>>(P, c->lat_xs.as<float>(), c->lat_ys.as<float>(),
                                                             c->wlat.as<float>(), h, grad, map_h, map_g, use_tma, tx,
                                                             ntiles);
  else
    k_eval_grid_tc<64><<<nblk, GTHREADS, Lay<64>::SMEM, s>>>(P, c->lat_xs.as<float>(), c->lat_ys.as<float>(),
                                                             c->wlat.as<float>(), h, grad, map_h, map_g, use_tma, tx,
                                                             ntiles);
  ::rbf::note_launch();
  RBF_CUDA(cudaGetLastError());
  return RBF_OK;
}
