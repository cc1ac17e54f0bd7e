// Internal declarations shared by the translation units of librbfgb.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rbfgb.h"

namespace rbf {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
rbf_status fail(rbf_status st, const char* fmt, ...);
rbf_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define RBF_CUDA(call)                                                         \
  do {                                                                         \
    cudaError_t _e = (call);                                                   \
    if (_e != cudaSuccess) return ::rbf::cuda_fail(_e, #call, __FILE__, __LINE__); \
  } while (0)

#define RBF_TRY(expr)                   \
  do {                                  \
    rbf_status _s = (expr);             \
    if (_s != RBF_OK) return _s;        \
  } while (0)

// Device-side status words (one int per context): kernels record a failure by
// atomically OR-ing a flag; the host reads the word at the next sync point.
enum DevFlag : int {
  DEV_NOT_SPD = 1,
  DEV_TIMEOUT = 2,
  DEV_BAD_INDEX = 4,
};

// ---------------------------------------------------------------------------
// Grow-only device buffer
// ---------------------------------------------------------------------------
struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
  template <class T>
  T* as() const { return reinterpret_cast<T*>(p); }
  rbf_status ensure(size_t nbytes);
  void release();
};

// ---------------------------------------------------------------------------
// Hash grid of centers (counting sort by cell, ids ascending within a cell)
// ---------------------------------------------------------------------------
struct Grid {
  float x0, y0;     // lower-left corner of cell (0, 0)
  float cs, inv_cs; // cell size and its reciprocal
  int nx, ny;       // number of cells
};

constexpr int64_t BW_DENSE_CTX = INT64_MAX / 4;  // "dense" half-bandwidth

// Compressed-row copy of a float64 matrix: every exactly nonzero entry,
// ascending columns (sparse.cu).
constexpr int64_t SPH_MAX = 4096;  // largest order kept (capacity n^2 entries)
struct SpH {
  Buf rp, col, val;  // int32 (n + 1), int32 and double (capacity n * n)
  int64_t n = 0;
  bool valid = false;
};

struct Lattice {
  bool on = false;  // every center sits on (x0 + (i + 0.5) h, y0 + (j + 0.5) h)
  double x0, y0, h;
  int nx, ny;
};

// Where the covariance of a center outside the active block is stored: the
// block of its latest departure starts at arena[base] (d x d, row-major) and
// the center is its row pos; base < 0: the center never left a block.
struct BlkRef {
  long long base;
  int d, pos;
};

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct Ctx {
  rbf_config cfg;
  int device = 0;
  int64_t M = 0;

  Buf c64;           // M x 2 float64 centers
  Buf w;             // M float64 weights
  Grid grid{};
  Lattice lat{};
  Buf cell_start;    // int32 (nx*ny + 1)
  Buf sorted_id;     // int32 M  (slot -> center id)
  Buf sorted_xyw;    // float4 M (x, y, w, 0) in slot order, float32
  Buf wlat;          // float32 lattice weights (lat.ny x lat.nx), 0 where no center
  Buf lat_xs, lat_ys; // float32 lattice node coordinates (fl32 of the float64 centers)
  Buf wlat2;          // padded pairs (W[j][i], W[j][i+1]) for the fixed-window kernel
  Buf lat_xhl, lat_yhl; // float2 (hi, lo) node coordinates, hi + lo = the float64 coordinate, for
                        // nodes -(lat_rc + 1) .. n + lat_rc - 1 of each axis (fixed-window kernel)
  int lat_rc = 0;     // window half-width in nodes (0: kernel not applicable)

  // recursive update state: the active block is held in information form
  int64_t a = 0;     // size of the current active block
  Buf A;             // int32 M   active ids (ascending)
  Buf g2l;           // int32 M   center id -> local index in A, -1 if not active
  Buf H;             // float64 a x a   information matrix of the active block
  Buf L;             // float64 a x a   its Cholesky factor (lower)
  int64_t ldH = 0;   // leading dimension of H and L
  Buf Lf;            // float32 factor of H (mixed precision), a x a, leading dimension ldw
  Buf Zd;            // float32 inverses of its 64 x 64 diagonal blocks
  Buf Zi;            // float32 L^{-1} of the whole factor (valid when zi_valid)
  bool zi_valid = false;
  int64_t inv_max = 4096;  // form L^{-1} for active blocks up to this size
  bool gacc_dirty = false; // the Gram accumulators may hold values of an unfinished update
  int64_t bw_lf = BW_DENSE_CTX;  // half-bandwidth of the float32 factor Lf
  int64_t nbr_cap = 0;           // neighbour-list capacity of rbf_update (0: read the total first)
  cudaStream_t bs[3] = {};           // side streams of the block stage (bs[2]: high priority)
  cudaEvent_t bev[4] = {};           // fork and joins of the block stage
  bool la_ok = true;                 // look-ahead factorization allowed
  bool df_ok = true;                 // one-launch dataflow factorization allowed
  int8_t fchoice[64] = {};           // per size bucket of 256: 0 untimed, 1 launch chain, 2 dataflow
  Buf df_flags;                      // its per-tile ready flags and abort word
  uint32_t df_epoch = 0;
  cudaStream_t la_stream = nullptr;  // side stream of the look-ahead factorization
  cudaEvent_t la_ev[5] = {};          // panel ready (2), trailing done (2), join
  SpH Hs;            // compressed rows of H (mixed update)
  SpH Hs_next;       // compressed rows of the information matrix being built
  int64_t ldw = 0;
  int refine_sweeps = 3;      // float64 refinement sweeps of the weight solve (mixed precision)
  int refine_sweeps_cov = 2;  // ... of the covariance solves (leaving centers, rbf_get_cov)
  // Covariance of the centers outside the active block.  It is block
  // diagonal: every departure stores its d x d block P_DD once, in an arena,
  // and each center that left refers to the block of its latest departure
  // (BlkRef); two centers are coupled only if they refer to the same block.
  Buf blkref;        // BlkRef M
  Buf arena;         // float64 blocks, arena_used entries in use
  int64_t arena_used = 0;
  Buf departed;      // int32 M: 1 once a center has left an active block (its P may be coupled)
  bool pg_on = false;  // some center has left a block

  // device status word + epoch counter for flag-based waits
  Buf dflag;         // int32[4]
  Buf sync_flags;    // int32 flags for sync-free triangular solves
  uint32_t epoch = 0;
  // test hooks (rbf_test_hook): failure statuses driven from the host
  long long spin_limit = 0;  // iterations of the solves' bounded waits (0: default)
  int wait_xor = 0;          // nonzero: the solves wait for a flag value no block writes
  double diag_shift = 0.0;   // added to the diagonal of H' before it is factored

  // scratch buffers, addressed by slot (slots 48.. are used by the scans)
  static constexpr int NSLOT = 100;
  Buf ws[NSLOT];
  Buf& scratch(int i) { return ws[i < NSLOT ? i : NSLOT - 1]; }

  // host pinned staging for small readbacks
  int64_t* host_small = nullptr;

  void* batch = nullptr;  // state of rbf_batch_update_eval (streams, workspaces, graphs)

  // stage timing (rbf_profile_enable)
  bool prof = false;
  struct Mark {
    int stage;
    cudaEvent_t a, b;
    double work;
  };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> ev_pool;
  double prof_ms[RBF_NSTAGE] = {};
  double prof_work[RBF_NSTAGE] = {};
  int64_t prof_count[RBF_NSTAGE] = {};
};

// Scoped stage interval: records an event pair on stream s when profiling is on.
struct StageTimer {
  Ctx* c;
  int stage;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  double work;
  StageTimer(Ctx* c_, int stage_, cudaStream_t s_, double work_ = 0.0);
  ~StageTimer();
};

rbf_status check_ctx(rbf_ctx* c, bool need_centers);

// float32 / float64 radii for the neighbour rule
double assembly_radius(const rbf_config& cfg, double noise);
double eval_radius(const rbf_config& cfg);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
// x added exactly to a 128-bit fixed-point accumulator U[0..1] with 2^64
// units per 1 (low word first; the carry of the low word goes to the high
// word): order-independent sums of float64 terms of magnitude below 2^63.
static __device__ __forceinline__ void add_u128(unsigned long long* U, double x) {
  double hi = floor(x);
  double fr = x - hi;  // exact, in [0, 1)
  unsigned long long lo = __double2ull_rz(ldexp(fr, 64));  // fr * 2^64 < 2^64
  unsigned long long old = atomicAdd(U, lo);
  unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
  long long h = (long long)hi + (long long)carry;
  if (h != 0) atomicAdd(U + 1, (unsigned long long)h);
}

// Neighbour rule: dx, dy, d2 each rounded once to float32, no contraction.
__device__ __forceinline__ float d2_rn(float qx, float qy, float cx, float cy) {
  float dx = __fsub_rn(qx, cx);
  float dy = __fsub_rn(qy, cy);
  return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
}

// Candidate cells of the row band j of the grid for a disc of radius rc (in
// cell units) around (fx, fy) (cell units): returns false if the band misses.
__device__ __forceinline__ bool row_range(const Grid& g, float fx, float fy, float rc, int j,
                                          int& ilo, int& ihi) {
  float gap = fmaxf(0.f, fmaxf((float)j - fy, fy - (float)(j + 1)));
  float hw2 = rc * rc - gap * gap;
  if (hw2 < -1e-3f) return false;
  float hw = sqrtf(fmaxf(hw2, 0.f)) + 2e-3f;
  float lo = floorf(fx - hw), hi = floorf(fx + hw);
  lo = fmaxf(lo, 0.f);
  hi = fminf(hi, (float)(g.nx - 1));
  if (!(lo <= hi)) return false;
  ilo = (int)lo;
  ihi = (int)hi;
  return true;
}

__device__ __forceinline__ bool rows_range(const Grid& g, float fy, float rc, int& jlo, int& jhi) {
  float lo = floorf(fy - rc - 2e-3f), hi = floorf(fy + rc + 2e-3f);
  lo = fmaxf(lo, 0.f);
  hi = fminf(hi, (float)(g.ny - 1));
  if (!(lo <= hi)) return false;
  jlo = (int)lo;
  jhi = (int)hi;
  return true;
}

// Regression row m(x) in float64 (Sec. III-B): Wendland phi(r), or the
// Gaussian moment row (s^2/st^2) exp(-r^2 / 2 st^2).
__device__ __forceinline__ double row_value(int kernel, double r2, double inv_rho,
                                            double g_scale, double g_inv2s2) {
  if (kernel == RBF_KERNEL_WENDLAND) {
    double s = sqrt(r2) * inv_rho;
    double t = fmax(1.0 - s, 0.0);
    double t2 = t * t;
    return t2 * t2 * (4.0 * s + 1.0);
  }
  return g_scale * exp(-r2 * g_inv2s2);
}

// ---------------------------------------------------------------------------
// Host-side helpers implemented in the .cu files
// ---------------------------------------------------------------------------
// exclusive scan of int32 counts -> int64 offsets (n + 1 entries, out[n] = total)
rbf_status scan_i32_to_i64(Ctx* c, const int32_t* in, int64_t* out, int64_t n,
                           cudaStream_t s, int scratch_slot);
// exclusive scan of int32 -> int32 (n + 1 entries)
rbf_status scan_i32(Ctx* c, const int32_t* in, int32_t* out, int64_t n, cudaStream_t s,
                    int scratch_slot);

rbf_status build_center_grid(Ctx* c, cudaStream_t s);
rbf_status refresh_center_weights(Ctx* c, cudaStream_t s);
rbf_status install_centers(Ctx* c, const double* cxy_dev, int64_t M, cudaStream_t s);
rbf_status reset_update_state(Ctx* c);

// neighbour lists (point-major CSR, ids ascending) under radius r
// (defer_cap > 0: the total is not read; rows past defer_cap entries stay
// unfilled and *nnz = -1, the caller reads row_ptr[n] and the flags later)
rbf_status neighbor_lists(Ctx* c, const float* pts, int64_t n, int stride_floats, double radius,
                          Buf& row_ptr, Buf& col, int64_t* nnz, cudaStream_t s, int64_t defer_cap = 0);

rbf_status read_dev_flag(Ctx* c, cudaStream_t s, int* flag);

// number of kernels this library has launched (all contexts, all threads)
void note_launch();
inline cudaError_t cooperative_launch(const void* f, dim3 g, dim3 b, void** args, size_t smem,
                                      cudaStream_t s) {
  cudaError_t e = cudaLaunchCooperativeKernel(f, g, b, args, smem, s);
  if (e == cudaSuccess) note_launch();
  return e;
}

// dense FP64 / mixed-precision linear algebra (dense.cu)
// bw: half-bandwidth of the matrix (entries with |i - j| > bw are zero and
// stay zero in the factor); the default treats it as dense
constexpr int64_t BW_DENSE = BW_DENSE_CTX;
rbf_status potrf_lower(Ctx* c, double* A, int64_t n, int64_t lda, int64_t nfactor,
                       bool mixed, cudaStream_t s, int64_t bw = BW_DENSE);
rbf_status trsm_lower(Ctx* c, const double* L, int64_t n, int64_t ldl, double* B, int64_t m,
                      int64_t ldb, bool transpose, cudaStream_t s, int64_t bw = BW_DENSE);
rbf_status gemm_f64(Ctx* c, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                    const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                    double* Cm, int64_t ldc, cudaStream_t s, int slot = 28);
// mixed precision (mixed.cu)
rbf_status potrf_mixed(Ctx* c, const double* H, int64_t ldh, int64_t n, float* W, int64_t ldw, float* Zd,
                       cudaStream_t s, int64_t bw = BW_DENSE);
rbf_status trsm32(Ctx* c, const float* L, int64_t n, int64_t ldl, const float* Zd, float* B, int64_t m,
                  int64_t ldb, bool transpose, cudaStream_t s, int64_t bw = BW_DENSE);
rbf_status mixed_solve(Ctx* c, const double* H, int64_t ldh, const SpH* Hs, const float* W, int64_t ldw,
                       const float* Zd, const float* Zi, int64_t n, double* B, int64_t m, int sweeps,
                       cudaStream_t s, int64_t bw = BW_DENSE);
rbf_status mixed_cov(Ctx* c, const double* H, int64_t ldh, const SpH* Hs, const float* W, int64_t ldw,
                     const float* Zd, const float* Zi, int64_t n, double* B, int64_t k, const int32_t* pos,
                     int sweeps, double* P, cudaStream_t s, int64_t bw = BW_DENSE);
// compressed rows of the information matrix (sparse.cu)
rbf_status build_csr(Ctx* c, const double* H, int64_t ld, int64_t n, SpH& out, cudaStream_t s);
rbf_status csr_bandwidth(Ctx* c, int64_t n, int64_t* bw, cudaStream_t s);
rbf_status dense_bandwidth(Ctx* c, const double* H, int64_t ld, int64_t n, int64_t* bw, cudaStream_t s);
rbf_status csr_residual(const SpH& A, const double* X, const double* B, int64_t m, double* R, cudaStream_t s);
// float64 in and out, float-float arithmetic inside (ffgemm.cu)
rbf_status gemm_ff(Ctx* c, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                   int64_t lda, const double* B, int64_t ldb, double beta, double* Cm, int64_t ldc, cudaStream_t s,
                   int slot, bool lower = false);
rbf_status csr_residual_ff(Ctx* c, const SpH& A, const double* X, const double* B, int64_t m, double* R,
                           cudaStream_t s, int slot);
// explicit inverse of the float32 factor and solves with it (inverse.cu)
rbf_status trtri_mixed(Ctx* c, const float* W, int64_t ldw, int64_t n, const float* Zd, float* Z, int64_t ldz,
                       cudaStream_t s);
rbf_status inv_solve(Ctx* c, const float* Z, int64_t ldz, int64_t n, float* F, int64_t m, cudaStream_t s);
// X += Z^T (Z R), float64 R and X, at most 8 right-hand sides (inverse.cu)
rbf_status inv_solve_acc(Ctx* c, const float* Z, int64_t ldz, int64_t n, const double* R, double* X, int64_t m,
                         cudaStream_t s);
rbf_status inv_solve_unit(Ctx* c, const float* Z, int64_t ldz, int64_t n, const int32_t* pos, int64_t m, float* F,
                          cudaStream_t s);
constexpr int SPD_SMALL_MAX = 128;  // largest order of spd_inverse_small (one CTA, shared memory)
rbf_status spd_inverse_small(Ctx* c, double* G, int64_t m, cudaStream_t s);
// the same in float-float arithmetic (ffgemm.cu), for the mixed-precision update
rbf_status spd_inverse_small_ff(Ctx* c, double* G, int64_t m, cudaStream_t s);
rbf_status chol_solve(Ctx* c, const double* H, const double* L, int64_t a, int64_t ld, double* b, bool refine,
                      cudaStream_t s, int64_t bw = BW_DENSE);
void batch_destroy(Ctx* c);
// the mixed-precision batch in persistent launches (bqueue.cu)
rbf_status bq_run(Ctx* c, void** state, const rbf_patch* patches, int32_t npatch, cudaStream_t s, bool* handled);
void bq_destroy(void* state);
// forget the cached device address of rbf_soft_cost_noalloc's scratch on `dev`
void noalloc_forget(int dev);
rbf_status symv_residual(const double* H, int64_t n, int64_t ld, const double* x,
                         const double* b, double* r, cudaStream_t s);

}  // namespace rbf

struct rbf_ctx {
  rbf::Ctx impl;
};

namespace rbf {
inline Ctx* C(rbf_ctx* c) { return &c->impl; }
}  // namespace rbf
