/*
 * rbfgb.h -- C ABI of the GB300 RBF terrain library (librbfgb.so).
 *
 * The library evaluates the radial-basis-function terrain model of
 * Sec. III-A, f(x; w) = sum_i w_i phi(||x - c_i||) (Eq. RBF_fml), with its
 * gradient, runs the recursive ridge update of the weights restricted to the
 * active rows (Sec. III-C, Eq. H_update, Eq. kf_w_update,
 * Eq. active_rows_weights_update, Eq. H_inverse_update), selects centers
 * adaptively (Sec. III-A), and computes the soft-constraint cost of
 * Sec. IV-C (Eq. residual_manifold_left_wheel, Eq. manifold_derivative) with
 * its gradients.
 *
 * Conventions (every entry point):
 *  - Array arguments are DEVICE pointers on the context's GPU, owned by the
 *    caller, unless the comment says "host".  The context owns only its
 *    internal state (centers, weights, the covariance store and workspaces).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    stream-ordered and asynchronous, except where a comment says the call
 *    synchronizes (calls that return a data-dependent size to the host).
 *  - Errors are returned as a status and never trapped on the device; the
 *    message of the last failure on the calling thread is rbf_last_error().
 *    A failed call leaves the context in the state it had before the call
 *    unless the comment says otherwise.
 *  - Empty inputs (n = 0, Q = 0) are valid no-ops.
 *  - Points are float32 (x, y, z) triples, row-major n x 3; queries are
 *    float32 (x, y) pairs, Q x 2; centers and weights are float64.
 *  - One context must not be used from two host threads at the same time.
 */
#ifndef RBFGB_H
#define RBFGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rbf_ctx rbf_ctx;

typedef enum {
  RBF_OK = 0,
  RBF_EINVAL = -1,    /* bad argument (null pointer, negative size, bad config) */
  RBF_ENOMEM = -2,    /* device allocation failed */
  RBF_ECUDA = -3,     /* a CUDA runtime call failed */
  RBF_ENOTSPD = -4,   /* a Cholesky pivot was not positive */
  RBF_ETIMEOUT = -5,  /* a bounded device-side wait gave up */
  RBF_ESTATE = -6,    /* call not valid in the current state (e.g. no centers) */
  RBF_ERANGE = -7     /* an output buffer is too small */
} rbf_status;

enum { RBF_KERNEL_WENDLAND = 0, RBF_KERNEL_GAUSSIAN = 1 };
enum { RBF_UPDATE_FP64 = 0, RBF_UPDATE_MIXED = 1 };
enum { RBF_LOSS_HUBER = 0, RBF_LOSS_L2 = 1 };

/* Parameters of a terrain model.  All lengths in metres. */
typedef struct rbf_config {
  int32_t kernel;           /* RBF_KERNEL_WENDLAND: phi = (1-r/rho)_+^4 (4 r/rho + 1);
                               RBF_KERNEL_GAUSSIAN: phi = exp(-r^2 / 2 sigma^2) (Eq. RBF_def) */
  int32_t update_precision; /* RBF_UPDATE_FP64: every step of rbf_update in FP64;
                               RBF_UPDATE_MIXED: factorizations on the tensor cores,
                               FP64 accumulation and FP64 iterative refinement */
  double rho;               /* Wendland support radius */
  double sigma;             /* Gaussian bandwidth sigma */
  double cutoff_mult;       /* Gaussian truncation: evaluation uses cutoff_mult*sigma,
                               the regression rows cutoff_mult*sqrt(sigma^2+noise^2) */
  double lambda;            /* ridge weight lambda (Sec. III-B); prior covariance I/lambda */
  int32_t loss;             /* soft-constraint loss: RBF_LOSS_HUBER or RBF_LOSS_L2 */
  int32_t min_count;        /* center selection: accept a candidate iff count >= min_count */
  double huber_delta;       /* Huber threshold delta */
  double lambda_m;          /* weight of the L2 loss (the paper's lambda_M) */
  double wheel_offset;      /* r in Eq. residual_manifold_left_wheel */
  double mesh_x0, mesh_y0;  /* candidate mesh of rbf_build_centers: candidate (i, j) sits at */
  double mesh_h;            /*   (mesh_x0 + (i + 0.5) mesh_h, mesh_y0 + (j + 0.5) mesh_h) */
  int32_t mesh_nx, mesh_ny; /*   0 <= i < mesh_nx, 0 <= j < mesh_ny, row-major (j outer) */
  double r_kd;              /* center selection radius (Sec. III-A) */
  int32_t refine_sweeps;    /* RBF_UPDATE_MIXED: float64 refinement sweeps of the solves with
                               the float32 factor (0 = defaults: 3 for the weights, 2 for
                               covariance blocks; n > 0: n for both; 1 = no refinement) */
  int32_t inverse_max;      /* RBF_UPDATE_MIXED: largest active block for which the update forms
                               L^{-1} of the float32 factor and solves by two products with it
                               (0 = default 4096; negative = never: blocked substitution only) */
  int32_t exact;            /* 0: the paper's block recursion (Sec. III-C: only the rows touched by
                                  the frame are updated, P[A, not A] = 0 afterwards);
                               1: the exact recursion with the full covariance (Eq. kf_w_update and
                                  Eq. H_inverse_update on all M rows): every center is in the active
                                  block of every update, so after any sequence of updates the
                                  weights equal the batch ridge estimate of Sec. III-B */
  int32_t reserved1;        /* must be 0 */
} rbf_config;

/* Create a context on the current CUDA device.  Validates cfg (positive radii,
 * lambda > 0, known enums).  No centers yet. */
rbf_status rbf_create(const rbf_config* cfg, rbf_ctx** out);

/* Free every device buffer of the context.  Synchronizes the device. */
rbf_status rbf_destroy(rbf_ctx* ctx);

/* Message of the last failing call on this host thread ("" if none). */
const char* rbf_last_error(void);

/* Install M centers (cxy: M x 2 float64).  Resets the weights to the prior
 * w = 0 and the covariance to P = I / lambda, and rebuilds the center hash
 * grid (a counting sort of the centers by cell).  The update's device
 * workspaces are kept, so calling it again with the same centers restarts the
 * recursion without new allocations.  Synchronizes. */
rbf_status rbf_set_centers(rbf_ctx* ctx, const double* cxy, int64_t M, void* stream);

/* Adaptive center selection (Sec. III-A): count the points (pts: n x 3, x and
 * y used) within r_kd of every candidate of the configured mesh, with the
 * float32 distance test d2 < r_kd^2, and install the candidates whose count is
 * >= min_count, in ascending row-major order, as the centers (as
 * rbf_set_centers does).  counts (optional, may be NULL): mesh_nx*mesh_ny int32
 * per-candidate counts.  *M_out = number of accepted centers.  Synchronizes. */
rbf_status rbf_build_centers(rbf_ctx* ctx, const float* pts, int64_t n, int32_t* counts,
                             int64_t* M_out, void* stream);

/* Number of installed centers (host). */
rbf_status rbf_num_centers(rbf_ctx* ctx, int64_t* M_out);

/* Copy the centers (M x 2 float64) / weights (M float64) to device buffers. */
rbf_status rbf_get_centers(rbf_ctx* ctx, double* cxy, void* stream);
rbf_status rbf_get_weights(rbf_ctx* ctx, double* w, void* stream);

/* Overwrite the weights (M float64) without touching the covariance. */
rbf_status rbf_set_weights(rbf_ctx* ctx, const double* w, void* stream);

/* One recursive ridge update (Sec. III-C) with the n points of one frame,
 * expressed in the world frame (pts: n x 3 float32).  noise = sigma_eps of
 * Sec. III-B (enters the Gaussian regression rows; unused for Wendland).
 * Active rows A = sorted union of the points' neighbour lists
 * (Eq. mfk_m_approx); only w_A and the covariance block P[A, A] change and
 * P[A, not A] becomes 0 (block-diagonal form of Eq. H_inverse_update).
 * Synchronizes a few times per call to read data-dependent sizes (of A, of
 * the leaving, staying and entering sets, of the coupled rows) and, before
 * the commit, the status word.  RBF_ENOTSPD if a factorization meets a
 * non-positive pivot; the state is then left unchanged. */
rbf_status rbf_update(rbf_ctx* ctx, const float* pts, int64_t n, double noise, void* stream);

/* h(q) and grad h(q) at Q query points (q: Q x 2 float32; h: Q float32;
 * grad: Q x 2 float32, may be NULL).  Eq. RBF_fml and Eq. manidolf_grad_detail,
 * summed over the centers within the support (Wendland) or within
 * cutoff_mult*sigma (Gaussian), in float32. */
rbf_status rbf_eval(rbf_ctx* ctx, const float* q, int64_t Q, float* h, float* grad, void* stream);

/* h and grad h on the regular raster q_kl = (qx0 + k dq, qy0 + l dq),
 * k < nqx, l < nqy (Eq. RBF_fml, Eq. manidolf_grad_detail), for the Gaussian
 * kernel with the centers on a square lattice: the Gaussian factorises per
 * axis, and the sums over a tile of 128 x 128 raster points become products
 * of small matrices, run on the tensor cores with every float32 operand split
 * into two bfloat16 parts (float32 accuracy of each term, about 2^-16).
 * Truncation is per axis: center j contributes iff |q_x - c_x| < r and
 * |q_y - c_y| < r, r = cutoff_mult * sigma, each decided in float32 as for
 * rbf_eval.  This keeps every term rbf_eval keeps plus the corners of the
 * square, each below exp(-cutoff_mult^2 / 2) |w_j|.
 * h: nqy x nqx float32, row l = raster row (device); grad: nqy x nqx x 2
 * float32 (d/dx, d/dy), 8-byte aligned, may be NULL (device).  The coordinates are rounded to
 * float32 after qx0 + k dq is formed in float64.
 * RBF_EINVAL: not the Gaussian kernel, centers not on a lattice, dq <= 0 or
 * non-finite arguments.  RBF_ERANGE: 127 dq + 2 r exceeds 60.5 lattice
 * spacings (a tile's window must fit in 64 nodes; evaluate coarser rasters
 * with rbf_eval).  Asynchronous; a tile whose bounded wait for the tensor
 * cores gives up (which a correct launch never does) is written as NaN. */
rbf_status rbf_eval_grid(rbf_ctx* ctx, double qx0, double qy0, double dq, int64_t nqx, int64_t nqy, float* h,
                         float* grad, void* stream);

/* Soft-constraint cost (Sec. IV-C) over n body-frame points (pts: n x 3
 * float32) under the pose R (host, 3x3 row-major float64), t (host, 3 float64):
 * q_i = R p_i + t, r_i = q_z - wheel_offset - f(q_xy),
 * cost = sum Huber_delta(r_i)  (or lambda_m sum r_i^2 for RBF_LOSS_L2),
 * grad6 = d cost / d [theta, t] with R <- R Exp(theta), t <- t + dt
 * (Eq. manifold_derivative, Eq. manifold_grad_2).
 * cost: 1 float64 (device); grad6: 6 float64 (device); resid: n float32
 * (device, optional, may be NULL).  Reductions are deterministic. */
rbf_status rbf_soft_cost(rbf_ctx* ctx, const double* R, const double* t, const float* pts,
                         int64_t n, double* cost, double* grad6, float* resid, void* stream);

/* The soft-constraint cost, its gradient and the Gauss-Newton matrix of the
 * pose, for a Levenberg-Marquardt step on the 6-DoF pose (Sec. IV-C: the
 * cost J_M is minimised by LM; here over all points of the frame).
 * out28 (device, 28 doubles): out28[0] = cost, out28[1..6] = gradient g (as
 * rbf_soft_cost), out28[7..27] = A = sum_i omega_i J_i J_i^T, the upper
 * triangle row by row (A00 A01 .. A05 A11 .. A55), with J_i the pose
 * Jacobian row of point i (same perturbation as the gradient) and the
 * iteratively reweighted least-squares weight omega_i = psi(r_i) / r_i
 * (1 inside the Huber zone, delta / |r_i| outside; 2 lambda_M for the L2
 * loss).  rbf_lm_step takes the step from these on the device.
 * Asynchronous on stream.  Errors: RBF_EINVAL (negative n, null output,
 * null points with n > 0, non-finite pose), RBF_ESTATE (no centers). */
rbf_status rbf_soft_cost_normal(rbf_ctx* ctx, const double* R, const double* t, const float* pts,
                                int64_t n, double* out28, void* stream);

/* One Levenberg-Marquardt step on the 6-DoF pose, entirely on the device
 * (Sec. IV-C: the soft-constraint cost J_M is minimised by LM; Eq.
 * manifold_derivative, Eq. manifold_grad_2 give the Jacobian).  Forms the
 * cost, the gradient g and the Gauss-Newton matrix A at the pose (R, t) as
 * rbf_soft_cost_normal does, solves (A + mu diag(A)) delta = -g in float64
 * (Cholesky of the damped 6 x 6 matrix) and applies the step on the manifold:
 * R_out = R Exp(delta_theta), t_out = t + delta_t.
 * R: host 3 x 3 row-major float64; t: host 3 float64; pts: device n x 3
 * float32 body-frame points; mu >= 0 the damping.
 * out20 (device, 20 float64): [0..8] R_out row-major, [9..11] t_out,
 * [12] the cost at the input pose, [13] 0, or 1 if the damped matrix was not
 * positive definite (no step: R_out = R, t_out = t), [14..19] delta
 * (theta, then t).  Asynchronous on stream.  Errors: RBF_EINVAL (negative n,
 * null output, null points with n > 0, non-finite pose, mu < 0),
 * RBF_ESTATE (no centers). */
rbf_status rbf_lm_step(rbf_ctx* ctx, const double* R, const double* t, const float* pts, int64_t n,
                       double mu, double* out20, void* stream);

/* rbf_soft_cost that allocates nothing, for callers that cannot allocate
 * device memory while they run: a scan-matching loop with a hard per-frame
 * deadline (cudaMalloc / cudaFree can synchronize the device and take
 * milliseconds) or a process that reserves its GPU memory once at start-up.
 * The paper has no counterpart; the arguments, results and launch are those
 * of rbf_soft_cost.  Its only scratch, the per-block partial sums, lives in a
 * fixed device array of 128 KiB (2,048 blocks x 8 float64) that every GPU
 * which loads the library holds until the process exits.  The launch uses
 * min(ceil(n / 256), 4 x number of SMs) blocks, so any n is accepted on GPUs
 * with up to 512 SMs; a launch that would need more blocks returns RBF_ERANGE.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The address is cached per process and device;
 * rbf_create drops the cached address of its device, so after a
 * cudaDeviceReset create the contexts anew before calling this again.  All calls share the one array: calls whose
 * work overlaps on the GPU (other streams, other threads, other contexts)
 * race on it and must be serialized by the caller.  Each call overwrites
 * every slot it later reads, so nothing of an earlier call leaks into a
 * result. */
rbf_status rbf_soft_cost_noalloc(rbf_ctx* ctx, const double* R, const double* t, const float* pts,
                                 int64_t n, double* cost, double* grad6, float* resid, void* stream);

/* Backward of gout * cost: gradients with respect to the weights (dw: M
 * float32), the centers (dc: M x 2 float32) and the pose (dpose6: 6 float64).
 * gout: device pointer to one float64 (NULL means 1).  Any of dw, dc, dpose6
 * may be NULL.  Center-major gather: deterministic, no atomics. */
rbf_status rbf_soft_cost_backward(rbf_ctx* ctx, const double* R, const double* t,
                                  const float* pts, int64_t n, const double* gout,
                                  float* dw, float* dc, double* dpose6, void* stream);

/* Covariance entries P[ids, ids] (ids: host, k int32 center ids; Pk: device,
 * k x k float64 row-major).  Synchronizes. */
rbf_status rbf_get_cov(rbf_ctx* ctx, const int32_t* ids, int64_t k, double* Pk, void* stream);

/* Active rows of the last update: A (device, capacity cap int32), *a_out =
 * their number (host).  RBF_ERANGE if cap < a.  Synchronizes. */
rbf_status rbf_get_active(rbf_ctx* ctx, int32_t* A, int64_t cap, int64_t* a_out, void* stream);

/* Neighbour lists of n points under the regression-row radius for the given
 * noise (rho for Wendland), with the float32 rule d2 < r^2, ids ascending:
 * row_ptr (device, n+1 int64), col (device, capacity cap int32).
 * *nnz_out = total entries (host).  RBF_ERANGE if cap < nnz (row_ptr is still
 * written).  Synchronizes. */
rbf_status rbf_get_neighbors(rbf_ctx* ctx, const float* pts, int64_t n, double noise,
                             int64_t* row_ptr, int32_t* col, int64_t cap, int64_t* nnz_out,
                             void* stream);

/* One terrain patch of a batch (lattice centers, see rbf_batch_update_eval). */
typedef struct rbf_patch {
  double x0, y0;      /* center id = j * nx + i sits at */
  double spacing;     /*   (x0 + (i + 0.5) spacing, y0 + (j + 0.5) spacing) */
  int32_t nx;         /* nodes per lattice row */
  int32_t pad0;
  int64_t M;          /* the patch's centers are ids 0 .. M-1 (rows of nx, the last may be partial) */
  int64_t n;          /* points (world frame), device float32 n x 3 */
  const float* pts;
  int64_t Q;          /* queries, device float32 Q x 2 */
  const float* q;
  double* w;          /* out: device float64 M weights */
  float* h;           /* out: device float32 Q heights */
  float* grad;        /* out: device float32 Q x 2 gradients (may be NULL) */
} rbf_patch;

/* A batch of independent terrain patches (no counterpart beyond Sec. III:
 * every patch is its own terrain model).  For every patch: prior w = 0,
 * P = I / lambda; one recursive update with its n points (Sec. III-C; from
 * the prior this equals batch ridge, Sec. III-B); then h and grad h at its Q
 * queries (Eq. RBF_fml).  The context supplies the kernel parameters and the
 * update precision; its own centers and state are not used or changed.
 * The regression rows use noise 0 (sigma~ = sigma for the Gaussian kernel).
 * patches: host array of npatch descriptors (device pointers inside).  The
 * patches run concurrently on internal streams forked from `stream`; the
 * whole batch is recorded once into a CUDA graph per distinct batch shape and
 * replayed.  The call synchronizes at its end and returns RBF_ENOTSPD or
 * RBF_EINVAL (non-finite point) if any patch failed. */
rbf_status rbf_batch_update_eval(rbf_ctx* ctx, const rbf_patch* patches, int32_t npatch, void* stream);

/* Stage timing.  While enabled, every call records CUDA events on its own
 * stream around each stage below and adds the stage's algorithmic work
 * (floating-point operations, or bytes for the memory-bound stages).
 * rbf_profile_read synchronizes, returns the accumulated milliseconds,
 * work and number of timed intervals per stage (arrays of RBF_NSTAGE) and
 * optionally resets them.  Tracing is host bookkeeping only: it changes no
 * result. */
enum {
  RBF_STAGE_NEIGHBORS = 0,  /* neighbour lists + active set (bytes: 12 per point) */
  RBF_STAGE_ASSEMBLY = 1,   /* m~ entries, innovation, m~ m~^T rows (flops) */
  RBF_STAGE_BLOCK = 2,      /* leaving/entering centers: Schur complement, stored blocks */
  RBF_STAGE_PANEL = 3,      /* Cholesky diagonal tiles + panel solves (flops) */
  RBF_STAGE_TRAILING = 4,   /* Cholesky trailing updates, one interval per launch (flops) */
  RBF_STAGE_SOLVE = 5,      /* triangular solves and refinement (flops) */
  RBF_STAGE_EVAL = 6,       /* rbf_eval (bytes: 8 in + 12 out per query) */
  RBF_STAGE_SOFTCOST = 7,   /* rbf_soft_cost (bytes: 12 in per point) */
  RBF_STAGE_BACKWARD = 8,   /* rbf_soft_cost_backward (bytes: 12 in + 12 out) */
  RBF_STAGE_TRSM32 = 9,     /* float32 sync-free triangular solves, one interval per launch
                               (flops: n^2 per right-hand side), nested inside SOLVE/BLOCK */
  RBF_STAGE_INVERSE = 10,   /* explicit inverse of the float32 factor (flops: a^3/3) */
  RBF_STAGE_INVAPPLY = 11,  /* solves by products with that inverse (flops: 2 a^2 per right-hand side),
                               nested inside SOLVE/BLOCK */
  RBF_STAGE_COVBLOCK = 12,  /* covariance block of the leaving centers (nested inside BLOCK) */
  RBF_STAGE_SCHUR = 13,     /* information of the staying centers (nested inside BLOCK) */
  RBF_STAGE_ENTER = 14,     /* information of the entering centers (nested inside BLOCK) */
  RBF_STAGE_EVAL_GRID = 15, /* rbf_eval_grid (bytes: 4 out per raster point, 12 with the gradient) */
  RBF_NSTAGE = 16
};
rbf_status rbf_profile_enable(rbf_ctx* ctx, int on);
/* Number of CUDA kernels librbfgb.so has launched since it was loaded (all
 * contexts and threads; host counter, no synchronization). */
rbf_status rbf_launch_count(int64_t* n);
rbf_status rbf_profile_read(rbf_ctx* ctx, double* ms, double* work, int64_t* count, int reset);

/* Test hooks.  They exist so that tests can drive the failure statuses from the
 * host without faulting the GPU; the paper has no counterpart.  Each setting
 * holds for the later calls on this context until it is set back to 0.
 *  RBF_HOOK_DIAG_SHIFT (value: a finite float64): added to every diagonal
 *    entry of the information matrix of the active block before rbf_update
 *    factors it.  A large negative shift makes the block indefinite: the
 *    update returns RBF_ENOTSPD and leaves the state unchanged.
 *  RBF_HOOK_WAIT_LIMIT (value: iterations in [0, 1e12], 0 = the default of
 *    about 4 million): limit of the bounded waits of the sync-free triangular
 *    solves (FP64 solves, and the float32 substitution solves of the mixed
 *    path used above inverse_max) and of the dataflow factorization.
 *  RBF_HOOK_WAIT_NEVER (value 0 or 1): with 1 those waits wait for a flag
 *    value that no block writes, so each runs out after the limit; the call
 *    then returns RBF_ETIMEOUT and an update leaves the state unchanged.
 *  RBF_HOOK_FACTOR_CHAIN (value 0 or 1): with 1 the mixed update factors
 *    with one launch per block column (the path that serves batched patches
 *    and stream capture) instead of the single dataflow launch, so that the
 *    two can be compared on the same frames.
 * RBF_EINVAL for an unknown hook or a value out of range.  Host only. */
enum { RBF_HOOK_DIAG_SHIFT = 1, RBF_HOOK_WAIT_LIMIT = 2, RBF_HOOK_WAIT_NEVER = 3, RBF_HOOK_FACTOR_CHAIN = 4 };
rbf_status rbf_test_hook(rbf_ctx* ctx, int32_t hook, double value);

#ifdef __cplusplus
}
#endif

#endif /* RBFGB_H */
