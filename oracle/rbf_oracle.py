"""FP64 CPU oracle for the RBF terrain hot path -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the CPU-baseline leg of the benchmark
use this module.  The product path (the CUDA library and its Python binding)
never imports it, and this module imports nothing from the product path.

Everything here is plain, slow and written to be checked against the paper by
eye:

* Sec. III-A, Eq. (RBF_fml), Eq. (RBF_def): the terrain model
  f(x; w) = sum_i w_i phi(||x - c_i||) and its basis function.
* Sec. III-A (center selection): a mesh of candidate centers, accepted when
  the number of points within r_kd reaches a threshold (brute-force count
  here; the paper uses a k-d tree).
* Sec. III-B, Eq. (moment_equality), Eq. (RBF_estimator) and the ridge
  estimator that follows it: the regression rows m(x) and batch ridge.
* Sec. III-C, Eq. (H_update), Eq. (kf_w_update), Eq. (mfk_m_approx),
  Eq. (active_rows_weights_update), Eq. (H_inverse_update): the recursive
  update restricted to the active rows, with the covariance kept block
  diagonal (the "block mode" the library implements), and an exact mode that
  keeps the full covariance (used only to pin the block mode).
* Sec. IV-C, Eq. (residual_manifold_left_wheel), Eq. (manifold_derivative),
  Eq. (manidolf_grad_detail), Eq. (manifold_grad_2): the soft-constraint
  residual, its cost and its gradients, generalised from two wheel points to
  many points.

Readings of passages that are silent, garbled or inconsistent (each is listed
in the design notes with its justification):

* G2  the regression row for the Gaussian kernel is (s^2/st^2) k_st(x; c) with
      st^2 = s^2 + noise^2 (the derivation of Sec. III-B), not k_s.
* G3  the innovation is p_z - m~^T w (Eq. active_rows_weights_update prints m~ w).
* G4  the block inverse on the right of Eq. (H_inverse_update) is the prior block.
* G5  df/dp_x = -sum_j w_j (x - x_j)/s^2 k_s (Eq. manidolf_grad_detail lacks the sign).
* G6  d xi / d eta = [-R [p]_x, I] with the right perturbation R <- R Exp(dtheta)
      (Eq. manifold_grad_2 prints [t]_x).
* G8  for the Wendland kernel (not in the paper) m(x) = phi(x); noise is unused.
* G9  the Gaussian is truncated at cutoff_mult * sigma for evaluation and at
      cutoff_mult * sigma~ for the regression rows.
* G10 observation noise covariance R = I (unweighted ridge).
* G11 prior w0 = 0, P0 = I / lambda, so the first update equals batch ridge.
* G13 a candidate center is accepted iff count >= min_count; the distance test
      is d^2 < r_kd^2 in the neighbour arithmetic below.
* G14 neighbour membership: dx = q_x - c_x, dy = q_y - c_y, d2 = dx*dx + dy*dy,
      each operation rounded to float32 (no fused multiply-add), member iff
      d2 < r*r with r rounded to float32 and r*r rounded to float32.
      Lists are in ascending center id.
* G17 Huber_delta(r) = r^2/2 if |r| <= delta else delta (|r| - delta/2);
      loss "l2" gives the paper's lambda_M r^2.
* G18 residual r_i = (R p_i + t)_z - wheel_offset - f((R p_i + t)_xy).
* G21 evaluation on a regular raster (the separable form of the Gaussian on a
      lattice): the truncation is per axis, |dx| < r and |dy| < r with
      r = cutoff_mult * sigma, each decided by the float32 rule of G14.  It keeps
      every term of the circular rule of G9 and adds corner terms, each below
      exp(-cutoff_mult^2 / 2) |w_j|.
"""
from __future__ import annotations

import math

import numpy as np

WENDLAND = 0
GAUSSIAN = 1

__all__ = [
    "WENDLAND", "GAUSSIAN", "phi", "grad_coef", "support_radius_eval",
    "support_radius_assembly", "fl32", "member_f32", "neighbors", "eval_h", "raster_coords", "eval_grid",
    "select_centers", "design_rows", "batch_ridge", "ridge_sparse", "CovStore", "BlockState",
    "block_update", "ExactState", "exact_update", "skew", "huber", "huber_psi",
    "soft_cost", "soft_cost_backward", "soft_cost_normal", "so3_exp", "lm_step",
]


# ---------------------------------------------------------------------------
# Basis functions (Sec. III-A, Eq. RBF_def; Wendland C2 as the compact kernel)
# ---------------------------------------------------------------------------
def phi(r, kind, rho=0.6, sigma=0.04):
    """phi(r).  Gaussian: exp(-r^2 / (2 sigma^2)) (Eq. RBF_def).
    Wendland C2 with support rho: (1 - r/rho)_+^4 (4 r/rho + 1)."""
    r = np.asarray(r, dtype=np.float64)
    if kind == GAUSSIAN:
        return np.exp(-(r * r) / (2.0 * sigma * sigma))
    s = r / rho
    t = np.clip(1.0 - s, 0.0, None)
    return t ** 4 * (4.0 * s + 1.0)


def grad_coef(r, kind, rho=0.6, sigma=0.04):
    """g(r) with grad_x phi(||x - c||) = g(r) (x - c).

    Gaussian: -phi(r) / sigma^2 (Eq. manidolf_grad_detail, sign per reading G5).
    Wendland C2: phi'(r) / r = -20 (1 - r/rho)_+^3 / rho^2.
    """
    r = np.asarray(r, dtype=np.float64)
    if kind == GAUSSIAN:
        return -phi(r, kind, rho, sigma) / (sigma * sigma)
    t = np.clip(1.0 - r / rho, 0.0, None)
    return -20.0 * t ** 3 / (rho * rho)


def support_radius_eval(kind, rho=0.6, sigma=0.04, cutoff_mult=4.0):
    """Radius of the neighbour rule for evaluating f: rho (Wendland) or
    cutoff_mult * sigma (Gaussian, reading G9)."""
    return rho if kind == WENDLAND else cutoff_mult * sigma


def support_radius_assembly(kind, rho=0.6, sigma=0.04, cutoff_mult=4.0, noise=0.0):
    """Radius of the neighbour rule for the regression rows m(x): rho
    (Wendland) or cutoff_mult * sqrt(sigma^2 + noise^2) (Gaussian, G2 + G9)."""
    if kind == WENDLAND:
        return rho
    return cutoff_mult * math.sqrt(sigma * sigma + noise * noise)


# ---------------------------------------------------------------------------
# Neighbour rule (reading G14) -- float32 arithmetic, one rounding per op
# ---------------------------------------------------------------------------
def fl32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def member_f32(q32, c32, radius):
    """Boolean matrix [i, j]: is center j a neighbour of point i?

    q32: (n, 2) float32, c32: (M, 2) float32.  Every operation below is a
    separate float32 operation, so each result is rounded once.
    """
    r32 = np.float32(radius)
    r2 = np.float32(r32 * r32)
    dx = (q32[:, None, 0] - c32[None, :, 0]).astype(np.float32)
    dy = (q32[:, None, 1] - c32[None, :, 1]).astype(np.float32)
    d2 = (dx * dx).astype(np.float32) + (dy * dy).astype(np.float32)
    return d2.astype(np.float32) < r2


def neighbors(q_xy, c_xy, radius, chunk=2048):
    """Neighbour lists by brute force over every (point, center) pair.

    Returns (row_ptr (n+1,), col (nnz,)) with each row's center ids ascending.
    """
    q32 = fl32(q_xy)
    c32 = fl32(c_xy)
    n = q32.shape[0]
    rows = []
    counts = np.zeros(n, dtype=np.int64)
    for s in range(0, n, chunk):
        m = member_f32(q32[s:s + chunk], c32, radius)
        for i in range(m.shape[0]):
            ids = np.nonzero(m[i])[0]
            rows.append(ids)
            counts[s + i] = ids.size
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = np.concatenate(rows).astype(np.int32) if rows else np.zeros(0, np.int32)
    return row_ptr, col


# ---------------------------------------------------------------------------
# Evaluation of f and grad f (Sec. III-A Eq. RBF_fml; Sec. IV-C Eq. manidolf_grad_detail)
# ---------------------------------------------------------------------------
def eval_h(q_xy, c_xy, w, kind, rho=0.6, sigma=0.04, cutoff_mult=4.0,
           truncate=True, chunk=1024):
    """h(q) = sum_j w_j phi(||q - c_j||) and grad h(q) for every query.

    Sums over every center in FP64.  The Wendland terms vanish outside the
    support by definition.  The Gaussian is truncated with the float32
    neighbour rule at cutoff_mult * sigma when ``truncate`` (reading G9).
    Returns (h, gx, gy, abs_h, abs_gx, abs_gy) where abs_* are the sums of the
    absolute values of the terms, used as the scale of a cancellation-safe
    relative tolerance.
    """
    q = np.asarray(q_xy, dtype=np.float64)
    c = np.asarray(c_xy, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    n = q.shape[0]
    out = [np.zeros(n) for _ in range(6)]
    radius = support_radius_eval(kind, rho, sigma, cutoff_mult)
    for s in range(0, n, chunk):
        qq = q[s:s + chunk]
        dx = qq[:, None, 0] - c[None, :, 0]
        dy = qq[:, None, 1] - c[None, :, 1]
        r = np.sqrt(dx * dx + dy * dy)
        p = phi(r, kind, rho, sigma)
        g = grad_coef(r, kind, rho, sigma)
        if kind == GAUSSIAN and truncate:
            mask = member_f32(fl32(qq), fl32(c), radius)
            p = np.where(mask, p, 0.0)
            g = np.where(mask, g, 0.0)
        th = w[None, :] * p
        tx = w[None, :] * g * dx
        ty = w[None, :] * g * dy
        out[0][s:s + chunk] = th.sum(1)
        out[1][s:s + chunk] = tx.sum(1)
        out[2][s:s + chunk] = ty.sum(1)
        out[3][s:s + chunk] = np.abs(th).sum(1)
        out[4][s:s + chunk] = np.abs(tx).sum(1)
        out[5][s:s + chunk] = np.abs(ty).sum(1)
    return tuple(out)


def raster_coords(q0, dq, nq):
    """Raster coordinates q0 + k dq, k = 0..nq-1, in float64 (the product and
    the sum each rounded once); the membership rule uses their float32 copies."""
    k = np.arange(nq, dtype=np.float64)
    return q0 + k * dq


def eval_grid(qx0, qy0, dq, nqx, nqy, c_xy, w, sigma=0.04, cutoff_mult=4.0, chunk=256):
    """Gaussian h and grad h on the raster (qx0 + k dq, qy0 + l dq),
    k < nqx, l < nqy, truncated per axis (reading G21): center j contributes
    to raster point q iff |q_x - c_x| < r and |q_y - c_y| < r with
    r = cutoff_mult * sigma, each axis decided by the float32 rule of G14
    (dx = q_x - c_x and dx * dx rounded to float32, member iff dx*dx < r*r).
    The terms are Eq. RBF_fml with Eq. RBF_def and their gradients
    (Eq. manidolf_grad_detail, sign per G5), summed in FP64 over every center.

    Returns arrays of shape (nqy, nqx), row l = y index:
    (h, gx, gy, abs_h, abs_gx, abs_gy), abs_* the sums of |term| (the scale of
    the cancellation-safe tolerance).
    """
    c = np.asarray(c_xy, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    xs = raster_coords(qx0, dq, nqx)
    ys = raster_coords(qy0, dq, nqy)
    r32 = np.float32(cutoff_mult * sigma)
    r2 = np.float32(r32 * r32)
    cx32, cy32 = fl32(c[:, 0]), fl32(c[:, 1])
    out = [np.zeros((nqy, nqx)) for _ in range(6)]
    inv_s2 = 1.0 / (sigma * sigma)
    for l in range(nqy):
        y = ys[l]
        dy32 = (np.float32(y) - cy32).astype(np.float32)
        in_y = (dy32 * dy32).astype(np.float32) < r2
        if not in_y.any():
            continue
        cj = c[in_y]
        wj = w[in_y]
        dy = y - cj[:, 1]
        cx32j = cx32[in_y]
        for s in range(0, nqx, chunk):
            x = xs[s:s + chunk]
            dx32 = (fl32(x)[:, None] - cx32j[None, :]).astype(np.float32)
            in_x = (dx32 * dx32).astype(np.float32) < r2
            dx = x[:, None] - cj[None, :, 0]
            k = np.exp(-(dx * dx + dy[None, :] * dy[None, :]) * (0.5 * inv_s2))
            th = np.where(in_x, wj[None, :] * k, 0.0)
            tx = -th * dx * inv_s2
            ty = -th * dy[None, :] * inv_s2
            out[0][l, s:s + chunk] = th.sum(1)
            out[1][l, s:s + chunk] = tx.sum(1)
            out[2][l, s:s + chunk] = ty.sum(1)
            out[3][l, s:s + chunk] = np.abs(th).sum(1)
            out[4][l, s:s + chunk] = np.abs(tx).sum(1)
            out[5][l, s:s + chunk] = np.abs(ty).sum(1)
    return tuple(out)


# ---------------------------------------------------------------------------
# Adaptive center selection (Sec. III-A)
# ---------------------------------------------------------------------------
def candidate_mesh(x0, y0, h, nx, ny):
    """Candidate (i, j) at (x0 + (i + 0.5) h, y0 + (j + 0.5) h), row-major
    (j outer).  Each coordinate: one FP64 multiply, then one FP64 add."""
    i = np.arange(nx, dtype=np.float64)
    j = np.arange(ny, dtype=np.float64)
    cx = x0 + (i + 0.5) * h
    cy = y0 + (j + 0.5) * h
    X, Y = np.meshgrid(cx, cy)
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def select_centers(pts_xy, x0, y0, h, nx, ny, r_kd, min_count, chunk=512):
    """Count the points within r_kd of every candidate (float32 rule G14) and
    accept the candidates whose count reaches min_count (reading G13).

    Returns (centers (M, 2) in ascending row-major order, counts (nx*ny,) int32).
    """
    cand = candidate_mesh(x0, y0, h, nx, ny)
    p32 = fl32(pts_xy)
    c32 = fl32(cand)
    counts = np.zeros(cand.shape[0], dtype=np.int64)
    for s in range(0, cand.shape[0], chunk):
        m = member_f32(c32[s:s + chunk], p32, r_kd)
        counts[s:s + chunk] = m.sum(1)
    keep = counts >= min_count
    return cand[keep], counts.astype(np.int32)


# ---------------------------------------------------------------------------
# Regression rows and batch ridge (Sec. III-B)
# ---------------------------------------------------------------------------
def design_rows(x_xy, c_xy, kind, rho=0.6, sigma=0.04, cutoff_mult=4.0, noise=0.0,
                cols=None):
    """Dense matrix Phi (n, M) of regression rows m(x_i)^T.

    Wendland: m(x) = phi(||x - c||) (reading G8).
    Gaussian: m(x) = (sigma^2 / st^2) k_st(x; c), st^2 = sigma^2 + noise^2
    (Sec. III-B, after Eq. mm_corresponding_obj_fun; reading G2), truncated
    with the float32 rule at cutoff_mult * st (G9).
    ``cols`` restricts the matrix to those center ids (in that order).
    """
    x = np.asarray(x_xy, dtype=np.float64)
    c = np.asarray(c_xy, dtype=np.float64)
    if cols is not None:
        c = c[cols]
    dx = x[:, None, 0] - c[None, :, 0]
    dy = x[:, None, 1] - c[None, :, 1]
    r = np.sqrt(dx * dx + dy * dy)
    if kind == WENDLAND:
        return phi(r, WENDLAND, rho)
    st2 = sigma * sigma + noise * noise
    st = math.sqrt(st2)
    m = (sigma * sigma / st2) * np.exp(-(r * r) / (2.0 * st2))
    mask = member_f32(fl32(x), fl32(c), cutoff_mult * st)
    return np.where(mask, m, 0.0)


def batch_ridge(points_xyz, c_xy, lam, kind, rho=0.6, sigma=0.04, cutoff_mult=4.0,
                noise=0.0):
    """w = (sum_i m_i m_i^T + lambda I)^{-1} sum_i m_i z_i (ridge estimator of Sec. III-B)."""
    p = np.asarray(points_xyz, dtype=np.float64)
    Phi = design_rows(p[:, :2], c_xy, kind, rho, sigma, cutoff_mult, noise)
    H = Phi.T @ Phi + lam * np.eye(Phi.shape[1])
    b = Phi.T @ p[:, 2]
    return np.linalg.solve(H, b)


def ridge_sparse(points_xyz, c_xy, lam, kind, rho=0.6, sigma=0.04, cutoff_mult=4.0,
                 noise=0.0, cov_ids=None):
    """The ridge estimator of Sec. III-B with a sparse design matrix, for
    center counts where the dense rows of ``batch_ridge`` do not fit.

    Same estimator: H = sum_i m_i m_i^T + lambda I, w = H^{-1} sum_i m_i z_i.
    The nonzeros of each row m(x_i) are the centers of the float32 neighbour
    rule at the assembly radius (G14); their values are the FP64 regression
    entries of ``design_rows``.  H is factored by a sparse LU (SuperLU, a
    library primitive).  With ``cov_ids`` it also returns P[ids, ids] for
    P = H^{-1}, which is the covariance after one update from the prior (G11).
    """
    from scipy.sparse import csr_matrix, identity
    from scipy.sparse.linalg import splu

    p = np.asarray(points_xyz, dtype=np.float64)
    c = np.asarray(c_xy, dtype=np.float64)
    n, M = p.shape[0], c.shape[0]
    radius = support_radius_assembly(kind, rho, sigma, cutoff_mult, noise)
    row_ptr, col = neighbors(p[:, :2], c, radius)
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    dx = p[rows, 0] - c[col, 0]
    dy = p[rows, 1] - c[col, 1]
    r = np.sqrt(dx * dx + dy * dy)
    if kind == WENDLAND:
        val = phi(r, WENDLAND, rho)
    else:
        st2 = sigma * sigma + noise * noise
        val = (sigma * sigma / st2) * np.exp(-(r * r) / (2.0 * st2))
    Phi = csr_matrix((val, col.astype(np.int64), row_ptr), shape=(n, M))
    H = (Phi.T @ Phi + lam * identity(M, format="csr")).tocsc()
    lu = splu(H)
    w = lu.solve(Phi.T @ p[:, 2])
    if cov_ids is None:
        return w
    ids = np.asarray(cov_ids, dtype=np.int64)
    E = np.zeros((M, ids.size))
    E[ids, np.arange(ids.size)] = 1.0
    X = lu.solve(E)
    Pk = X[ids, :]
    return w, 0.5 * (Pk + Pk.T)


# ---------------------------------------------------------------------------
# Recursive update, block mode (Sec. III-C)
# ---------------------------------------------------------------------------
class CovStore:
    """The covariance P = H^{-1} of all M weights.

    Centers never touched keep the prior P_jj = 1/lambda with no coupling
    (reading G11); the touched ones are held as a dense matrix over the
    touched set.  ``block(A)`` returns P[A, A]; ``set_block(A, PA)`` writes
    P[A, A] = PA and P[A, not A] = P[not A, A] = 0 (the block-diagonal form
    of Eq. H_inverse_update).
    """

    def __init__(self, M, lam):
        self.M = M
        self.lam = lam
        self.pos = np.full(M, -1, dtype=np.int64)
        self.ids = np.zeros(0, dtype=np.int64)
        self.D = np.zeros((0, 0))

    def _grow(self, A):
        new = A[self.pos[A] < 0]
        if new.size == 0:
            return
        k0 = self.ids.size
        k1 = k0 + new.size
        D = np.zeros((k1, k1))
        D[:k0, :k0] = self.D
        D[np.arange(k0, k1), np.arange(k0, k1)] = 1.0 / self.lam
        self.D = D
        self.pos[new] = np.arange(k0, k1)
        self.ids = np.concatenate([self.ids, new])

    def block(self, A):
        A = np.asarray(A, dtype=np.int64)
        out = np.eye(A.size) / self.lam
        known = self.pos[A] >= 0
        kp = self.pos[A][known]
        kk = np.nonzero(known)[0]
        out[np.ix_(kk, kk)] = self.D[np.ix_(kp, kp)]
        return out

    def set_block(self, A, PA):
        A = np.asarray(A, dtype=np.int64)
        self._grow(A)
        ia = self.pos[A]
        self.D[ia, :] = 0.0
        self.D[:, ia] = 0.0
        self.D[np.ix_(ia, ia)] = PA

    def dense(self):
        """Full M x M matrix (small M only)."""
        return self.block(np.arange(self.M))


class BlockState:
    """State of the recursive ridge update in block mode: weights w and the
    covariance store, starting from the prior w0 = 0, P0 = I / lambda (G11)."""

    def __init__(self, c_xy, lam, kind=WENDLAND, rho=0.6, sigma=0.04, cutoff_mult=4.0):
        self.c = np.asarray(c_xy, dtype=np.float64)
        self.M = self.c.shape[0]
        self.lam = lam
        self.kind = kind
        self.rho = rho
        self.sigma = sigma
        self.cutoff_mult = cutoff_mult
        self.w = np.zeros(self.M)
        self.P = CovStore(self.M, lam)
        self.last_active = np.zeros(0, dtype=np.int64)


def active_set(points_xy, c_xy, radius):
    """Active rows of Eq. (mfk_m_approx): the sorted union of every point's
    neighbour list (reading G15: ascending center id)."""
    _, col = neighbors(points_xy, c_xy, radius)
    return np.unique(col).astype(np.int64)


def block_update(st: BlockState, points_xyz, noise=0.0, form="info", joseph=False):
    """One frame of the active-rows recursion (Sec. III-C).

    1. A = active rows (Eq. mfk_m_approx); Phi~ = rows of m(x_i) over A.
    2. P_A = P[A, A] of the stored covariance.
    3. e = z - Phi~^T w_A (Eq. kf_w_update / active_rows_weights_update, G3).
    4. P_new = (P_A^{-1} + Phi~ Phi~^T)^{-1} (Eq. H_update on the block, form
       "info") or, identically, the Woodbury form of Eq. H_inverse_update
       P_A - P_A Phi~ (I + Phi~^T P_A Phi~)^{-1} Phi~^T P_A (form "woodbury").
       With ``joseph`` the covariance is instead
       (I - K Phi~^T) P_A (I - K Phi~^T)^T + K K^T with R = I (G10).
    5. w_A += K e with K = P_new Phi~ (Eq. active_rows_weights_update).
    6. P[A, A] = P_new; P[A, not A] = 0 (block-diagonal form of Eq. H_inverse_update).
    Returns the active set A.
    """
    p = np.asarray(points_xyz, dtype=np.float64)
    if p.shape[0] == 0:
        return np.zeros(0, dtype=np.int64)
    radius = support_radius_assembly(st.kind, st.rho, st.sigma, st.cutoff_mult, noise)
    A = active_set(p[:, :2], st.c, radius)
    st.last_active = A
    if A.size == 0:
        return A
    PhiT = design_rows(p[:, :2], st.c, st.kind, st.rho, st.sigma, st.cutoff_mult, noise,
                       cols=A)            # (n, a) = Phi~^T
    Phi = PhiT.T                          # (a, n)
    PA = st.P.block(A)
    wA = st.w[A]
    e = p[:, 2] - PhiT @ wA
    if form == "woodbury":
        U = PA @ Phi                      # (a, n)
        S = np.eye(p.shape[0]) + Phi.T @ U
        K = U @ np.linalg.inv(S)          # P_A Phi~ S^{-1}
        Pnew = PA - K @ U.T
    else:
        Hnew = np.linalg.inv(PA) + Phi @ PhiT
        Pnew = np.linalg.inv(Hnew)
        K = Pnew @ Phi
    if joseph:
        IKH = np.eye(A.size) - K @ PhiT
        Pnew = IKH @ PA @ IKH.T + K @ K.T
    Pnew = 0.5 * (Pnew + Pnew.T)
    st.w[A] = wA + K @ e
    st.P.set_block(A, Pnew)
    return A


# ---------------------------------------------------------------------------
# Exact recursion with the full covariance (used only to pin the block mode)
# ---------------------------------------------------------------------------
class ExactState:
    def __init__(self, c_xy, lam, kind=WENDLAND, rho=0.6, sigma=0.04, cutoff_mult=4.0):
        self.c = np.asarray(c_xy, dtype=np.float64)
        self.M = self.c.shape[0]
        self.kind, self.rho, self.sigma, self.cutoff_mult = kind, rho, sigma, cutoff_mult
        self.w = np.zeros(self.M)
        self.P = np.eye(self.M) / lam


def exact_update(st: ExactState, points_xyz, noise=0.0):
    """Eq. (kf_w_update) and Eq. (H_inverse_update) on the full matrices."""
    p = np.asarray(points_xyz, dtype=np.float64)
    m = design_rows(p[:, :2], st.c, st.kind, st.rho, st.sigma, st.cutoff_mult, noise).T
    U = st.P @ m
    S = np.eye(p.shape[0]) + m.T @ U
    K = U @ np.linalg.inv(S)
    st.w = st.w + K @ (p[:, 2] - m.T @ st.w)
    st.P = st.P - K @ U.T
    st.P = 0.5 * (st.P + st.P.T)


# ---------------------------------------------------------------------------
# Soft constraint (Sec. IV-C)
# ---------------------------------------------------------------------------
def skew(v):
    """[v]_x, the skew-symmetric matrix with [v]_x u = v x u."""
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])


def huber(r, delta):
    a = np.abs(r)
    return np.where(a <= delta, 0.5 * r * r, delta * (a - 0.5 * delta))


def huber_psi(r, delta):
    return np.clip(r, -delta, delta)


def soft_cost(R, t, body_xyz, c_xy, w, kind, rho=0.6, sigma=0.04, cutoff_mult=4.0,
              delta=0.05, wheel_offset=0.0, loss="huber", lam_m=1.0):
    """Soft-constraint cost over many points and its pose gradient.

    q_i = R p_i + t; r_i = q_z - wheel_offset - f(q_xy) (Eq.
    residual_manifold_left_wheel, G18); cost = sum Huber_delta(r_i) (G17) or
    lam_m sum r_i^2 (the paper's J_M).  Pose gradient [d/dtheta, d/dt] with
    R <- R Exp(dtheta), t <- t + dt: dr/dq = [-f_x, -f_y, 1]
    (Eq. manifold_derivative), dq/dtheta = -R [p]_x, dq/dt = I (G6).
    Returns dict(cost, grad6, r, J (n, 6), psi).
    """
    R = np.asarray(R, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    p = np.asarray(body_xyz, dtype=np.float64)
    q = p @ R.T + t[None, :]
    h, gx, gy, *_ = eval_h(q[:, :2], c_xy, w, kind, rho, sigma, cutoff_mult)
    r = q[:, 2] - wheel_offset - h
    drdq = np.stack([-gx, -gy, np.ones_like(gx)], axis=1)     # (n, 3)
    J = np.zeros((p.shape[0], 6))
    for i in range(p.shape[0]):
        J[i, :3] = drdq[i] @ (-R @ skew(p[i]))
        J[i, 3:] = drdq[i]
    if loss == "l2":
        cost = lam_m * float(np.sum(r * r))
        psi = 2.0 * lam_m * r
    else:
        cost = float(np.sum(huber(r, delta)))
        psi = huber_psi(r, delta)
    grad6 = psi @ J
    return dict(cost=cost, grad6=grad6, r=r, J=J, psi=psi, q=q)


def soft_cost_normal(R, t, body_xyz, c_xy, w, kind, rho=0.6, sigma=0.04, cutoff_mult=4.0,
                     delta=0.05, wheel_offset=0.0, loss="huber", lam_m=1.0):
    """Gauss-Newton matrix of the pose for a Levenberg-Marquardt step on the
    soft-constraint cost (Sec. IV-C minimises J_M by LM):
    A = sum_i omega_i J_i^T J_i with the iteratively reweighted least-squares
    weight omega_i = psi(r_i) / r_i (1 inside the Huber zone, delta / |r_i|
    outside; 2 lam_m for the L2 loss).  Returns dict(cost, grad6, A)."""
    d = soft_cost(R, t, body_xyz, c_xy, w, kind, rho, sigma, cutoff_mult, delta, wheel_offset, loss, lam_m)
    r, J = d["r"], d["J"]
    if loss == "l2":
        om = np.full(r.shape, 2.0 * lam_m)
    else:
        a = np.abs(r)
        om = np.where(a <= delta, 1.0, delta / np.maximum(a, 1e-300))
    A = (J * om[:, None]).T @ J
    return dict(cost=d["cost"], grad6=d["grad6"], A=A)


def so3_exp(v):
    """exp([v]_x) by Rodrigues' formula (the right perturbation R <- R Exp(dtheta))."""
    v = np.asarray(v, dtype=np.float64)
    a = float(np.linalg.norm(v))
    K = skew(v)
    if a < 1e-12:
        return np.eye(3) + K
    return np.eye(3) + math.sin(a) / a * K + (1.0 - math.cos(a)) / (a * a) * (K @ K)


def lm_step(R, t, body_xyz, c_xy, w, kind, mu=1e-3, **kw):
    """One Levenberg-Marquardt step on the pose: (A + mu diag(A)) d = -g,
    R <- R Exp(d_theta), t <- t + d_t."""
    d = soft_cost_normal(R, t, body_xyz, c_xy, w, kind, **kw)
    A = d["A"]
    step = np.linalg.solve(A + mu * np.diag(np.diag(A)), -d["grad6"])
    return np.asarray(R) @ so3_exp(step[:3]), np.asarray(t) + step[3:], d["cost"]


def soft_cost_backward(R, t, body_xyz, c_xy, w, kind, rho=0.6, sigma=0.04,
                       cutoff_mult=4.0, delta=0.05, wheel_offset=0.0, loss="huber",
                       lam_m=1.0, gout=1.0):
    """Gradient of gout * cost with respect to the weights, the centers and the pose.

    With r_i = q_z - off - sum_j w_j phi(||q_i - c_j||):
      dr_i/dw_j = -phi(||q_i - c_j||),
      dr_i/dc_j = +w_j g(||q_i - c_j||) (q_i - c_j)   (chain rule of Eq. manidolf_grad_detail),
    so dC/dw_j = -sum_i psi_i phi_ij and dC/dc_j = sum_i psi_i w_j g_ij (q_i - c_j).

    Also returns, per center, the sums of the absolute values of those terms
    (dw_abs, dc_abs) and of the terms without psi (phi_abs = sum_i |phi_ij|,
    gq_abs = sum_i |w_j g_ij (q_i - c_j)|): the scales of a per-entry,
    cancellation-safe tolerance.
    """
    fw = soft_cost(R, t, body_xyz, c_xy, w, kind, rho, sigma, cutoff_mult, delta,
                   wheel_offset, loss, lam_m)
    q = fw["q"]
    psi = fw["psi"] * gout
    c = np.asarray(c_xy, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    dw = np.zeros(c.shape[0])
    dc = np.zeros((c.shape[0], 2))
    dw_abs = np.zeros(c.shape[0])
    dc_abs = np.zeros((c.shape[0], 2))
    phi_abs = np.zeros(c.shape[0])
    gq_abs = np.zeros((c.shape[0], 2))
    radius = support_radius_eval(kind, rho, sigma, cutoff_mult)
    chunk = 1024
    for s in range(0, q.shape[0], chunk):
        qq = q[s:s + chunk, :2]
        dx = qq[:, None, 0] - c[None, :, 0]
        dy = qq[:, None, 1] - c[None, :, 1]
        r = np.sqrt(dx * dx + dy * dy)
        p = phi(r, kind, rho, sigma)
        g = grad_coef(r, kind, rho, sigma)
        if kind == GAUSSIAN:
            mask = member_f32(fl32(qq), fl32(c), radius)
            p = np.where(mask, p, 0.0)
            g = np.where(mask, g, 0.0)
        ps = psi[s:s + chunk, None]
        dw -= (ps * p).sum(0)
        dc[:, 0] += (ps * g * dx).sum(0) * w
        dc[:, 1] += (ps * g * dy).sum(0) * w
        dw_abs += np.abs(ps * p).sum(0)
        dc_abs[:, 0] += np.abs(ps * g * dx).sum(0) * np.abs(w)
        dc_abs[:, 1] += np.abs(ps * g * dy).sum(0) * np.abs(w)
        phi_abs += np.abs(p).sum(0)
        gq_abs[:, 0] += np.abs(g * dx).sum(0) * np.abs(w)
        gq_abs[:, 1] += np.abs(g * dy).sum(0) * np.abs(w)
    return dict(dw=dw, dc=dc, dpose6=fw["grad6"] * gout, cost=fw["cost"] * gout, fw=fw,
                dw_abs=dw_abs, dc_abs=dc_abs, phi_abs=phi_abs, gq_abs=gq_abs)
