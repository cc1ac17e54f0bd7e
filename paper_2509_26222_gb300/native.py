"""Thin ctypes binding of librbfgb.so (argument marshalling only).

Every computation runs in the library's CUDA kernels; this module only turns
torch CUDA tensors into device pointers and the current torch stream into a
cudaStream_t.  It raises when the library is missing: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

_LIB = None

RBF_OK = 0
STATUS = {0: "RBF_OK", -1: "RBF_EINVAL", -2: "RBF_ENOMEM", -3: "RBF_ECUDA", -4: "RBF_ENOTSPD",
          -5: "RBF_ETIMEOUT", -6: "RBF_ESTATE", -7: "RBF_ERANGE"}
KERNEL_WENDLAND, KERNEL_GAUSSIAN = 0, 1
UPDATE_FP64, UPDATE_MIXED = 0, 1
LOSS_HUBER, LOSS_L2 = 0, 1


class RBFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class RbfConfig(ctypes.Structure):
    """Mirror of ``rbf_config`` in include/rbfgb.h (same field order)."""
    _fields_ = [
        ("kernel", ctypes.c_int32),
        ("update_precision", ctypes.c_int32),
        ("rho", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("cutoff_mult", ctypes.c_double),
        ("lambda_", ctypes.c_double),
        ("loss", ctypes.c_int32),
        ("min_count", ctypes.c_int32),
        ("huber_delta", ctypes.c_double),
        ("lambda_m", ctypes.c_double),
        ("wheel_offset", ctypes.c_double),
        ("mesh_x0", ctypes.c_double),
        ("mesh_y0", ctypes.c_double),
        ("mesh_h", ctypes.c_double),
        ("mesh_nx", ctypes.c_int32),
        ("mesh_ny", ctypes.c_int32),
        ("r_kd", ctypes.c_double),
        ("refine_sweeps", ctypes.c_int32),
        ("inverse_max", ctypes.c_int32),
        ("exact", ctypes.c_int32),
        ("reserved1", ctypes.c_int32),
    ]


class RbfPatch(ctypes.Structure):
    """Mirror of ``rbf_patch`` in include/rbfgb.h."""
    _fields_ = [
        ("x0", ctypes.c_double),
        ("y0", ctypes.c_double),
        ("spacing", ctypes.c_double),
        ("nx", ctypes.c_int32),
        ("pad0", ctypes.c_int32),
        ("M", ctypes.c_int64),
        ("n", ctypes.c_int64),
        ("pts", ctypes.c_void_p),
        ("Q", ctypes.c_int64),
        ("q", ctypes.c_void_p),
        ("w", ctypes.c_void_p),
        ("h", ctypes.c_void_p),
        ("grad", ctypes.c_void_p),
    ]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double
_SIGS = {
    "rbf_create": [ctypes.POINTER(RbfConfig), ctypes.POINTER(_P)],
    "rbf_destroy": [_P],
    "rbf_set_centers": [_P, _P, _I64, _P],
    "rbf_build_centers": [_P, _P, _I64, _P, ctypes.POINTER(_I64), _P],
    "rbf_num_centers": [_P, ctypes.POINTER(_I64)],
    "rbf_get_centers": [_P, _P, _P],
    "rbf_get_weights": [_P, _P, _P],
    "rbf_set_weights": [_P, _P, _P],
    "rbf_update": [_P, _P, _I64, _D, _P],
    "rbf_eval": [_P, _P, _I64, _P, _P, _P],
    "rbf_eval_grid": [_P, _D, _D, _D, _I64, _I64, _P, _P, _P],
    "rbf_soft_cost": [_P, _P, _P, _P, _I64, _P, _P, _P, _P],
    "rbf_soft_cost_backward": [_P, _P, _P, _P, _I64, _P, _P, _P, _P, _P],
    "rbf_get_cov": [_P, _P, _I64, _P, _P],
    "rbf_get_active": [_P, _P, _I64, ctypes.POINTER(_I64), _P],
    "rbf_get_neighbors": [_P, _P, _I64, _D, _P, _P, _I64, ctypes.POINTER(_I64), _P],
    "rbf_profile_enable": [_P, ctypes.c_int],
    "rbf_profile_read": [_P, _P, _P, _P, ctypes.c_int],
    "rbf_launch_count": [ctypes.POINTER(_I64)],
    "rbf_soft_cost_normal": [_P, _P, _P, _P, _I64, _P, _P],
    "rbf_batch_update_eval": [_P, _P, ctypes.c_int32, _P],
    "rbf_lm_step": [_P, _P, _P, _P, _I64, _D, _P, _P],
    "rbf_test_hook": [_P, ctypes.c_int32, _D],
    "rbf_soft_cost_noalloc": [_P, _P, _P, _P, _I64, _P, _P, _P, _P],
}
HOOK_DIAG_SHIFT, HOOK_WAIT_LIMIT, HOOK_WAIT_NEVER, HOOK_FACTOR_CHAIN = 1, 2, 3, 4

STAGES = ["neighbors", "assembly", "block", "panel", "trailing", "solve", "eval", "softcost", "backward",
          "trsm32", "inverse", "invapply", "covblock", "schur", "enter", "evalgrid"]


def _out_tensor(t, n, device, dtype=torch.float32):
    """A caller's output buffer: contiguous `dtype` on the context's device
    with room for n values (the kernels write through its raw pointer)."""
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"output buffers must be contiguous {dtype} tensors")
    if t.device != torch.device(device):
        raise ValueError(f"output buffer on {t.device}, expected {device}")
    if t.numel() < n:
        raise ValueError(f"output buffer holds {t.numel()} values, {n} needed")
    return t


def launch_count() -> int:
    """Kernels launched by librbfgb.so since it was loaded."""
    n = ctypes.c_int64()
    _check(load().rbf_launch_count(ctypes.byref(n)))
    return n.value


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load librbfgb.so (building it first if asked).  Raises if absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"{path} is missing: run paper_2509_26222_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.rbf_last_error.argtypes = []
    lib.rbf_last_error.restype = ctypes.c_char_p
    _LIB = lib
    return lib


def _check(st):
    if st != RBF_OK:
        raise RBFError(st, _LIB.rbf_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev_tensor(x, dtype, cols=None):
    if not isinstance(x, torch.Tensor):
        x = torch.as_tensor(x)
    if x.device.type != "cuda":
        raise ValueError("device tensors only (use .cuda()): the library has no host path")
    x = x.to(dtype).contiguous()
    if cols is not None and (x.dim() != 2 or x.shape[1] != cols):
        raise ValueError(f"expected shape (n, {cols}), got {tuple(x.shape)}")
    return x


class Terrain:
    """One terrain model (a context of librbfgb.so) on the current CUDA device."""

    def __init__(self, kernel=KERNEL_WENDLAND, rho=0.6, sigma=0.04, cutoff_mult=4.0, lam=1e-3,
                 update_precision=UPDATE_FP64, loss=LOSS_HUBER, huber_delta=0.05, lambda_m=1.0,
                 wheel_offset=0.0, mesh=None, r_kd=0.1, min_count=1, refine_sweeps=0, inverse_max=0,
                 exact=False):
        self.lib = load()
        cfg = RbfConfig()
        cfg.kernel = kernel
        cfg.update_precision = update_precision
        cfg.rho = rho
        cfg.sigma = sigma
        cfg.cutoff_mult = cutoff_mult
        cfg.lambda_ = lam
        cfg.loss = loss
        cfg.min_count = min_count
        cfg.huber_delta = huber_delta
        cfg.lambda_m = lambda_m
        cfg.wheel_offset = wheel_offset
        x0, y0, h, nx, ny = mesh if mesh is not None else (0.0, 0.0, 1.0, 1, 1)
        cfg.mesh_x0, cfg.mesh_y0, cfg.mesh_h, cfg.mesh_nx, cfg.mesh_ny = x0, y0, h, nx, ny
        cfg.r_kd = r_kd
        cfg.refine_sweeps = refine_sweeps
        cfg.inverse_max = inverse_max
        cfg.exact = 1 if exact else 0
        self.cfg = cfg
        self.device = torch.cuda.current_device()
        h_ = ctypes.c_void_p()
        _check(self.lib.rbf_create(ctypes.byref(cfg), ctypes.byref(h_)))
        self._h = h_

    def close(self):
        if getattr(self, "_h", None):
            self.lib.rbf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- centers ----------------------------------------------------------
    def set_centers(self, cxy):
        c = _dev_tensor(cxy, torch.float64, 2)
        _check(self.lib.rbf_set_centers(self._h, _ptr(c), c.shape[0], _stream()))

    def build_centers(self, pts, return_counts=False):
        p = _dev_tensor(pts, torch.float32, 3)
        counts = None
        if return_counts:
            counts = torch.empty(self.cfg.mesh_nx * self.cfg.mesh_ny, dtype=torch.int32, device=p.device)
        M = ctypes.c_int64()
        _check(self.lib.rbf_build_centers(self._h, _ptr(p), p.shape[0], _ptr(counts), ctypes.byref(M),
                                          _stream()))
        return (M.value, counts) if return_counts else M.value

    @property
    def M(self):
        m = ctypes.c_int64()
        _check(self.lib.rbf_num_centers(self._h, ctypes.byref(m)))
        return m.value

    def centers(self):
        out = torch.empty(self.M, 2, dtype=torch.float64, device="cuda")
        _check(self.lib.rbf_get_centers(self._h, _ptr(out), _stream()))
        return out

    def weights(self):
        out = torch.empty(self.M, dtype=torch.float64, device="cuda")
        _check(self.lib.rbf_get_weights(self._h, _ptr(out), _stream()))
        return out

    def set_weights(self, w):
        w = _dev_tensor(w, torch.float64)
        _check(self.lib.rbf_set_weights(self._h, _ptr(w), _stream()))

    # -- hot path ---------------------------------------------------------
    def update(self, pts, noise=0.0):
        p = _dev_tensor(pts, torch.float32, 3)
        _check(self.lib.rbf_update(self._h, _ptr(p), p.shape[0], float(noise), _stream()))

    def eval(self, q, out_h=None, out_grad=None, with_grad=True):
        q = _dev_tensor(q, torch.float32, 2)
        Q = q.shape[0]
        h = _out_tensor(out_h, Q, q.device) if out_h is not None else torch.empty(Q, dtype=torch.float32,
                                                                                   device=q.device)
        g = None
        if with_grad:
            g = (_out_tensor(out_grad, 2 * Q, q.device) if out_grad is not None
                 else torch.empty(Q, 2, dtype=torch.float32, device=q.device))
        _check(self.lib.rbf_eval(self._h, _ptr(q), Q, _ptr(h), _ptr(g), _stream()))
        return h, g

    def eval_grid(self, qx0, qy0, dq, nqx, nqy, out_h=None, out_grad=None, with_grad=True):
        """h (nqy x nqx) and grad h (nqy x nqx x 2) on the raster (qx0 + k dq, qy0 + l dq):
        Gaussian kernel, centers on a lattice, per-axis truncation (rbf_eval_grid)."""
        dev = torch.device("cuda", torch.cuda.current_device())
        n = int(nqx) * int(nqy)
        h = _out_tensor(out_h, n, dev) if out_h is not None else torch.empty(nqy, nqx, dtype=torch.float32, device=dev)
        g = None
        if with_grad:
            g = (_out_tensor(out_grad, 2 * n, dev) if out_grad is not None
                 else torch.empty(nqy, nqx, 2, dtype=torch.float32, device=dev))
        _check(self.lib.rbf_eval_grid(self._h, float(qx0), float(qy0), float(dq), int(nqx), int(nqy), _ptr(h),
                                      _ptr(g), _stream()))
        return h, g

    def soft_cost(self, R, t, pts, with_resid=False, out=None):
        R = torch.as_tensor(R, dtype=torch.float64).cpu().contiguous()
        t = torch.as_tensor(t, dtype=torch.float64).cpu().contiguous()
        p = _dev_tensor(pts, torch.float32, 3)
        buf = _out_tensor(out, 7, p.device, torch.float64) if out is not None else torch.empty(
            7, dtype=torch.float64, device=p.device)
        resid = torch.empty(p.shape[0], dtype=torch.float32, device=p.device) if with_resid else None
        _check(self.lib.rbf_soft_cost(self._h, _ptr(R), _ptr(t), _ptr(p), p.shape[0], _ptr(buf[:1]),
                                      ctypes.c_void_p(buf.data_ptr() + 8), _ptr(resid), _stream()))
        return buf[0], buf[1:7], resid

    def soft_cost_normal(self, R, t, pts, out=None):
        """(cost, gradient (6), Gauss-Newton matrix A (6 x 6)) of the pose, device tensors."""
        R = torch.as_tensor(R, dtype=torch.float64).cpu().contiguous()
        t = torch.as_tensor(t, dtype=torch.float64).cpu().contiguous()
        p = _dev_tensor(pts, torch.float32, 3)
        buf = _out_tensor(out, 28, p.device, torch.float64) if out is not None else torch.empty(
            28, dtype=torch.float64, device=p.device)
        _check(self.lib.rbf_soft_cost_normal(self._h, _ptr(R), _ptr(t), _ptr(p), p.shape[0], _ptr(buf), _stream()))
        iu = torch.triu_indices(6, 6, device=p.device)
        A = torch.zeros(6, 6, dtype=torch.float64, device=p.device)
        A[iu[0], iu[1]] = buf[7:28]
        A = A + A.T - torch.diag(torch.diagonal(A))
        return buf[0], buf[1:7], A

    def lm_step(self, R, t, pts, mu=1e-3, out=None):
        """One Levenberg-Marquardt step on the pose (rbf_lm_step, on the device).
        Returns (R_out, t_out, cost at the input pose) as host float64 arrays;
        the full 20-value result stays in ``out`` when given."""
        R = torch.as_tensor(R, dtype=torch.float64).cpu().contiguous()
        t = torch.as_tensor(t, dtype=torch.float64).cpu().contiguous()
        p = _dev_tensor(pts, torch.float32, 3)
        buf = _out_tensor(out, 20, p.device, torch.float64) if out is not None else torch.empty(
            20, dtype=torch.float64, device=p.device)
        _check(self.lib.rbf_lm_step(self._h, _ptr(R), _ptr(t), _ptr(p), p.shape[0], float(mu), _ptr(buf), _stream()))
        h = buf.cpu().numpy()
        return h[:9].reshape(3, 3).copy(), h[9:12].copy(), float(h[12])

    def test_hook(self, hook, value):
        """Set a test hook of the context (rbf_test_hook)."""
        _check(self.lib.rbf_test_hook(self._h, int(hook), float(value)))

    def soft_cost_backward(self, R, t, pts, gout=None):
        R = torch.as_tensor(R, dtype=torch.float64).cpu().contiguous()
        t = torch.as_tensor(t, dtype=torch.float64).cpu().contiguous()
        p = _dev_tensor(pts, torch.float32, 3)
        M = self.M
        dw = torch.empty(M, dtype=torch.float32, device=p.device)
        dc = torch.empty(M, 2, dtype=torch.float32, device=p.device)
        dpose = torch.empty(6, dtype=torch.float64, device=p.device)
        g = None if gout is None else _dev_tensor(gout, torch.float64).reshape(1)
        _check(self.lib.rbf_soft_cost_backward(self._h, _ptr(R), _ptr(t), _ptr(p), p.shape[0], _ptr(g),
                                               _ptr(dw), _ptr(dc), _ptr(dpose), _stream()))
        return dw, dc, dpose

    # -- batched patches --------------------------------------------------
    def batch_update_eval(self, patches):
        """patches: list of dicts with keys x0, y0, spacing, nx, M, pts (device n x 3
        float32), q (device Q x 2 float32).  Returns a list of (w, h, grad) device
        tensors.  Each patch is its own terrain updated once from the prior."""
        arr = (RbfPatch * len(patches))()
        outs = []
        keep = []
        for k, p in enumerate(patches):
            pts = _dev_tensor(p["pts"], torch.float32, 3)
            q = _dev_tensor(p["q"], torch.float32, 2)
            M = int(p["M"])
            w = torch.empty(M, dtype=torch.float64, device=pts.device)
            h = torch.empty(q.shape[0], dtype=torch.float32, device=pts.device)
            g = torch.empty(q.shape[0], 2, dtype=torch.float32, device=pts.device)
            keep += [pts, q]
            outs.append((w, h, g))
            d = arr[k]
            d.x0, d.y0, d.spacing, d.nx = float(p["x0"]), float(p["y0"]), float(p["spacing"]), int(p["nx"])
            d.M, d.n, d.Q = M, pts.shape[0], q.shape[0]
            d.pts, d.q = pts.data_ptr(), q.data_ptr()
            d.w, d.h, d.grad = w.data_ptr(), h.data_ptr(), g.data_ptr()
        _check(self.lib.rbf_batch_update_eval(self._h, ctypes.cast(arr, ctypes.c_void_p), len(patches), _stream()))
        self._batch_keep = keep
        return outs

    def batch_update_eval_into(self, arr, count):
        """Run a prepared RbfPatch array (buffers owned by the caller)."""
        _check(self.lib.rbf_batch_update_eval(self._h, ctypes.cast(arr, ctypes.c_void_p), count, _stream()))

    # -- stage timing -----------------------------------------------------
    def profile(self, on=True):
        _check(self.lib.rbf_profile_enable(self._h, 1 if on else 0))

    def profile_read(self, reset=True):
        """{stage: (ms, work, intervals)} accumulated since the last reset."""
        k = len(STAGES)
        ms = (ctypes.c_double * k)()
        work = (ctypes.c_double * k)()
        cnt = (ctypes.c_int64 * k)()
        _check(self.lib.rbf_profile_read(self._h, ms, work, cnt, 1 if reset else 0))
        return {STAGES[i]: (ms[i], work[i], cnt[i]) for i in range(k)}

    # -- inspection -------------------------------------------------------
    def cov(self, ids):
        ids = torch.as_tensor(ids, dtype=torch.int32).cpu().contiguous()
        k = ids.numel()
        out = torch.empty(k, k, dtype=torch.float64, device="cuda")
        _check(self.lib.rbf_get_cov(self._h, _ptr(ids), k, _ptr(out), _stream()))
        return out

    def active(self):
        a = ctypes.c_int64()
        buf = torch.empty(max(self.M, 1), dtype=torch.int32, device="cuda")
        _check(self.lib.rbf_get_active(self._h, _ptr(buf), buf.numel(), ctypes.byref(a), _stream()))
        return buf[:a.value].clone()

    def neighbors(self, pts, noise=0.0):
        p = _dev_tensor(pts, torch.float32, 3)
        n = p.shape[0]
        rp = torch.empty(n + 1, dtype=torch.int64, device=p.device)
        nnz = ctypes.c_int64()
        st = self.lib.rbf_get_neighbors(self._h, _ptr(p), n, float(noise), _ptr(rp), None, 0,
                                        ctypes.byref(nnz), _stream())
        if st not in (RBF_OK, -7):
            _check(st)
        col = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=p.device)
        _check(self.lib.rbf_get_neighbors(self._h, _ptr(p), n, float(noise), _ptr(rp), _ptr(col),
                                          col.numel(), ctypes.byref(nnz), _stream()))
        return rp, col[:nnz.value]


class SoftCost(torch.autograd.Function):
    """cost = sum_i loss(r_i) with r_i = (R p_i + t)_z - off - h((R p_i + t)_xy).

    Inputs: (terrain, R (3x3, host), t (3, host), pts (device), w (M, device,
    float64), c (M x 2, device, float64), pose6 (6, device, float64)).  ``w``,
    ``c`` and ``pose6`` are the differentiable leaves: the weights, the centers
    and a zero pose increment [theta, t] applied as R Exp(theta), t + dt.  The
    kernels read the weights and centers from the terrain, so ``w`` and ``c``
    must equal the terrain's own (checked: ValueError otherwise), and
    ``pose6`` must be zero (the pose is R, t).
    """

    @staticmethod
    def forward(ctx, terrain, R, t, pts, w, c, pose6):
        if not torch.equal(w.detach().to(torch.float64).reshape(-1), terrain.weights()):
            raise ValueError("w differs from the terrain's weights: install it with set_weights first")
        if not torch.equal(c.detach().to(torch.float64).reshape(-1, 2), terrain.centers()):
            raise ValueError("c differs from the terrain's centers: install them with set_centers first")
        if torch.count_nonzero(pose6.detach()).item() != 0:
            raise ValueError("pose6 must be the zero increment; pass the pose as R, t")
        cost, _, _ = terrain.soft_cost(R, t, pts)
        ctx.terrain = terrain
        ctx.R, ctx.t = R, t
        ctx.save_for_backward(pts)
        return cost.clone()

    @staticmethod
    def backward(ctx, gout):
        (pts,) = ctx.saved_tensors
        dw, dc, dpose = ctx.terrain.soft_cost_backward(ctx.R, ctx.t, pts, gout=gout.detach().reshape(1))
        return None, None, None, None, dw.double(), dc.double(), dpose
