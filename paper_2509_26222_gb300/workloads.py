"""Seeded synthetic inputs for the RBF terrain hot path.

This module only draws random numbers and evaluates the *ground-truth* terrain
shapes used to make synthetic scans.  It contains none of the method's
arithmetic (no RBF kernel, no neighbour search, no regression), so that the
CPU oracle and the CUDA path receive identical inputs without sharing code.

The paper's own data (real Mid360 scans of a legged-wheel robot, Sec. VI-A)
is not available; the shapes below stand in for it:

* ``config1``  -- 16x16 centers at 0.25 m, 2,000 noisy points on a
  sinusoid-plus-step surface, 10,000 uniform queries (Sec. III, small case).
* ``config2_centers`` / ``config2_frame`` -- a 64x64 center grid at 0.2 m and
  a 200-frame sequence of Mid360-like scans over a staircase with bumps
  (ground returns ray-marched to the height field, range noise along the ray).
* ``config3`` -- soft-constraint workload: 65,536 body-frame points under a
  random SE(3) pose, weights for the 64x64 grid (Sec. IV-C).
* ``config4_patch`` -- one of 256 independent patches of uneven size.
* ``config5`` -- 256x256 centers at 0.1 m, one 128x64 active block touched by
  32,768 points, and 1,048,576 queries.

All arrays are float64 unless stated; callers cast to the dtype an interface
needs (points and queries are float32 on the device path).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "KernelSpec", "Config1", "config1", "config2_centers", "config2_frame",
    "config3", "config4_patch", "config5", "uniform_queries", "grid_centers",
    "surface_c1", "surface_c2", "random_pose",
]


@dataclass
class KernelSpec:
    """Parameters of the basis function (Sec. III-A, Eq. RBF_def).

    kind 0 = Wendland C2 with support ``rho``; kind 1 = Gaussian with
    bandwidth ``sigma`` truncated at ``cutoff_mult * sigma``.
    """
    kind: int = 0
    rho: float = 0.6
    sigma: float = 0.04
    cutoff_mult: float = 4.0
    lam: float = 1e-3


def grid_centers(nx: int, ny: int, x0: float, y0: float, h: float) -> np.ndarray:
    """Centers of a regular nx x ny mesh, row-major (y outer, x inner).

    Center (i, j) sits at (x0 + (i + 0.5) h, y0 + (j + 0.5) h); id = j*nx + i.
    """
    i = np.arange(nx, dtype=np.float64)
    j = np.arange(ny, dtype=np.float64)
    cx = x0 + (i + 0.5) * h
    cy = y0 + (j + 0.5) * h
    X, Y = np.meshgrid(cx, cy)  # shape (ny, nx), row-major
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def surface_c1(x, y):
    """Config-1 ground truth: 0.1 sin(2x) cos(1.5y) plus a 0.15 m step at x = 2."""
    return 0.1 * np.sin(2.0 * x) * np.cos(1.5 * y) + 0.15 * (x >= 2.0)


def surface_c2(x, y):
    """Config-2 ground truth: flat for x < 0, then 10 stairs (tread 0.30 m,
    rise 0.15 m, top at 1.5 m), plus bumps of +-2 cm everywhere."""
    steps = np.zeros_like(np.asarray(x, dtype=np.float64))
    for k in range(10):
        steps = steps + 0.15 * (x >= 0.3 * k)
    bumps = 0.02 * np.sin(2.0 * np.pi * x / 0.5) * np.cos(2.0 * np.pi * y / 0.7)
    return steps + bumps


def uniform_queries(rng: np.random.Generator, q: int, lo: float, hi: float,
                    lo_y: float | None = None, hi_y: float | None = None) -> np.ndarray:
    lo_y = lo if lo_y is None else lo_y
    hi_y = hi if hi_y is None else hi_y
    x = rng.uniform(lo, hi, q)
    y = rng.uniform(lo_y, hi_y, q)
    return np.stack([x, y], axis=1)


@dataclass
class Config1:
    centers: np.ndarray
    points: np.ndarray      # (n, 3) world frame
    queries: np.ndarray     # (Q, 2)
    kernel: KernelSpec = field(default_factory=KernelSpec)
    noise: float = 0.02


def config1(seed: int = 0, n: int = 2000, q: int = 10_000) -> Config1:
    """16x16 centers at 0.25 m on [0,4]^2, Wendland rho = 0.6, lambda = 1e-3."""
    rng = np.random.default_rng(seed)
    centers = grid_centers(16, 16, 0.0, 0.0, 0.25)
    xy = rng.uniform(0.0, 4.0, size=(n, 2))
    z = surface_c1(xy[:, 0], xy[:, 1]) + rng.normal(0.0, 0.02, n)
    pts = np.concatenate([xy, z[:, None]], axis=1)
    qs = uniform_queries(rng, q, 0.0, 4.0)
    return Config1(centers, pts, qs, KernelSpec(kind=0, rho=0.6, lam=1e-3), 0.02)


# ----------------------------------------------------------------------------
# Config 2: LIO sequence over a staircase
# ----------------------------------------------------------------------------
C2_NX = 64
C2_H = 0.2
C2_X0 = -6.4
C2_FRAMES = 200
C2_GROUND = 8000
C2_OTHER = 12000
C2_SENSOR_HEIGHT = 0.6
C2_RANGE_SIGMA = 0.03


def config2_centers() -> np.ndarray:
    """64x64 centers at 0.2 m covering [-6.4, 6.4]^2 (M = 4,096)."""
    return grid_centers(C2_NX, C2_NX, C2_X0, C2_X0, C2_H)


def config2_sensor(k: int) -> np.ndarray:
    """Sensor position of frame k: moves +4 cm per frame along x, 0.6 m above ground."""
    x = -3.0 + 0.04 * k
    y = 0.0
    z = float(surface_c2(np.array([x]), np.array([y]))[0]) + C2_SENSOR_HEIGHT
    return np.array([x, y, z])


def _ray_march(origin, dirs, surface, t_max=12.0, dt=0.02, iters=30):
    """First crossing of each ray with the height field z = surface(x, y).

    Coarse march with step dt, then bisection on the bracketing interval.
    Rays that never cross return NaN.
    """
    n = dirs.shape[0]
    t_prev = np.zeros(n)
    hit_hi = np.full(n, np.nan)
    alive = np.ones(n, dtype=bool)
    t = 0.0
    while t < t_max and alive.any():
        t += dt
        p = origin[None, :] + t * dirs
        below = p[:, 2] <= surface(p[:, 0], p[:, 1])
        newly = alive & below
        hit_hi[newly] = t
        t_prev[alive & ~below] = t
        alive &= ~below
    ok = ~np.isnan(hit_hi)
    lo = t_prev.copy()
    hi = np.where(ok, hit_hi, 0.0)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        p = origin[None, :] + mid[:, None] * dirs
        below = p[:, 2] <= surface(p[:, 0], p[:, 1])
        hi = np.where(below, mid, hi)
        lo = np.where(below, lo, mid)
    out = np.where(ok, hi, np.nan)
    return out


def config2_frame(k: int, n_ground: int = C2_GROUND, n_other: int = C2_OTHER,
                  with_other: bool = False):
    """Frame k of the staircase sequence (seed = k).

    Returns ``(ground_world (n_ground, 3), sensor (3,), other_world)`` where the
    ground returns come from an inverted Mid360-like pattern: azimuth
    U[0, 2pi), elevation U[-52 deg, -7 deg], ray-marched to the height field,
    with N(0, 0.03^2) range noise along the ray.  Non-ground returns
    (elevation U[-7, 7] deg hitting a cylinder wall 8 m away) are only built
    when ``with_other`` is set; they are discarded before the update.
    """
    rng = np.random.default_rng(k)
    s = config2_sensor(k)
    pts = []
    need = n_ground
    while need > 0:
        m = int(need * 1.2) + 16
        az = rng.uniform(0.0, 2.0 * math.pi, m)
        el = np.deg2rad(rng.uniform(-52.0, -7.0, m))
        d = np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], axis=1)
        t = _ray_march(s, d, surface_c2)
        ok = ~np.isnan(t)
        t = t[ok] + rng.normal(0.0, C2_RANGE_SIGMA, ok.sum())
        p = s[None, :] + t[:, None] * d[ok]
        pts.append(p[:need])
        need -= min(need, p.shape[0])
    ground = np.concatenate(pts, axis=0)
    other = None
    if with_other:
        az = rng.uniform(0.0, 2.0 * math.pi, n_other)
        el = np.deg2rad(rng.uniform(-7.0, 7.0, n_other))
        rr = 8.0 / np.cos(el)
        d = np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], axis=1)
        other = s[None, :] + rr[:, None] * d
    return ground, s, other


# ----------------------------------------------------------------------------
# Config 3: soft-constraint workload
# ----------------------------------------------------------------------------
def rotation_zyx(yaw: float, pitch: float, roll: float) -> np.ndarray:
    cy, sy = math.cos(yaw), math.sin(yaw)
    cp, sp = math.cos(pitch), math.sin(pitch)
    cr, sr = math.cos(roll), math.sin(roll)
    Rz = np.array([[cy, -sy, 0], [sy, cy, 0], [0, 0, 1]])
    Ry = np.array([[cp, 0, sp], [0, 1, 0], [-sp, 0, cp]])
    Rx = np.array([[1, 0, 0], [0, cr, -sr], [0, sr, cr]])
    return Rz @ Ry @ Rx


def random_pose(rng: np.random.Generator):
    """Yaw U[0, 2pi), roll/pitch U[-5, 5] deg, translation U[-0.5, 0.5] m."""
    yaw = rng.uniform(0.0, 2.0 * math.pi)
    pitch = math.radians(rng.uniform(-5.0, 5.0))
    roll = math.radians(rng.uniform(-5.0, 5.0))
    R = rotation_zyx(yaw, pitch, roll)
    t = rng.uniform(-0.5, 0.5, 3)
    return R, t


# Weights of the config-3 terrain: a quasi-interpolant of the config-1 surface
# on the config-2 grid, w_j = f(c_j) * h^2 / V, where V = pi rho^2 / 7 is the
# integral over the plane of the Wendland C2 function with support rho
# (2 pi rho^2 * int_0^1 (1-s)^4 (4s+1) s ds = 2 pi rho^2 / 14).  This only
# shapes the synthetic terrain; it is not part of the method.
def config3(seed: int = 0, n: int = 65_536, outlier_frac: float = 0.05):
    rng = np.random.default_rng(seed)
    centers = config2_centers()
    rho = 0.6
    V = math.pi * rho * rho / 7.0
    w = surface_c1(centers[:, 0], centers[:, 1]) * (C2_H * C2_H) / V
    R, t = random_pose(rng)
    xy = rng.uniform(-5.5, 5.5, size=(n, 2))
    z = surface_c1(xy[:, 0], xy[:, 1]) + rng.normal(0.0, 0.03, n)
    nout = int(round(outlier_frac * n))
    idx = rng.choice(n, nout, replace=False)
    z[idx] += rng.choice([-0.3, 0.3], nout)
    world = np.concatenate([xy, z[:, None]], axis=1)
    body = (world - t[None, :]) @ R  # R^T (p - t), row-vector form
    return dict(centers=centers, w=w, R=R, t=t, body=body, world=world,
                kernel=KernelSpec(kind=0, rho=rho), delta=0.05, wheel_offset=0.0)


# ----------------------------------------------------------------------------
# Config 4: batched patches
# ----------------------------------------------------------------------------
def config4_patch(pid: int, m_lo=64, m_hi=4096, n_lo=500, n_hi=50_000):
    """Patch pid (seed = pid): M log-uniform, n log-uniform, a sinusoid+step surface."""
    rng = np.random.default_rng(pid)
    M = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
    n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
    gx = int(math.ceil(math.sqrt(M)))
    gy = int(math.ceil(M / gx))
    h = 0.2
    centers = grid_centers(gx, gy, 0.0, 0.0, h)[:M]
    # points cover the rows actually holding centers
    full_rows = M // gx
    ymax = (full_rows if full_rows > 0 else 1) * h
    amp = rng.uniform(0.02, 0.2)
    fx, fy = rng.uniform(0.5, 3.0, 2)
    step_x = rng.uniform(0.2, 0.8) * gx * h
    step_h = rng.uniform(-0.2, 0.2)
    xy = np.stack([rng.uniform(0.0, gx * h, n), rng.uniform(0.0, ymax, n)], axis=1)
    z = amp * np.sin(fx * xy[:, 0]) * np.cos(fy * xy[:, 1]) + step_h * (xy[:, 0] >= step_x)
    z = z + rng.normal(0.0, 0.02, n)
    pts = np.concatenate([xy, z[:, None]], axis=1)
    return dict(centers=centers, points=pts, M=M, n=n, kernel=KernelSpec(kind=0, rho=0.6))


# ----------------------------------------------------------------------------
# Config 5: precision and scale
# ----------------------------------------------------------------------------
def config5(seed: int = 0, n: int = 32_768, q: int = 1_048_576, rho: float = 0.3):
    """256x256 centers at 0.1 m on [0, 25.6]^2; an active block of 128 x 64
    centers (columns 64..191, rows 96..159) touched by n points drawn inside
    the block inset by rho - h, so that no center outside the block lies within
    rho of a point; the 4 corners of the inset rectangle are always included so
    that the block's corner centers are touched.  Then q uniform queries."""
    rng = np.random.default_rng(seed)
    h = 0.1
    centers = grid_centers(256, 256, 0.0, 0.0, h)
    i0, i1, j0, j1 = 64, 191, 96, 159
    xa, xb = (i0 + 0.5) * h, (i1 + 0.5) * h
    ya, yb = (j0 + 0.5) * h, (j1 + 0.5) * h
    inset = rho - h
    lo_x, hi_x = xa + inset + 1e-4, xb - inset - 1e-4
    lo_y, hi_y = ya + inset + 1e-4, yb - inset - 1e-4
    xy = np.stack([rng.uniform(lo_x, hi_x, n), rng.uniform(lo_y, hi_y, n)], axis=1)
    xy[0] = (lo_x, lo_y)
    xy[1] = (hi_x, lo_y)
    xy[2] = (lo_x, hi_y)
    xy[3] = (hi_x, hi_y)
    z = 0.1 * np.sin(0.7 * xy[:, 0]) * np.cos(0.9 * xy[:, 1]) + rng.normal(0.0, 0.02, n)
    pts = np.concatenate([xy, z[:, None]], axis=1)
    qs = uniform_queries(rng, q, 0.0, 25.6)
    block = (i0, i1, j0, j1)
    return dict(centers=centers, points=pts, queries=qs, block=block,
                kernel=KernelSpec(kind=0, rho=rho), noise=0.02)


# ----------------------------------------------------------------------------
# Raster evaluation of the paper's Gaussian terrain
# ----------------------------------------------------------------------------
def raster_gaussian(n_lat: int = 366, h: float = 0.07, sigma: float = 0.04, dq: float = 0.005,
                    n_q: int = 5120):
    """The paper's Gaussian parameters (sigma = 0.04 m on a 0.07 m mesh,
    Sec. VI-B) on an n_lat x n_lat lattice (25.6 m square by default), with
    the weights of the quasi-interpolant of the staircase surface,
    w_ij = f(c_ij) h^2 / (2 pi sigma^2) (a smooth stand-in for fitted
    weights), and an n_q x n_q raster at dq over the same square (5 mm and
    26.2 M points by default)."""
    centers = grid_centers(n_lat, n_lat, 0.0, 0.0, h)
    w = surface_c2(centers[:, 0] - 6.0, centers[:, 1]) * (h * h / (2.0 * np.pi * sigma * sigma))
    return dict(centers=centers, w=w, sigma=sigma, cutoff_mult=4.0, qx0=0.0, qy0=0.0, dq=dq, nqx=n_q, nqy=n_q)
