"""Pins of the oracle's raster evaluation (separable Gaussian, reading G21).

Each pin is independent of the oracle's own formula:
* Poisson summation (Jacobi theta): on an unbounded lattice of unit weights the
  Gaussian sum has a closed form;
* central finite differences of h against the gradient;
* the oracle's scattered-query evaluation (itself pinned elsewhere) when the
  cutoff covers every center, on a raster with nqx != nqy;
* the per-axis window contains the circular one, so the difference is bounded
  by the corner terms.
"""
import math

import numpy as np
import pytest

from oracle import rbf_oracle as o


def theta_sum(x, h, sigma, m_max=6):
    # sum_i exp(-(x - (i + 1/2) h)^2 / (2 sigma^2)) over all integers i, by
    # Poisson summation: (sqrt(2 pi) sigma / h) sum_m exp(-2 pi^2 sigma^2 m^2 / h^2)
    # cos(2 pi m (x - h/2) / h)
    s = np.ones_like(x)
    for m in range(1, m_max + 1):
        s = s + 2.0 * math.exp(-2.0 * math.pi ** 2 * sigma ** 2 * m ** 2 / h ** 2) * np.cos(2.0 * math.pi * m * (x - 0.5 * h) / h)
    return math.sqrt(2.0 * math.pi) * sigma / h * s


def lattice(nx, ny, h, x0=0.0, y0=0.0):
    i, j = np.meshgrid(np.arange(nx), np.arange(ny))
    return np.stack([x0 + (i.ravel() + 0.5) * h, y0 + (j.ravel() + 0.5) * h], 1)


def test_poisson_summation_unit_lattice():
    # unit weights on a lattice far larger than the cutoff around the raster:
    # h(q) = S(q_x) S(q_y) with S the theta sum above (truncation at 12 sigma
    # leaves exp(-72) per term)
    sigma, h = 0.05, 0.07
    c = lattice(60, 60, h)
    w = np.ones(len(c))
    qx0, qy0, dq = 1.5, 1.7, 0.013
    nqx, nqy = 23, 17
    H, GX, GY, *_ = o.eval_grid(qx0, qy0, dq, nqx, nqy, c, w, sigma=sigma, cutoff_mult=12.0)
    xs = qx0 + np.arange(nqx) * dq
    ys = qy0 + np.arange(nqy) * dq
    ref = theta_sum(ys, h, sigma)[:, None] * theta_sum(xs, h, sigma)[None, :]
    assert np.max(np.abs(H - ref)) < 1e-10 * np.max(np.abs(ref))


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    sigma, h = 0.04, 0.07
    c = lattice(20, 18, h)
    w = rng.normal(0.0, 0.3, len(c))
    qx0, qy0, dq, nqx, nqy = 0.31, 0.27, 0.017, 9, 7
    e = 1e-6
    cm = 30.0  # no center near the window edge: membership cannot change under the shift
    H, GX, GY, *_ = o.eval_grid(qx0, qy0, dq, nqx, nqy, c, w, sigma=sigma, cutoff_mult=cm)
    hp = o.eval_grid(qx0 + e, qy0, dq, nqx, nqy, c, w, sigma=sigma, cutoff_mult=cm)[0]
    hm = o.eval_grid(qx0 - e, qy0, dq, nqx, nqy, c, w, sigma=sigma, cutoff_mult=cm)[0]
    assert np.max(np.abs((hp - hm) / (2 * e) - GX)) < 1e-6 * np.max(np.abs(GX))
    hp = o.eval_grid(qx0, qy0 + e, dq, nqx, nqy, c, w, sigma=sigma, cutoff_mult=cm)[0]
    hm = o.eval_grid(qx0, qy0 - e, dq, nqx, nqy, c, w, sigma=sigma, cutoff_mult=cm)[0]
    assert np.max(np.abs((hp - hm) / (2 * e) - GY)) < 1e-6 * np.max(np.abs(GY))


def test_equals_scattered_evaluation_without_truncation():
    rng = np.random.default_rng(5)
    sigma, h = 0.04, 0.07
    c = lattice(16, 11, h, x0=-0.3, y0=0.2)
    w = rng.normal(0.0, 0.5, len(c))
    qx0, qy0, dq, nqx, nqy = -0.35, 0.15, 0.029, 41, 30
    H, GX, GY, *_ = o.eval_grid(qx0, qy0, dq, nqx, nqy, c, w, sigma=sigma, cutoff_mult=40.0)
    xs = o.raster_coords(qx0, dq, nqx)
    ys = o.raster_coords(qy0, dq, nqy)
    q = np.stack(np.meshgrid(xs, ys), -1).reshape(-1, 2)  # row l = y index
    ref = o.eval_h(q, c, w, o.GAUSSIAN, sigma=sigma, truncate=False)
    for a, b in ((H, ref[0]), (GX, ref[1]), (GY, ref[2])):
        assert np.max(np.abs(a.ravel() - b)) < 1e-12 * (1.0 + np.max(np.abs(b)))


def test_square_window_bounds_the_circular_rule():
    rng = np.random.default_rng(7)
    sigma, h, cm = 0.04, 0.07, 4.0
    c = lattice(14, 14, h)
    w = rng.normal(0.0, 1.0, len(c))
    qx0, qy0, dq, nqx, nqy = 0.05, 0.08, 0.011, 60, 55
    H, GX, GY, AH, *_ = o.eval_grid(qx0, qy0, dq, nqx, nqy, c, w, sigma=sigma, cutoff_mult=cm)
    xs = o.raster_coords(qx0, dq, nqx)
    ys = o.raster_coords(qy0, dq, nqy)
    q = np.stack(np.meshgrid(xs, ys), -1).reshape(-1, 2)
    circ = o.eval_h(q, c, w, o.GAUSSIAN, sigma=sigma, cutoff_mult=cm, truncate=True)
    diff = np.abs(H.ravel() - circ[0])
    # corner terms: at most (2 r / h + 1)^2 centers per point, each below |w| exp(-cm^2 / 2)
    n_sq = (2 * cm * sigma / h + 1) ** 2
    bound = n_sq * np.max(np.abs(w)) * math.exp(-cm * cm / 2.0) * 1.001
    assert np.all(diff <= bound)
    assert np.any(diff > 0.0)  # the corners do contribute somewhere
    # and the square window keeps every circular term: |h_square| sums dominate
    assert np.all(AH.ravel() >= circ[3] - 1e-12)


def test_empty_and_degenerate_rasters():
    c = lattice(4, 4, 0.07)
    w = np.ones(len(c))
    for nqx, nqy in ((0, 5), (5, 0), (0, 0)):
        out = o.eval_grid(0.0, 0.0, 0.01, nqx, nqy, c, w)
        assert out[0].shape == (nqy, nqx)
    # a raster far from every center is zero
    H = o.eval_grid(50.0, 50.0, 0.01, 4, 3, c, w)[0]
    assert np.all(H == 0.0)
