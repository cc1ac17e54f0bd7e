"""Pins for evaluation of f, grad f (Sec. III-A, IV-C) and for the float32
neighbour rule (reading G14) and center selection (Sec. III-A)."""
import struct

import numpy as np
import pytest

from oracle import rbf_oracle as O


def f32(v):
    return struct.unpack("f", struct.pack("f", float(v)))[0]


def member_py(q, c, radius):
    """Independent float32 emulation: each exact FP64 result rounded once to
    float32 (exact for sums/products of float32 values of similar scale)."""
    qx, qy = f32(q[0]), f32(q[1])
    cx, cy = f32(c[0]), f32(c[1])
    dx = f32(qx - cx); dy = f32(qy - cy)
    d2 = f32(f32(dx * dx) + f32(dy * dy))
    r = f32(radius)
    return d2 < f32(r * r)


def test_neighbors_match_python_float32_emulation():
    rng = np.random.default_rng(5)
    c = rng.uniform(0, 2, (40, 2)); q = rng.uniform(0, 2, (60, 2))
    rp, col = O.neighbors(q, c, 0.37)
    for i in range(q.shape[0]):
        want = [j for j in range(c.shape[0]) if member_py(q[i], c[j], 0.37)]
        got = list(col[rp[i]:rp[i + 1]])
        assert got == want


def test_neighbor_boundary_is_excluded():
    c = np.array([[0.0, 0.0], [1.0, 0.0]])
    q = np.array([[0.5, 0.0], [0.25, 0.0], [0.75, 0.0]])
    rp, col = O.neighbors(q, c, 0.5)
    # distance exactly 0.5 from both centers: excluded (d2 < r2 is strict)
    assert rp[1] - rp[0] == 0
    assert list(col[rp[1]:rp[2]]) == [0]
    assert list(col[rp[2]:rp[3]]) == [1]


def test_single_center_closed_form():
    c = np.array([[0.2, -0.1]]); w = np.array([1.7])
    q = np.array([[0.2, -0.1], [0.2 + 0.6, -0.1], [0.2, 0.6]])
    h, gx, gy, *_ = O.eval_h(q, c, w, O.WENDLAND, rho=0.6)
    assert h[0] == pytest.approx(1.7) and gx[0] == 0 and gy[0] == 0
    assert h[1] == 0 and h[2] == 0


@pytest.mark.parametrize("kind", [O.WENDLAND, O.GAUSSIAN])
def test_eval_gradient_matches_finite_difference(kind):
    rng = np.random.default_rng(7)
    c = rng.uniform(0, 1, (30, 2)); w = rng.normal(size=30)
    q = rng.uniform(0.1, 0.9, (40, 2))
    kw = dict(rho=0.4, sigma=0.08, cutoff_mult=40.0)
    h, gx, gy, *_ = O.eval_h(q, c, w, kind, **kw)
    e = 1e-6
    for k, g in ((0, gx), (1, gy)):
        d = np.zeros(2); d[k] = e
        hp = O.eval_h(q + d, c, w, kind, **kw)[0]
        hm = O.eval_h(q - d, c, w, kind, **kw)[0]
        assert np.allclose((hp - hm) / (2 * e), g, rtol=1e-6, atol=1e-7)


def test_eval_is_linear_in_w_and_reflects():
    rng = np.random.default_rng(8)
    c = rng.uniform(-1, 1, (25, 2)); q = rng.uniform(-1, 1, (30, 2))
    w1 = rng.normal(size=25); w2 = rng.normal(size=25)
    a = O.eval_h(q, c, w1, O.WENDLAND, rho=0.7)
    b = O.eval_h(q, c, w2, O.WENDLAND, rho=0.7)
    s = O.eval_h(q, c, 2 * w1 - 3 * w2, O.WENDLAND, rho=0.7)
    for k in range(3):
        assert np.allclose(s[k], 2 * a[k] - 3 * b[k], atol=1e-12)
    # mirror x -> -x: h unchanged, dh/dx flips, dh/dy unchanged
    m = np.array([-1.0, 1.0])
    r = O.eval_h(q * m, c * m, w1, O.WENDLAND, rho=0.7)
    assert np.allclose(r[0], a[0]) and np.allclose(r[1], -a[1]) and np.allclose(r[2], a[2])


def test_gaussian_truncation_within_bound():
    rng = np.random.default_rng(9)
    c = rng.uniform(0, 1, (80, 2)); w = rng.normal(size=80); q = rng.uniform(0, 1, (50, 2))
    sig, cm = 0.05, 4.0
    ht = O.eval_h(q, c, w, O.GAUSSIAN, sigma=sig, cutoff_mult=cm, truncate=True)[0]
    hu = O.eval_h(q, c, w, O.GAUSSIAN, sigma=sig, cutoff_mult=cm, truncate=False)[0]
    bound = np.abs(w).sum() * np.exp(-cm * cm / 2) * (1 + 1e-6)
    assert np.all(np.abs(ht - hu) <= bound)
    assert np.any(ht != hu)


def test_select_centers_counts_brute_force():
    rng = np.random.default_rng(11)
    pts = rng.uniform(0, 1, (150, 2))
    cents, counts = O.select_centers(pts, 0.0, 0.0, 0.1, 10, 10, 0.12, 3)
    k = 0
    for j in range(10):
        for i in range(10):
            cx, cy = (i + 0.5) * 0.1, (j + 0.5) * 0.1
            n = sum(member_py(p, (cx, cy), 0.12) for p in pts)
            assert counts[k] == n
            k += 1
    keep = counts >= 3
    assert cents.shape[0] == keep.sum()
    assert np.all(np.diff(np.nonzero(keep)[0]) > 0)


def test_select_centers_handcrafted():
    # 3 points around candidate (0,0) -> center at (0.05, 0.05); one far point
    pts = np.array([[0.05, 0.05], [0.06, 0.05], [0.05, 0.04], [0.95, 0.95]])
    cents, counts = O.select_centers(pts, 0.0, 0.0, 0.1, 10, 10, 0.02, 3)
    assert counts[0] == 3 and counts[99] == 1 and counts.sum() == 4
    assert cents.shape == (1, 2) and np.allclose(cents[0], [0.05, 0.05])
    # threshold is inclusive (reading G13)
    cents2, _ = O.select_centers(pts, 0.0, 0.0, 0.1, 10, 10, 0.02, 1)
    assert cents2.shape[0] == 2
