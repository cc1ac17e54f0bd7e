"""GPU parity of the raster evaluation (rbf_eval_grid, tensor cores) against
the FP64 oracle's raster evaluation (per-axis truncation, reading G21).

Tolerance: the float32 evaluation bound of the other evaluation tests,
|h - h_ref| <= 1e-3 (sum_j |w_j phi_j| + 1e-12) per raster point, and the same
bound with the sums of |terms| for each gradient component.
"""
import math

import numpy as np
import pytest
import torch

from oracle import rbf_oracle as O
from paper_2509_26222_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EVAL_TOL = 1e-3
SIGMA, MESH, CUT = 0.04, 0.07, 4.0


@pytest.fixture(scope="module")
def N():
    from paper_2509_26222_gb300 import native
    native.load(build_if_missing=True)
    torch.cuda.set_device(0)
    return native


def dev(x, dt=torch.float32):
    return torch.tensor(np.asarray(x), dtype=dt, device="cuda")


def check(h, g, ref):
    ho, gxo, gyo, ah, ax, ay = ref
    h = h.cpu().double().numpy()
    assert h.shape == ho.shape
    assert np.all(np.abs(h - ho) <= EVAL_TOL * (ah + 1e-12)), np.max(np.abs(h - ho) / (ah + 1e-12))
    if g is not None:
        g = g.cpu().double().numpy()
        assert np.all(np.abs(g[..., 0] - gxo) <= EVAL_TOL * (ax + 1e-12))
        assert np.all(np.abs(g[..., 1] - gyo) <= EVAL_TOL * (ay + 1e-12))


def lattice_terrain(N, nx, ny, drop=0.1, seed=0):
    """Gaussian terrain on an nx x ny lattice at the paper's mesh with a share
    of the lattice nodes left without a center."""
    rng = np.random.default_rng(seed)
    c = W.grid_centers(nx, ny, 0.0, 0.0, MESH)
    keep = rng.uniform(size=len(c)) >= drop
    keep[0] = keep[-1] = True  # the lattice extent stays the same
    c = c[keep]
    w = rng.normal(0.0, 0.1, len(c))
    T = N.Terrain(kernel=N.KERNEL_GAUSSIAN, sigma=SIGMA, cutoff_mult=CUT)
    T.set_centers(dev(c, torch.float64))
    T.set_weights(dev(w, torch.float64))
    return T, c, w


@pytest.mark.parametrize("nqx,nqy", [(300, 211), (301, 129), (128, 128), (1, 1), (7, 300)])
def test_eval_grid_parity_ragged(N, nqx, nqy):
    # tiles of 128 x 128 with ragged last tiles, a raster that overhangs the
    # lattice on every side, missing lattice nodes; nqx % 4 == 0 takes the
    # vector stores, the others the scalar ones
    T, c, w = lattice_terrain(N, 40, 30)
    qx0, qy0, dq = -0.13, -0.11, 0.0123
    h, g = T.eval_grid(qx0, qy0, dq, nqx, nqy)
    ref = O.eval_grid(qx0, qy0, dq, nqx, nqy, c, w, sigma=SIGMA, cutoff_mult=CUT)
    check(h, g, ref)
    h2, _ = T.eval_grid(qx0, qy0, dq, nqx, nqy, with_grad=False)
    check(h2, None, ref)


@pytest.mark.parametrize("nqx", [140, 141])
def test_eval_grid_coarsest_raster(N, nqx):
    # the largest spacing the 64-node windows accept; nqx = 140 takes the bulk
    # tensor stores, 141 the transposing stores
    T, c, w = lattice_terrain(N, 50, 50, seed=1)
    dq = (60.5 * MESH - 2.0 * CUT * SIGMA) / 127.0 * 0.999
    ref = O.eval_grid(0.02, 0.03, dq, nqx, 133, c, w, sigma=SIGMA, cutoff_mult=CUT)
    h, g = T.eval_grid(0.02, 0.03, dq, nqx, 133)
    check(h, g, ref)
    h2, _ = T.eval_grid(0.02, 0.03, dq, nqx, 133, with_grad=False)
    check(h2, None, ref)


def test_eval_grid_matches_scattered_eval_up_to_corners(N):
    # rbf_eval keeps the disc, rbf_eval_grid the square: they differ by the
    # corner terms only, each below |w| exp(-cutoff^2 / 2)
    T, c, w = lattice_terrain(N, 30, 30, seed=2)
    qx0, qy0, dq, nqx, nqy = 0.1, 0.2, 0.0071, 256, 200
    h, _ = T.eval_grid(qx0, qy0, dq, nqx, nqy, with_grad=False)
    xs = O.raster_coords(qx0, dq, nqx).astype(np.float32)
    ys = O.raster_coords(qy0, dq, nqy).astype(np.float32)
    q = np.stack(np.meshgrid(xs, ys), -1).reshape(-1, 2)
    hs, _ = T.eval(dev(q))
    n_sq = (2 * CUT * SIGMA / MESH + 1) ** 2
    bound = n_sq * np.max(np.abs(w)) * math.exp(-CUT * CUT / 2.0) + 1e-5
    assert np.max(np.abs(h.cpu().numpy().ravel() - hs.cpu().numpy())) <= bound


def test_eval_grid_empty_outside_and_errors(N):
    T, c, w = lattice_terrain(N, 10, 10, seed=3)
    h, g = T.eval_grid(0.0, 0.0, 0.01, 0, 5)
    assert h.numel() == 0
    h, g = T.eval_grid(0.0, 0.0, 0.01, 5, 0)
    assert h.numel() == 0
    h, g = T.eval_grid(40.0, -30.0, 0.01, 130, 3)  # far from every center
    assert torch.all(h == 0) and torch.all(g == 0)
    with pytest.raises(N.RBFError):
        T.eval_grid(0.0, 0.0, 0.0, 4, 4)  # spacing must be > 0
    with pytest.raises(N.RBFError):
        T.eval_grid(0.0, 0.0, -0.01, 4, 4)
    with pytest.raises(N.RBFError):
        T.eval_grid(0.0, 0.0, 0.04, 4, 4)  # 127 dq + 2 r > 60.5 h: windows of 64 nodes do not cover a tile
    with pytest.raises(N.RBFError):
        T.eval_grid(float("nan"), 0.0, 0.01, 4, 4)
    Tw = N.Terrain(rho=0.6)  # Wendland: not separable
    Tw.set_centers(dev(W.grid_centers(8, 8, 0.0, 0.0, 0.2), torch.float64))
    with pytest.raises(N.RBFError):
        Tw.eval_grid(0.0, 0.0, 0.01, 4, 4)
    Tg = N.Terrain(kernel=N.KERNEL_GAUSSIAN, sigma=SIGMA)  # centers off any lattice
    rng = np.random.default_rng(4)
    Tg.set_centers(dev(rng.uniform(0, 1, (50, 2)), torch.float64))
    with pytest.raises(N.RBFError):
        Tg.eval_grid(0.0, 0.0, 0.01, 4, 4)


def test_eval_grid_full_size_sampled_rows(N):
    """The raster the benchmark times (366 x 366 lattice, 5120 x 5120 points at
    5 mm), in the same launch; 12 raster rows checked point by point."""
    cfg = W.raster_gaussian()
    T = N.Terrain(kernel=N.KERNEL_GAUSSIAN, sigma=cfg["sigma"], cutoff_mult=cfg["cutoff_mult"])
    T.set_centers(dev(cfg["centers"], torch.float64))
    T.set_weights(dev(cfg["w"], torch.float64))
    h, g = T.eval_grid(cfg["qx0"], cfg["qy0"], cfg["dq"], cfg["nqx"], cfg["nqy"])
    assert torch.isfinite(h).all() and torch.isfinite(g).all()
    rng = np.random.default_rng(12)
    rows = np.sort(rng.choice(cfg["nqy"], 12, replace=False))
    for l in rows:
        y0 = cfg["qy0"] + l * cfg["dq"]  # the raster row's coordinate, formed as the kernel forms it
        ref = O.eval_grid(cfg["qx0"], y0, cfg["dq"], cfg["nqx"], 1, cfg["centers"], cfg["w"],
                          sigma=cfg["sigma"], cutoff_mult=cfg["cutoff_mult"], chunk=1024)
        check(h[l:l + 1], g[l:l + 1], ref)


def test_eval_grid_many_tiles_sampled_rows(N):
    # more tiles than CTAs, so that each persistent CTA runs through
    # consecutive tiles of a raster column (Ex, Ex' kept between them) and
    # across column boundaries; ragged last tiles, bulk stores (nqx % 4 == 0)
    T, c, w = lattice_terrain(N, 100, 80, seed=6)
    qx0, qy0, dq, nqx, nqy = -0.1, -0.1, 0.0041, 1752, 1400
    h, g = T.eval_grid(qx0, qy0, dq, nqx, nqy)
    rng = np.random.default_rng(7)
    rows = np.unique(np.concatenate([[0, nqy - 1], rng.choice(nqy, 28, replace=False)]))
    for l in rows:
        ref = O.eval_grid(qx0, qy0 + l * dq, dq, nqx, 1, c, w, sigma=SIGMA, cutoff_mult=CUT, chunk=1024)
        check(h[l:l + 1], g[l:l + 1], ref)
