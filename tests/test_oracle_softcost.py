"""Pins for the soft-constraint cost and its gradients (Sec. IV-C)."""
import numpy as np
import pytest
from scipy.linalg import expm

from oracle import rbf_oracle as O
from paper_2509_26222_gb300 import workloads as W


def _setup(seed=0, n=300, kind=O.WENDLAND):
    rng = np.random.default_rng(seed)
    c = W.grid_centers(8, 8, 0, 0, 0.25)
    w = rng.normal(0, 0.1, 64)
    R, t = W.random_pose(rng)
    world = np.c_[rng.uniform(0.3, 1.7, (n, 2)), rng.normal(0, 0.08, n)]
    body = (world - t) @ R
    kw = dict(rho=0.6, sigma=0.15, cutoff_mult=40.0)
    # keep points away from the Huber kink so that central differences apply
    fw = O.soft_cost(R, t, body, c, w, kind, delta=0.05, **kw)
    keep = np.abs(np.abs(fw["r"]) - 0.05) > 2e-3
    return R, t, body[keep], c, w, kw


@pytest.mark.parametrize("kind", [O.WENDLAND, O.GAUSSIAN])
@pytest.mark.parametrize("loss", ["huber", "l2"])
def test_pose_gradient_matches_finite_difference(kind, loss):
    R, t, body, c, w, kw = _setup(kind=kind)
    fw = O.soft_cost(R, t, body, c, w, kind, delta=0.05, loss=loss, lam_m=0.7, **kw)
    e = 1e-6
    fd = np.zeros(6)
    for k in range(6):
        d = np.zeros(6); d[k] = e
        cp = O.soft_cost(R @ expm(O.skew(d[:3])), t + d[3:], body, c, w, kind, delta=0.05,
                         loss=loss, lam_m=0.7, **kw)["cost"]
        cm = O.soft_cost(R @ expm(O.skew(-d[:3])), t - d[3:], body, c, w, kind, delta=0.05,
                         loss=loss, lam_m=0.7, **kw)["cost"]
        fd[k] = (cp - cm) / (2 * e)
    assert np.allclose(fw["grad6"], fd, rtol=1e-6, atol=1e-7 * np.abs(fd).max())


@pytest.mark.parametrize("kind", [O.WENDLAND, O.GAUSSIAN])
def test_weight_and_center_gradients_match_finite_difference(kind):
    R, t, body, c, w, kw = _setup(seed=1, n=200, kind=kind)
    bw = O.soft_cost_backward(R, t, body, c, w, kind, delta=0.05, gout=1.3, **kw)
    cost = lambda cc, ww: 1.3 * O.soft_cost(R, t, body, cc, ww, kind, delta=0.05, **kw)["cost"]
    e = 1e-6
    for j in (0, 9, 27, 45, 63):
        d = np.zeros(64); d[j] = e
        assert (cost(c, w + d) - cost(c, w - d)) / (2 * e) == pytest.approx(bw["dw"][j], rel=1e-6, abs=1e-9)
        for k in range(2):
            cp = c.copy(); cm = c.copy(); cp[j, k] += e; cm[j, k] -= e
            assert (cost(cp, w) - cost(cm, w)) / (2 * e) == pytest.approx(bw["dc"][j, k], rel=1e-6, abs=1e-9)


def test_huber_pieces():
    d = 0.05
    r = np.array([-0.2, -d, -0.01, 0.0, 0.03, d, 0.4])
    v = O.huber(r, d)
    assert np.allclose(v[[2, 3, 4]], 0.5 * r[[2, 3, 4]] ** 2)
    assert np.allclose(v[[0, 6]], d * (np.abs(r[[0, 6]]) - d / 2))
    # continuity and derivative at the kink
    e = 1e-7
    for x in (d, -d):
        assert abs(O.huber(np.array([x + e]), d)[0] - O.huber(np.array([x - e]), d)[0]) <= 2 * e * d * 1.001
    xs = np.linspace(-0.3, 0.3, 61)
    fd = (O.huber(xs + e, d) - O.huber(xs - e, d)) / (2 * e)
    assert np.allclose(fd, O.huber_psi(xs, d), atol=1e-6)


def test_flat_terrain_closed_form():
    # w = 0: r_i = (R p_i + t)_z - off; d cost/d t = (0, 0, sum psi);
    # d cost/d theta = sum psi_i (-R [p_i]_x)[2, :]
    rng = np.random.default_rng(4)
    c = W.grid_centers(4, 4, 0, 0, 0.25); w = np.zeros(16)
    R, t = W.random_pose(rng)
    body = rng.normal(0, 0.3, (50, 3))
    fw = O.soft_cost(R, t, body, c, w, O.WENDLAND, delta=0.05, wheel_offset=0.1)
    q = body @ R.T + t
    r = q[:, 2] - 0.1
    assert np.allclose(fw["r"], r)
    psi = np.clip(r, -0.05, 0.05)
    assert np.allclose(fw["grad6"][3:], [0, 0, psi.sum()])
    gth = sum(psi[i] * (-(R @ O.skew(body[i])))[2] for i in range(50))
    assert np.allclose(fw["grad6"][:3], gth)


def _on_surface(seed=1, n=400, kind=O.WENDLAND):
    """Points lying exactly on the surface f under a known pose (zero residuals)."""
    rng = np.random.default_rng(seed)
    c = W.grid_centers(8, 8, 0, 0, 0.25)
    w = rng.normal(0, 0.1, 64)
    kw = dict(rho=0.6, sigma=0.15, cutoff_mult=40.0)
    R, t = W.random_pose(rng)
    xy = rng.uniform(0.4, 1.6, (n, 2))
    z = O.eval_h(xy, c, w, kind, rho=kw["rho"], sigma=kw["sigma"], cutoff_mult=kw["cutoff_mult"])[0]
    world = np.c_[xy, z]
    body = (world - t) @ R
    return R, t, body, c, w, kw


@pytest.mark.parametrize("kind", [O.WENDLAND, O.GAUSSIAN])
@pytest.mark.parametrize("loss", ["huber", "l2"])
def test_gauss_newton_matrix_is_the_hessian_at_zero_residual(kind, loss):
    """With every residual zero, the Hessian of the cost is sum psi'(0) J^T J,
    which is the Gauss-Newton matrix A; checked against central differences
    of the (finite-difference-pinned) pose gradient."""
    R, t, body, c, w, kw = _on_surface(kind=kind)
    nm = O.soft_cost_normal(R, t, body, c, w, kind, delta=0.05, loss=loss, lam_m=0.7, **kw)
    assert nm["cost"] < 1e-20
    e = 1e-6
    Hfd = np.zeros((6, 6))
    for k in range(6):
        d = np.zeros(6); d[k] = e
        gp = O.soft_cost(R @ expm(O.skew(d[:3])), t + d[3:], body, c, w, kind, delta=0.05, loss=loss,
                         lam_m=0.7, **kw)["grad6"]
        gm = O.soft_cost(R @ expm(O.skew(-d[:3])), t - d[3:], body, c, w, kind, delta=0.05, loss=loss,
                         lam_m=0.7, **kw)["grad6"]
        Hfd[:, k] = (gp - gm) / (2 * e)
    Hfd = 0.5 * (Hfd + Hfd.T)
    assert np.allclose(nm["A"], Hfd, rtol=1e-5, atol=1e-6 * np.abs(Hfd).max())


@pytest.mark.parametrize("loss", ["huber", "l2"])
def test_lm_steps_recover_the_pose(loss):
    R, t, body, c, w, kw = _on_surface(seed=2)
    Rp = R @ O.so3_exp([0.02, -0.015, 0.03])
    tp = t + np.array([0.04, -0.03, 0.02])
    for _ in range(12):
        Rp, tp, cost = O.lm_step(Rp, tp, body, c, w, O.WENDLAND, mu=1e-4, delta=0.05, loss=loss, **kw)
    assert np.max(np.abs(Rp - R)) < 1e-7 and np.max(np.abs(tp - t)) < 1e-7
