"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: neighbour lists, active sets and center counts bit-exact; FP64
update steps 1e-5 norm-wise relative; float32 evaluation
|h - h_ref| <= 1e-3 * (sum_j |w_j phi_j| + 1e-12) per query (the same bound,
with the sums of |terms|, for each gradient component).
"""
import math

import numpy as np
import pytest
import torch

from oracle import rbf_oracle as O
from paper_2509_26222_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EVAL_TOL = 1e-3
F64_TOL = 1e-5


@pytest.fixture(scope="module")
def N():
    from paper_2509_26222_gb300 import native
    native.load(build_if_missing=True)
    torch.cuda.set_device(0)
    return native


def dev(x, dt=torch.float32):
    return torch.tensor(np.asarray(x), dtype=dt, device="cuda")


def rel_inf(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def check_eval(h, g, ref):
    ho, gxo, gyo, ah, ax, ay = ref
    h = h.cpu().double().numpy()
    g = g.cpu().double().numpy()
    assert np.all(np.abs(h - ho) <= EVAL_TOL * (ah + 1e-12)), np.max(np.abs(h - ho) / (ah + 1e-12))
    assert np.all(np.abs(g[:, 0] - gxo) <= EVAL_TOL * (ax + 1e-12))
    assert np.all(np.abs(g[:, 1] - gyo) <= EVAL_TOL * (ay + 1e-12))


# ---------------------------------------------------------------------------
# evaluation (Sec. III-A, IV-C)
# ---------------------------------------------------------------------------
def test_eval_config1(N):
    c1 = W.config1()
    w = O.batch_ridge(c1.points.astype(np.float32).astype(np.float64), c1.centers, 1e-3, O.WENDLAND, rho=0.6)
    T = N.Terrain(rho=0.6)
    T.set_centers(dev(c1.centers, torch.float64))
    T.set_weights(dev(w, torch.float64))
    q = c1.queries.astype(np.float32)
    for Q in (10_000, 10_001 - 256, 1, 0):
        h, g = T.eval(dev(q[:Q]).reshape(Q, 2))
        if Q:
            check_eval(h, g, O.eval_h(q[:Q].astype(np.float64), c1.centers, w, O.WENDLAND, rho=0.6))


def test_eval_outside_and_nonfinite_queries(N):
    c1 = W.config1()
    T = N.Terrain(rho=0.6)
    T.set_centers(dev(c1.centers, torch.float64))
    T.set_weights(dev(np.ones(256), torch.float64))
    q = np.array([[100.0, 100.0], [-50.0, 2.0], [4.3, 2.0], [np.nan, 1.0], [1.0, np.inf]], np.float32)
    h, g = T.eval(dev(q))
    h = h.cpu().numpy()
    assert h[0] == 0 and h[1] == 0
    ref = O.eval_h(q[2:3].astype(np.float64), c1.centers, np.ones(256), O.WENDLAND, rho=0.6)
    assert abs(h[2] - ref[0][0]) <= EVAL_TOL * ref[3][0]
    assert np.isnan(h[3]) and np.isnan(h[4])


def test_eval_gaussian_paper_parameters(N):
    # sigma = 0.04, mesh 0.07 (Sec. VI-B), truncation at 4 sigma (reading G9)
    rng = np.random.default_rng(3)
    c = W.grid_centers(20, 20, 0.0, 0.0, 0.07)
    w = rng.normal(0, 0.1, 400)
    T = N.Terrain(kernel=N.KERNEL_GAUSSIAN, sigma=0.04, cutoff_mult=4.0)
    T.set_centers(dev(c, torch.float64))
    T.set_weights(dev(w, torch.float64))
    q = rng.uniform(-0.1, 1.5, (5000, 2)).astype(np.float32)
    h, g = T.eval(dev(q))
    check_eval(h, g, O.eval_h(q.astype(np.float64), c, w, O.GAUSSIAN, sigma=0.04, cutoff_mult=4.0))


def test_eval_config5_full_size_sampled(N):
    """M = 65,536 centers, 1,048,576 queries in the launch the benchmark times;
    4,000 sampled outputs checked one by one against the oracle."""
    cfg = W.config5()
    rng = np.random.default_rng(11)
    w = rng.normal(0, 0.1, cfg["centers"].shape[0])
    T = N.Terrain(rho=0.3)
    T.set_centers(dev(cfg["centers"], torch.float64))
    T.set_weights(dev(w, torch.float64))
    q = cfg["queries"].astype(np.float32)
    h, g = T.eval(dev(q))
    idx = np.sort(rng.choice(q.shape[0], 4000, replace=False))
    ref = O.eval_h(q[idx].astype(np.float64), cfg["centers"], w, O.WENDLAND, rho=0.3, chunk=32)
    check_eval(h[idx], g[idx], ref)


# ---------------------------------------------------------------------------
# neighbour lists and center selection: bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("frame", [0, 120])
def test_neighbor_lists_bit_exact_config2(N, frame):
    c = W.config2_centers()
    pts, _, _ = W.config2_frame(frame)
    p32 = pts.astype(np.float32)
    T = N.Terrain(rho=0.6)
    T.set_centers(dev(c, torch.float64))
    rp, col = T.neighbors(dev(p32))
    rpo, colo = O.neighbors(p32, c, 0.6)
    assert np.array_equal(rp.cpu().numpy(), rpo)
    assert np.array_equal(col.cpu().numpy(), colo)


def test_neighbor_lists_gaussian_assembly_radius(N):
    rng = np.random.default_rng(5)
    c = W.grid_centers(30, 30, 0.0, 0.0, 0.07)
    p = np.c_[rng.uniform(-0.2, 2.3, (3000, 2)), rng.normal(0, 0.05, 3000)].astype(np.float32)
    T = N.Terrain(kernel=N.KERNEL_GAUSSIAN, sigma=0.04, cutoff_mult=4.0)
    T.set_centers(dev(c, torch.float64))
    rp, col = T.neighbors(dev(p), noise=0.1)
    rpo, colo = O.neighbors(p, c, O.support_radius_assembly(O.GAUSSIAN, sigma=0.04, cutoff_mult=4.0, noise=0.1))
    assert np.array_equal(rp.cpu().numpy(), rpo) and np.array_equal(col.cpu().numpy(), colo)


def test_neighbor_boundary_exact_distance(N):
    # centers on a 0.5 lattice, points exactly rho = 0.5 away along an axis
    c = W.grid_centers(4, 4, 0.0, 0.0, 0.5)
    p = np.array([[0.25 + 0.5, 0.25, 0.0], [0.25, 0.25 + 0.25, 0.0], [1.0, 1.0, 0.0]], np.float32)
    T = N.Terrain(rho=0.5)
    T.set_centers(dev(c, torch.float64))
    rp, col = T.neighbors(dev(p))
    rpo, colo = O.neighbors(p, c, 0.5)
    assert np.array_equal(rp.cpu().numpy(), rpo) and np.array_equal(col.cpu().numpy(), colo)


@pytest.mark.parametrize("min_count", [0, 3, 10_000])
def test_build_centers_bit_exact(N, min_count):
    rng = np.random.default_rng(2)
    xy = np.r_[rng.uniform(0, 4, (3000, 2)), rng.uniform(4.2, 5, (50, 2))]
    p = np.c_[xy, rng.normal(0, 0.05, xy.shape[0])].astype(np.float32)
    mesh = (0.0, 0.0, 0.07, 58, 58)
    T = N.Terrain(rho=0.3, mesh=mesh, r_kd=0.1, min_count=min_count)
    M, counts = T.build_centers(dev(p), return_counts=True)
    cents, co = O.select_centers(p[:, :2], 0.0, 0.0, 0.07, 58, 58, 0.1, min_count)
    assert np.array_equal(counts.cpu().numpy(), co)
    assert M == cents.shape[0]
    if M:
        assert np.array_equal(T.centers().cpu().numpy(), cents)


# ---------------------------------------------------------------------------
# recursive update (Sec. III-C)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [0, 1])
def test_update_config1_single_frame(N, prec):
    c1 = W.config1()
    p32 = c1.points.astype(np.float32)
    T = N.Terrain(rho=0.6, update_precision=prec)
    T.set_centers(dev(c1.centers, torch.float64))
    T.update(dev(p32), noise=0.02)
    st = O.BlockState(c1.centers, 1e-3, O.WENDLAND, rho=0.6)
    A = O.block_update(st, p32.astype(np.float64))
    assert np.array_equal(T.active().cpu().numpy(), A)
    assert rel_inf(T.weights().cpu().numpy(), st.w) < F64_TOL
    ids = A[::7]
    assert rel_inf(T.cov(ids).cpu().numpy(), st.P.block(ids)) < F64_TOL
    # equals batch ridge (closed form of one update from the prior)
    ref = O.batch_ridge(p32.astype(np.float64), c1.centers, 1e-3, O.WENDLAND, rho=0.6)
    assert rel_inf(T.weights().cpu().numpy(), ref) < F64_TOL


@pytest.mark.parametrize("prec", [0, 1])
def test_update_neighbour_lists_outgrow_capacity(N, prec):
    """After its first update the library fills the neighbour lists up to a
    capacity (twice the largest total seen) without reading the total first;
    an update whose lists do not fit starts over with a larger capacity.  A
    50-point batch followed by the full config-1 batch takes that path; both
    updates must still equal the oracle's recursion."""
    c1 = W.config1()
    p32 = c1.points.astype(np.float32)
    T = N.Terrain(rho=0.6, update_precision=prec)
    T.set_centers(dev(c1.centers, torch.float64))
    st = O.BlockState(c1.centers, 1e-3, O.WENDLAND, rho=0.6)
    for batch in (p32[:50], p32[50:]):
        T.update(dev(batch), noise=0.02)
        A = O.block_update(st, batch.astype(np.float64))
        assert np.array_equal(T.active().cpu().numpy(), A)
        assert rel_inf(T.weights().cpu().numpy(), st.w) < F64_TOL


@pytest.mark.parametrize("prec,inv", [(0, 0), (1, 0), (1, -1)])
def test_update_config2_sequence_with_departures(N, prec, inv):
    """Frames 0, 1, 2, 40, 41 of the staircase sequence: the later frames
    drop centers from the active block and bring new ones in.  The mixed
    update runs with the explicit factor inverse (inv = 0, default) and with
    blocked substitution only (inv = -1)."""
    c = W.config2_centers()
    T = N.Terrain(rho=0.6, update_precision=prec, inverse_max=inv)
    T.set_centers(dev(c, torch.float64))
    st = O.BlockState(c, 1e-3, O.WENDLAND, rho=0.6)
    rng = np.random.default_rng(0)
    for k in (0, 1, 2, 40, 41):
        pts, _, _ = W.config2_frame(k)
        p32 = pts.astype(np.float32)
        T.update(dev(p32), noise=0.03)
        A = O.block_update(st, p32.astype(np.float64))
        assert np.array_equal(T.active().cpu().numpy(), A)
        assert rel_inf(T.weights().cpu().numpy(), st.w) < F64_TOL
        ids = np.unique(np.r_[rng.choice(A, 40, replace=False), rng.choice(4096, 40, replace=False)])
        assert rel_inf(T.cov(ids).cpu().numpy(), st.P.block(ids)) < F64_TOL


@pytest.mark.parametrize("prec", [0, 1])
def test_update_config5_full_size(N, prec):
    """256x256 centers at 0.1 m, rho = 0.3 m: one update by 32,768 points that
    touch exactly the 128x64 block (a = 8192).  The oracle is the sparse ridge
    over the block plus a 3-center margin (one update from the prior equals
    ridge, G11); the GPU's active set must equal the oracle's."""
    cfg = W.config5(q=16)
    c = cfg["centers"]
    p32 = cfg["points"].astype(np.float32)
    i0, i1, j0, j1 = cfg["block"]
    T = N.Terrain(rho=0.3, update_precision=prec)
    T.set_centers(dev(c, torch.float64))
    T.update(dev(p32), noise=0.02)
    A = T.active().cpu().numpy()
    gi, gj = np.meshgrid(np.arange(i0 - 3, i1 + 4), np.arange(j0 - 3, j1 + 4))
    cand = np.sort((gj * 256 + gi).ravel())
    p64 = p32.astype(np.float64)
    A_ref = cand[O.active_set(p64[:, :2], c[cand], 0.3)]
    assert A.size == 8192 and np.array_equal(A, A_ref)
    rng = np.random.default_rng(5)
    ids = np.sort(rng.choice(A, 48, replace=False))
    w_ref, P_ref = O.ridge_sparse(p64, c[cand], 1e-3, O.WENDLAND, rho=0.3, cov_ids=np.searchsorted(cand, ids))
    w = T.weights().cpu().numpy()
    assert rel_inf(w[cand], w_ref) < F64_TOL
    outside = np.ones(c.shape[0], bool)
    outside[cand] = False
    assert np.all(w[outside] == 0.0)
    assert rel_inf(T.cov(ids).cpu().numpy(), P_ref) < F64_TOL


@pytest.mark.parametrize("prec", [0, 1])
def test_exact_mode_equals_exact_recursion_config1(N, prec):
    """Exact mode (every center updated every time, Eq. kf_w_update /
    H_inverse_update on the full matrices): ten batches of the config-1
    points against the oracle's full-covariance recursion, and the end
    result against batch ridge over all points."""
    c1 = W.config1()
    p32 = c1.points.astype(np.float32)
    T = N.Terrain(rho=0.6, update_precision=prec, exact=True)
    T.set_centers(dev(c1.centers, torch.float64))
    st = O.ExactState(c1.centers, 1e-3, O.WENDLAND, rho=0.6)
    ids = np.arange(0, 256, 5)
    for b in range(10):
        chunk = p32[b * 200:(b + 1) * 200]
        T.update(dev(chunk), noise=0.02)
        O.exact_update(st, chunk.astype(np.float64))
        assert T.active().numel() == 256
        assert rel_inf(T.weights().cpu().numpy(), st.w) < F64_TOL
    assert rel_inf(T.cov(ids).cpu().numpy(), st.P[np.ix_(ids, ids)]) < F64_TOL
    ref = O.batch_ridge(p32.astype(np.float64), c1.centers, 1e-3, O.WENDLAND, rho=0.6)
    assert rel_inf(T.weights().cpu().numpy(), ref) < F64_TOL


@pytest.mark.parametrize("prec", [0, 1])
def test_exact_mode_config2_frames_equal_batch_ridge(N, prec):
    """Exact mode over three staircase frames on the 64x64 grid (M = 4096):
    weights and a covariance block equal the ridge estimate over all the
    points of the three frames (sparse-design oracle)."""
    c = W.config2_centers()
    T = N.Terrain(rho=0.6, update_precision=prec, exact=True)
    T.set_centers(dev(c, torch.float64))
    allp = []
    for k in (0, 30, 60):
        pts, _, _ = W.config2_frame(k)
        p32 = pts.astype(np.float32)
        T.update(dev(p32), noise=0.03)
        allp.append(p32)
    p64 = np.concatenate(allp).astype(np.float64)
    rng = np.random.default_rng(3)
    ids = np.sort(rng.choice(4096, 40, replace=False))
    w_ref, P_ref = O.ridge_sparse(p64, c, 1e-3, O.WENDLAND, rho=0.6, cov_ids=ids)
    assert rel_inf(T.weights().cpu().numpy(), w_ref) < F64_TOL
    assert rel_inf(T.cov(ids).cpu().numpy(), P_ref) < F64_TOL


def test_update_gaussian_moment_rows(N):
    rng = np.random.default_rng(9)
    c = W.grid_centers(12, 12, 0.0, 0.0, 0.07)
    T = N.Terrain(kernel=N.KERNEL_GAUSSIAN, sigma=0.04, cutoff_mult=4.0, lam=1e-3)
    T.set_centers(dev(c, torch.float64))
    st = O.BlockState(c, 1e-3, O.GAUSSIAN, sigma=0.04, cutoff_mult=4.0)
    for k in range(3):
        xy = rng.uniform(0.1 * k, 0.5 + 0.1 * k, (400, 2))
        p32 = np.c_[xy, 0.05 * np.sin(9 * xy[:, 0])].astype(np.float32)
        T.update(dev(p32), noise=0.1)
        O.block_update(st, p32.astype(np.float64), noise=0.1)
        assert rel_inf(T.weights().cpu().numpy(), st.w) < F64_TOL


@pytest.mark.parametrize("prec", [0, 1])
def test_update_tiny_degenerate_cases(N, prec):
    # one point (a handful of active centers), then a second frame that moves
    # the block (departures); and a model with a single center
    c1 = W.config1()
    T = N.Terrain(rho=0.6, update_precision=prec)
    T.set_centers(dev(c1.centers, torch.float64))
    st = O.BlockState(c1.centers, 1e-3, O.WENDLAND, rho=0.6)
    for pts in (np.array([[1.03, 2.07, 0.11]], np.float32), np.array([[3.1, 0.4, -0.05], [3.2, 0.5, 0.02]], np.float32)):
        T.update(dev(pts), noise=0.02)
        A = O.block_update(st, pts.astype(np.float64))
        assert np.array_equal(T.active().cpu().numpy(), A)
        assert rel_inf(T.weights().cpu().numpy(), st.w) < F64_TOL
    c = np.array([[0.5, 0.5]])
    T1 = N.Terrain(rho=0.6, update_precision=prec)
    T1.set_centers(dev(c, torch.float64))
    pts = np.array([[0.4, 0.6, 0.3], [0.7, 0.45, 0.2], [0.55, 0.5, 0.25]], np.float32)
    T1.update(dev(pts), noise=0.02)
    ref = O.batch_ridge(pts.astype(np.float64), c, 1e-3, O.WENDLAND, rho=0.6)
    assert rel_inf(T1.weights().cpu().numpy(), ref) < F64_TOL


def test_update_empty_and_untouched_are_noops(N):
    c1 = W.config1()
    T = N.Terrain(rho=0.6)
    T.set_centers(dev(c1.centers, torch.float64))
    T.update(torch.zeros(0, 3, device="cuda"))
    T.update(dev(np.array([[50.0, 50.0, 1.0]], np.float32)))
    assert torch.all(T.weights() == 0)
    assert T.active().numel() == 0


def test_update_rejects_nonfinite_point(N):
    c1 = W.config1()
    T = N.Terrain(rho=0.6)
    T.set_centers(dev(c1.centers, torch.float64))
    with pytest.raises(N.RBFError) as e:
        T.update(dev(np.array([[1.0, 1.0, np.nan]], np.float32)))
    assert e.value.status == -1
    assert torch.all(T.weights() == 0)


# ---------------------------------------------------------------------------
# soft constraint (Sec. IV-C)
# ---------------------------------------------------------------------------
def _c3_terrain(N, **kw):
    cfg = W.config3()
    T = N.Terrain(rho=0.6, huber_delta=cfg["delta"], **kw)
    T.set_centers(dev(cfg["centers"], torch.float64))
    T.set_weights(dev(cfg["w"], torch.float64))
    return cfg, T


def test_soft_cost_forward_config3(N):
    cfg, T = _c3_terrain(N)
    p32 = cfg["body"].astype(np.float32)
    cost, g6, r = T.soft_cost(cfg["R"], cfg["t"], dev(p32), with_resid=True)
    fw = O.soft_cost(cfg["R"], cfg["t"], p32.astype(np.float64), cfg["centers"], cfg["w"], O.WENDLAND,
                     rho=0.6, delta=cfg["delta"])
    assert abs(float(cost) - fw["cost"]) <= 1e-4 * abs(fw["cost"])
    assert rel_inf(g6.cpu().numpy(), fw["grad6"]) < 1e-3
    assert np.max(np.abs(r.cpu().numpy() - fw["r"])) < 1e-4
    # both Huber branches are exercised
    assert np.any(np.abs(fw["r"]) > 0.05) and np.any(np.abs(fw["r"]) < 0.05)


@pytest.mark.parametrize("loss", ["huber", "l2"])
def test_soft_cost_normal_matrix_config3(N, loss):
    """Cost, gradient and the Gauss-Newton matrix of the pose (LM step of
    Sec. IV-C) on the 65,536 config-3 points, against the oracle."""
    kw = dict(loss=N.LOSS_L2, lambda_m=0.5) if loss == "l2" else {}
    cfg, T = _c3_terrain(N, **kw)
    p32 = cfg["body"].astype(np.float32)
    cost, g6, A = T.soft_cost_normal(cfg["R"], cfg["t"], dev(p32))
    ref = O.soft_cost_normal(cfg["R"], cfg["t"], p32.astype(np.float64), cfg["centers"], cfg["w"], O.WENDLAND,
                             rho=0.6, delta=cfg["delta"], loss=loss, lam_m=0.5)
    assert abs(float(cost) - ref["cost"]) <= 1e-4 * abs(ref["cost"])
    assert rel_inf(g6.cpu().numpy(), ref["grad6"]) < 1e-3
    assert rel_inf(A.cpu().numpy(), ref["A"]) < 1e-3


def test_lm_steps_recover_pose_on_gpu(N):
    """Ten GPU LM steps from a perturbed pose recover the pose of points that
    lie on the terrain (no noise, no outliers)."""
    cfg, T = _c3_terrain(N)
    rng = np.random.default_rng(4)
    xy = rng.uniform(-5.0, 5.0, (20000, 2))
    z = O.eval_h(xy, cfg["centers"], cfg["w"], O.WENDLAND, rho=0.6)[0]
    R, t = cfg["R"], cfg["t"]
    body = dev(((np.c_[xy, z] - t) @ R).astype(np.float32))
    Rp = R @ O.so3_exp([0.01, -0.01, 0.02])
    tp = t + np.array([0.03, -0.02, 0.02])
    for _ in range(10):
        Rp, tp, cost = T.lm_step(Rp, tp, body, mu=1e-4)
    assert np.max(np.abs(Rp - R)) < 2e-4 and np.max(np.abs(tp - t)) < 2e-4


def test_soft_cost_backward_config3(N):
    cfg, T = _c3_terrain(N)
    p32 = cfg["body"].astype(np.float32)
    gout = torch.tensor([0.7], dtype=torch.float64, device="cuda")
    dw, dc, dpose = T.soft_cost_backward(cfg["R"], cfg["t"], dev(p32), gout=gout)
    bw = O.soft_cost_backward(cfg["R"], cfg["t"], p32.astype(np.float64), cfg["centers"], cfg["w"],
                              O.WENDLAND, rho=0.6, delta=cfg["delta"], gout=0.7)
    assert rel_inf(dw.cpu().numpy(), bw["dw"]) < 1e-3
    assert rel_inf(dc.cpu().numpy(), bw["dc"]) < 1e-3
    assert rel_inf(dpose.cpu().numpy(), bw["dpose6"]) < 1e-3


def test_soft_cost_l2_loss_and_autograd(N):
    cfg, T = _c3_terrain(N, loss=N.LOSS_L2, lambda_m=0.5)
    p32 = cfg["body"][:5000].astype(np.float32)
    w = dev(cfg["w"], torch.float64).requires_grad_(True)
    c = dev(cfg["centers"], torch.float64).requires_grad_(True)
    pose = torch.zeros(6, dtype=torch.float64, device="cuda", requires_grad=True)
    cost = N.SoftCost.apply(T, cfg["R"], cfg["t"], dev(p32), w, c, pose)
    cost.backward()
    bw = O.soft_cost_backward(cfg["R"], cfg["t"], p32.astype(np.float64), cfg["centers"], cfg["w"],
                              O.WENDLAND, rho=0.6, loss="l2", lam_m=0.5)
    assert abs(cost.item() - bw["cost"]) <= 1e-4 * abs(bw["cost"])
    assert rel_inf(w.grad.cpu().numpy(), bw["dw"]) < 1e-3
    assert rel_inf(c.grad.cpu().numpy(), bw["dc"]) < 1e-3
    assert rel_inf(pose.grad.cpu().numpy(), bw["dpose6"]) < 1e-3


def test_status_codes(N):
    T = N.Terrain(rho=0.6)
    with pytest.raises(N.RBFError) as e:
        T.eval(torch.zeros(4, 2, device="cuda"))
    assert e.value.status == -6
    c1 = W.config1()
    T.set_centers(dev(c1.centers, torch.float64))
    T.update(dev(c1.points.astype(np.float32)))
    import ctypes
    a = ctypes.c_int64()
    buf = torch.empty(3, dtype=torch.int32, device="cuda")
    st = T.lib.rbf_get_active(T._h, ctypes.c_void_p(buf.data_ptr()), 3, ctypes.byref(a), None)
    assert st == -7 and a.value == 256


# ---------------------------------------------------------------------------
# batched patches (independent terrains, update from the prior + evaluation)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [0, 1])
def test_batch_patches_match_oracle_and_replay(N, prec):
    ids = [3, 17, 42, 77, 101, 150]
    specs = [W.config4_patch(pid, m_hi=900, n_hi=6000) for pid in ids]
    T = N.Terrain(rho=0.6, update_precision=prec)
    # descriptors with caller-owned buffers, so repeated calls see the same shape
    import ctypes
    arr = (N.RbfPatch * len(specs))()
    bufs = []
    for k, sp in enumerate(specs):
        M = sp["M"]
        gx = int(math.ceil(math.sqrt(M)))
        pts = dev(sp["points"].astype(np.float32))
        q = dev(sp["points"][:, :2].astype(np.float32)[::3].copy())
        w = torch.empty(M, dtype=torch.float64, device="cuda")
        h = torch.empty(q.shape[0], dtype=torch.float32, device="cuda")
        g = torch.empty(q.shape[0], 2, dtype=torch.float32, device="cuda")
        bufs.append((pts, q, w, h, g))
        d = arr[k]
        d.x0, d.y0, d.spacing, d.nx, d.M = 0.0, 0.0, 0.2, gx, M
        d.n, d.Q = pts.shape[0], q.shape[0]
        d.pts, d.q, d.w, d.h, d.grad = pts.data_ptr(), q.data_ptr(), w.data_ptr(), h.data_ptr(), g.data_ptr()
    results = []
    for call in range(3):  # eager, captured, replayed
        T.batch_update_eval_into(arr, len(specs))
        torch.cuda.synchronize()
        results.append([(b[2].cpu().numpy().copy(), b[3].cpu().numpy().copy()) for b in bufs])
    for call in (1, 2):
        for (w0, h0), (w1, h1) in zip(results[0], results[call]):
            assert np.array_equal(w0, w1) and np.array_equal(h0, h1)
    for sp, (pts, q, w, h, g) in zip(specs, bufs):
        p64 = sp["points"].astype(np.float32).astype(np.float64)
        ref = O.batch_ridge(p64, sp["centers"], 1e-3, O.WENDLAND, rho=0.6)
        assert rel_inf(w.cpu().numpy(), ref) < F64_TOL
        qq = q.cpu().numpy().astype(np.float64)
        check_eval(h, g, O.eval_h(qq, sp["centers"], ref, O.WENDLAND, rho=0.6))
