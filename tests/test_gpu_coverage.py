"""GPU parity of the paths the first parity suite left out: the hash-grid
evaluation of scattered centers, the lattice kernels at every window width and
wide supports, per-entry soft-cost gradients, map-scale translations, the LM
step on the device, the hand-worked overlapping-frames case, and the failure
statuses driven through the test hooks.

Tolerances as in test_gpu_parity: FP64 steps 1e-5 norm-wise relative; float32
evaluation |x - x_ref| <= 1e-3 (sum |terms| + 1e-12) per output.
"""
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
    assert np.all(np.abs(g[:, 0] - gxo) <= EVAL_TOL * (ax + 1e-12)), np.max(np.abs(g[:, 0] - gxo) / (ax + 1e-12))
    assert np.all(np.abs(g[:, 1] - gyo) <= EVAL_TOL * (ay + 1e-12)), np.max(np.abs(g[:, 1] - gyo) / (ay + 1e-12))


# ---------------------------------------------------------------------------
# evaluation kernels (Eq. RBF_fml, Eq. manidolf_grad_detail)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["wendland", "gaussian"])
def test_eval_scattered_centers_hash_grid(N, kind):
    """Centers off any lattice (jittered grid plus a random cloud) go through
    the hash-grid gather; queries cover the interior, the border and beyond."""
    rng = np.random.default_rng(21)
    if kind == "wendland":
        c = W.grid_centers(40, 30, 0.0, 0.0, 0.2) + rng.uniform(-0.07, 0.07, (1200, 2))
        c = np.r_[c, rng.uniform(0.0, 8.0, (300, 2))]
        kw = dict(rho=0.6)
        T = N.Terrain(rho=0.6)
        ok = O.WENDLAND
    else:
        c = W.grid_centers(40, 30, 0.0, 0.0, 0.07) + rng.uniform(-0.02, 0.02, (1200, 2))
        kw = dict(sigma=0.04, cutoff_mult=4.0)
        T = N.Terrain(kernel=N.KERNEL_GAUSSIAN, sigma=0.04, cutoff_mult=4.0)
        ok = O.GAUSSIAN
    w = rng.normal(0, 0.1, c.shape[0])
    T.set_centers(dev(c, torch.float64))
    T.set_weights(dev(w, torch.float64))
    lo, hi = c.min(0) - 0.3, c.max(0) + 0.3
    q = rng.uniform(lo, hi, (6001, 2)).astype(np.float32)
    h, g = T.eval(dev(q))
    check_eval(h, g, O.eval_h(q.astype(np.float64), c, w, ok, **kw))


@pytest.mark.parametrize("nx,ny", [(30, 30), (256, 256)])
def test_eval_lattice_wide_support(N, nx, ny):
    """Wendland support wider than four lattice spacings (rho / h = 6) takes the
    per-query lattice kernel instead of the fixed window: a lattice whose
    weights fit in shared memory (30 x 30) and one that does not (256 x 256)."""
    rng = np.random.default_rng(nx)
    c = W.grid_centers(nx, ny, 0.0, 0.0, 0.1)
    w = rng.normal(0, 0.1, c.shape[0])
    T = N.Terrain(rho=0.6)
    T.set_centers(dev(c, torch.float64))
    T.set_weights(dev(w, torch.float64))
    q = rng.uniform(-0.5, nx * 0.1 + 0.5, (20000, 2)).astype(np.float32)
    h, g = T.eval(dev(q))
    idx = np.sort(rng.choice(q.shape[0], 3000, replace=False))
    check_eval(h[idx], g[idx], O.eval_h(q[idx].astype(np.float64), c, w, O.WENDLAND, rho=0.6, chunk=128))


@pytest.mark.parametrize("rho", [0.2, 0.4, 0.8])
def test_eval_lattice_window_widths(N, rho):
    """The fixed-window lattice kernel at window half-widths of 1, 2 and 4
    lattice spacings (rho / h = 1, 2, 4 on a 0.2 m lattice)."""
    rng = np.random.default_rng(int(rho * 10))
    c = W.grid_centers(48, 40, -1.0, 2.0, 0.2)
    w = rng.normal(0, 0.1, c.shape[0])
    T = N.Terrain(rho=rho)
    T.set_centers(dev(c, torch.float64))
    T.set_weights(dev(w, torch.float64))
    q = rng.uniform([-1.5, 1.5], [9.1, 10.5], (8193, 2)).astype(np.float32)
    h, g = T.eval(dev(q))
    check_eval(h, g, O.eval_h(q.astype(np.float64), c, w, O.WENDLAND, rho=rho))


def test_eval_gaussian_lattice_beyond_shared_memory(N):
    """Gaussian lattice whose weights do not fit in shared memory (250 x 200
    nodes at the paper's 0.07 m mesh, sigma = 0.04)."""
    rng = np.random.default_rng(8)
    c = W.grid_centers(250, 200, 0.0, 0.0, 0.07)
    w = rng.normal(0, 0.1, c.shape[0])
    T = N.Terrain(kernel=N.KERNEL_GAUSSIAN, sigma=0.04, cutoff_mult=4.0)
    T.set_centers(dev(c, torch.float64))
    T.set_weights(dev(w, torch.float64))
    q = rng.uniform(-0.2, 17.7, (40000, 2)).astype(np.float32)
    h, g = T.eval(dev(q))
    idx = np.sort(rng.choice(q.shape[0], 3000, replace=False))
    check_eval(h[idx], g[idx], O.eval_h(q[idx].astype(np.float64), c, w, O.GAUSSIAN, sigma=0.04,
                                        cutoff_mult=4.0, chunk=128))


# ---------------------------------------------------------------------------
# soft constraint (Sec. IV-C)
# ---------------------------------------------------------------------------
def _c3_terrain(N, offset=(0.0, 0.0), **kw):
    cfg = W.config3()
    c = cfg["centers"] + np.asarray(offset)[None, :]
    T = N.Terrain(rho=0.6, huber_delta=cfg["delta"], **kw)
    T.set_centers(dev(c, torch.float64))
    T.set_weights(dev(cfg["w"], torch.float64))
    return cfg, c, T


def test_soft_cost_backward_per_entry_config3(N):
    """dC/dw_j and dC/dc_j entry by entry on the 65,536 config-3 points, each
    against its own scale: 1e-3 of the sum of |terms| plus 1e-5 of the sum of
    the terms without psi (psi comes from a float32 residual, accurate to
    about 1e-6 m, so 1e-5 m covers its rounding)."""
    cfg, c, T = _c3_terrain(N)
    p32 = cfg["body"].astype(np.float32)
    dw, dc, dpose = T.soft_cost_backward(cfg["R"], cfg["t"], dev(p32))
    bw = O.soft_cost_backward(cfg["R"], cfg["t"], p32.astype(np.float64), c, cfg["w"], O.WENDLAND,
                              rho=0.6, delta=cfg["delta"])
    dw = dw.cpu().double().numpy()
    dc = dc.cpu().double().numpy()
    tol_w = EVAL_TOL * bw["dw_abs"] + 1e-5 * bw["phi_abs"]
    tol_c = EVAL_TOL * bw["dc_abs"] + 1e-5 * bw["gq_abs"]
    assert np.all(np.abs(dw - bw["dw"]) <= tol_w), np.max(np.abs(dw - bw["dw"]) / (tol_w + 1e-300))
    assert np.all(np.abs(dc - bw["dc"]) <= tol_c), np.max(np.abs(dc - bw["dc"]) / (tol_c + 1e-300))
    # the small entries are checked at their own scale, not only against the largest
    small = np.abs(bw["dw"]) < 1e-3 * np.max(np.abs(bw["dw"]))
    assert small.sum() > 100
    g = dpose.cpu().numpy()
    assert np.all(np.abs(g - bw["dpose6"]) <= 1e-3 * np.max(np.abs(bw["dpose6"])))


def test_soft_cost_map_scale_translation(N):
    """The same terrain and body points 480 m east, 350 m south and 200 m up
    (wheel offset 200 m): the pose is applied in float64, so cost, gradient and
    residuals keep their tolerances."""
    off = np.array([480.0, -350.0])
    cfg, c, T = _c3_terrain(N, offset=off, wheel_offset=200.0)
    t = cfg["t"] + np.array([off[0], off[1], 200.0])
    p32 = cfg["body"].astype(np.float32)
    cost, g6, r = T.soft_cost(cfg["R"], t, dev(p32), with_resid=True)
    fw = O.soft_cost(cfg["R"], t, p32.astype(np.float64), c, cfg["w"], O.WENDLAND, rho=0.6,
                     delta=cfg["delta"], wheel_offset=200.0)
    assert abs(float(cost) - fw["cost"]) <= 1e-4 * abs(fw["cost"])
    assert rel_inf(g6.cpu().numpy(), fw["grad6"]) < 1e-3
    assert np.max(np.abs(r.cpu().numpy() - fw["r"])) < 1e-4


def test_lm_step_on_device_matches_oracle(N):
    """One LM step (rbf_lm_step: 6 x 6 damped solve and R Exp(dtheta) on the
    device) against the oracle's step from the same perturbed pose."""
    cfg, c, T = _c3_terrain(N)
    p32 = cfg["body"][:20000].astype(np.float32)
    R0 = cfg["R"] @ O.so3_exp([0.01, -0.01, 0.02])
    t0 = cfg["t"] + np.array([0.03, -0.02, 0.02])
    R1, t1, cost = T.lm_step(R0, t0, dev(p32), mu=1e-3)
    Rr, tr, cr = O.lm_step(R0, t0, p32.astype(np.float64), c, cfg["w"], O.WENDLAND, mu=1e-3, rho=0.6,
                           delta=cfg["delta"])
    assert abs(cost - cr) <= 1e-4 * abs(cr)
    step = max(np.max(np.abs(Rr - R0)), np.max(np.abs(tr - t0)))
    assert step > 1e-3
    assert np.max(np.abs(R1 - Rr)) <= 2e-3 * step
    assert np.max(np.abs(t1 - tr)) <= 2e-3 * step
    assert np.allclose(R1 @ R1.T, np.eye(3), atol=1e-12)


def test_soft_cost_autograd_rejects_foreign_leaves(N):
    cfg, c, T = _c3_terrain(N)
    p = dev(cfg["body"][:100].astype(np.float32))
    w = dev(cfg["w"] * 1.01, torch.float64).requires_grad_(True)
    cc = dev(c, torch.float64).requires_grad_(True)
    pose = torch.zeros(6, dtype=torch.float64, device="cuda", requires_grad=True)
    with pytest.raises(ValueError):
        N.SoftCost.apply(T, cfg["R"], cfg["t"], p, w, cc, pose)


# ---------------------------------------------------------------------------
# recursive update: hand-worked overlap, failure statuses (Sec. III-C)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [0, 1])
def test_update_overlapping_frames_hand_case(N, prec):
    """The three frames of golden/block_overlap_hand.txt (a center leaves and
    returns) through rbf_update: w and P against the hand-worked values."""
    from _fixtures import (OVERLAP_CENTERS, OVERLAP_FRAMES, OVERLAP_LAMBDA, OVERLAP_RHO,
                           overlap_expected)
    exp = overlap_expected()
    T = N.Terrain(rho=OVERLAP_RHO, lam=OVERLAP_LAMBDA, update_precision=prec)
    T.set_centers(dev(OVERLAP_CENTERS, torch.float64))
    for k, p in enumerate(OVERLAP_FRAMES, start=1):
        T.update(dev(p))
        if k in exp:
            w_ref, P_ref = exp[k]
            assert rel_inf(T.weights().cpu().numpy(), w_ref) < F64_TOL
            assert rel_inf(T.cov(np.arange(4)).cpu().numpy(), P_ref) < F64_TOL


def _state(T, ids):
    return (T.weights().cpu().numpy().copy(), T.active().cpu().numpy().copy(), T.cov(ids).cpu().numpy().copy())


@pytest.mark.parametrize("prec", [0, 1])
def test_update_not_spd_keeps_state(N, prec):
    """A diagonal shift set through the test hook makes the block indefinite:
    rbf_update returns RBF_ENOTSPD, the state is unchanged, and after the hook
    is cleared the same frame updates as the oracle does."""
    c1 = W.config1()
    p32 = c1.points.astype(np.float32)
    T = N.Terrain(rho=0.6, update_precision=prec)
    T.set_centers(dev(c1.centers, torch.float64))
    T.update(dev(p32[:1000]), noise=0.02)
    ids = np.arange(0, 256, 9)
    before = _state(T, ids)
    T.test_hook(N.HOOK_DIAG_SHIFT, -1e9)
    with pytest.raises(N.RBFError) as e:
        T.update(dev(p32[1000:]), noise=0.02)
    assert e.value.status == -4
    T.test_hook(N.HOOK_DIAG_SHIFT, 0.0)
    after = _state(T, ids)
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    assert np.allclose(before[2], after[2], rtol=1e-12, atol=0)
    T.update(dev(p32[1000:]), noise=0.02)
    st = O.BlockState(c1.centers, 1e-3, O.WENDLAND, rho=0.6)
    O.block_update(st, p32[:1000].astype(np.float64))
    O.block_update(st, p32[1000:].astype(np.float64))
    assert rel_inf(T.weights().cpu().numpy(), st.w) < F64_TOL


@pytest.mark.parametrize("prec,inv", [(0, 0), (1, -1)])
def test_update_wait_timeout_keeps_state(N, prec, inv):
    """The sync-free triangular solves wait on per-block flags with a bounded
    spin.  With the test hook they wait for a value no block writes, so every
    wait runs out (limit 2,000 spins): rbf_update returns RBF_ETIMEOUT and the
    state is unchanged; with the hook cleared the update proceeds."""
    c1 = W.config1()
    p32 = c1.points.astype(np.float32)
    T = N.Terrain(rho=0.6, update_precision=prec, inverse_max=inv)
    T.set_centers(dev(c1.centers, torch.float64))
    T.update(dev(p32[:1000]), noise=0.02)
    ids = np.arange(0, 256, 9)
    before = _state(T, ids)
    T.test_hook(N.HOOK_WAIT_LIMIT, 2000)
    T.test_hook(N.HOOK_WAIT_NEVER, 1)
    with pytest.raises(N.RBFError) as e:
        T.update(dev(p32[1000:]), noise=0.02)
    assert e.value.status == -5
    T.test_hook(N.HOOK_WAIT_NEVER, 0)
    T.test_hook(N.HOOK_WAIT_LIMIT, 0)
    after = _state(T, ids)
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    assert np.allclose(before[2], after[2], rtol=1e-12, atol=0)
    T.update(dev(p32[1000:]), noise=0.02)
    st = O.BlockState(c1.centers, 1e-3, O.WENDLAND, rho=0.6)
    O.block_update(st, p32[:1000].astype(np.float64))
    O.block_update(st, p32[1000:].astype(np.float64))
    assert rel_inf(T.weights().cpu().numpy(), st.w) < F64_TOL


def test_test_hook_validation(N):
    T = N.Terrain(rho=0.6)
    for hook, value in ((99, 0.0), (N.HOOK_WAIT_NEVER, 2.0), (N.HOOK_WAIT_LIMIT, -1.0),
                        (N.HOOK_DIAG_SHIFT, float("nan"))):
        with pytest.raises(N.RBFError) as e:
            T.test_hook(hook, value)
        assert e.value.status == -1


@pytest.mark.parametrize("prec", [0, 1])
def test_update_departures_at_65536_centers(N, prec):
    """256 x 256 centers at 0.1 m (M = 65,536, rho = 0.3 m): three overlapping
    frames -- the second shifted so that centers leave the active block, the
    third bringing most of them back -- against the oracle's block recursion
    (its covariance store); covariance blocks mix active, departed and
    never-touched centers.  The outside covariance is stored per departure,
    not as an M x M matrix (34 GB here)."""
    cfg = W.config5(q=16)
    c = cfg["centers"]
    rng = np.random.default_rng(41)

    def frame(x0, y0):
        xy = rng.uniform([x0, y0], [x0 + 2.0, y0 + 1.0], (3000, 2))
        z = 0.1 * np.sin(0.7 * xy[:, 0]) * np.cos(0.9 * xy[:, 1]) + rng.normal(0.0, 0.02, 3000)
        return np.c_[xy, z].astype(np.float32)

    frames = [frame(10.0, 12.0), frame(10.6, 12.3), frame(10.1, 12.05)]
    T = N.Terrain(rho=0.3, update_precision=prec)
    T.set_centers(dev(c, torch.float64))
    st = O.BlockState(c, 1e-3, O.WENDLAND, rho=0.3)
    for k, p32 in enumerate(frames):
        T.update(dev(p32), noise=0.02)
        A = O.block_update(st, p32.astype(np.float64))
        assert np.array_equal(T.active().cpu().numpy(), A)
        assert rel_inf(T.weights().cpu().numpy(), st.w) < F64_TOL
        left = np.setdiff1d(st.P.ids, A)
        ids = np.unique(np.r_[rng.choice(A, 40, replace=False),
                              rng.choice(left, min(30, left.size), replace=False) if left.size else [],
                              rng.choice(c.shape[0], 6, replace=False)]).astype(np.int32)
        assert rel_inf(T.cov(ids).cpu().numpy(), st.P.block(ids)) < F64_TOL
        if k > 0:
            assert left.size > 0
