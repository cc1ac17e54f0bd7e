"""Pins for batch ridge (Sec. III-B) and the recursive update (Sec. III-C)."""
import numpy as np
import pytest

from oracle import rbf_oracle as O
from paper_2509_26222_gb300 import workloads as W


def rel_inf(a, b):
    """||a - b||_inf / ||b||_inf, the norm-wise relative error used throughout."""
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def _pts(rng, n, lo=0.0, hi=1.0, f=None):
    xy = rng.uniform(lo, hi, (n, 2))
    z = (np.sin(3 * xy[:, 0]) * np.cos(2 * xy[:, 1]) if f is None else f(xy)) + rng.normal(0, 0.02, n)
    return np.c_[xy, z]


def test_batch_ridge_equals_lstsq_on_augmented_system():
    rng = np.random.default_rng(0)
    c = W.grid_centers(6, 6, 0, 0, 1 / 6)
    p = _pts(rng, 300)
    lam = 1e-3
    w = O.batch_ridge(p, c, lam, O.WENDLAND, rho=0.4)
    Phi = O.design_rows(p[:, :2], c, O.WENDLAND, rho=0.4)
    A = np.vstack([Phi, np.sqrt(lam) * np.eye(c.shape[0])])
    b = np.concatenate([p[:, 2], np.zeros(c.shape[0])])
    ref = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.allclose(w, ref, rtol=1e-9, atol=1e-11)


def test_self_consistency_recovers_generating_weights():
    rng = np.random.default_rng(1)
    c = W.grid_centers(16, 16, 0, 0, 0.25)
    xy = rng.uniform(0, 4, (4000, 2))
    ws = rng.normal(size=256)
    z = O.design_rows(xy, c, O.WENDLAND, rho=0.6) @ ws
    w = O.batch_ridge(np.c_[xy, z], c, 1e-12, O.WENDLAND, rho=0.6)
    assert np.max(np.abs(w - ws)) < 1e-8


def test_plane_is_approximated_in_the_interior():
    # the model has no polynomial term (Sec. III-A), so a plane is not exact
    rng = np.random.default_rng(0)
    c = W.grid_centers(16, 16, 0, 0, 0.25)
    xy = rng.uniform(0, 4, (4000, 2)); z = 0.3 * xy[:, 0] - 0.2 * xy[:, 1] + 0.1
    w = O.batch_ridge(np.c_[xy, z], c, 1e-6, O.WENDLAND, rho=0.6)
    q = rng.uniform(0.75, 3.25, (2000, 2))
    h = O.eval_h(q, c, w, O.WENDLAND, rho=0.6)[0]
    rms = np.sqrt(np.mean((h - (0.3 * q[:, 0] - 0.2 * q[:, 1] + 0.1)) ** 2))
    assert rms < 0.015


@pytest.mark.parametrize("form", ["info", "woodbury"])
def test_first_update_from_prior_equals_batch_ridge(form):
    rng = np.random.default_rng(2)
    c = W.grid_centers(8, 8, 0, 0, 0.125)
    p = _pts(rng, 400)
    st = O.BlockState(c, 1e-3, O.WENDLAND, rho=0.3)
    A = O.block_update(st, p, form=form)
    assert A.size == 64
    ref = O.batch_ridge(p, c, 1e-3, O.WENDLAND, rho=0.3)
    assert np.allclose(st.w, ref, rtol=1e-10, atol=1e-12)
    Phi = O.design_rows(p[:, :2], c, O.WENDLAND, rho=0.3)
    Pref = np.linalg.inv(Phi.T @ Phi + 1e-3 * np.eye(64))
    assert np.allclose(st.P.dense(), Pref, rtol=1e-9, atol=1e-9)


def test_forms_agree_info_woodbury_joseph():
    rng = np.random.default_rng(3)
    c = W.grid_centers(5, 5, 0, 0, 0.2)
    res = []
    for form, jos in (("info", False), ("woodbury", False), ("info", True)):
        st = O.BlockState(c, 1e-2, O.WENDLAND, rho=0.35)
        r2 = np.random.default_rng(30)
        for k in range(4):
            O.block_update(st, _pts(r2, 20, 0.2 * k, 0.2 * k + 0.5), form=form, joseph=jos)
        res.append((st.w.copy(), st.P.dense()))
    for w, P in res[1:]:
        assert np.allclose(w, res[0][0], rtol=1e-9, atol=1e-12)
        assert np.allclose(P, res[0][1], rtol=1e-8, atol=1e-10)


def test_all_active_batches_equal_exact_and_batch_ridge():
    rng = np.random.default_rng(4)
    c = W.grid_centers(6, 6, 0, 0, 1 / 6)
    batches = [_pts(rng, 200) for _ in range(5)]
    bs = O.BlockState(c, 1e-3, O.WENDLAND, rho=0.4)
    ex = O.ExactState(c, 1e-3, O.WENDLAND, rho=0.4)
    for b in batches:
        assert O.block_update(bs, b).size == 36
        O.exact_update(ex, b)
    ref = O.batch_ridge(np.vstack(batches), c, 1e-3, O.WENDLAND, rho=0.4)
    assert rel_inf(bs.w, ref) < 1e-9
    assert rel_inf(ex.w, ref) < 1e-9
    assert rel_inf(bs.P.dense(), ex.P) < 1e-9


def test_disjoint_active_sets_equal_exact():
    rng = np.random.default_rng(5)
    c = W.grid_centers(12, 4, 0, 0, 0.25)       # 3 m x 1 m strip
    bs = O.BlockState(c, 1e-3, O.WENDLAND, rho=0.3)
    ex = O.ExactState(c, 1e-3, O.WENDLAND, rho=0.3)
    seen = set()
    for k in range(3):
        p = _pts(rng, 150, 0.0, 1.0)
        p[:, 0] = 0.45 + 0.9 * (p[:, 0] / 1.0) * 0.2 + k * 1.0   # bands far apart
        A = O.block_update(bs, p)
        O.exact_update(ex, p)
        assert not (set(A.tolist()) & seen)
        seen |= set(A.tolist())
    assert np.allclose(bs.w, ex.w, rtol=1e-9, atol=1e-12)
    assert np.allclose(bs.P.dense(), ex.P, rtol=1e-8, atol=1e-10)


def test_overlapping_block_mode_keeps_P_spd_and_block_structure():
    rng = np.random.default_rng(6)
    c = W.grid_centers(10, 10, 0, 0, 0.1)
    st = O.BlockState(c, 1e-3, O.WENDLAND, rho=0.25)
    for k in range(6):
        p = _pts(rng, 80, 0.1 * k, 0.1 * k + 0.4)
        A = O.block_update(st, p)
        P = st.P.dense()
        assert np.allclose(P, P.T, atol=1e-12)
        assert np.linalg.eigvalsh(P).min() > 0
        notA = np.setdiff1d(np.arange(100), A)
        assert np.all(P[np.ix_(A, notA)] == 0)
    # the block mode differs from the exact recursion once active sets overlap
    ex = O.ExactState(c, 1e-3, O.WENDLAND, rho=0.25)
    rng = np.random.default_rng(6)
    for k in range(6):
        O.exact_update(ex, _pts(rng, 80, 0.1 * k, 0.1 * k + 0.4))
    assert not np.allclose(st.w, ex.w, rtol=1e-6)


def test_exact_update_equals_batch_ridge_gaussian():
    rng = np.random.default_rng(7)
    c = W.grid_centers(7, 7, 0, 0, 0.07)
    batches = [_pts(rng, 60, 0.0, 0.49) for _ in range(3)]
    ex = O.ExactState(c, 1e-3, O.GAUSSIAN, sigma=0.04, cutoff_mult=4.0)
    for b in batches:
        O.exact_update(ex, b, noise=0.1)
    ref = O.batch_ridge(np.vstack(batches), c, 1e-3, O.GAUSSIAN, sigma=0.04,
                        cutoff_mult=4.0, noise=0.1)
    assert np.allclose(ex.w, ref, rtol=1e-8, atol=1e-10)


def test_empty_and_untouched_updates_are_noops():
    c = W.grid_centers(4, 4, 0, 0, 0.25)
    st = O.BlockState(c, 1e-3, O.WENDLAND, rho=0.3)
    assert O.block_update(st, np.zeros((0, 3))).size == 0
    far = np.array([[10.0, 10.0, 1.0]])
    assert O.block_update(st, far).size == 0
    assert np.all(st.w == 0) and np.allclose(st.P.dense(), np.eye(16) * 1e3)


@pytest.mark.parametrize("kind", [O.WENDLAND, O.GAUSSIAN])
def test_sparse_ridge_equals_dense_ridge_and_inverse(kind):
    """The sparse-design ridge (used at 65,536 centers) against the dense
    normal equations and numpy's dense inverse; points cover only part of the
    grid, so untouched centers must keep w = 0 and P = I / lambda."""
    rng = np.random.default_rng(4)
    c = W.grid_centers(16, 16, 0, 0, 0.07 if kind == O.GAUSSIAN else 0.25)
    span = 0.6 if kind == O.GAUSSIAN else 2.5
    p = _pts(rng, 1500, 0.0, span)
    kw = dict(rho=0.6, sigma=0.04, cutoff_mult=4.0, noise=0.05)
    ids = np.array([0, 5, 17, 40, 200, 255])
    w, Pk = O.ridge_sparse(p, c, 1e-3, kind, cov_ids=ids, **kw)
    ref = O.batch_ridge(p, c, 1e-3, kind, **kw)
    assert rel_inf(w, ref) < 1e-9          # cond(H) is about 7e4 for the Gaussian rows
    Phi = O.design_rows(p[:, :2], c, kind, **kw)
    Pref = np.linalg.inv(Phi.T @ Phi + 1e-3 * np.eye(c.shape[0]))
    assert rel_inf(Pk, Pref[np.ix_(ids, ids)]) < 1e-9
    untouched = np.abs(Phi).sum(axis=0) == 0
    assert untouched.any() and np.all(w[untouched] == 0.0)
    assert Pk[-1, -1] == pytest.approx(1e3) and untouched[255]


@pytest.mark.parametrize("form,joseph", [("info", False), ("woodbury", False), ("info", True)])
def test_overlapping_frames_match_hand_derivation(form, joseph):
    """Three frames whose active sets overlap: a center leaves and later
    returns, reading back the variance stored when it left with its coupling
    zeroed (block-diagonal form of Eq. H_inverse_update).  Expected w and P
    after frames 2 and 3 are worked by hand in golden/block_overlap_hand.txt."""
    from _fixtures import (OVERLAP_CENTERS, OVERLAP_FRAMES, OVERLAP_LAMBDA, OVERLAP_RHO,
                           overlap_expected)
    exp = overlap_expected()
    st = O.BlockState(OVERLAP_CENTERS, OVERLAP_LAMBDA, O.WENDLAND, rho=OVERLAP_RHO)
    actives = [[0, 1], [1, 2], [0, 1]]
    for k, p in enumerate(OVERLAP_FRAMES, start=1):
        A = O.block_update(st, p, form=form, joseph=joseph)
        assert list(A) == actives[k - 1]
        if k in exp:
            w_ref, P_ref = exp[k]
            assert np.max(np.abs(st.w - w_ref)) < 1e-14
            assert np.max(np.abs(st.P.dense() - P_ref)) < 1e-14
