"""Batched terrain patches at the sizes the benchmark times: the 256 patches
of config 4 (M log-uniform 64-4,096 centers, n log-uniform 500-50,000 points)
in one rbf_batch_update_eval call, in both update precisions.  Every patch
with M > 2,048 or n > 20,000, plus the first patch of every log2(M) bucket
(where the path autotuner makes its choice), is compared with the oracle:
weights against the sparse-design ridge (one update from the prior equals
ridge, Sec. III-B / III-C), h and grad h at 1,000 sampled queries against the
oracle's evaluation with the oracle's weights (Eq. RBF_fml).  Replays of the
captured graph must equal the eager run bit for bit."""
import math

import numpy as np
import pytest
import torch

from oracle import rbf_oracle as O
from paper_2509_26222_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NPATCH = 256
EVAL_TOL = 1e-3
F64_TOL = 1e-5


def _selected():
    sel, buckets = set(), {}
    for pid in range(NPATCH):
        sp = W.config4_patch(pid)
        if sp["M"] > 2048 or sp["n"] > 20000:
            sel.add(pid)
        buckets.setdefault(int(math.floor(math.log2(sp["M"]))), pid)
    return sorted(sel | set(buckets.values()))


@pytest.fixture(scope="module")
def reference():
    """Oracle results of the selected patches (CPU only)."""
    out = {}
    for pid in _selected():
        sp = W.config4_patch(pid)
        p64 = sp["points"].astype(np.float32).astype(np.float64)
        w = O.ridge_sparse(p64, sp["centers"], 1e-3, O.WENDLAND, rho=0.6)
        rng = np.random.default_rng(7000 + pid)
        idx = np.sort(rng.choice(p64.shape[0], min(1000, p64.shape[0]), replace=False))
        ev = O.eval_h(p64[idx, :2], sp["centers"], w, O.WENDLAND, rho=0.6)
        out[pid] = (w, idx, ev)
    return out


@pytest.fixture(scope="module")
def N():
    from paper_2509_26222_gb300 import native
    native.load(build_if_missing=True)
    torch.cuda.set_device(0)
    return native


def rel_inf(a, b):
    return float(np.max(np.abs(np.asarray(a) - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_full_size_config4(reference, N, prec):
    T = N.Terrain(rho=0.6, lam=1e-3, update_precision=prec)
    arr = (N.RbfPatch * NPATCH)()
    bufs = []
    for k in range(NPATCH):
        sp = W.config4_patch(k)
        M = sp["M"]
        pts = torch.tensor(sp["points"].astype(np.float32), device="cuda")
        q = pts[:, :2].contiguous()
        w = torch.empty(M, dtype=torch.float64, device="cuda")
        h = torch.empty(q.shape[0], dtype=torch.float32, device="cuda")
        g = torch.empty(q.shape[0], 2, dtype=torch.float32, device="cuda")
        bufs.append((pts, q, w, h, g))
        d = arr[k]
        d.x0, d.y0, d.spacing, d.nx, d.M = 0.0, 0.0, 0.2, int(math.ceil(math.sqrt(M))), M
        d.n, d.Q = pts.shape[0], q.shape[0]
        d.pts, d.q, d.w, d.h, d.grad = pts.data_ptr(), q.data_ptr(), w.data_ptr(), h.data_ptr(), g.data_ptr()
    runs = []
    for call in range(3):  # eager (sizes workspaces, tunes), captured, replayed
        T.batch_update_eval_into(arr, NPATCH)
        torch.cuda.synchronize()
        runs.append([(b[2].cpu().numpy().copy(), b[3].cpu().numpy().copy(), b[4].cpu().numpy().copy())
                     for b in bufs])
    for call in (1, 2):
        for a, b in zip(runs[1], runs[call]):
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    for pid, (w_ref, idx, ev) in reference.items():
        w, h, g = runs[2][pid]
        assert rel_inf(w, w_ref) < F64_TOL, (pid, rel_inf(w, w_ref))
        ho, gxo, gyo, ah, ax, ay = ev
        hh, gg = h[idx].astype(np.float64), g[idx].astype(np.float64)
        assert np.all(np.abs(hh - ho) <= EVAL_TOL * (ah + 1e-12)), pid
        assert np.all(np.abs(gg[:, 0] - gxo) <= EVAL_TOL * (ax + 1e-12)), pid
        assert np.all(np.abs(gg[:, 1] - gyo) <= EVAL_TOL * (ay + 1e-12)), pid
    T.close()
