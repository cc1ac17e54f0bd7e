"""The whole 200-frame staircase sequence (config 2: 64 x 64 centers at 0.2 m,
8,000 ground returns per frame) through rbf_update in both precisions,
compared with the oracle's stored state at frames 60 (on the stairs), 120
(near the top) and 199 (the end): the active set bit for bit, the weights
and a covariance block (active, departed and never-touched centers) at 1e-5
norm-wise relative.  The stored state comes from tests/golden/make_c2_sequence.py,
which runs only the oracle (block recursion of Sec. III-C, Eq. kf_w_update and
the block-diagonal form of Eq. H_inverse_update)."""
import hashlib

import numpy as np
import pytest
import torch

from paper_2509_26222_gb300 import workloads as W

pytestmark = pytest.mark.gpu

F64_TOL = 1e-5
NOISE = 0.03


def rel_inf(a, b):
    return float(np.max(np.abs(np.asarray(a) - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def golden():
    from _fixtures import c2_sequence
    return c2_sequence()


@pytest.fixture(scope="module")
def frames(golden):
    out = []
    for k in range(200):
        p32 = W.config2_frame(k)[0].astype(np.float32)
        assert hashlib.sha256(p32.tobytes()).hexdigest() == golden["hashes"][k], (
            f"frame {k}: the input generator gives other points than when the stored state was written")
        out.append(p32)
    return out


@pytest.fixture(scope="module")
def N():
    from paper_2509_26222_gb300 import native
    native.load(build_if_missing=True)
    torch.cuda.set_device(0)
    return native


@pytest.mark.parametrize("prec", [0, 1])
def test_c2_sequence_all_frames(golden, frames, N, prec):
    stored = set(int(k) for k in golden["frames"])
    T = N.Terrain(rho=0.6, lam=1e-3, update_precision=prec)
    T.set_centers(torch.tensor(W.config2_centers(), dtype=torch.float64, device="cuda"))
    for k, p32 in enumerate(frames):
        T.update(torch.tensor(p32, device="cuda"), noise=NOISE)
        if k not in stored:
            continue
        assert np.array_equal(T.active().cpu().numpy(), golden[f"A_{k}"]), k
        err_w = rel_inf(T.weights().cpu().numpy(), golden[f"w_{k}"])
        assert err_w < F64_TOL, (k, err_w)
        ids = golden[f"ids_{k}"]
        err_p = rel_inf(T.cov(ids).cpu().numpy(), golden[f"P_{k}"])
        assert err_p < F64_TOL, (k, err_p)
    T.close()
