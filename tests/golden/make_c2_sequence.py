"""Write the oracle state of the 200-frame staircase sequence (config 2) at
frames 60, 120 and 199 to ``c2_sequence_oracle.npz``.

Test infrastructure: this script calls only the FP64 oracle (``oracle/``) and
the seeded input generator (``workloads``, which holds none of the method's
arithmetic).  The oracle runs the block recursion of Sec. III-C
(Eq. kf_w_update, Eq. H_inverse_update, block-diagonal form) over all 200
frames; at each stored frame it records
  * the weights w (all 4,096),
  * the active set A of that frame,
  * a covariance block P[ids, ids] over ids drawn from the active set, from
    centers that left an earlier block (their stored covariance) and from
    never-touched centers (the prior),
  * a SHA-256 of every frame's float32 points, so a test can tell a changed
    input generator from a changed result.
Run:  python tests/golden/make_c2_sequence.py   (about 10 minutes on 8 cores)
"""
from __future__ import annotations

import hashlib
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import rbf_oracle as O  # noqa: E402
from paper_2509_26222_gb300 import workloads as W  # noqa: E402

FRAMES = (60, 120, 199)
NOISE = 0.03
OUT = os.path.join(HERE, "c2_sequence_oracle.npz")


def frame_points(k):
    pts, _, _ = W.config2_frame(k)
    return pts.astype(np.float32)


def main():
    c = W.config2_centers()
    st = O.BlockState(c, 1e-3, O.WENDLAND, rho=0.6)
    out = {}
    hashes = []
    for k in range(200):
        p32 = frame_points(k)
        hashes.append(hashlib.sha256(p32.tobytes()).hexdigest())
        A = O.block_update(st, p32.astype(np.float64), noise=NOISE)
        if k in FRAMES:
            rng = np.random.default_rng(1000 + k)
            touched = st.P.ids
            left = np.setdiff1d(touched, A)
            never = np.setdiff1d(np.arange(c.shape[0]), touched)
            ids = np.unique(np.r_[rng.choice(A, 48, replace=False),
                                  rng.choice(left, min(24, left.size), replace=False),
                                  rng.choice(never, min(8, never.size), replace=False)]).astype(np.int32)
            out[f"w_{k}"] = st.w.copy()
            out[f"A_{k}"] = A.astype(np.int32)
            out[f"ids_{k}"] = ids
            out[f"P_{k}"] = st.P.block(ids)
            print(f"frame {k}: a={A.size} touched={touched.size} left={left.size}", flush=True)
    out["hashes"] = np.array(hashes)
    out["frames"] = np.array(FRAMES)
    np.savez_compressed(OUT, **out)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
