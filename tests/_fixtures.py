"""Readers of the stored expected values under tests/golden/ (no arithmetic of the method)."""
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# the tiny overlapping-frames case of golden/block_overlap_hand.txt
OVERLAP_CENTERS = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0], [3.0, 0.0]])
OVERLAP_FRAMES = [
    np.array([[0.0, 0.0, 0.2], [0.5, 0.0, 0.1]]),
    np.array([[1.5, 0.0, -0.1]]),
    np.array([[0.5, 0.0, 0.3]]),
]
OVERLAP_RHO = 1.0
OVERLAP_LAMBDA = 1.0


def overlap_expected():
    """{after_frame: (w (4,), P (4, 4))} from the hand-worked fixture."""
    out = {}
    with open(os.path.join(GOLDEN, "block_overlap_hand.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            fr, kind, i, j, val = line.split()
            fr, i, j = int(fr), int(i), int(j)
            v = float(Fraction(val))
            w, P = out.setdefault(fr, (np.zeros(4), np.zeros((4, 4))))
            if kind == "w":
                w[i] = v
            else:
                P[i, j] = v
                P[j, i] = v
    return out


def c2_sequence():
    """The oracle's stored state of the staircase sequence (tests/golden/make_c2_sequence.py)."""
    return np.load(os.path.join(GOLDEN, "c2_sequence_oracle.npz"))
