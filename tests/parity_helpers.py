"""Shared helpers of the GPU parity tests (host side, oracle only)."""
import numpy as np


def accounted_pair(oracle_lib, s, params, src, tgt, Xi, Xj, gpu_mask, r):
    """The oracle's sums of one pair with every flagged point that the GPU
    decided the other way moved to the GPU's side: its contribution (from the
    oracle, or from the oracle's other-branch evaluation when the oracle
    rejected it) is removed or added.  Returns (H, b, cost, count, n_flipped,
    n_unexplained)."""
    H, b, cost, count = r["H"].copy(), r["b"].copy(), r["cost"], r["count"]
    n = r["n_points"]
    diff = np.unpackbits((gpu_mask ^ r["mask"]).view(np.uint8), bitorder="little")[:n]
    ok_o = np.unpackbits(r["mask"].view(np.uint8), bitorder="little")[:n]
    idx = np.nonzero(diff)[0]
    unexplained = 0
    if idx.size:
        pts, _ = oracle_lib.frame_points(s, params, src)
        for k in idx.tolist():
            c = oracle_lib.point_contribution(s, params, tgt, Xi, Xj, pts[k], other_branch=not ok_o[k])
            if c is None:
                unexplained += 1
                continue
            sign = -1.0 if ok_o[k] else 1.0
            H += sign * c[0]
            b += sign * c[1]
            cost += sign * c[2]
            count += int(sign)
    return H, b, cost, count, int(idx.size), unexplained
