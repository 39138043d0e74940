"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.maximum(1.0, np.abs(b))


def path_mismatches(x_gpu, x_orc, margin, anchor, M, tol, nwl=None):
    """Compare worldlines in the order they were drawn (slices a+M-1 .. a+1).

    Up to its first difference a worldline must agree exactly; the first difference
    is allowed only where the oracle's uniform landed within `tol` (relative) of a
    CDF edge.  Returns (draws compared, first differences, offending list)."""
    bad, draws, firsts = [], 0, 0
    n = x_gpu.shape[1] if nwl is None else nwl
    for sg in range(2):
        for p in range(n):
            for i in range(M - 1, 0, -1):
                l = (anchor + i) % M
                draws += 1
                if x_gpu[sg, p, l] != x_orc[sg, p, l]:
                    firsts += 1
                    if not (margin[sg, p, l] < tol):
                        bad.append((sg, p, l, int(x_gpu[sg, p, l]), int(x_orc[sg, p, l]), margin[sg, p, l]))
                    break
    return draws, firsts, bad
