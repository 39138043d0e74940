"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.maximum(1.0, np.abs(b))


def path_mismatches(x_gpu, x_orc, margin, anchor, M, tol, nwl=None, block=0):
    """Compare worldlines in the order they were drawn.

    The loop is resampled as blocks of `block` slices from the anchor (0 or >= M: one
    block of M slices), each drawn from its last interior slice back to its first and
    independent of the others given the held end sites.  Within a block a worldline
    must agree exactly up to its first difference, which is allowed only where the
    oracle's uniform landed within `tol` (relative) of a CDF edge; the held block starts
    must agree exactly.  Returns (draws compared, first differences, offending list)."""
    B = block if 0 < block < M else M
    bad, draws, firsts = [], 0, 0
    n = x_gpu.shape[1] if nwl is None else nwl
    for sg in range(2):
        for p in range(n):
            for b0 in range(0, M, B):
                l0 = (anchor + b0) % M
                if x_gpu[sg, p, l0] != x_orc[sg, p, l0]:
                    bad.append((sg, p, l0, "held site changed"))
                for i in range(min(B, M - b0) - 1, 0, -1):
                    l = (l0 + i) % M
                    draws += 1
                    if x_gpu[sg, p, l] != x_orc[sg, p, l]:
                        firsts += 1
                        if not (margin[sg, p, l] < tol):
                            bad.append((sg, p, l, int(x_gpu[sg, p, l]), int(x_orc[sg, p, l]), margin[sg, p, l]))
                        break
    return draws, firsts, bad
