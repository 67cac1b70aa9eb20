"""Shared helpers for the GPU parity tests (comparison only, no transform math)."""
import numpy as np


def normwise(got, ref):
    """max |got - ref| / max |ref| over the whole array (the parity measure)."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    scale = np.abs(ref).max()
    if scale == 0:
        return float(np.abs(got).max())
    return float(np.abs(got - ref).max() / scale)


def fp64_bound(lmax):
    """Normwise tolerance of the FP64 path: 1e-11, the accuracy the method
    reaches for N < 2048 (Sec. 3.5)."""
    return 1e-11
