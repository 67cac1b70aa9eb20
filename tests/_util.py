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


def fp32_bound(lmax):
    """Normwise tolerance of the FP32 path.

    The FP32 recurrence carries a relative error that grows at most linearly
    with the number of steps (~ (N+1) u, u = 2^-24) and each Legendre sum adds
    ~ sqrt(N+1) u; the FFT adds ~ log2(nphi) u.  The bound used is
    8 (N + 1) u + 1e-6."""
    u = 2.0 ** -24
    return 8.0 * (lmax + 1) * u + 1e-6


FP64_TOL = {31: 1e-13, 255: 1e-12, 1023: 1e-11}


def fp64_bound(lmax):
    """Normwise tolerance of the FP64 path: 1e-11 at N <= 1023 (the paper's
    accuracy statement of Sec. 3.5), tighter at small N."""
    for n, tol in sorted(FP64_TOL.items()):
        if lmax <= n:
            return tol
    return 1e-11
