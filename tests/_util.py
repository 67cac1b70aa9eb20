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

    Near the poles (x -> 1) the three-term recurrence of Sec. 3.2 has a nearly
    double characteristic root, so rounding errors introduced at each step are
    carried forward with a linearly growing factor; summed over N steps as a
    random walk this gives a relative error ~ (N+1)^1.5 u with u = 2^-24
    (measured on the CPU by running the recurrence in float32: 7e-3 at the
    polemost node for N = 1023, m = 0; 5.8e-4 normwise for a full synthesis).
    The bound used is (N+1)^1.5 u + 2e-6."""
    u = 2.0 ** -24
    return (lmax + 1) ** 1.5 * u + 2e-6


def fp64_bound(lmax):
    """Normwise tolerance of the FP64 path: 1e-11, the accuracy the method
    reaches for N < 2048 (Sec. 3.5)."""
    return 1e-11


def tc_bound(lmax):
    """Normwise tolerance of the tensor-core path (bf16 hi+lo split of both
    operands, hi*hi + hi*lo + lo*hi products, FP32 accumulation).  Each product
    carries a relative error <= 2^-15 (the dropped lo*lo term, 2^-16, plus the
    two split remainders, 2^-17 each); allowing a factor 4 for cancellation in
    the Legendre sums gives 2^-13.  The panels come from the FP64 recurrence,
    so, unlike the FP32 path, this bound does not grow with N."""
    return 2.0 ** -13
