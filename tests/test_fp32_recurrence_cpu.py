"""FP32 evaluation of the P_n^m recurrence, simulated on the CPU (no GPU).

The FP32 path of the library runs the recurrence of Sec. 3.2 in single
precision.  This file shows, at N = 1023 against the oracle's P_n^m, why it
needs both of its measures, and pins the constant B_F32_REC that bounds its
error in the GPU parity tests:

1. Without the exponent scale of Sec. 3.5, P_m^m underflows FP32 near the
   poles for high orders, and whole (order, latitude) blocks whose values are
   well above FP32's resolution come out as zero.
2. With the exponent scale but one FP32 chain over all N degrees, rounding
   errors grow with N (the recurrence has a nearly double characteristic
   root near the poles); at N = 1023 the relative error is far above
   B_F32_REC.
3. With the exponent scale and the chain restarted every 32 degrees from the
   FP64 state (what the library's FP32 kernels do), the error stays below
   B_F32_REC for every sampled order and node.

Error measure per (order m, node x_j): the RSS over n of the error of
P_n^m(x_j) divided by the RSS over n of P_n^m(x_j) -- the factor by which a
Legendre sum over n with random coefficients is perturbed.  Nodes whose RSS is
below 1e-7 of the order's largest do not enter FP32 results and are skipped.

The simulation rounds every operation to FP32 (an FMA is computed in FP64 and
rounded once to FP32); values with a positive exponent counter are left out,
as in the kernels.
"""
import math

import numpy as np

import oracle
from _bounds import B_F32_REC

N = 1023
NLAT = 1024
S32 = 64          # exponent step of the FP32 scale (Sec. 3.5)
SEG = 32          # degrees between restarts
ORDERS = (0, 10, 100, 400, 800)


def f32(v):
    return np.asarray(v, dtype=np.float64).astype(np.float32).astype(np.float64)


def fma32(a, b, c):
    return f32(a * b + c)


def coefficients(m):
    """(a_n^m, b_n^m) of the recurrence of Sec. 3.2 for n = m .. N, FP32; the
    first step (n = m) is P_m^m = 0 x P_{m-1} + 1 x P_m^m, the start value."""
    n = np.arange(m, N + 1, dtype=np.float64)
    a = np.zeros_like(n)
    b = np.zeros_like(n)
    b[0] = 1.0
    if len(n) > 1:
        a[1] = math.sqrt(2 * m + 3)
    nn = n[2:]
    a[2:] = np.sqrt((4 * nn * nn - 1) / (nn * nn - m * m))
    b[2:] = -np.sqrt((2 * nn + 1) / (2 * nn - 3) * ((nn - 1) ** 2 - m * m) / (nn * nn - m * m))
    return f32(a), f32(b)


def log2_pmm(m, x):
    """log2 P_m^m(x) = log2 sqrt(1/4pi) + sum_k log2 sqrt((2k+1)/(2k)) + m log2 sin(theta)."""
    k = np.arange(1, m + 1, dtype=np.float64)
    c = 0.5 * math.log2(1 / (4 * math.pi)) + 0.5 * float(np.sum(np.log2((2 * k + 1) / (2 * k))))
    return c + m * 0.5 * np.log2((1 - x) * (1 + x))


def to_scaled(log2v):
    """y, k with value = y 2^(-64 k), y in [2^-65, 1) when k > 0 (Sec. 3.5 form)."""
    e = np.floor(log2v) + 1
    k = np.where(e >= 1 - S32, 0, np.floor(-e / S32)).astype(np.int64)
    return f32(np.exp2(log2v + S32 * k)), k


def simulate(m, x, true, scaled, restart):
    """FP32 values of P_n^m(x_j) for n = m .. N (rows) at the nodes x (cols)."""
    a, b = coefficients(m)
    xf = f32(x)
    L = N - m + 1
    y1 = np.zeros_like(xf)
    if scaled:
        y2, k = to_scaled(log2_pmm(m, x))
    else:
        y2, k = f32(np.exp2(log2_pmm(m, x))), np.zeros(len(x), dtype=np.int64)
    out = np.zeros((L, len(x)))
    for i in range(L):
        if restart and i % SEG == 0 and i > 0:
            # state (P_{n0-1}, P_{n0-2}) from FP64, in the scaled FP32 form
            t1, t2 = true[i - 1], true[i - 2] if i >= 2 else np.zeros_like(xf)
            mx = np.maximum(np.abs(t1), np.abs(t2))
            with np.errstate(divide="ignore"):
                e = np.where(mx > 0, np.floor(np.log2(np.where(mx > 0, mx, 1.0))) + 1, 0)
            k = np.where((mx == 0) | (e >= 1 - S32), 0, np.floor(-e / S32)).astype(np.int64)
            y1 = f32(np.ldexp(t1, S32 * k))
            y2 = f32(np.ldexp(t2, S32 * k))
        yn = fma32(f32(a[i] * xf), y1, f32(b[i] * y2))
        y2, y1 = y1, yn
        if scaled:
            resc = (k > 0) & (np.abs(yn) >= 1.0)
            y1 = np.where(resc, f32(np.ldexp(y1, -S32)), y1)
            y2 = np.where(resc, f32(np.ldexp(y2, -S32)), y2)
            k = k - resc
        out[i] = np.where(k == 0, y1, 0.0)
    return out


_cache = {}


def true_values():
    """The oracle's P_n^m(x_j) for the sampled orders at the northern nodes."""
    if "p" not in _cache:
        x, _ = oracle.gauss(NLAT)
        xs = x[: NLAT // 2]
        blocks = {m: oracle.plm_order(N, m, xs).T for m in ORDERS}      # [n - m, node]
        _cache["p"] = (xs, blocks)
    return _cache["p"]


def worst_ratio(scaled, restart):
    xs, blocks = true_values()
    worst = 0.0
    for m in ORDERS:
        true = blocks[m]
        got = simulate(m, xs, true, scaled, restart)
        rss = np.sqrt(np.sum(true ** 2, axis=0))
        live = rss >= 1e-7 * rss.max()
        err = np.sqrt(np.sum((got - true) ** 2, axis=0))
        worst = max(worst, float((err[live] / rss[live]).max()))
    return worst


def test_fp32_without_exponent_scale_loses_blocks():
    r = worst_ratio(scaled=False, restart=False)
    assert r > 0.99, r          # some significant (m, x_j) block is lost entirely


def test_fp32_scaled_chain_error_grows_with_n():
    r = worst_ratio(scaled=True, restart=False)
    assert r > 10 * B_F32_REC, r


def test_fp32_scaled_restarted_chain_within_constant():
    r = worst_ratio(scaled=True, restart=True)
    assert r <= B_F32_REC, r
