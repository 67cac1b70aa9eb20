"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws random numbers and lays them out; it holds none of the
transform's arithmetic.  The paper measures on random spectral coefficients
(Sec. 3.5), so these generators stand in for its workloads:

* spectra: Re and Im of every packed coefficient drawn from N(0, 1) with
  ``numpy.random.default_rng(seed)`` (all real parts in packed m-major order,
  then all imaginary parts), multiplied by (n+1)^-power, Im zeroed at m = 0;
* grids: N(0, 1) samples, shape [..., nlat, nphi];
* uniform spectra in [-1, 1] as in the accuracy test of Sec. 3.5.
"""
from __future__ import annotations

import numpy as np


def packed_degrees_orders(lmax: int, mmax: int | None = None):
    """Degree n and order m of every packed coefficient (m-major, n = m..lmax)."""
    mmax = lmax if mmax is None else mmax
    ns, ms = [], []
    for m in range(mmax + 1):
        for n in range(m, lmax + 1):
            ns.append(n)
            ms.append(m)
    return np.asarray(ns, dtype=np.int64), np.asarray(ms, dtype=np.int64)


def spectrum(lmax: int, mmax: int | None = None, batch: int | None = None,
             seed: int = 0, power: float = 1.0, uniform: bool = False) -> np.ndarray:
    """Seeded complex128 spectra of shape [nlm] (batch None) or [batch, nlm]."""
    ns, ms = packed_degrees_orders(lmax, mmax)
    nlm = ns.size
    rng = np.random.default_rng(seed)
    nb = 1 if batch is None else batch
    if uniform:
        re = rng.uniform(-1.0, 1.0, size=(nb, nlm))
        im = rng.uniform(-1.0, 1.0, size=(nb, nlm))
    else:
        re = rng.standard_normal((nb, nlm))
        im = rng.standard_normal((nb, nlm))
    scale = (ns + 1.0) ** (-power)
    a = (re + 1j * im) * scale
    a[:, ms == 0] = a[:, ms == 0].real
    return a[0] if batch is None else a


def grid(nlat: int, nphi: int, batch: int | None = None, seed: int = 1) -> np.ndarray:
    """Seeded float64 N(0,1) grid of shape [nlat, nphi] or [batch, nlat, nphi]."""
    rng = np.random.default_rng(seed)
    shape = (nlat, nphi) if batch is None else (batch, nlat, nphi)
    return rng.standard_normal(shape)


def uneven_truncations(nfields: int = 96, choices=(63, 127, 255, 511), seed: int = 0):
    """Truncations drawn uniformly from ``choices`` for an uneven batch."""
    rng = np.random.default_rng(seed)
    return [int(c) for c in rng.choice(np.asarray(choices), size=nfields)]
