"""Plain FP64 CPU oracle for the Gauss-Legendre spherical harmonic transform.

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, obviously correct reference
that the CUDA library is checked against (Sec. 2 of Schaeffer's SHTns paper:
Eq. "synth_direct" for synthesis, Eq. "gauss" for analysis; the P_n^m
recurrence of Sec. 3.2).  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA path: it is a separate C file (``sht_oracle.c``) compiled with gcc and
loaded here through ctypes.

All arrays are numpy float64.  Spectral arrays are complex128 of length
nlm (packed m-major, idx(n,m) = m(2 lmax+3-m)/2 + n-m); grids are
float64 [nlat, nphi].  Batched inputs are handled by looping in Python.

Every function documents the passage it follows; see the C file header for
the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sht_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile sht_oracle.c with gcc (-O2 -fopenmp, no fast-math) into _build/."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
               "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        I = ctypes.POINTER(ctypes.c_int)
        c_int = ctypes.c_int
        lib.oracle_gauss.argtypes = [c_int, D, D]
        lib.oracle_gauss.restype = c_int
        lib.oracle_plm.argtypes = [c_int, c_int, ctypes.c_double, D]
        lib.oracle_dplm.argtypes = [c_int, c_int, ctypes.c_double, D]
        lib.oracle_plm_order.argtypes = [c_int, c_int, ctypes.c_double, D, D]
        lib.oracle_nlm.argtypes = [c_int, c_int]
        lib.oracle_nlm.restype = ctypes.c_long
        lib.oracle_threads.restype = c_int
        lib.oracle_set_threads.argtypes = [c_int]
        for name in ("oracle_synth", "oracle_analys_adj"):
            getattr(lib, name).argtypes = [c_int] * 4 + [D, D, I, c_int]
        for name in ("oracle_analys", "oracle_synth_adj"):
            getattr(lib, name).argtypes = [c_int] * 4 + [D, D, I, c_int]
        for name in ("oracle_synth_vec", "oracle_analys_vec_adj"):
            getattr(lib, name).argtypes = [c_int] * 4 + [D, D, D, D, I, c_int]
        for name in ("oracle_analys_vec", "oracle_synth_vec_adj"):
            getattr(lib, name).argtypes = [c_int] * 4 + [D, D, D, D, I, c_int]
        _lib = lib
        return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _sel(sel):
    if sel is None:
        return None, 0, None
    arr = np.ascontiguousarray(np.asarray(sel, dtype=np.int32))
    return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(arr.size), arr


def threads() -> int:
    """Number of OpenMP threads the oracle uses."""
    return int(_load().oracle_threads())


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def nlm(lmax: int, mmax: int | None = None) -> int:
    mmax = lmax if mmax is None else mmax
    return int(_load().oracle_nlm(lmax, mmax))


def gauss(nlat: int):
    """Gauss-Legendre nodes (descending, north to south) and weights (Sec. 2.3)."""
    x = np.zeros(nlat)
    w = np.zeros(nlat)
    if _load().oracle_gauss(nlat, _dp(x), _dp(w)) != 0:
        raise ValueError("nlat must be >= 1")
    return x, w


def plm(lmax: int, mmax: int, x: float) -> np.ndarray:
    """P_n^m(x) (Sec. 3.2 recurrence, no Condon-Shortley phase), packed."""
    out = np.zeros(nlm(lmax, mmax))
    _load().oracle_plm(lmax, mmax, float(x), _dp(out))
    return out


def plm_order(lmax: int, m: int, x, deriv: bool = False) -> np.ndarray:
    """P_n^m(x_j) (or dP_n^m/dtheta) of one order m, n = m..lmax, at the nodes
    x (scalar or 1-D): array [len(x), lmax - m + 1] -- the same recurrence as
    plm, one column of its packed layout."""
    xs = np.atleast_1d(np.asarray(x, dtype=np.float64))
    L = lmax - m + 1
    p = np.zeros(L)
    d = np.zeros(L)
    out = np.zeros((xs.size, L))
    lib = _load()
    for i, xv in enumerate(xs):
        lib.oracle_plm_order(lmax, m, float(xv), _dp(p), _dp(d) if deriv else None)
        out[i] = d if deriv else p
    return out


def dplm_dtheta(lmax: int, mmax: int, x: float) -> np.ndarray:
    """dP_n^m(cos theta)/dtheta at x = cos theta, packed."""
    out = np.zeros(nlm(lmax, mmax))
    _load().oracle_dplm(lmax, mmax, float(x), _dp(out))
    return out


def _spec_in(a, n):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    if a.shape[-1] != n:
        raise ValueError(f"spectral array must have {n} coefficients, got {a.shape}")
    return a


def _grid_in(g, nlat, nphi):
    g = np.ascontiguousarray(np.asarray(g, dtype=np.float64))
    if g.shape[-2:] != (nlat, nphi):
        raise ValueError(f"grid must be [..., {nlat}, {nphi}], got {g.shape}")
    return g


def _spec_to_grid(fname, lmax, mmax, nlat, nphi, specs, rows):
    lib = _load()
    n = nlm(lmax, mmax)
    specs = [_spec_in(s, n) for s in specs]
    lead = specs[0].shape[:-1]
    flat = [s.reshape(-1, n) for s in specs]
    nb = flat[0].shape[0]
    outs = [np.zeros((nb, nlat, nphi)) for _ in range(2 if len(specs) == 2 else 1)]
    rp, nr, keep = _sel(rows)
    for b in range(nb):
        ins = [np.ascontiguousarray(f[b]).view(np.float64) for f in flat]
        if len(specs) == 1:
            getattr(lib, fname)(lmax, mmax, nlat, nphi, _dp(ins[0]), _dp(outs[0][b]), rp, nr)
        else:
            getattr(lib, fname)(lmax, mmax, nlat, nphi, _dp(ins[0]), _dp(ins[1]),
                                _dp(outs[0][b]), _dp(outs[1][b]), rp, nr)
    del keep
    res = [o.reshape(lead + (nlat, nphi)) for o in outs]
    return res[0] if len(res) == 1 else tuple(res)


def _grid_to_spec(fname, lmax, mmax, nlat, nphi, grids, ms):
    lib = _load()
    n = nlm(lmax, mmax)
    grids = [_grid_in(g, nlat, nphi) for g in grids]
    lead = grids[0].shape[:-2]
    flat = [g.reshape(-1, nlat, nphi) for g in grids]
    nb = flat[0].shape[0]
    outs = [np.zeros((nb, n), dtype=np.complex128) for _ in grids]
    mp, nm, keep = _sel(ms)
    for b in range(nb):
        ins = [np.ascontiguousarray(f[b]) for f in flat]
        ov = [o[b].view(np.float64) for o in outs]
        if len(grids) == 1:
            getattr(lib, fname)(lmax, mmax, nlat, nphi, _dp(ins[0]), _dp(ov[0]), mp, nm)
        else:
            getattr(lib, fname)(lmax, mmax, nlat, nphi, _dp(ins[0]), _dp(ins[1]),
                                _dp(ov[0]), _dp(ov[1]), mp, nm)
    del keep
    res = [o.reshape(lead + (n,)) for o in outs]
    return res[0] if len(res) == 1 else tuple(res)


def synth(lmax, mmax, nlat, nphi, spec, rows=None):
    """Scalar synthesis, Sec. 2.2 (Eq. synth_direct) + Hermitian Fourier sum.

    rows: optional list of latitude indices; other rows are returned as 0."""
    return _spec_to_grid("oracle_synth", lmax, mmax, nlat, nphi, [spec], rows)


def analys(lmax, mmax, nlat, nphi, grid, ms=None):
    """Scalar analysis, Sec. 2.3 (Eq. gauss).  ms: optional orders to compute."""
    return _grid_to_spec("oracle_analys", lmax, mmax, nlat, nphi, [grid], ms)


def synth_adj(lmax, mmax, nlat, nphi, grid, ms=None):
    """Adjoint of synth under <a,b> = sum Re(conj a b), <f,g> = sum f g."""
    return _grid_to_spec("oracle_synth_adj", lmax, mmax, nlat, nphi, [grid], ms)


def analys_adj(lmax, mmax, nlat, nphi, spec, rows=None):
    """Adjoint of analys under the same inner products."""
    return _spec_to_grid("oracle_analys_adj", lmax, mmax, nlat, nphi, [spec], rows)


def synth_vec(lmax, mmax, nlat, nphi, S, T, rows=None):
    """Spheroidal/toroidal synthesis v = grad S + r x grad T -> (v_theta, v_phi)."""
    return _spec_to_grid("oracle_synth_vec", lmax, mmax, nlat, nphi, [S, T], rows)


def analys_vec(lmax, mmax, nlat, nphi, vt, vp, ms=None):
    """Vector analysis (v_theta, v_phi) -> (S, T), divided by n(n+1)."""
    return _grid_to_spec("oracle_analys_vec", lmax, mmax, nlat, nphi, [vt, vp], ms)


def synth_vec_adj(lmax, mmax, nlat, nphi, gt, gp, ms=None):
    return _grid_to_spec("oracle_synth_vec_adj", lmax, mmax, nlat, nphi, [gt, gp], ms)


def analys_vec_adj(lmax, mmax, nlat, nphi, S, T, rows=None):
    return _spec_to_grid("oracle_analys_vec_adj", lmax, mmax, nlat, nphi, [S, T], rows)


def lm_index(lmax: int, n: int, m: int) -> int:
    """Packed m-major index (layout of the spectral arrays)."""
    return m * (2 * lmax + 3 - m) // 2 + (n - m)


def eps_max_rms(R: np.ndarray, Q: np.ndarray, lmax: int):
    """Error measures of Sec. 3.5: eps_max = max |R - Q|,
    eps_rms = sqrt(2/((N+1)(N+2)) sum |R - Q|^2) over the packed m >= 0 set."""
    d = np.abs(np.asarray(R) - np.asarray(Q))
    emax = float(d.max()) if d.size else 0.0
    erms = float(np.sqrt(2.0 / ((lmax + 1) * (lmax + 2)) * np.sum(d * d)))
    return emax, erms
