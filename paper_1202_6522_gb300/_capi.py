"""ctypes binding of libsht's C ABI (include/sht.h), with the same names.

Argument marshalling only: every function takes plain integers (device
pointers, stream handles) and returns the library's status code.  The library
is built in-tree by ``paper_1202_6522_gb300.build``; if it is missing this
module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

SHT_OK = 0
SHT_EINVAL = -1
SHT_ENOMEM = -2
SHT_ECUDA = -3
SHT_ETIMEOUT = -4
SHT_EUNSUPPORTED = -5

SHT_F64 = 0
SHT_F32 = 1
SHT_TC_BF16X3 = 2
SHT_F32_AUTO = 3
SHT_TC_OTF = 4
SHT_TC_F64 = 5

_lib = None
_lock = threading.Lock()

_VP = ctypes.c_void_p
_I = ctypes.c_int

# name -> (argtypes, restype); mirrors include/sht.h
SIGNATURES = {
    "sht_create": ([_I, _I, _I, _I, ctypes.POINTER(_VP)], _I),
    "sht_create_mres": ([_I, _I, _I, _I, _I, ctypes.POINTER(_VP)], _I),
    "sht_destroy": ([_VP], None),
    "sht_reserve": ([_VP, _I, _I], _I),
    "sht_synth": ([_VP, _VP, _VP, _I, _I, _VP], _I),
    "sht_analys": ([_VP, _VP, _VP, _I, _I, _VP], _I),
    "sht_synth_vec": ([_VP, _VP, _VP, _VP, _VP, _I, _I, _VP], _I),
    "sht_analys_vec": ([_VP, _VP, _VP, _VP, _VP, _I, _I, _VP], _I),
    "sht_synth_adj": ([_VP, _VP, _VP, _I, _I, _VP], _I),
    "sht_analys_adj": ([_VP, _VP, _VP, _I, _I, _VP], _I),
    "sht_synth_vec_adj": ([_VP, _VP, _VP, _VP, _VP, _I, _I, _VP], _I),
    "sht_analys_vec_adj": ([_VP, _VP, _VP, _VP, _VP, _I, _I, _VP], _I),
    "sht_nlm": ([_VP], _I),
    "sht_lm_index": ([_VP, _I, _I], _I),
    "sht_gauss": ([_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], _I),
    "sht_sync_status": ([_VP, _VP], _I),
    "sht_synth_static": ([_VP, _VP, _VP, _I, _I, _VP], _I),
    "sht_batch_create": ([_I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_VP)], _I),
    "sht_batch_create_mode": ([_I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), _I,
                               ctypes.POINTER(_VP)], _I),
    "sht_batch_mode": ([_VP, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)], _I),
    "sht_batch_destroy": ([_VP], None),
    "sht_batch_synth": ([_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I, _VP], _I),
    "sht_batch_analys": ([_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I, _VP], _I),
    "sht_tune": ([_VP, _I, _I, ctypes.POINTER(ctypes.c_double), _VP], _I),
    "sht_selftest_timeout": ([_VP, _I, _VP], _I),
    "sht_set_polar_threshold": ([_VP, ctypes.c_double], _I),
    "sht_alu_peaks": ([ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _VP], _I),
    "sht_tc_polar_skip": ([_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], _I),
    "sht_cc_polar_skip": ([_VP, _I, ctypes.POINTER(ctypes.c_double)], _I),
    "sht_profile": ([_VP, _I], _I),
    "sht_profile_read": ([_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I), _I], _I),
    "sht_kernel_name": ([_I], ctypes.c_char_p),
    "sht_last_error": ([], ctypes.c_char_p),
}

SHT_NKERNELS = 10


def library_path() -> str:
    return _build.LIB


def load():
    """Load libsht.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(
                f"libsht.so not found at {path}; build it with "
                "`python -m paper_1202_6522_gb300.build` (the transform has no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


class SHTError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libsht error {code}: {msg}")
        self.code = code


def check(code: int) -> int:
    if code is not None and code < 0:
        msg = load().sht_last_error()
        msg = msg.decode() if msg else ""
        if code == SHT_EINVAL:
            raise ValueError(f"libsht: {msg}")
        raise SHTError(code, msg)
    return code


def _call(name, *args):
    return getattr(load(), name)(*args)


def sht_create(lmax: int, mmax: int, nlat: int, nphi: int) -> int:
    h = _VP()
    check(_call("sht_create", lmax, mmax, nlat, nphi, ctypes.byref(h)))
    return h.value


def sht_create_mres(lmax: int, mmax: int, mres: int, nlat: int, nphi: int) -> int:
    h = _VP()
    check(_call("sht_create_mres", lmax, mmax, mres, nlat, nphi, ctypes.byref(h)))
    return h.value


def sht_destroy(h: int) -> None:
    _call("sht_destroy", h)


def sht_reserve(h, batch, mode):
    return check(_call("sht_reserve", h, batch, mode))


def sht_synth(h, spec, grid, batch, mode, stream):
    return check(_call("sht_synth", h, spec, grid, batch, mode, stream))


def sht_analys(h, grid, spec, batch, mode, stream):
    return check(_call("sht_analys", h, grid, spec, batch, mode, stream))


def sht_synth_vec(h, S, T, vt, vp, batch, mode, stream):
    return check(_call("sht_synth_vec", h, S, T, vt, vp, batch, mode, stream))


def sht_analys_vec(h, vt, vp, S, T, batch, mode, stream):
    return check(_call("sht_analys_vec", h, vt, vp, S, T, batch, mode, stream))


def sht_synth_adj(h, grid, spec, batch, mode, stream):
    return check(_call("sht_synth_adj", h, grid, spec, batch, mode, stream))


def sht_analys_adj(h, spec, grid, batch, mode, stream):
    return check(_call("sht_analys_adj", h, spec, grid, batch, mode, stream))


def sht_synth_vec_adj(h, gt, gp, S, T, batch, mode, stream):
    return check(_call("sht_synth_vec_adj", h, gt, gp, S, T, batch, mode, stream))


def sht_analys_vec_adj(h, S, T, gt, gp, batch, mode, stream):
    return check(_call("sht_analys_vec_adj", h, S, T, gt, gp, batch, mode, stream))


def sht_nlm(h) -> int:
    return check(_call("sht_nlm", h))


def sht_lm_index(h, n, m) -> int:
    return _call("sht_lm_index", h, n, m)


def sht_gauss(h, nlat: int):
    x = (ctypes.c_double * nlat)()
    w = (ctypes.c_double * nlat)()
    check(_call("sht_gauss", h, x, w))
    return list(x), list(w)


def sht_sync_status(h, stream):
    return check(_call("sht_sync_status", h, stream))


def sht_synth_static(h, spec, grid, batch, mode, stream):
    """sht_synth without any device allocation (intermediate in a fixed 16 MiB array)."""
    return check(_call("sht_synth_static", h, spec, grid, batch, mode, stream))


SHT_STATIC_SCRATCH_BYTES = 16 * 1024 * 1024


def _ints(v):
    arr = (ctypes.c_int * len(v))(*[int(x) for x in v])
    return arr


def _ptrs(v):
    return (_VP * len(v))(*[int(x) for x in v])


def sht_batch_create(lmax, nlat, nphi) -> int:
    """Uneven batch plan over len(lmax) fields (mmax = lmax each)."""
    h = _VP()
    n = len(lmax)
    check(_call("sht_batch_create", n, _ints(lmax), _ints(nlat), _ints(nphi), ctypes.byref(h)))
    return h.value


def sht_batch_create_mode(lmax, nlat, nphi, mode) -> int:
    """Uneven batch plan with a path: SHT_F32, SHT_TC_BF16X3 or SHT_F32_AUTO."""
    h = _VP()
    n = len(lmax)
    check(_call("sht_batch_create_mode", n, _ints(lmax), _ints(nlat), _ints(nphi), int(mode), ctypes.byref(h)))
    return h.value


def sht_batch_mode(b):
    """(path in use, measured ms of the CUDA-core path, of the tensor-core path)."""
    a, c = ctypes.c_float(0.0), ctypes.c_float(0.0)
    mode = check(_call("sht_batch_mode", b, ctypes.byref(a), ctypes.byref(c)))
    return mode, a.value, c.value


def sht_batch_destroy(b) -> None:
    _call("sht_batch_destroy", b)


def sht_batch_synth(b, spec_ptrs, grid_ptrs, use_graph, stream):
    return check(_call("sht_batch_synth", b, _ptrs(spec_ptrs), _ptrs(grid_ptrs), int(bool(use_graph)), stream))


def sht_batch_analys(b, grid_ptrs, spec_ptrs, use_graph, stream):
    return check(_call("sht_batch_analys", b, _ptrs(grid_ptrs), _ptrs(spec_ptrs), int(bool(use_graph)), stream))


def sht_tune(h, batch, mode, stream):
    """Runtime tuning; returns the three timings of the report (ms)."""
    rep = (ctypes.c_double * 3)()
    check(_call("sht_tune", h, batch, mode, rep, stream))
    return rep[0], rep[1], rep[2]


def sht_tc_polar_skip(h):
    a, b = ctypes.c_double(), ctypes.c_double()
    check(_call("sht_tc_polar_skip", h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def sht_set_polar_threshold(h, threshold):
    return check(_call("sht_set_polar_threshold", h, float(threshold)))


def sht_cc_polar_skip(h, mode):
    """Share of the CUDA-core scalar terms before their first live segment (-1: no table)."""
    f = ctypes.c_double()
    check(_call("sht_cc_polar_skip", h, mode, ctypes.byref(f)))
    return f.value


def sht_selftest_timeout(h, timeout_us, stream):
    return check(_call("sht_selftest_timeout", h, timeout_us, stream))


def sht_alu_peaks(stream):
    """Measured (FP32, FP64) FMA throughput in TFLOP/s."""
    a, b = ctypes.c_double(), ctypes.c_double()
    check(_call("sht_alu_peaks", ctypes.byref(a), ctypes.byref(b), stream))
    return a.value, b.value


def sht_profile(h, enable):
    return check(_call("sht_profile", h, int(bool(enable))))


def sht_profile_read(h):
    """{kernel name: (total ms, launches)} since the last read; synchronises."""
    ms = (ctypes.c_double * SHT_NKERNELS)()
    cnt = (ctypes.c_int * SHT_NKERNELS)()
    check(_call("sht_profile_read", h, ms, cnt, SHT_NKERNELS))
    return {sht_kernel_name(k): (ms[k], cnt[k]) for k in range(SHT_NKERNELS) if cnt[k]}


def sht_kernel_name(kind) -> str:
    n = _call("sht_kernel_name", kind)
    return n.decode() if n else ""


def sht_last_error() -> str:
    msg = load().sht_last_error()
    return msg.decode() if msg else ""
