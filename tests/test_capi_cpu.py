"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol include/sht.h declares, and rejects bad arguments on the host."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sht.h")


def _declared():
    txt = open(HEADER).read()
    names = re.findall(r"^SHT_API[^;(]*?\b(sht_\w+)\s*\(", txt, flags=re.M)
    assert names, "no declarations found"
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1202_6522_gb300 import _capi, build
    build.build()
    return _capi.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("sht_create", "sht_destroy", "sht_synth", "sht_analys", "sht_synth_vec", "sht_analys_vec",
                 "sht_synth_adj", "sht_analys_adj", "sht_synth_vec_adj", "sht_analys_vec_adj"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_binding_covers_every_symbol(lib):
    from paper_1202_6522_gb300 import _capi
    for name in _declared():
        assert name in _capi.SIGNATURES, name
        assert callable(getattr(_capi, name)), name


@pytest.mark.parametrize("args,code", [
    ((-1, 0, 4, 8), -1),     # lmax < 0
    ((10, 11, 16, 32), -1),  # mmax > lmax
    ((10, 10, 10, 32), -1),  # nlat < lmax + 1 (quadrature not exact)
    ((10, 10, 11, 20), -1),  # nphi < 2 mmax + 1
    ((10, 10, 11, 28), -5),  # nphi / 2 = 14 has the factor 7 (FFT lengths are 2^a 3^b 5^c)
    ((10, 10, 11, 25), -5),  # nphi odd
])
def test_create_rejects_bad_sizes_on_host(lib, args, code):
    h = ctypes.c_void_p()
    assert lib.sht_create(*args, ctypes.byref(h)) == code
    assert h.value is None
    assert lib.sht_last_error()


def test_null_handle_and_pointers(lib):
    assert lib.sht_synth(None, None, None, 1, 0, None) == -1
    assert lib.sht_nlm(None) == -1
    assert lib.sht_create(3, 3, 4, 8, None) == -1
    lib.sht_destroy(None)


def test_python_errors_map_to_exceptions(lib):
    from paper_1202_6522_gb300 import _capi
    with pytest.raises(ValueError):
        _capi.sht_create(10, 11, 16, 32)


def _ints(v):
    return (ctypes.c_int * len(v))(*v)


@pytest.mark.parametrize("mode,nphi,code", [
    (7, 16, -1),     # not a batch path (SHT_F32, SHT_TC_BF16X3 or SHT_F32_AUTO)
    (0, 16, -1),     # SHT_F64 has no uneven-batch form
    (2, 28, -5),     # a field whose FFT length 14 has the factor 7
    (3, 8192, -5),   # nphi above the batch FFT limit
])
def test_batch_create_mode_rejects_on_host(lib, mode, nphi, code):
    b = ctypes.c_void_p()
    assert lib.sht_batch_create_mode(2, _ints([7, 7]), _ints([8, 8]), _ints([16, nphi]), mode, ctypes.byref(b)) == code
    assert b.value is None
    assert lib.sht_last_error()


def test_batch_mode_null_handle(lib):
    assert lib.sht_batch_mode(None, None, None) == -1


@pytest.mark.parametrize("args,code", [
    ((31, 7, 0, 32, 16), -1),       # mres < 1
    ((31, 8, 4, 32, 32), -1),       # mmax mres = 32 > lmax
    ((31, 7, 4, 31, 16), -1),       # nlat < lmax + 1
    ((31, 7, 4, 32, 14), -1),       # nphi < 2 mmax + 1 (orders counted by index)
    ((31, 7, 4, 32, 22), -5),       # nphi / 2 = 11
    ((5000, 10, 4, 5001, 32), -5),  # lmax above 4095
])
def test_create_mres_rejects_on_host(lib, args, code):
    h = ctypes.c_void_p()
    assert lib.sht_create_mres(*args, ctypes.byref(h)) == code
    assert h.value is None
