"""The synthesis entry point that allocates nothing (sht_synth_static).

Some callers cannot ask the CUDA runtime for memory when they call the
transform: a host framework that owns a fixed device-memory budget, or a loop
that cannot afford the device-wide synchronisation cudaMalloc/cudaFree bring.
For them sht_synth_static keeps its intermediate in a fixed array inside the
library.  These tests call it through the C ABI and check that

* its output equals the ordinary sht_synth's bit for bit (both run the same
  kernels on the same inputs), twice in a row with different inputs (the array
  keeps the previous call's contents, which must not leak into the next
  result), on plain and m-stride plans;
* on a handle that has never run another transform, the device's free memory
  is the same before and after two calls (after one warm-up call, which may
  load the kernels' code), and the results still equal sht_synth's;
* calls too large for the array, and calls on a plan whose restart states
  (and, in FP64, polar table) were never built, are refused on the host.

The file is named so that pytest collects it last.
"""
import pytest

from paper_1202_6522_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def C():
    from paper_1202_6522_gb300 import build
    build.build()
    from paper_1202_6522_gb300 import _capi
    _capi.load()
    return _capi


def _types(C, prec):
    if prec == "f64":
        return torch.complex128, torch.float64, C.SHT_F64
    return torch.complex64, torch.float32, C.SHT_F32


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("lmax,mmax,mres,nlat,nphi,batch",
                         [(255, 255, 1, 256, 512, 2), (40, 40, 1, 41, 128, 3), (1023, 1023, 1, 1024, 2048, 1),
                          (63, 15, 4, 64, 32, 2)])
def test_static_synthesis_equals_synth(C, prec, lmax, mmax, mres, nlat, nphi, batch):
    from paper_1202_6522_gb300 import SHT
    sht = SHT(lmax, mmax, nlat, nphi, mres=mres, device=DEV)
    cdt, rdt, mode = _types(C, prec)
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (0, 1):  # two calls in a row on different inputs
        a = torch.from_numpy(synthetic.spectrum(lmax, mmax, batch=batch, seed=seed)[:, : sht.nlm]).to(DEV, cdt)
        ref = torch.empty(batch, nlat, nphi, dtype=rdt, device=DEV)
        got = torch.full((batch, nlat, nphi), float("nan"), dtype=rdt, device=DEV)
        C.sht_synth(sht._h, a.data_ptr(), ref.data_ptr(), batch, mode, stream)
        C.sht_synth_static(sht._h, a.data_ptr(), got.data_ptr(), batch, mode, stream)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_static_synthesis_on_a_fresh_handle_allocates_nothing(C, prec):
    lmax, nlat, nphi, batch = 100, 101, 256, 3
    cdt, rdt, mode = _types(C, prec)
    stream = torch.cuda.current_stream().cuda_stream
    h = C.sht_create(lmax, lmax, nlat, nphi)
    try:
        a = [torch.from_numpy(synthetic.spectrum(lmax, batch=batch, seed=s)).to(DEV, cdt) for s in (5, 6)]
        got = [torch.full((batch, nlat, nphi), float("nan"), dtype=rdt, device=DEV) for _ in a]
        with pytest.raises(C.SHTError):                     # restart states not built yet
            C.sht_synth_static(h, a[0].data_ptr(), got[0].data_ptr(), batch, mode, stream)
        C.sht_reserve(h, 1, mode)                           # builds them (and a 1-field scratch)
        # a first call may load the kernels' code (lazy module loading takes
        # device memory for it); the allocation-free property is about the calls
        C.sht_synth_static(h, a[1].data_ptr(), got[0].data_ptr(), batch, mode, stream)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for x, g in zip(a, got):
            C.sht_synth_static(h, x.data_ptr(), g.data_ptr(), batch, mode, stream)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        for x, g in zip(a, got):
            ref = torch.empty_like(g)
            C.sht_synth(h, x.data_ptr(), ref.data_ptr(), batch, mode, stream)   # allocates its scratch
            torch.cuda.synchronize()
            assert torch.equal(g, ref)
    finally:
        C.sht_destroy(h)


def test_static_synthesis_refuses_oversized_calls(C):
    from paper_1202_6522_gb300 import SHT
    sht = SHT(1023, 1023, 1024, 2048, device=DEV)
    batch = 2  # 2 fields of N = 1023 in FP64 need 32 MiB of intermediate storage
    a = torch.zeros(batch, sht.nlm, dtype=torch.complex128, device=DEV)
    g = torch.zeros(batch, 1024, 2048, dtype=torch.float64, device=DEV)
    with pytest.raises(ValueError, match="fixed"):
        C.sht_synth_static(sht._h, a.data_ptr(), g.data_ptr(), batch, C.SHT_F64,
                           torch.cuda.current_stream().cuda_stream)
