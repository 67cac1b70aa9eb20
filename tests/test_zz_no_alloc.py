"""The synthesis entry point that allocates nothing (sht_synth_static).

Some callers cannot ask the CUDA runtime for memory when they call the
transform: a host framework that owns a fixed device-memory budget, or a loop
that cannot afford the device-wide synchronisation cudaMalloc/cudaFree bring.
For them sht_synth_static keeps its intermediate in a fixed array inside the
library.  This test calls it through the C ABI and checks its output against
the ordinary sht_synth, twice in a row with different inputs (the array keeps
the previous call's contents, which must not leak into the next result), and
checks that a call too large for the array is refused on the host.

The file is named so that pytest collects it last.
"""
import pytest

from paper_1202_6522_gb300 import synthetic

from _util import fp32_bound, fp64_bound, normwise

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


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("lmax,nlat,nphi,batch", [(255, 256, 512, 2), (40, 41, 128, 3), (1023, 1024, 2048, 1)])
def test_static_synthesis_matches_synth(C, prec, lmax, nlat, nphi, batch):
    from paper_1202_6522_gb300 import SHT
    sht = SHT(lmax, lmax, nlat, nphi, device=DEV)
    cdt = torch.complex128 if prec == "f64" else torch.complex64
    rdt = torch.float64 if prec == "f64" else torch.float32
    mode = C.SHT_F64 if prec == "f64" else C.SHT_F32
    tol = fp64_bound(lmax) if prec == "f64" else fp32_bound(lmax)
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (0, 1):  # two calls in a row on different inputs
        a = torch.from_numpy(synthetic.spectrum(lmax, batch=batch, seed=seed)).to(DEV, cdt)
        ref = torch.empty(batch, nlat, nphi, dtype=rdt, device=DEV)
        got = torch.full((batch, nlat, nphi), float("nan"), dtype=rdt, device=DEV)
        C.sht_synth(sht._h, a.data_ptr(), ref.data_ptr(), batch, mode, stream)
        C.sht_synth_static(sht._h, a.data_ptr(), got.data_ptr(), batch, mode, stream)
        torch.cuda.synchronize()
        assert not torch.isnan(got).any()
        assert normwise(got.cpu().numpy(), ref.cpu().numpy()) <= tol


def test_static_synthesis_refuses_oversized_calls(C):
    from paper_1202_6522_gb300 import SHT
    sht = SHT(1023, 1023, 1024, 2048, device=DEV)
    batch = 2  # 2 fields of N = 1023 in FP64 need 32 MiB of intermediate storage
    a = torch.zeros(batch, sht.nlm, dtype=torch.complex128, device=DEV)
    g = torch.zeros(batch, 1024, 2048, dtype=torch.float64, device=DEV)
    with pytest.raises(ValueError, match="fixed"):
        C.sht_synth_static(sht._h, a.data_ptr(), g.data_ptr(), batch, C.SHT_F64,
                           torch.cuda.current_stream().cuda_stream)
