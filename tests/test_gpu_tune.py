"""Runtime tuning (the analogue of the paper's runtime tuning in Sec. 3.2):
tuned kernel shapes must leave results unchanged within tolerance, and the
automatic FP32 mode must pick one of its two paths and stay accurate."""
import numpy as np
import pytest

import oracle
from paper_1202_6522_gb300 import synthetic

import _bounds as B
from _util import fp64_bound, normwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def lib():
    from paper_1202_6522_gb300 import build
    build.build()
    import paper_1202_6522_gb300 as P
    from paper_1202_6522_gb300 import _capi
    return P, _capi


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_tuned_shapes_keep_results(lib, prec):
    P, C = lib
    lmax, nlat, nphi, batch = 95, 96, 256, 5
    sht = P.SHT(lmax, lmax, nlat, nphi)
    mode = C.SHT_F64 if prec == "f64" else C.SHT_F32
    syn_ms, ana_ms, none = C.sht_tune(sht._h, batch, mode, torch.cuda.current_stream().cuda_stream)
    assert syn_ms > 0 and ana_ms > 0 and none == -1.0
    cdt = torch.complex128 if prec == "f64" else torch.complex64
    a = synthetic.spectrum(lmax, batch=batch, seed=3)
    if prec == "f32":
        a = a.astype(np.complex64).astype(np.complex128)
    g = sht.synth_(torch.from_numpy(a).to(DEV, cdt))
    ref = oracle.synth(lmax, lmax, nlat, nphi, a)
    r = sht.analys_(g)
    gn = g.cpu().numpy().astype(np.float64)
    refa = oracle.analys(lmax, lmax, nlat, nphi, gn)
    if prec == "f64":
        assert normwise(g.cpu().numpy(), ref) < fp64_bound(lmax)
        assert normwise(r.cpu().numpy(), refa) < fp64_bound(lmax)
    else:
        B.assert_synth(g.cpu().numpy(), a, lmax, lmax, nlat, nphi, "f32", ref=ref, what="tuned f32 synth")
        B.assert_analys(r.cpu().numpy(), gn, lmax, lmax, nlat, nphi, "f32", ref=refa, what="tuned f32 analys")


def test_auto_mode_chooses_a_path(lib):
    P, C = lib
    lmax, nlat, nphi, batch = 127, 128, 256, 8
    sht = P.SHT(lmax, lmax, nlat, nphi)
    f32_ms, tc_ms, otf_ms = C.sht_tune(sht._h, batch, C.SHT_F32_AUTO, torch.cuda.current_stream().cuda_stream)
    assert f32_ms > 0 and tc_ms > 0 and otf_ms > 0
    sht.fp32_mode = C.SHT_F32_AUTO
    a = synthetic.spectrum(lmax, batch=batch, seed=4).astype(np.complex64)
    g = sht.synth_(torch.from_numpy(a).to(DEV))
    chosen = min((f32_ms, "f32"), (tc_ms, "tc"), (otf_ms, "otf"))[1]
    B.assert_synth(g.cpu().numpy(), a.astype(np.complex128), lmax, lmax, nlat, nphi, chosen,
                   what=f"auto ({chosen}) synth")
