"""Longitude grids whose FFT length nphi/2 is not a power of two (2^a 3^b 5^c).

The mixed-radix FFT (radix-16/8/4/2 passes, then 3 and 5) serves every path
for such grids; each case is compared with the FP64 oracle, whose Fourier sums
are direct and take any nphi.  Cases: H = nphi/2 = 48 (16 x 3), 60 (4 x 3 x 5),
75 (3 x 5 x 5, odd), 384 (128 x 3) and 1536 (512 x 3), in FP64, FP32, the
tensor-core paths, the vector transform, an adjoint and an uneven batch."""
import numpy as np
import pytest

import oracle
from paper_1202_6522_gb300 import synthetic

import _bounds as B
from _util import fp64_bound, normwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

CASES = [
    (31, 31, 32, 96, 2),
    (40, 40, 41, 120, 2),
    (63, 50, 64, 150, 1),
    (191, 191, 192, 768, 3),
    (511, 511, 512, 3072, 1),
]
IDS = [f"N{c[0]}m{c[1]}lat{c[2]}phi{c[3]}b{c[4]}" for c in CASES]


@pytest.fixture(scope="module")
def lib():
    from paper_1202_6522_gb300 import build
    build.build()
    import paper_1202_6522_gb300 as pkg
    return pkg


def _np(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_fp64_mixed_radix(lib, case):
    lmax, mmax, nlat, nphi, batch = case
    sht = lib.SHT(lmax, mmax, nlat, nphi)
    a = synthetic.spectrum(lmax, mmax, batch=batch, seed=0)
    got = _np(sht.synth_(torch.from_numpy(a).to(DEV)))
    assert normwise(got, oracle.synth(lmax, mmax, nlat, nphi, a)) < fp64_bound(lmax)
    g = synthetic.grid(nlat, nphi, batch=batch, seed=1)
    got = _np(sht.analys_(torch.from_numpy(g).to(DEV)))
    assert normwise(got, oracle.analys(lmax, mmax, nlat, nphi, g)) < fp64_bound(lmax)


@pytest.mark.parametrize("path", ["f32", "tc", "otf"])
@pytest.mark.parametrize("case", CASES[:4], ids=IDS[:4])
def test_fp32_paths_mixed_radix(lib, case, path):
    lmax, mmax, nlat, nphi, batch = case
    sht = lib.SHT(lmax, mmax, nlat, nphi, fp32_path=path)
    a = synthetic.spectrum(lmax, mmax, batch=batch, seed=2).astype(np.complex64)
    got = _np(sht.synth_(torch.from_numpy(a).to(DEV)))
    B.assert_synth(got, a.astype(np.complex128), lmax, mmax, nlat, nphi, path, what=f"{path} synth nphi{nphi}")
    g = synthetic.grid(nlat, nphi, batch=batch, seed=3).astype(np.float32)
    got = _np(sht.analys_(torch.from_numpy(g).to(DEV)))
    B.assert_analys(got, g.astype(np.float64), lmax, mmax, nlat, nphi, path, what=f"{path} analys nphi{nphi}")


def test_fp64_tensor_core_mixed_radix(lib):
    lmax, mmax, nlat, nphi, batch = CASES[3]
    sht = lib.SHT(lmax, mmax, nlat, nphi, fp64_path="tc")
    a = synthetic.spectrum(lmax, mmax, batch=batch, seed=4)
    got = _np(sht.synth_(torch.from_numpy(a).to(DEV)))
    assert normwise(got, oracle.synth(lmax, mmax, nlat, nphi, a)) < fp64_bound(lmax)
    g = synthetic.grid(nlat, nphi, batch=batch, seed=5)
    got = _np(sht.analys_(torch.from_numpy(g).to(DEV)))
    assert normwise(got, oracle.analys(lmax, mmax, nlat, nphi, g)) < fp64_bound(lmax)


def test_vector_and_adjoint_mixed_radix(lib):
    lmax, mmax, nlat, nphi, batch = CASES[1]
    sht = lib.SHT(lmax, mmax, nlat, nphi)
    S = synthetic.spectrum(lmax, mmax, batch=batch, seed=6)
    T = synthetic.spectrum(lmax, mmax, batch=batch, seed=7)
    vt, vp = sht.synth_vec_(torch.from_numpy(S).to(DEV), torch.from_numpy(T).to(DEV))
    rt, rp = oracle.synth_vec(lmax, mmax, nlat, nphi, S, T)
    assert normwise(_np(vt), rt) < fp64_bound(lmax) and normwise(_np(vp), rp) < fp64_bound(lmax)
    g = synthetic.grid(nlat, nphi, batch=batch, seed=8)
    got = _np(sht.synth_adj_(torch.from_numpy(g).to(DEV)))
    assert normwise(got, oracle.synth_adj(lmax, mmax, nlat, nphi, g)) < fp64_bound(lmax)


def test_uneven_batch_mixed_radix_matches_per_field(lib):
    """Fields on 3 x 2^k and 5 x 2^k grids in one batch: the batched synthesis
    equals the per-field launches bitwise (same tile function)."""
    lmaxs = [31, 47, 63, 95]
    nphis = [96, 120, 192, 240]
    ub = lib.UnevenBatch(lmaxs, nphi=nphis)
    specs = [torch.from_numpy(synthetic.spectrum(l, seed=i).astype(np.complex64)).to(DEV)
             for i, l in enumerate(lmaxs)]
    got = ub.synth_(specs)
    for l, n, s, g in zip(lmaxs, nphis, specs, got):
        ref = lib.SHT(l, l, l + 1, n).synth_(s)
        torch.cuda.synchronize()
        assert torch.equal(g, ref)
        B.assert_synth(g.cpu().numpy(), s.cpu().numpy().astype(np.complex128), l, l, l + 1, n, "f32",
                       what=f"f32 batch synth nphi{n}")


def test_unsupported_nphi_refused(lib):
    from paper_1202_6522_gb300 import _capi as C
    for nphi in (14, 2 * 7 * 16, 2 * 11):   # FFT lengths with a factor 7 or 11
        with pytest.raises(C.SHTError):
            lib.SHT(5, 5, 6, nphi)
