"""Parity of the CUDA transforms (through the C ABI) with the FP64 CPU oracle.

Each case draws seeded synthetic inputs, runs the GPU path and the oracle on
the same values and compares element by element: the FP64 path normwise
(max |gpu - oracle| over max |oracle| below 1e-11, Sec. 3.5), the FP32 path
against the per-element bound derived from its arithmetic (tests/_bounds.py).
Sizes span several latitude blocks and ragged tails; full-size cases compare
sampled rows/orders the oracle computes one by one.
"""
import numpy as np
import pytest

import oracle
from paper_1202_6522_gb300 import synthetic

import _bounds as B
from _util import fp64_bound, normwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def SHT():
    from paper_1202_6522_gb300 import build
    build.build()
    from paper_1202_6522_gb300 import SHT as cls
    return cls


DEV = "cuda:0"

# (lmax, mmax, nlat, nphi, batch): tiny, odd nlat, mmax < lmax, ragged batch,
# several pair blocks with a ragged tail, and N = 255
CASES = [
    (0, 0, 1, 2, 1),
    (1, 1, 2, 4, 1),
    (7, 7, 8, 16, 1),
    (31, 31, 32, 64, 1),
    (31, 31, 33, 64, 3),
    (31, 20, 40, 64, 2),
    (40, 40, 41, 128, 5),
    (300, 300, 301, 1024, 1),
    (255, 255, 256, 512, 2),
]
IDS = [f"N{c[0]}m{c[1]}lat{c[2]}phi{c[3]}b{c[4]}" for c in CASES]


def _tol(lmax, prec):
    return fp64_bound(lmax)


def _spec(lmax, mmax, batch, seed, prec, power=1.0):
    a = synthetic.spectrum(lmax, mmax, batch=batch, seed=seed, power=power)
    if prec == "f32":
        a = a.astype(np.complex64).astype(np.complex128)
    return a


def _grid(nlat, nphi, batch, seed, prec):
    g = synthetic.grid(nlat, nphi, batch=batch, seed=seed)
    if prec == "f32":
        g = g.astype(np.float32).astype(np.float64)
    return g


def _to_dev(a, prec):
    if np.iscomplexobj(a):
        return torch.from_numpy(a.astype(np.complex128 if prec == "f64" else np.complex64)).to(DEV)
    return torch.from_numpy(a.astype(np.float64 if prec == "f64" else np.float32)).to(DEV)


def _np(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_scalar_synthesis(SHT, case, prec):
    lmax, mmax, nlat, nphi, batch = case
    sht = SHT(lmax, mmax, nlat, nphi)
    a = _spec(lmax, mmax, batch, 0, prec)
    got = _np(sht.synth_(_to_dev(a, prec)))
    ref = oracle.synth(lmax, mmax, nlat, nphi, a)
    if prec == "f64":
        assert normwise(got, ref) < _tol(lmax, prec)
    else:
        B.assert_synth(got, a, lmax, mmax, nlat, nphi, "f32", ref=ref, what=f"f32 synth N{lmax}")


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_scalar_analysis(SHT, case, prec):
    lmax, mmax, nlat, nphi, batch = case
    sht = SHT(lmax, mmax, nlat, nphi)
    g = _grid(nlat, nphi, batch, 1, prec)
    got = _np(sht.analys_(_to_dev(g, prec)))
    ref = oracle.analys(lmax, mmax, nlat, nphi, g)
    if prec == "f64":
        assert normwise(got, ref) < _tol(lmax, prec)
    else:
        B.assert_analys(got, g, lmax, mmax, nlat, nphi, "f32", ref=ref, what=f"f32 analys N{lmax}")


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_scalar_adjoints(SHT, case, prec):
    lmax, mmax, nlat, nphi, batch = case
    sht = SHT(lmax, mmax, nlat, nphi)
    g = _grid(nlat, nphi, batch, 2, prec)
    a = _spec(lmax, mmax, batch, 3, prec)
    got_sa = _np(sht.synth_adj_(_to_dev(g, prec)))
    got_aa = _np(sht.analys_adj_(_to_dev(a, prec)))
    if prec == "f64":
        assert normwise(got_sa, oracle.synth_adj(lmax, mmax, nlat, nphi, g)) < _tol(lmax, prec)
        assert normwise(got_aa, oracle.analys_adj(lmax, mmax, nlat, nphi, a)) < _tol(lmax, prec)
    else:
        B.check_scalar_adjoints(got_sa, got_aa, g, a, lmax, mmax, nlat, nphi, "f32", "f32")


VEC_CASES = [c for c in CASES if c[0] >= 1]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("case", VEC_CASES, ids=[i for c, i in zip(CASES, IDS) if c[0] >= 1])
def test_vector_synthesis_and_analysis(SHT, case, prec):
    lmax, mmax, nlat, nphi, batch = case
    sht = SHT(lmax, mmax, nlat, nphi)
    S = _spec(lmax, mmax, batch, 4, prec, power=1.5)
    T = _spec(lmax, mmax, batch, 5, prec, power=1.5)
    vt, vp = sht.synth_vec_(_to_dev(S, prec), _to_dev(T, prec))
    rt, rp = oracle.synth_vec(lmax, mmax, nlat, nphi, S, T)
    gt = _grid(nlat, nphi, batch, 6, prec)
    gp = _grid(nlat, nphi, batch, 7, prec)
    S2, T2 = sht.analys_vec_(_to_dev(gt, prec), _to_dev(gp, prec))
    rS, rT = oracle.analys_vec(lmax, mmax, nlat, nphi, gt, gp)
    if prec == "f64":
        tol = _tol(lmax, prec)
        assert normwise(_np(vt), rt) < tol
        assert normwise(_np(vp), rp) < tol
        assert normwise(_np(S2), rS) < tol
        assert normwise(_np(T2), rT) < tol
    else:
        B.check_vector(_np(vt), _np(vp), rt, rp, S, T, _np(S2), _np(T2), rS, rT, gt, gp,
                     lmax, mmax, nlat, nphi, "f32", "f32")


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("case", VEC_CASES, ids=[i for c, i in zip(CASES, IDS) if c[0] >= 1])
def test_vector_adjoints(SHT, case, prec):
    lmax, mmax, nlat, nphi, batch = case
    sht = SHT(lmax, mmax, nlat, nphi)
    gt = _grid(nlat, nphi, batch, 8, prec)
    gp = _grid(nlat, nphi, batch, 9, prec)
    S, T = sht.synth_vec_adj_(_to_dev(gt, prec), _to_dev(gp, prec))
    rS, rT = oracle.synth_vec_adj(lmax, mmax, nlat, nphi, gt, gp)
    A = _spec(lmax, mmax, batch, 10, prec)
    Bs = _spec(lmax, mmax, batch, 11, prec)
    ht, hp = sht.analys_vec_adj_(_to_dev(A, prec), _to_dev(Bs, prec))
    rt, rp = oracle.analys_vec_adj(lmax, mmax, nlat, nphi, A, Bs)
    if prec == "f64":
        tol = _tol(lmax, prec)
        assert normwise(_np(S), rS) < tol
        assert normwise(_np(T), rT) < tol
        assert normwise(_np(ht), rt) < tol
        assert normwise(_np(hp), rp) < tol
    else:
        B.check_vector_adjoints(_np(S), _np(T), rS, rT, gt, gp, _np(ht), _np(hp), rt, rp, A, Bs,
                              lmax, mmax, nlat, nphi, "f32", "f32")


def test_round_trip_accuracy_fp64_n255(SHT):
    """Sec. 3.5: eps_max < 1e-11 for N < 2048 -- checked on the GPU FP64 path."""
    lmax = 255
    sht = SHT(lmax, lmax, 256, 512)
    Q = synthetic.spectrum(lmax, seed=0, uniform=True)
    R = _np(sht.analys_(sht.synth_(_to_dev(Q, "f64"))))
    emax, erms = oracle.eps_max_rms(R, Q, lmax)
    assert emax < 1e-11 and erms < 1e-12


def test_outputs_fully_written_and_deterministic(SHT):
    lmax, nlat, nphi, batch = 40, 41, 128, 3
    sht = SHT(lmax, lmax, nlat, nphi)
    a = _to_dev(_spec(lmax, lmax, batch, 12, "f64"), "f64")
    g1 = torch.full((batch, nlat, nphi), float("nan"), dtype=torch.float64, device=DEV)
    from paper_1202_6522_gb300 import _capi as C
    C.sht_synth(sht._h, a.data_ptr(), g1.data_ptr(), batch, C.SHT_F64, torch.cuda.current_stream().cuda_stream)
    g2 = sht.synth_(a)
    torch.cuda.synchronize()
    assert not torch.isnan(g1).any()
    assert torch.equal(g1, g2)
    s1 = sht.analys_(g1)
    s2 = sht.analys_(g1)
    assert torch.equal(s1, s2)


# --------------------------------------------------------------------------
# Full-size cases: N = 1023, nlat = 1024, nphi = 2048, batch 16 (sampled)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_full_size_n1023_sampled(SHT, prec):
    lmax, nlat, nphi, batch = 1023, 1024, 2048, 16
    sht = SHT(lmax, lmax, nlat, nphi)
    a = _spec(lmax, lmax, batch, 0, prec)
    grid = _np(sht.synth_(_to_dev(a, prec)))
    rows = [0, 1, 255, 511, 512, 1000, 1023]
    tol = _tol(lmax, prec)
    for b in (0, 7, 15):
        ref = oracle.synth(lmax, lmax, nlat, nphi, a[b], rows=rows)
        if prec == "f64":
            assert normwise(grid[b][rows], ref[rows]) < tol, b
        else:
            B.assert_synth(grid[b], a[b], lmax, lmax, nlat, nphi, "f32", rows=rows, ref=ref,
                           what=f"f32 synth N{lmax} field {b}")
    g = _grid(nlat, nphi, batch, 1, prec)
    spec = _np(sht.analys_(_to_dev(g, prec)))
    ms = [0, 1, 100, 511, 900, 1023]
    idx = np.concatenate([[oracle.lm_index(lmax, n, m) for n in range(m, lmax + 1)] for m in ms])
    for b in (0, 15):
        ref = oracle.analys(lmax, lmax, nlat, nphi, g[b], ms=ms)
        if prec == "f64":
            assert normwise(spec[b][idx], ref[idx]) < tol, b
        else:
            B.assert_analys(spec[b], g[b], lmax, lmax, nlat, nphi, "f32", ms_sel=ms, ref=ref,
                            what=f"f32 analys N{lmax} field {b}")


def test_full_size_round_trip_fp64_n1023(SHT):
    """eps_max < 1e-11 (Sec. 3.5) for a full N = 1023 round trip on the GPU."""
    lmax = 1023
    sht = SHT(lmax, lmax, 1024, 2048)
    Q = synthetic.spectrum(lmax, seed=0, uniform=True)
    R = _np(sht.analys_(sht.synth_(_to_dev(Q, "f64"))))
    emax, erms = oracle.eps_max_rms(R, Q, lmax)
    assert emax < 1e-11, emax


def test_fp32_round_trip_n1023_equals_fp64_within_bound(SHT):
    """N = 1023 in FP32 (P_m^m far below the FP32 range near the poles, so the
    exponent scale of Sec. 3.5 is in use, and the recurrence restarted every 32
    degrees): the round trip of uniform spectra (Sec. 3.5) equals the FP64 GPU
    path's, coefficient by coefficient on sampled orders, within the bound
    derived from the FP32 arithmetic."""
    lmax = 1023
    sht = SHT(lmax, lmax, 1024, 2048)
    Q = synthetic.spectrum(lmax, seed=0, uniform=True).astype(np.complex64).astype(np.complex128)
    R32 = _np(sht.analys_(sht.synth_(torch.from_numpy(Q.astype(np.complex64)).to(DEV))))
    R64 = _np(sht.analys_(sht.synth_(_to_dev(Q, "f64"))))
    assert oracle.eps_max_rms(R64, Q, lmax)[0] < 1e-11
    ms = [0, 1, 10, 100, 511, 1000, 1023]
    ns_, ms_ = synthetic.packed_degrees_orders(lmax)
    sel = np.isin(ms_, ms)
    sig = B.product_sigma("f32", lmax)
    bnd = B.round_trip_bounds(lmax, 1024, 2048, Q, sig, sig, ms)
    B.check(R32[sel], R64[sel], bnd[sel], "f32 round trip N1023")


def test_invalid_arguments_raise(SHT):
    with pytest.raises(ValueError):
        SHT(10, 11, 16, 32)
    sht = SHT(7, 7, 8, 16)
    with pytest.raises(ValueError):
        sht.synth_(torch.zeros(5, dtype=torch.complex128, device=DEV))
