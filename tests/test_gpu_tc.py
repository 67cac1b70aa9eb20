"""Parity of the tensor-core modes (SHT_TC_BF16X3, SHT_TC_OTF) with the FP64 oracle.

The per-order Legendre contraction runs on tcgen05 against P_n^m panels
built once by the FP64 recurrence (or generated on the fly in FP32); data are
FP32.  Every comparison is element by element against the bound derived from
the split-bf16 arithmetic (tests/_bounds.py).  Cases cover several 128-row
tiles and ragged tails, mmax < lmax, odd nlat, batches split into several
chunks, the vector transforms, the adjoints, and sampled rows/orders of the
full N = 1023, batch 16 scalar and N = 511, batch 64 vector workloads."""
import numpy as np
import pytest

import oracle
from paper_1202_6522_gb300 import synthetic

import _bounds as B

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

CASES = [
    (7, 7, 8, 16, 2),
    (31, 20, 40, 64, 2),
    (40, 40, 41, 128, 3),
    (300, 300, 301, 1024, 1),
    (255, 255, 256, 512, 16),
    (100, 100, 101, 256, 40),   # 80 data columns: three 32-column slices
]
IDS = [f"N{c[0]}m{c[1]}lat{c[2]}phi{c[3]}b{c[4]}" for c in CASES]


@pytest.fixture(scope="module")
def SHT():
    from paper_1202_6522_gb300 import build
    build.build()
    from paper_1202_6522_gb300 import SHT as cls
    return cls


def _spec(lmax, mmax, batch, seed):
    return synthetic.spectrum(lmax, mmax, batch=batch, seed=seed).astype(np.complex64).astype(np.complex128)


def _grid(nlat, nphi, batch, seed):
    return synthetic.grid(nlat, nphi, batch=batch, seed=seed).astype(np.float32).astype(np.float64)


def _dev(a):
    return torch.from_numpy(a.astype(np.complex64 if np.iscomplexobj(a) else np.float32)).to(DEV)


def _np(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


@pytest.mark.parametrize("path", ["tc", "otf"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_tc_synthesis_and_analysis(SHT, case, path):
    """Panels ("tc") and on-the-fly P ("otf") against the oracle."""
    lmax, mmax, nlat, nphi, batch = case
    sht = SHT(lmax, mmax, nlat, nphi, fp32_path=path)
    a = _spec(lmax, mmax, batch, 0)
    got = _np(sht.synth_(_dev(a)))
    B.assert_synth(got, a, lmax, mmax, nlat, nphi, path, what=f"{path} synth N{lmax}b{batch}")
    g = _grid(nlat, nphi, batch, 1)
    got = _np(sht.analys_(_dev(g)))
    B.assert_analys(got, g, lmax, mmax, nlat, nphi, path, what=f"{path} analys N{lmax}b{batch}")
    assert sht.sync_status() == 0


@pytest.mark.parametrize("path", ["tc", "otf"])
@pytest.mark.parametrize("case", CASES[:4], ids=IDS[:4])
def test_tc_adjoints(SHT, case, path):
    lmax, mmax, nlat, nphi, batch = case
    sht = SHT(lmax, mmax, nlat, nphi, fp32_path=path)
    g = _grid(nlat, nphi, batch, 2)
    a = _spec(lmax, mmax, batch, 3)
    B.check_scalar_adjoints(_np(sht.synth_adj_(_dev(g))), _np(sht.analys_adj_(_dev(a))), g, a,
                            lmax, mmax, nlat, nphi, path, path)


@pytest.mark.parametrize("path", ["tc", "otf"])
def test_tc_full_size_n1023_b16_sampled(SHT, path):
    lmax, nlat, nphi, batch = 1023, 1024, 2048, 16
    sht = SHT(lmax, lmax, nlat, nphi, fp32_path=path)
    a = _spec(lmax, lmax, batch, 0)
    grid = _np(sht.synth_(_dev(a)))
    rows = [0, 1, 127, 128, 511, 512, 900, 1023]
    for b in (0, 9, 15):
        B.assert_synth(grid[b], a[b], lmax, lmax, nlat, nphi, path, rows=rows,
                       what=f"{path} synth N1023 field {b}")
    g = _grid(nlat, nphi, batch, 1)
    spec = _np(sht.analys_(_dev(g)))
    ms = [0, 1, 127, 300, 1000, 1023]
    for b in (0, 15):
        B.assert_analys(spec[b], g[b], lmax, lmax, nlat, nphi, path, ms_sel=ms,
                        what=f"{path} analys N1023 field {b}")
    assert sht.sync_status() == 0


@pytest.mark.parametrize("path", ["tc", "otf"])
def test_tc_adjoints_full_size_n1023_b16_sampled(SHT, path):
    """The adjoints at the full differentiable workload (N = 1023, batch 16):
    synth^T on sampled orders, analys^T on sampled rows, of three fields."""
    lmax, nlat, nphi, batch = 1023, 1024, 2048, 16
    sht = SHT(lmax, lmax, nlat, nphi, fp32_path=path)
    g = _grid(nlat, nphi, batch, 2)
    a = _spec(lmax, lmax, batch, 3)
    sa = _np(sht.synth_adj_(_dev(g)))
    aa = _np(sht.analys_adj_(_dev(a)))
    rows = [0, 2, 255, 511, 512, 1023]
    ms = [0, 1, 200, 777, 1023]
    for b in (0, 8, 15):
        B.check_scalar_adjoints(sa[b], aa[b], g[b], a[b], lmax, lmax, nlat, nphi, path,
                                f"{path} field {b}", rows=rows, ms_sel=ms)
    assert sht.sync_status() == 0


@pytest.mark.parametrize("path", ["tc", "otf"])
def test_tc_round_trip_error_n1023(SHT, path):
    """Sec. 3.5 error measures of the tensor-core round trip of uniform spectra:
    per coefficient on sampled orders within the bound derived from the
    arithmetic of both directions; eps_max and eps_rms over all coefficients
    stated."""
    lmax = 1023
    sht = SHT(lmax, lmax, 1024, 2048, fp32_path=path)
    Q = synthetic.spectrum(lmax, seed=0, uniform=True).astype(np.complex64).astype(np.complex128)
    R = _np(sht.analys_(sht.synth_(torch.from_numpy(Q.astype(np.complex64)).to(DEV))))
    ms = [0, 1, 10, 100, 511, 1000, 1023]
    ns_, ms_ = synthetic.packed_degrees_orders(lmax)
    sel = np.isin(ms_, ms)
    sig = B.product_sigma(path, lmax)
    bnd = B.round_trip_bounds(lmax, 1024, 2048, Q, sig, sig, ms, sigma_rep=B.data_sigma(path))
    B.check(R[sel], Q[sel], bnd[sel], f"{path} round trip N1023")
    emax, erms = oracle.eps_max_rms(R, Q, lmax)
    assert np.isfinite(emax) and erms <= emax


@pytest.mark.parametrize("path", ["tc", "otf"])
def test_tc_deterministic(SHT, path):
    sht = SHT(255, 255, 256, 512, fp32_path=path)
    a = _dev(_spec(255, 255, 4, 5))
    g1 = sht.synth_(a)
    g2 = sht.synth_(a)
    assert torch.equal(g1, g2)


VEC_CASES = [
    (7, 7, 8, 16, 2),
    (31, 20, 40, 64, 2),
    (40, 40, 41, 128, 3),
    (255, 255, 256, 512, 16),
    (100, 100, 101, 256, 40),   # one launch: field halves of 32 + 8 as adjacent CTAs
    (31, 31, 32, 64, 70),       # two launches: 64 (two full halves) + 6 fields
]
VEC_IDS = [f"N{c[0]}m{c[1]}lat{c[2]}phi{c[3]}b{c[4]}" for c in VEC_CASES]


@pytest.mark.parametrize("case", VEC_CASES, ids=VEC_IDS)
def test_tc_vector_synthesis_and_analysis(SHT, case):
    """Spheroidal/toroidal transforms with P and sin(theta) dP/dtheta panels."""
    lmax, mmax, nlat, nphi, batch = case
    sht = SHT(lmax, mmax, nlat, nphi, fp32_path="tc")
    S = synthetic.spectrum(lmax, mmax, batch=batch, seed=4, power=1.5).astype(np.complex64).astype(np.complex128)
    T = synthetic.spectrum(lmax, mmax, batch=batch, seed=5, power=1.5).astype(np.complex64).astype(np.complex128)
    vt, vp = sht.synth_vec_(_dev(S), _dev(T))
    rt, rp = oracle.synth_vec(lmax, mmax, nlat, nphi, S, T)
    gt = _grid(nlat, nphi, batch, 6)
    gp = _grid(nlat, nphi, batch, 7)
    S2, T2 = sht.analys_vec_(_dev(gt), _dev(gp))
    rS, rT = oracle.analys_vec(lmax, mmax, nlat, nphi, gt, gp)
    B.check_vector(_np(vt), _np(vp), rt, rp, S, T, _np(S2), _np(T2), rS, rT, gt, gp, lmax, mmax, nlat, nphi,
                   "tc", f"tc N{lmax}b{batch}")
    assert sht.sync_status() == 0


@pytest.mark.parametrize("case", VEC_CASES[:3], ids=VEC_IDS[:3])
def test_tc_vector_adjoints(SHT, case):
    lmax, mmax, nlat, nphi, batch = case
    sht = SHT(lmax, mmax, nlat, nphi, fp32_path="tc")
    gt = _grid(nlat, nphi, batch, 8)
    gp = _grid(nlat, nphi, batch, 9)
    S, T = sht.synth_vec_adj_(_dev(gt), _dev(gp))
    rS, rT = oracle.synth_vec_adj(lmax, mmax, nlat, nphi, gt, gp)
    A = _spec(lmax, mmax, batch, 10)
    Bs = _spec(lmax, mmax, batch, 11)
    ht, hp = sht.analys_vec_adj_(_dev(A), _dev(Bs))
    rt, rp = oracle.analys_vec_adj(lmax, mmax, nlat, nphi, A, Bs)
    B.check_vector_adjoints(_np(S), _np(T), rS, rT, gt, gp, _np(ht), _np(hp), rt, rp, A, Bs,
                            lmax, mmax, nlat, nphi, "tc", f"tc N{lmax}")


def test_tc_vector_full_size_n511_b64_sampled(SHT):
    """The vector workload (N = 511, 512 x 1024 grid, 64 fields) on sampled
    rows and orders of the oracle."""
    lmax, nlat, nphi, batch = 511, 512, 1024, 64
    sht = SHT(lmax, lmax, nlat, nphi, fp32_path="tc")
    S = synthetic.spectrum(lmax, batch=batch, seed=4, power=1.5).astype(np.complex64).astype(np.complex128)
    T = synthetic.spectrum(lmax, batch=batch, seed=5, power=1.5).astype(np.complex64).astype(np.complex128)
    vt, vp = sht.synth_vec_(_dev(S), _dev(T))
    vt, vp = _np(vt), _np(vp)
    gt = _grid(nlat, nphi, batch, 6)
    gp = _grid(nlat, nphi, batch, 7)
    S2, T2 = sht.analys_vec_(_dev(gt), _dev(gp))
    S2, T2 = _np(S2), _np(T2)
    rows = [0, 1, 127, 255, 256, 400, 511]
    ms = [0, 1, 200, 510, 511]
    for b in (0, 33, 63):
        rt, rp = oracle.synth_vec(lmax, lmax, nlat, nphi, S[b], T[b], rows=rows)
        rS, rT = oracle.analys_vec(lmax, lmax, nlat, nphi, gt[b], gp[b], ms=ms)
        B.check_vector(vt[b], vp[b], rt, rp, S[b], T[b], S2[b], T2[b], rS, rT, gt[b], gp[b],
                       lmax, lmax, nlat, nphi, "tc", f"tc vector N511 field {b}", rows=rows, ms_sel=ms)
    assert sht.sync_status() == 0


def test_tc_static_polar_skip_fraction(SHT):
    """Sec. 3.1 polar optimisation: at N = 1023 a share of the panel chunks holds
    only values below 2^-40 and is skipped; results above stay within the bound."""
    from paper_1202_6522_gb300 import _capi as C
    sht = SHT(1023, 1023, 1024, 2048, fp32_path="tc")
    assert C.sht_tc_polar_skip(sht._h) == (-1.0, -1.0)
    a = _spec(1023, 1023, 1, 0)
    g = _np(sht.synth_(_dev(a)))
    rows = [0, 5, 40, 300]
    B.assert_synth(g, a, 1023, 1023, 1024, 2048, "tc", rows=rows, what="tc polar-skip synth N1023")
    fs, fa = C.sht_tc_polar_skip(sht._h)
    assert 0.02 < fs < 0.5 and 0.02 < fa < 0.5, (fs, fa)


def test_tc_polar_threshold_api(SHT):
    """The threshold of the polar optimisation (Sec. 3.1): 0 skips nothing; a
    larger threshold skips more chunks; results stay within the bound."""
    from paper_1202_6522_gb300 import _capi as C
    lmax, nlat, nphi = 255, 256, 512
    sht = SHT(lmax, lmax, nlat, nphi, fp32_path="tc")
    a = _spec(lmax, lmax, 2, 7)
    ref = oracle.synth(lmax, lmax, nlat, nphi, a)

    def syn(what):
        B.assert_synth(_np(sht.synth_(_dev(a))), a, lmax, lmax, nlat, nphi, "tc", ref=ref, what=what)
    syn("tc polar default")
    fs0, fa0 = C.sht_tc_polar_skip(sht._h)
    C.sht_set_polar_threshold(sht._h, 0.0)
    assert C.sht_tc_polar_skip(sht._h) == (0.0, 0.0)
    syn("tc polar 0")
    # 2^-20 drops terms up to 2^-20 |P| -- above the split's rounding, so the
    # derived bound is widened by the dropped terms (at most 2^-20 each)
    C.sht_set_polar_threshold(sht._h, 2.0 ** -20)
    fs1, fa1 = C.sht_tc_polar_skip(sht._h)
    assert fs1 >= fs0 and fa1 >= fa0 and fa1 > 0
    got = _np(sht.synth_(_dev(a)))
    ns, ms = synthetic.packed_degrees_orders(lmax)
    cm = np.where(ms == 0, 1.0, 2.0)
    # dropped terms: |P| < 2^-20 each, random signs through the coefficients
    drop = B.LAMBDA * 2.0 ** -20 * np.sqrt(np.sum((cm * np.abs(a)) ** 2, axis=-1))
    bnd = B.synth_row_bounds(lmax, lmax, nlat, nphi, a, B.product_sigma("tc", lmax))
    B.check(got, ref, bnd[:, :, None] + drop[:, None, None], "tc polar 2^-20")
    g = _grid(nlat, nphi, 2, 8)
    got = _np(sht.analys_(_dev(g)))
    ref_a = oracle.analys(lmax, lmax, nlat, nphi, g)
    bnd = B.analys_coeff_bounds(lmax, lmax, nlat, nphi, g, B.product_sigma("tc", lmax))
    _, w = oracle.gauss(nlat)
    F = (2 * np.pi / nphi) * np.fft.rfft(g, axis=-1)[..., : lmax + 1]          # [b, nlat, m]
    dm = B.LAMBDA * 2.0 ** -20 * np.sqrt(np.sum((w[None, :, None] * np.abs(F)) ** 2, axis=1))
    dropa = dm[:, ms]
    B.check(got, ref_a, bnd + dropa, "tc polar 2^-20 analysis")
    for bad in (-1.0, 2.0, float("nan")):
        with pytest.raises((C.SHTError, ValueError)):
            C.sht_set_polar_threshold(sht._h, bad)


def test_alu_peaks_measured(SHT):
    from paper_1202_6522_gb300 import _capi as C
    f32, f64 = C.sht_alu_peaks(torch.cuda.current_stream().cuda_stream)
    assert 10.0 < f32 < 200.0 and 0.05 < f64 < 100.0, (f32, f64)


def test_otf_polar_threshold_and_skip(SHT):
    """The on-the-fly mode keeps its own polar-skip tables (first live chunk per
    tile, from the FP64 seeds); a threshold change rebuilds them."""
    from paper_1202_6522_gb300 import _capi as C
    lmax, nlat, nphi = 511, 512, 1024
    sht = SHT(lmax, lmax, nlat, nphi, fp32_path="otf")
    a = _spec(lmax, lmax, 2, 9)
    rows = [0, 3, 100, 255]
    ref = oracle.synth(lmax, lmax, nlat, nphi, a, rows=rows)
    B.assert_synth(_np(sht.synth_(_dev(a))), a, lmax, lmax, nlat, nphi, "otf", rows=rows, ref=ref,
                   what="otf polar default")
    fs, fa = C.sht_tc_polar_skip(sht._h)
    assert 0.0 < fs < 0.5 and 0.0 < fa < 0.5, (fs, fa)
    C.sht_set_polar_threshold(sht._h, 0.0)
    assert C.sht_tc_polar_skip(sht._h) == (0.0, 0.0)
    B.assert_synth(_np(sht.synth_(_dev(a))), a, lmax, lmax, nlat, nphi, "otf", rows=rows, ref=ref,
                   what="otf polar 0")
    g = _grid(nlat, nphi, 2, 10)
    ms = [0, 7, 300, 511]
    B.assert_analys(_np(sht.analys_(_dev(g))), g, lmax, lmax, nlat, nphi, "otf", ms_sel=ms, what="otf polar 0 analys")


def test_otf_vector_runs_panels(SHT):
    """Vector transforms in the on-the-fly mode run on the panels."""
    lmax, nlat, nphi = 31, 40, 64
    sht = SHT(lmax, 20, nlat, nphi, fp32_path="otf")
    S = synthetic.spectrum(lmax, 20, batch=2, seed=4, power=1.5).astype(np.complex64).astype(np.complex128)
    vt, vp = sht.synth_vec_(_dev(S), _dev(S))
    rt, rp = oracle.synth_vec(lmax, 20, nlat, nphi, S, S)
    bt, bp = B.synth_vec_row_bounds(lmax, 20, nlat, nphi, S, S, B.product_sigma("tc", lmax))
    B.check(_np(vt), rt, bt[:, :, None], "otf vector on panels theta")
    B.check(_np(vp), rp, bp[:, :, None], "otf vector on panels phi")
