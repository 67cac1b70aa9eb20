"""Static polar optimisation of the on-the-fly CUDA-core kernels (Sec. 3.1).

Per (order, latitude pair) the plan keeps the first 32-degree segment in
which |P_n^m| reaches a threshold; the kernels run neither the recurrence nor
the sums of a segment for a group of 32 pairs (one per lane of a warp) none of
which is live yet.  Checked against the FP64 oracle, FP64 and
FP32, synthesis and analysis (the FP64 analysis at 8 fields runs the
warp-per-segment kernel):

* with the default thresholds (2^-64 FP64, 2^-40 FP32) and with threshold 0
  (nothing skipped) the results stay within the paths' usual bounds;
* at 2^-20 terms are dropped -- the results move away from those at 0 -- but
  by no more than the dropped terms allow: |P| < 2^-20 each, so at most
  2^-20 sum c_m |f_n^m| for a synthesis value and 2^-20 sum_j w_j |F_m(x_j)|
  for an analysis coefficient (hard bounds, no statistical factor).
"""
import numpy as np
import pytest

import oracle
from paper_1202_6522_gb300 import synthetic

import _bounds as B
from _util import fp64_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
LMAX, NLAT, NPHI, BATCH = 255, 256, 512, 8
THR = 2.0 ** -20


@pytest.fixture(scope="module")
def SHT():
    from paper_1202_6522_gb300 import build
    build.build()
    from paper_1202_6522_gb300 import SHT as cls
    return cls


@pytest.fixture(scope="module")
def data():
    a = synthetic.spectrum(LMAX, batch=BATCH, seed=31)
    g = synthetic.grid(NLAT, NPHI, batch=BATCH, seed=32)
    return a, g, oracle.synth(LMAX, LMAX, NLAT, NPHI, a), oracle.analys(LMAX, LMAX, NLAT, NPHI, g)


def _dev(x, prec):
    if np.iscomplexobj(x):
        return torch.from_numpy(x.astype(np.complex128 if prec == "f64" else np.complex64)).to(DEV)
    return torch.from_numpy(x.astype(np.float64 if prec == "f64" else np.float32)).to(DEV)


def _np(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


def _inputs(a, g, prec):
    if prec == "f32":   # the FP32 path sees FP32 inputs; the oracle the same values
        a = a.astype(np.complex64).astype(np.complex128)
        g = g.astype(np.float32).astype(np.float64)
    return a, g


def _drops(a, g):
    ns, ms = synthetic.packed_degrees_orders(LMAX)
    cm = np.where(ms == 0, 1.0, 2.0)
    drop_s = THR * np.sum(cm * np.abs(a), axis=-1)                       # [B]
    _, w = oracle.gauss(NLAT)
    F = (2 * np.pi / NPHI) * np.fft.rfft(g, axis=-1)[..., : LMAX + 1]   # [B, nlat, m]
    drop_a = THR * np.sum(w[None, :, None] * np.abs(F), axis=1)[:, ms]   # [B, nlm]
    return drop_s, drop_a


def _check(prec, got_s, got_a, a, g, ref_s, ref_a, drop_s=0.0, drop_a=0.0, what=""):
    if prec == "f64":
        tol_s = fp64_bound(LMAX) * np.abs(ref_s).max()
        tol_a = fp64_bound(LMAX) * np.abs(ref_a).max()
        B.check(got_s, ref_s, tol_s + np.asarray(drop_s).reshape(-1, 1, 1), what + " synthesis")
        B.check(got_a, ref_a, tol_a + drop_a, what + " analysis")
    else:
        bs = B.synth_row_bounds(LMAX, LMAX, NLAT, NPHI, a, B.product_sigma("f32", LMAX))
        ba = B.analys_coeff_bounds(LMAX, LMAX, NLAT, NPHI, g, B.product_sigma("f32", LMAX))
        B.check(got_s, ref_s, bs[:, :, None] + np.asarray(drop_s).reshape(-1, 1, 1), what + " synthesis")
        B.check(got_a, ref_a, ba + drop_a, what + " analysis")


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_cuda_core_polar_threshold(SHT, data, prec):
    from paper_1202_6522_gb300 import _capi as C
    a0, g0, ref_s0, ref_a0 = data
    a, g = _inputs(a0, g0, prec)
    ref_s = ref_s0 if prec == "f64" else oracle.synth(LMAX, LMAX, NLAT, NPHI, a)
    ref_a = ref_a0 if prec == "f64" else oracle.analys(LMAX, LMAX, NLAT, NPHI, g)
    sht = SHT(LMAX, LMAX, NLAT, NPHI, device=DEV)

    def run():
        return _np(sht.synth_(_dev(a, prec))), _np(sht.analys_(_dev(g, prec)))

    mode = C.SHT_F64 if prec == "f64" else C.SHT_F32
    assert C.sht_cc_polar_skip(sht._h, mode) == -1.0           # no table before the first call
    s_def, a_def = run()
    f_def = C.sht_cc_polar_skip(sht._h, mode)
    assert 0.0 < f_def < 0.5, f_def
    _check(prec, s_def, a_def, a, g, ref_s, ref_a, what=f"{prec} polar default")
    C.sht_set_polar_threshold(sht._h, 0.0)
    assert C.sht_cc_polar_skip(sht._h, mode) == 0.0
    s_0, a_0 = run()
    _check(prec, s_0, a_0, a, g, ref_s, ref_a, what=f"{prec} polar 0")
    C.sht_set_polar_threshold(sht._h, THR)
    assert C.sht_cc_polar_skip(sht._h, mode) > f_def
    s_t, a_t = run()
    drop_s, drop_a = _drops(a, g)
    _check(prec, s_t, a_t, a, g, ref_s, ref_a, drop_s, drop_a, what=f"{prec} polar 2^-20")
    # terms were dropped: the results differ from those with nothing skipped
    assert np.abs(s_t - s_0).max() > 0 and np.abs(a_t - a_0).max() > 0


def test_fp64_segment_analysis_field_groups(SHT, data):
    """The warp-per-segment FP64 analysis at every field-group width (1, 2,
    4, 8 fields per CTA) and a ragged batch: the same coefficients as the
    oracle, and bitwise the same across repeated calls."""
    from paper_1202_6522_gb300 import _capi as C
    _, g, _, ref_a = data
    sht = SHT(LMAX, LMAX, NLAT, NPHI, device=DEV)
    for nb in (1, 2, 3, 5, 8):
        x = _dev(g[:nb], "f64")
        got = _np(sht.analys_(x))
        again = _np(sht.analys_(x))
        assert np.array_equal(got, again)
        B.check(got, ref_a[:nb], fp64_bound(LMAX) * np.abs(ref_a[:nb]).max(), f"f64 segment analysis b{nb}")
    C.sht_tune(sht._h, 8, C.SHT_F64, torch.cuda.current_stream().cuda_stream)
    B.check(_np(sht.analys_(_dev(g, "f64"))), ref_a, fp64_bound(LMAX) * np.abs(ref_a).max(), "f64 tuned analysis")


def test_fp64_team_analysis_beyond_512_pairs(SHT):
    """More latitude pairs than one warp holds (551 here): each segment is
    summed by a team of warps whose partial sums meet in shared memory.
    Sampled orders against the oracle at every field-group width (1, 2 and 4
    fields per CTA, ragged batches), bitwise the same across repeated calls."""
    lmax, nlat, nphi = 1100, 1101, 2304
    ms = [0, 1, 257, 550, 1100]
    g = synthetic.grid(nlat, nphi, batch=5, seed=41)
    ref = oracle.analys(lmax, lmax, nlat, nphi, g, ms=ms)
    ns, mm = synthetic.packed_degrees_orders(lmax)
    sel = np.isin(mm, ms)
    sht = SHT(lmax, lmax, nlat, nphi, device=DEV)
    for nb in (1, 3, 5):
        x = _dev(g[:nb], "f64")
        got = _np(sht.analys_(x))
        assert np.array_equal(got, _np(sht.analys_(x)))
        r = ref.reshape(5, -1)[:nb][:, sel]
        B.check(got[:, sel], r, fp64_bound(lmax) * np.abs(r).max(), f"f64 team analysis b{nb}")
