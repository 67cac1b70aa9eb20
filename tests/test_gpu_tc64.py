"""Parity of the FP64-accurate tensor-core mode (SHT_TC_F64) with the FP64 oracle.

Both operands of each per-order contraction are split into signed 7-bit digit
slices (7 for P per row, 8 for the data per field) whose integer products the
tensor core sums exactly; the bound is the FP64 path's, 1e-11 normwise.  Cases cover
several 128-row tiles and ragged tails, mmax < lmax, odd nlat, batches of more
than 16 fields (several launches), the adjoints, sampled rows/orders of the
full N = 1023, batch 16 workload, exact power-of-two scaling and the size
limit."""
import numpy as np
import pytest

import oracle
from paper_1202_6522_gb300 import synthetic

from _util import fp64_bound, normwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

CASES = [
    (7, 7, 8, 16, 2),
    (31, 20, 40, 64, 2),
    (40, 40, 41, 128, 3),
    (300, 300, 301, 1024, 1),
    (255, 255, 256, 512, 16),
    (100, 100, 101, 256, 20),   # two launches: 16 + 4 fields
]
IDS = [f"N{c[0]}m{c[1]}lat{c[2]}phi{c[3]}b{c[4]}" for c in CASES]


@pytest.fixture(scope="module")
def SHT():
    from paper_1202_6522_gb300 import build
    build.build()
    from paper_1202_6522_gb300 import SHT as cls
    return cls


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_tc64_synthesis_and_analysis(SHT, case):
    lmax, mmax, nlat, nphi, batch = case
    sht = SHT(lmax, mmax, nlat, nphi, fp64_path="tc")
    a = synthetic.spectrum(lmax, mmax, batch=batch, seed=0)
    got = _np(sht.synth_(torch.from_numpy(a).to(DEV)))
    assert normwise(got, oracle.synth(lmax, mmax, nlat, nphi, a)) < fp64_bound(lmax)
    g = synthetic.grid(nlat, nphi, batch=batch, seed=1)
    got = _np(sht.analys_(torch.from_numpy(g).to(DEV)))
    assert normwise(got, oracle.analys(lmax, mmax, nlat, nphi, g)) < fp64_bound(lmax)
    assert sht.sync_status() == 0


@pytest.mark.parametrize("case", CASES[:4], ids=IDS[:4])
def test_tc64_adjoints(SHT, case):
    lmax, mmax, nlat, nphi, batch = case
    sht = SHT(lmax, mmax, nlat, nphi, fp64_path="tc")
    g = synthetic.grid(nlat, nphi, batch=batch, seed=2)
    a = synthetic.spectrum(lmax, mmax, batch=batch, seed=3)
    got = _np(sht.synth_adj_(torch.from_numpy(g).to(DEV)))
    assert normwise(got, oracle.synth_adj(lmax, mmax, nlat, nphi, g)) < fp64_bound(lmax)
    got = _np(sht.analys_adj_(torch.from_numpy(a).to(DEV)))
    assert normwise(got, oracle.analys_adj(lmax, mmax, nlat, nphi, a)) < fp64_bound(lmax)


def test_tc64_full_size_n1023_b16_sampled(SHT):
    lmax, nlat, nphi, batch = 1023, 1024, 2048, 16
    sht = SHT(lmax, lmax, nlat, nphi, fp64_path="tc")
    a = synthetic.spectrum(lmax, batch=batch, seed=0)
    grid = _np(sht.synth_(torch.from_numpy(a).to(DEV)))
    rows = [0, 1, 127, 128, 511, 512, 900, 1023]
    for b in (0, 15):
        ref = oracle.synth(lmax, lmax, nlat, nphi, a[b], rows=rows)
        assert normwise(grid[b][rows], ref[rows]) < fp64_bound(lmax), b
    g = synthetic.grid(nlat, nphi, batch=batch, seed=1)
    spec = _np(sht.analys_(torch.from_numpy(g).to(DEV)))
    ms = [0, 1, 127, 300, 1000, 1023]
    idx = np.concatenate([[oracle.lm_index(lmax, n, m) for n in range(m, lmax + 1)] for m in ms])
    for b in (0, 15):
        ref = oracle.analys(lmax, lmax, nlat, nphi, g[b], ms=ms)
        assert normwise(spec[b][idx], ref[idx]) < fp64_bound(lmax), b
    assert sht.sync_status() == 0
    # all-zero digit chunks (high orders near the poles) are reported and skipped
    from paper_1202_6522_gb300 import _capi as C
    fs, fa = C.sht_tc_polar_skip(sht._h)
    assert 0.0 < fs < 0.5 and 0.0 < fa < 0.5


def test_tc64_n511_b16_sampled(SHT):
    """N = 511, batch 16 (panels larger than L2): sampled rows and orders."""
    lmax, nlat, nphi, batch = 511, 512, 1024, 16
    sht = SHT(lmax, lmax, nlat, nphi, fp64_path="tc")
    a = synthetic.spectrum(lmax, batch=batch, seed=4)
    grid = _np(sht.synth_(torch.from_numpy(a).to(DEV)))
    rows = [0, 5, 255, 256, 400, 511]
    ref = oracle.synth(lmax, lmax, nlat, nphi, a[7], rows=rows)
    assert normwise(grid[7][rows], ref[rows]) < fp64_bound(lmax)
    g = synthetic.grid(nlat, nphi, batch=batch, seed=5)
    spec = _np(sht.analys_(torch.from_numpy(g).to(DEV)))
    ms = [0, 3, 200, 511]
    idx = np.concatenate([[oracle.lm_index(lmax, n, m) for n in range(m, lmax + 1)] for m in ms])
    ref = oracle.analys(lmax, lmax, nlat, nphi, g[11], ms=ms)
    assert normwise(spec[11][idx], ref[idx]) < fp64_bound(lmax)
    assert sht.sync_status() == 0


def test_tc64_round_trip_error_n1023(SHT):
    """Sec. 3.5 error measures of the round trip, at the FP64 path's level."""
    lmax = 1023
    sht = SHT(lmax, lmax, 1024, 2048, fp64_path="tc")
    Q = synthetic.spectrum(lmax, seed=0, uniform=True)
    R = _np(sht.analys_(sht.synth_(torch.from_numpy(Q).to(DEV))))
    emax, erms = oracle.eps_max_rms(R, Q, lmax)
    assert emax < 1e-11 and erms < 1e-12


def test_tc64_matches_fp64_path_and_is_deterministic(SHT):
    sht_tc = SHT(255, 255, 256, 512, fp64_path="tc")
    sht_64 = SHT(255, 255, 256, 512)
    a = torch.from_numpy(synthetic.spectrum(255, batch=4, seed=5)).to(DEV)
    g1 = sht_tc.synth_(a)
    g2 = sht_tc.synth_(a)
    assert torch.equal(g1, g2)
    assert normwise(_np(g1), _np(sht_64.synth_(a))) < fp64_bound(255)


def test_tc64_vector_runs_fp64_recurrence(SHT):
    """Vector transforms in this mode take the FP64 recurrence path."""
    lmax, nlat, nphi = 31, 32, 64
    sht_tc = SHT(lmax, lmax, nlat, nphi, fp64_path="tc")
    sht_64 = SHT(lmax, lmax, nlat, nphi)
    S = torch.from_numpy(synthetic.spectrum(lmax, batch=2, seed=6)).to(DEV)
    T = torch.from_numpy(synthetic.spectrum(lmax, batch=2, seed=7)).to(DEV)
    vt1, vp1 = sht_tc.synth_vec_(S, T)
    vt2, vp2 = sht_64.synth_vec_(S, T)
    assert torch.equal(vt1, vt2) and torch.equal(vp1, vp2)


def test_tc64_size_limit(SHT):
    """lmax > 1023 would let a level's integer sum pass 2^24: refused."""
    from paper_1202_6522_gb300 import _capi as C
    sht = SHT(1100, 1100, 1101, 4096, fp64_path="tc")
    a = torch.zeros(1, sht.nlm, dtype=torch.complex128, device=DEV)
    with pytest.raises(C.SHTError):
        sht.synth_(a)


def test_tc64_power_of_two_scaling_is_exact(SHT):
    """Inputs scaled by 2^-600 or 2^600 (far outside FP32's range) give outputs
    scaled by the same power, bit for bit: the contraction scales each field and
    the double-float FFT each latitude pair by a power of two taken from the
    FP64 exponents, so only those exponents move."""
    lmax, nlat, nphi = 63, 64, 128
    sht = SHT(lmax, lmax, nlat, nphi, fp64_path="tc")
    a = torch.from_numpy(synthetic.spectrum(lmax, batch=3, seed=8)).to(DEV)
    g = sht.synth_(a)
    x = torch.from_numpy(synthetic.grid(nlat, nphi, batch=3, seed=9)).to(DEV)
    s = sht.analys_(x)
    for k in (-600, 600):
        assert torch.equal(sht.synth_(a * 2.0 ** k), g * 2.0 ** k), k
        assert torch.equal(sht.analys_(x * 2.0 ** k), s * 2.0 ** k), k
    assert normwise(_np(g), oracle.synth(lmax, lmax, nlat, nphi, _np(a))) < fp64_bound(lmax)
