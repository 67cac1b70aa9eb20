"""High degree (N = 2047, nlat = 2048, nphi = 4096): the regime where P_m^m
underflows double precision near the poles and the rescaling of Sec. 3.5 is
needed.  Sampled rows/orders against the oracle (which carries an exact
extended exponent), and the Sec. 3.5 round-trip bound eps_max < 1e-11 for
N < 2048 on the FP64 path."""
import numpy as np
import pytest

import oracle
from paper_1202_6522_gb300 import synthetic

import _bounds as B
from _util import fp64_bound, normwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
N, NLAT, NPHI = 2047, 2048, 4096


@pytest.fixture(scope="module")
def SHT():
    from paper_1202_6522_gb300 import build
    build.build()
    from paper_1202_6522_gb300 import SHT as cls
    return cls


def test_n2047_fp64_sampled_and_round_trip(SHT):
    sht = SHT(N, N, NLAT, NPHI)
    Q = synthetic.spectrum(N, seed=0, uniform=True)
    g = sht.synth_(torch.from_numpy(Q).to(DEV))
    grid = g.cpu().numpy()
    rows = [0, 1, 2, 700, 1023, 1024, 2046, 2047]
    ref = oracle.synth(N, N, NLAT, NPHI, Q, rows=rows)
    assert normwise(grid[rows], ref[rows]) < fp64_bound(N)
    R = sht.analys_(g).cpu().numpy()
    emax, erms = oracle.eps_max_rms(R, Q, N)
    assert emax < 1e-11, emax
    ms = [0, 5, 1500, 2047]
    idx = np.concatenate([[oracle.lm_index(N, n, m) for n in range(m, N + 1)] for m in ms])
    refa = oracle.analys(N, N, NLAT, NPHI, grid.astype(np.float64), ms=ms)
    assert normwise(R[idx], refa[idx]) < fp64_bound(N)


def test_n2047_tensor_core_sampled(SHT):
    """The tensor-core panels come from the FP64 recurrence: the error bound
    does not grow with N."""
    sht = SHT(N, N, NLAT, NPHI, fp32_path="tc")
    a = synthetic.spectrum(N, batch=2, seed=1).astype(np.complex64)
    g = sht.synth_(torch.from_numpy(a).to(DEV)).cpu().numpy()
    rows = [0, 3, 1000, 2047]
    for b in range(2):
        B.assert_synth(g[b], a[b].astype(np.complex128), N, N, NLAT, NPHI, "tc", rows=rows,
                       what=f"tc synth N2047 field {b}")


def test_n4095_fp64_and_fp32_sampled(SHT):
    """N = 4095 (nlat 4096, nphi 8192): P_m^m spans ~13000 decimal orders of
    magnitude near the poles.  FP64 rows against the oracle and the round-trip
    error (the paper's 1e-11 statement covers N < 2048 only; bounded here by
    1e-10).  The FP32 path (exponent scale S = 64, recurrence restarted every 32
    degrees) on rows at the poles and the equator and on sampled orders of its
    analysis, within the bounds derived from its arithmetic -- the restarts
    keep the error from growing with N."""
    n, nlat, nphi = 4095, 4096, 8192
    sht = SHT(n, n, nlat, nphi)
    Q = synthetic.spectrum(n, seed=0, uniform=True)
    g = sht.synth_(torch.from_numpy(Q).to(DEV))
    grid = g.cpu().numpy()
    rows = [0, 1, 2047, 4095]
    ref = oracle.synth(n, n, nlat, nphi, Q, rows=rows)
    assert normwise(grid[rows], ref[rows]) < fp64_bound(n)
    R = sht.analys_(g).cpu().numpy()
    emax, erms = oracle.eps_max_rms(R, Q, n)
    assert emax < 1e-10 and erms < 1e-11, (emax, erms)
    del g
    Q32 = Q.astype(np.complex64).astype(np.complex128)
    g32 = sht.synth_(torch.from_numpy(Q32.astype(np.complex64)).to(DEV))
    G32 = g32.cpu().numpy()
    rows32 = [0, 1, 700, 2047, 4095]
    B.assert_synth(G32, Q32, n, n, nlat, nphi, "f32", rows=rows32, what="f32 synth N4095")
    grid32 = synthetic.grid(nlat, nphi, seed=5).astype(np.float32).astype(np.float64)
    S32 = sht.analys_(torch.from_numpy(grid32.astype(np.float32)).to(DEV)).cpu().numpy()
    B.assert_analys(S32, grid32, n, n, nlat, nphi, "f32", ms_sel=[0, 1, 2000, 4095], what="f32 analys N4095")


def test_n4095_tensor_core_sampled(SHT):
    """Tensor-core panels at N = 4095 (about 69 GB per direction): sampled rows
    of the synthesis and sampled orders of the analysis within the bound of
    the split-bf16 arithmetic (the panels come from the FP64 recurrence with
    the rescaling of Sec. 3.5, so the bound does not grow with N)."""
    n, nlat, nphi = 4095, 4096, 8192
    sht = SHT(n, n, nlat, nphi, fp32_path="tc")
    a = synthetic.spectrum(n, batch=2, seed=3).astype(np.complex64)
    g = sht.synth_(torch.from_numpy(a).to(DEV)).cpu().numpy()
    rows = [0, 1, 1500, 2047, 4095]
    for b in range(2):
        B.assert_synth(g[b], a[b].astype(np.complex128), n, n, nlat, nphi, "tc", rows=rows,
                       what=f"tc synth N4095 field {b}")
    grid = synthetic.grid(nlat, nphi, batch=2, seed=4).astype(np.float32)
    S = sht.analys_(torch.from_numpy(grid).to(DEV)).cpu().numpy()
    for b in range(2):
        B.assert_analys(S[b], grid[b].astype(np.float64), n, n, nlat, nphi, "tc", ms_sel=[0, 2, 3000, 4095],
                        what=f"tc analys N4095 field {b}")
    assert sht.sync_status() == 0
