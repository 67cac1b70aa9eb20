"""The m-stride variant (orders m = k mres only, one 2 pi / mres sector of longitudes),
on the FP64, FP32 and every tensor-core path (panels, on-the-fly P, FP64-accurate).

Such a field is an ordinary field whose orders off the stride vanish, and its
grid repeats every 2 pi / mres.  So the oracle is the plain one on the full
circle: synthesis of the spectrum spread onto every order (zeros off the
stride) on nphi mres longitudes, of which the first nphi are the sector; and
analysis of the sector tiled mres times, read at the strided orders."""
import numpy as np
import pytest

import oracle
from paper_1202_6522_gb300 import synthetic

import _bounds as B
from _util import fp64_bound, normwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

# (lmax, mmax in order indices, mres, nlat, nphi of the sector, batch)
CASES = [
    (31, 7, 4, 32, 16, 2),
    (40, 13, 3, 41, 30, 1),
    (127, 25, 5, 128, 60, 2),
    (255, 127, 2, 256, 256, 1),
]
IDS = [f"N{c[0]}k{c[1]}mres{c[2]}lat{c[3]}phi{c[4]}b{c[5]}" for c in CASES]


@pytest.fixture(scope="module")
def SHT():
    from paper_1202_6522_gb300 import build
    build.build()
    from paper_1202_6522_gb300 import SHT as cls
    return cls


def _np(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


def _strided_index(lmax, mmax, mres):
    """Packed index of each (n, m = k mres) of the strided layout in the full
    (mres = 1, mmax_full = mmax mres) layout, in the strided layout's order."""
    idx = []
    for k in range(mmax + 1):
        m = k * mres
        idx.extend(oracle.lm_index(lmax, n, m) for n in range(m, lmax + 1))
    return np.array(idx)


def _spread(a, lmax, mmax, mres):
    full = np.zeros(a.shape[:-1] + (oracle.nlm(lmax, mmax * mres),), dtype=a.dtype)
    full[..., _strided_index(lmax, mmax, mres)] = a
    return full


@pytest.mark.parametrize("path", ["f64", "f32", "tc", "otf", "tc64"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_mres_scalar(SHT, case, path):
    lmax, mmax, mres, nlat, nphi, batch = case
    sht = SHT(lmax, mmax, nlat, nphi, mres=mres, fp32_path=path if path in ("tc", "otf") else "f32",
              fp64_path="tc" if path == "tc64" else "f64")
    assert sht.nlm == len(_strided_index(lmax, mmax, mres))
    rng = np.random.default_rng(7)
    a = (rng.standard_normal((batch, sht.nlm)) + 1j * rng.standard_normal((batch, sht.nlm))) * 0.3
    a[:, : lmax + 1] = a[:, : lmax + 1].real          # order 0 is real
    g = synthetic.grid(nlat, nphi, batch=batch, seed=3)
    cdt, fdt = (np.complex128, np.float64) if path in ("f64", "tc64") else (np.complex64, np.float32)
    a = a.astype(cdt)
    g = g.astype(fdt)
    full = _spread(a.astype(np.complex128), lmax, mmax, mres)
    tiled = np.tile(g.astype(np.float64), (1, 1, mres))
    idx = _strided_index(lmax, mmax, mres)
    got = _np(sht.synth_(torch.from_numpy(a).to(DEV)))
    ref = oracle.synth(lmax, mmax * mres, nlat, nphi * mres, full)
    gota = _np(sht.analys_(torch.from_numpy(g).to(DEV)))
    refa = oracle.analys(lmax, mmax * mres, nlat, nphi * mres, tiled)
    if path in ("f64", "tc64"):
        assert normwise(got, ref[..., :nphi]) < fp64_bound(lmax)
        assert normwise(gota, refa[..., idx]) < fp64_bound(lmax)
        return
    # the bounds of the full-circle transform the oracle computes
    sig = B.product_sigma(path, lmax)
    bnd = B.synth_row_bounds(lmax, mmax * mres, nlat, nphi * mres, full, sig)
    B.check(got, ref[..., :nphi], bnd[:, :, None], f"{path} mres{mres} synth")
    bnd = B.analys_coeff_bounds(lmax, mmax * mres, nlat, nphi * mres, tiled, sig)
    B.check(gota, refa[..., idx], bnd[:, idx], f"{path} mres{mres} analys")


@pytest.mark.parametrize("path", ["f64", "tc"])
def test_mres_vector_and_adjoint(SHT, path):
    lmax, mmax, mres, nlat, nphi, batch = CASES[1]
    sht = SHT(lmax, mmax, nlat, nphi, mres=mres, fp32_path="tc")
    rng = np.random.default_rng(11)
    S = rng.standard_normal((batch, sht.nlm)) + 1j * rng.standard_normal((batch, sht.nlm))
    T = rng.standard_normal((batch, sht.nlm)) + 1j * rng.standard_normal((batch, sht.nlm))
    S[:, : lmax + 1] = S[:, : lmax + 1].real
    T[:, : lmax + 1] = T[:, : lmax + 1].real
    rt, rp = oracle.synth_vec(lmax, mmax * mres, nlat, nphi * mres, _spread(S, lmax, mmax, mres),
                              _spread(T, lmax, mmax, mres))
    if path == "tc":
        # the tensor-core vector path (FP32 data); its analysis against the oracle's
        S32 = S.astype(np.complex64)
        T32 = T.astype(np.complex64)
        rt, rp = oracle.synth_vec(lmax, mmax * mres, nlat, nphi * mres, _spread(S32.astype(np.complex128), lmax, mmax, mres),
                                  _spread(T32.astype(np.complex128), lmax, mmax, mres))
        vt, vp = sht.synth_vec_(torch.from_numpy(S32).to(DEV), torch.from_numpy(T32).to(DEV))
        sig = B.product_sigma("tc", lmax)
        bt, bp = B.synth_vec_row_bounds(lmax, mmax * mres, nlat, nphi * mres,
                                        _spread(S32.astype(np.complex128), lmax, mmax, mres),
                                        _spread(T32.astype(np.complex128), lmax, mmax, mres), sig)
        B.check(_np(vt), rt[..., :nphi], bt[:, :, None], "tc mres vector theta")
        B.check(_np(vp), rp[..., :nphi], bp[:, :, None], "tc mres vector phi")
        gt = synthetic.grid(nlat, nphi, batch=batch, seed=12).astype(np.float32).astype(np.float64)
        gp = synthetic.grid(nlat, nphi, batch=batch, seed=13).astype(np.float32).astype(np.float64)
        Sg, Tg = sht.analys_vec_(torch.from_numpy(gt.astype(np.float32)).to(DEV),
                                 torch.from_numpy(gp.astype(np.float32)).to(DEV))
        tt, tp = np.tile(gt, (1, 1, mres)), np.tile(gp, (1, 1, mres))
        rS, rT = oracle.analys_vec(lmax, mmax * mres, nlat, nphi * mres, tt, tp)
        idx = _strided_index(lmax, mmax, mres)
        bnd = B.analys_vec_coeff_bounds(lmax, mmax * mres, nlat, nphi * mres, tt, tp, sig)
        B.check(_np(Sg), rS[..., idx], bnd[:, idx], "tc mres vector S")
        B.check(_np(Tg), rT[..., idx], bnd[:, idx], "tc mres vector T")
        return
    vt, vp = sht.synth_vec_(torch.from_numpy(S).to(DEV), torch.from_numpy(T).to(DEV))
    assert normwise(_np(vt), rt[..., :nphi]) < fp64_bound(lmax)
    assert normwise(_np(vp), rp[..., :nphi]) < fp64_bound(lmax)
    # adjoint of synthesis: the sector grid's transposed synthesis, which on the
    # full circle sees the sector once (the tiled copies are not part of the sector)
    g = synthetic.grid(nlat, nphi, batch=batch, seed=9)
    full = np.zeros((batch, nlat, nphi * mres))
    full[..., :nphi] = g
    got = _np(sht.synth_adj_(torch.from_numpy(g).to(DEV)))
    ref = oracle.synth_adj(lmax, mmax * mres, nlat, nphi * mres, full)
    assert normwise(got, ref[..., _strided_index(lmax, mmax, mres)]) < fp64_bound(lmax)


def test_mres_index_and_refusals(SHT):
    sht = SHT(31, 7, 32, 16, mres=4)
    assert sht.lm_index(4, 4) == 32                 # order index 1 starts after the 32 degrees of m = 0
    assert sht.lm_index(5, 2) == -1                 # m off the stride
    with pytest.raises(ValueError):
        SHT(31, 8, 32, 32, mres=4)                  # mmax mres > lmax (SHT_EINVAL)
