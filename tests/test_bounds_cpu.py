"""The error-bound machinery of the GPU parity tests, checked on the CPU.

* Every check helper accepts the oracle's own outputs (zero error) and rejects
  them with a planted relative error of 1e-3, far above any bound of the
  FP32 or tensor-core paths.
* The RMS relative error of a split-bf16 product (hi*hi + hi*lo + lo*hi of
  two values split into bf16 hi = bf16(x), lo = bf16(x - hi)), measured on a
  numpy emulation of round-to-nearest bf16 over random operands spanning ten
  binades, stays within 10 % of the derived SIGMA_SPLIT and its worst case
  below 3 x 2^-16; the representation error alone matches SIGMA_REP.
"""
import numpy as np
import pytest

import oracle
from paper_1202_6522_gb300 import synthetic

import _bounds as B

L, M, NL, NPH = 15, 15, 16, 32


def _bf16(v):
    """Round float32 values to bf16 (nearest, ties to even), as float64."""
    u = np.asarray(v, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _split(v):
    v32 = np.asarray(v, dtype=np.float32).astype(np.float64)
    hi = _bf16(v32)
    return hi, _bf16((v32 - hi).astype(np.float32))


def test_split_bf16_rounding_model():
    rng = np.random.default_rng(0)
    p = rng.uniform(-1, 1, 400000) * np.exp2(rng.uniform(-5, 5, 400000))
    a = rng.uniform(-1, 1, 400000).astype(np.float32).astype(np.float64)
    p = p.astype(np.float32).astype(np.float64)
    ph, pl = _split(p)
    ah, al = _split(a)
    rel = (ph * ah + ph * al + pl * ah - p * a) / (p * a)
    rms = float(np.sqrt(np.mean(rel ** 2)))
    assert 0.8 * B.SIGMA_SPLIT < rms < 1.1 * B.SIGMA_SPLIT, (rms, B.SIGMA_SPLIT)
    assert np.abs(rel).max() < 3 * 2.0 ** -16
    rep = float(np.sqrt(np.mean(((ph + pl - p) / p) ** 2)))
    assert 0.8 * B.SIGMA_REP < rep < 1.1 * B.SIGMA_REP, (rep, B.SIGMA_REP)


@pytest.fixture(scope="module")
def data():
    g = synthetic.grid(NL, NPH, batch=2, seed=1)
    a = synthetic.spectrum(L, batch=2, seed=2)
    S = synthetic.spectrum(L, batch=2, seed=3)
    T = synthetic.spectrum(L, batch=2, seed=4)
    return g, a, S, T


@pytest.mark.parametrize("err", [0.0, 1e-3])
def test_scalar_checks(data, err):
    g, a, _, _ = data
    f = 1.0 + err
    syn = oracle.synth(L, M, NL, NPH, a)
    ana = oracle.analys(L, M, NL, NPH, g)
    cases = [
        lambda: B.assert_synth(syn * f, a, L, M, NL, NPH, "tc"),
        lambda: B.assert_analys(ana * f, g, L, M, NL, NPH, "f32"),
        lambda: B.check_scalar_adjoints(oracle.synth_adj(L, M, NL, NPH, g) * f,
                                        oracle.analys_adj(L, M, NL, NPH, a) * f, g, a, L, M, NL, NPH, "tc", "cpu"),
    ]
    for c in cases:
        if err == 0.0:
            assert c() == 0.0
        else:
            with pytest.raises(AssertionError):
                c()


@pytest.mark.parametrize("err", [0.0, 1e-3])
def test_vector_checks(data, err):
    g, _, S, T = data
    f = 1.0 + err
    rt, rp = oracle.synth_vec(L, M, NL, NPH, S, T)
    rS, rT = oracle.analys_vec(L, M, NL, NPH, g, g)
    sa, ta = oracle.synth_vec_adj(L, M, NL, NPH, g, g)
    ha, hp = oracle.analys_vec_adj(L, M, NL, NPH, S, T)

    def run():
        B.check_vector(rt * f, rp * f, rt, rp, S, T, rS * f, rT * f, rS, rT, g, g, L, M, NL, NPH, "tc", "cpu")
        B.check_vector_adjoints(sa * f, ta * f, sa, ta, g, g, ha * f, hp * f, ha, hp, S, T, L, M, NL, NPH, "tc",
                                "cpu")
    if err == 0.0:
        run()
    else:
        with pytest.raises(AssertionError):
            run()


def test_round_trip_and_gradient_bounds_positive():
    Q = synthetic.spectrum(L, seed=0, uniform=True)
    ns, ms = synthetic.packed_degrees_orders(L)
    b = B.round_trip_bounds(L, NL, NPH, Q, 1e-5, 1e-5, [0, 3], sigma_rep=B.SIGMA_REP)
    assert (b[np.isin(ms, [0, 3])] > 0).all() and (b[~np.isin(ms, [0, 3])] == 0).all()
    resid = oracle.synth(L, M, NL, NPH, Q) - synthetic.grid(NL, NPH, seed=5)
    gb = B.loss_grad_bounds(L, NL, NPH, Q, resid, 1e-5, [1, 2], sigma_rep=B.SIGMA_REP)
    assert (gb[np.isin(ms, [1, 2])] > 0).all()
