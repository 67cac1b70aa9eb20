"""Uneven batches: fields of different truncations in one persistent,
graph-captured launch, checked field by field against the FP64 oracle and
against the per-field path."""
import numpy as np
import pytest

import oracle
from paper_1202_6522_gb300 import synthetic

from _util import fp32_bound, normwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def lib():
    from paper_1202_6522_gb300 import build
    build.build()
    import paper_1202_6522_gb300 as P
    return P


@pytest.mark.parametrize("use_graph", [True, False])
def test_uneven_batch_matches_oracle(lib, use_graph):
    lmaxs = [7, 31, 15, 63, 0, 40, 127, 31]
    ub = lib.UnevenBatch(lmaxs, use_graph=use_graph)
    specs = [synthetic.spectrum(l, seed=i).astype(np.complex64) for i, l in enumerate(lmaxs)]
    for rep in range(2):  # replays reuse the captured graph with new pointers
        sp = [torch.from_numpy(s * (1 + rep)).to(DEV) for s in specs]
        grids = ub.synth_(sp)
        torch.cuda.synchronize()
        for l, la, ph, s, g in zip(lmaxs, ub.nlat, ub.nphi, specs, grids):
            ref = oracle.synth(l, l, la, ph, (s * (1 + rep)).astype(np.complex128))
            assert normwise(g.cpu().numpy(), ref) < fp32_bound(l), l
        gs = [torch.from_numpy(synthetic.grid(la, ph, seed=10 + i).astype(np.float32)).to(DEV)
              for i, (la, ph) in enumerate(zip(ub.nlat, ub.nphi))]
        out = ub.analys_(gs)
        torch.cuda.synchronize()
        for l, la, ph, g, o in zip(lmaxs, ub.nlat, ub.nphi, gs, out):
            ref = oracle.analys(l, l, la, ph, g.cpu().numpy().astype(np.float64))
            assert normwise(o.cpu().numpy(), ref) < fp32_bound(l), l


def test_config4_batch_matches_per_field_path(lib):
    """96 fields with N drawn from {63, 127, 255, 511}: the batched synthesis
    equals the per-field launches bitwise (same tile function and order)."""
    lmaxs = synthetic.uneven_truncations(96)
    ub = lib.UnevenBatch(lmaxs)
    plans = {l: lib.SHT(l, l, l + 1, 2 * (l + 1)) for l in set(lmaxs)}
    specs = [torch.from_numpy(synthetic.spectrum(l, seed=i).astype(np.complex64)).to(DEV) for i, l in enumerate(lmaxs)]
    got = ub.synth_(specs)
    ref = [plans[l].synth_(s) for l, s in zip(lmaxs, specs)]
    torch.cuda.synchronize()
    for g, r in zip(got, ref):
        assert torch.equal(g, r)
    back = ub.analys_(got)
    ref2 = [plans[l].analys_(g) for l, g in zip(lmaxs, got)]
    torch.cuda.synchronize()
    # analysis splits the latitude sum over threads differently in the two
    # paths, so the results agree to rounding, not bitwise
    for l, a, b in zip(lmaxs, back, ref2):
        assert normwise(a.cpu().numpy(), b.cpu().numpy()) < fp32_bound(l)
    # spot-check two fields against the oracle
    for i in (0, 95):
        l = lmaxs[i]
        refo = oracle.synth(l, l, l + 1, 2 * (l + 1), specs[i].cpu().numpy().astype(np.complex128))
        assert normwise(got[i].cpu().numpy(), refo) < fp32_bound(l)


def test_batch_rejects_bad_shapes(lib):
    with pytest.raises(ValueError):
        lib.UnevenBatch([10], nlat=[5], nphi=[32])


@pytest.mark.parametrize("use_graph", [True, False])
def test_tc_uneven_batch_matches_oracle(lib, use_graph):
    """Tensor-core mode: fields grouped by shape, one contraction per group.
    Shapes with an odd nlm (5, 9: spectra gathered through the prep pass),
    repeated shapes (groups of several fields), a single-field group and a
    3 x 2^k longitude grid."""
    from _util import tc_bound
    lmaxs = [9, 31, 5, 63, 31, 9, 47, 31]
    nphis = [20, 64, 12, 128, 64, 20, 96, 64]
    ub = lib.UnevenBatch(lmaxs, nphi=nphis, use_graph=use_graph, path="tc")
    assert ub.path == "tc"
    specs = [synthetic.spectrum(l, seed=i).astype(np.complex64) for i, l in enumerate(lmaxs)]
    for rep in range(2):  # replays with new pointers and values
        sp = [torch.from_numpy(s * (1 + rep)).to(DEV) for s in specs]
        grids = ub.synth_(sp)
        torch.cuda.synchronize()
        for l, la, ph, s, g in zip(lmaxs, ub.nlat, ub.nphi, specs, grids):
            ref = oracle.synth(l, l, la, ph, (s * (1 + rep)).astype(np.complex128))
            assert normwise(g.cpu().numpy(), ref) < tc_bound(l), l
        gs = [torch.from_numpy(synthetic.grid(la, ph, seed=10 + i + rep).astype(np.float32)).to(DEV)
              for i, (la, ph) in enumerate(zip(ub.nlat, ub.nphi))]
        out = ub.analys_(gs)
        torch.cuda.synchronize()
        for l, la, ph, g, o in zip(lmaxs, ub.nlat, ub.nphi, gs, out):
            ref = oracle.analys(l, l, la, ph, g.cpu().numpy().astype(np.float64))
            assert normwise(o.cpu().numpy(), ref) < tc_bound(l), l


def test_tc_config4_batch_equals_batched_tensor_core_path(lib):
    """96 fields, N from {63, 127, 255, 511}, tensor-core mode: each field's
    result equals, bitwise, the regular batched tensor-core call on its shape
    group stacked in field order (same contraction over the same batch, same
    FFT tile function); one field per shape against the oracle."""
    from _util import tc_bound
    lmaxs = synthetic.uneven_truncations(96)
    ub = lib.UnevenBatch(lmaxs, path="tc")
    specs = [torch.from_numpy(synthetic.spectrum(l, seed=i).astype(np.complex64)).to(DEV) for i, l in enumerate(lmaxs)]
    got = ub.synth_(specs)
    back = ub.analys_(got)
    torch.cuda.synchronize()
    for l in sorted(set(lmaxs)):
        idx = [i for i, v in enumerate(lmaxs) if v == l]
        sht = lib.SHT(l, l, l + 1, 2 * (l + 1), fp32_path="tc")
        g = sht.synth_(torch.stack([specs[i] for i in idx]))
        b = sht.analys_(torch.stack([got[i] for i in idx]))
        torch.cuda.synchronize()
        for k, i in enumerate(idx):
            assert torch.equal(got[i], g[k]), (l, i)
            assert torch.equal(back[i], b[k]), (l, i)
        i = idx[0]
        refo = oracle.synth(l, l, l + 1, 2 * (l + 1), specs[i].cpu().numpy().astype(np.complex128))
        assert normwise(got[i].cpu().numpy(), refo) < tc_bound(l), l


def test_auto_batch_chooses_a_timed_path(lib):
    from _util import tc_bound
    lmaxs = [63, 127, 63, 31]
    ub = lib.UnevenBatch(lmaxs, path="auto")
    assert ub.path in ("f32", "tc")
    assert ub.tuned_ms["f32"] > 0 and ub.tuned_ms["tc"] > 0
    faster = "tc" if ub.tuned_ms["tc"] < ub.tuned_ms["f32"] else "f32"
    assert ub.path == faster
    specs = [torch.from_numpy(synthetic.spectrum(l, seed=i).astype(np.complex64)).to(DEV) for i, l in enumerate(lmaxs)]
    grids = ub.synth_(specs)
    torch.cuda.synchronize()
    for l, s, g in zip(lmaxs, specs, grids):
        ref = oracle.synth(l, l, l + 1, 2 * (l + 1), s.cpu().numpy().astype(np.complex128))
        assert normwise(g.cpu().numpy(), ref) < max(tc_bound(l), fp32_bound(l)), l
    with pytest.raises(ValueError):
        lib.UnevenBatch(lmaxs, path="f64")
