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
