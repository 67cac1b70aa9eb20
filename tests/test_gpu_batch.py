"""Uneven batches: fields of different truncations in one persistent,
graph-captured launch, checked field by field against the FP64 oracle and
against the per-field path."""
import numpy as np
import pytest

import oracle
from paper_1202_6522_gb300 import synthetic

import _bounds as B

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
            B.assert_synth(g.cpu().numpy(), (s * (1 + rep)).astype(np.complex128), l, l, la, ph, "f32",
                           what=f"f32 batch synth N{l}")
        gs = [torch.from_numpy(synthetic.grid(la, ph, seed=10 + i).astype(np.float32)).to(DEV)
              for i, (la, ph) in enumerate(zip(ub.nlat, ub.nphi))]
        out = ub.analys_(gs)
        torch.cuda.synchronize()
        for l, la, ph, g, o in zip(lmaxs, ub.nlat, ub.nphi, gs, out):
            B.assert_analys(o.cpu().numpy(), g.cpu().numpy().astype(np.float64), l, l, la, ph, "f32",
                            what=f"f32 batch analys N{l}")


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
    # paths, so the results agree to rounding, not bitwise: each is within the
    # derived bound of the exact result, so they are within twice it of each other
    for l, a, b, g in zip(lmaxs, back, ref2, got):
        gn = g.cpu().numpy().astype(np.float64)
        bnd = B.analys_coeff_bounds(l, l, l + 1, 2 * (l + 1), gn, B.product_sigma("f32", l))
        B.check(a.cpu().numpy()[None], b.cpu().numpy()[None], 2 * bnd, f"f32 batch vs per-field analys N{l}")
    # spot-check two fields against the oracle
    for i in (0, 95):
        l = lmaxs[i]
        B.assert_synth(got[i].cpu().numpy(), specs[i].cpu().numpy().astype(np.complex128), l, l, l + 1,
                       2 * (l + 1), "f32", what=f"f32 batch synth N{l}")


def test_batch_rejects_bad_shapes(lib):
    with pytest.raises(ValueError):
        lib.UnevenBatch([10], nlat=[5], nphi=[32])


@pytest.mark.parametrize("use_graph", [True, False])
def test_tc_uneven_batch_matches_oracle(lib, use_graph):
    """Tensor-core mode: fields grouped by shape, one contraction per group.
    Shapes with an odd nlm (5, 9: spectra gathered through the prep pass),
    repeated shapes (groups of several fields), a single-field group and a
    3 x 2^k longitude grid."""
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
            B.assert_synth(g.cpu().numpy(), (s * (1 + rep)).astype(np.complex128), l, l, la, ph, "tc",
                           what=f"tc batch synth N{l}")
        gs = [torch.from_numpy(synthetic.grid(la, ph, seed=10 + i + rep).astype(np.float32)).to(DEV)
              for i, (la, ph) in enumerate(zip(ub.nlat, ub.nphi))]
        out = ub.analys_(gs)
        torch.cuda.synchronize()
        for l, la, ph, g, o in zip(lmaxs, ub.nlat, ub.nphi, gs, out):
            B.assert_analys(o.cpu().numpy(), g.cpu().numpy().astype(np.float64), l, l, la, ph, "tc",
                            what=f"tc batch analys N{l}")


def test_tc_config4_batch_equals_batched_tensor_core_path(lib):
    """96 fields, N from {63, 127, 255, 511}, tensor-core mode: each field's
    result equals, bitwise, the regular batched tensor-core call on its shape
    group stacked in field order (same contraction over the same batch, same
    FFT tile function); one field per shape against the oracle."""
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
        B.assert_synth(got[i].cpu().numpy(), specs[i].cpu().numpy().astype(np.complex128), l, l, l + 1,
                       2 * (l + 1), "tc", what=f"tc batch synth N{l}")


def test_auto_batch_chooses_a_timed_path(lib):
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
        B.assert_synth(g.cpu().numpy(), s.cpu().numpy().astype(np.complex128), l, l, l + 1, 2 * (l + 1),
                       ub.path, what=f"auto batch synth N{l}")
    with pytest.raises(ValueError):
        lib.UnevenBatch(lmaxs, path="f64")
