"""Differentiation through the transforms: the autograd Functions call the
hand-written adjoint kernels; checked by gradcheck (finite differences), by
dot-product identities and against the oracle's adjoints."""
import numpy as np
import pytest

import oracle
from paper_1202_6522_gb300 import synthetic

from _util import fp64_bound, normwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def SHT():
    from paper_1202_6522_gb300 import build
    build.build()
    from paper_1202_6522_gb300 import SHT as cls
    return cls


def _real_dof_spec(sht, lmax, batch, seed):
    """Spectra whose m = 0 imaginary parts are zero (they are not degrees of freedom)."""
    a = synthetic.spectrum(lmax, sht.mmax, batch=batch, seed=seed)
    return torch.from_numpy(a).to(DEV)


@pytest.mark.parametrize("lmax,nlat,nphi", [(5, 6, 16), (9, 11, 32)])
def test_gradcheck_scalar(SHT, lmax, nlat, nphi):
    sht = SHT(lmax, lmax, nlat, nphi)
    ns, ms = synthetic.packed_degrees_orders(lmax)
    mask = torch.from_numpy(ms > 0).to(DEV)
    a = _real_dof_spec(sht, lmax, 2, 1).requires_grad_(True)

    def f(a):
        # keep Im a_n^0 out of the function (the transform ignores it)
        a = torch.where(mask, a, a.real.to(a.dtype))
        return sht.synth(a)

    assert torch.autograd.gradcheck(f, (a,), eps=1e-6, atol=1e-8, rtol=1e-6)
    g = torch.from_numpy(synthetic.grid(nlat, nphi, batch=2, seed=2)).to(DEV).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda g: sht.analys(g), (g,), eps=1e-6, atol=1e-8, rtol=1e-6)


@pytest.mark.parametrize("lmax,nlat,nphi", [(5, 6, 16)])
def test_gradcheck_vector(SHT, lmax, nlat, nphi):
    sht = SHT(lmax, lmax, nlat, nphi)
    ns, ms = synthetic.packed_degrees_orders(lmax)
    mask = torch.from_numpy(ms > 0).to(DEV)
    S = _real_dof_spec(sht, lmax, 1, 3).requires_grad_(True)
    T = _real_dof_spec(sht, lmax, 1, 4).requires_grad_(True)

    def f(S, T):
        S = torch.where(mask, S, S.real.to(S.dtype))
        T = torch.where(mask, T, T.real.to(T.dtype))
        return sht.synth_vec(S, T)

    assert torch.autograd.gradcheck(f, (S, T), eps=1e-6, atol=1e-8, rtol=1e-6)
    gt = torch.from_numpy(synthetic.grid(nlat, nphi, seed=5)).to(DEV).requires_grad_(True)
    gp = torch.from_numpy(synthetic.grid(nlat, nphi, seed=6)).to(DEV).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda a, b: sht.analys_vec(a, b), (gt, gp), eps=1e-6, atol=1e-8, rtol=1e-6)


def test_loss_gradient_matches_oracle_and_directional_fd(SHT):
    """loss = ||synth(a) - target||^2: the gradient 2 synth^T(synth(a) - target)
    against the oracle, and against a directional central difference."""
    lmax, nlat, nphi = 63, 64, 128
    sht = SHT(lmax, lmax, nlat, nphi)
    a0 = synthetic.spectrum(lmax, batch=2, seed=7)
    tgt = synthetic.grid(nlat, nphi, batch=2, seed=8)
    a = torch.from_numpy(a0).to(DEV).requires_grad_(True)
    t = torch.from_numpy(tgt).to(DEV)
    loss = ((sht.synth(a) - t) ** 2).sum()
    loss.backward()
    g = a.grad.cpu().numpy()
    resid = oracle.synth(lmax, lmax, nlat, nphi, a0) - tgt
    ref = 2 * oracle.synth_adj(lmax, lmax, nlat, nphi, resid)
    assert normwise(g, ref) < fp64_bound(lmax)
    d = synthetic.spectrum(lmax, batch=2, seed=9)
    h = 1e-6

    def L(x):
        with torch.no_grad():
            return float(((sht.synth(torch.from_numpy(x).to(DEV)) - t) ** 2).sum())
    fd = (L(a0 + h * d) - L(a0 - h * d)) / (2 * h)
    an = float(np.sum(g.real * d.real + g.imag * d.imag))
    assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_dot_product_identities_on_gpu(SHT, prec):
    lmax, nlat, nphi = 47, 50, 128
    sht = SHT(lmax, lmax, nlat, nphi)
    cdt = torch.complex128 if prec == "f64" else torch.complex64
    rdt = torch.float64 if prec == "f64" else torch.float32
    a = torch.from_numpy(synthetic.spectrum(lmax, seed=10)).to(DEV, cdt)
    g = torch.from_numpy(synthetic.grid(nlat, nphi, seed=11)).to(DEV, rdt)

    def sdot(x, y):
        return float((x.real.double() * y.real.double() + x.imag.double() * y.imag.double()).sum())
    lhs = float((sht.synth_(a).double() * g.double()).sum())
    rhs = sdot(a, sht.synth_adj_(g))
    tol = 1e-12 if prec == "f64" else 1e-4
    assert abs(lhs - rhs) <= tol * max(1.0, abs(lhs))
    lhs = sdot(sht.analys_(g), a)
    rhs = float((g.double() * sht.analys_adj_(a).double()).sum())
    assert abs(lhs - rhs) <= tol * max(1.0, abs(lhs))


def test_config5_loss_gradient_n1023_b16_tensor_cores(SHT):
    """The differentiable workload at its own size and precision: loss =
    ||synth(a) - target||^2 at N = 1023 (1024 x 2048 grid), batch 16, on the
    split-bf16 tensor-core path.  The gradient from the adjoint kernels against
    2 synth^T(synth(a) - target) of the oracle, on sampled orders of three
    fields, within the bound derived from the split-bf16 arithmetic of both
    the synthesis and its adjoint; and against a directional central
    difference, which for this quadratic loss is exact for any step, so a
    step of 1 keeps the FP32 rounding of the loss small against the signal."""
    import _bounds as B
    lmax, nlat, nphi, batch = 1023, 1024, 2048, 16
    sht = SHT(lmax, lmax, nlat, nphi, fp32_path="tc")
    a0 = synthetic.spectrum(lmax, batch=batch, seed=2).astype(np.complex64).astype(np.complex128)
    tgt = synthetic.grid(nlat, nphi, batch=batch, seed=2).astype(np.float32).astype(np.float64)
    a = torch.from_numpy(a0.astype(np.complex64)).to(DEV).requires_grad_(True)
    t = torch.from_numpy(tgt.astype(np.float32)).to(DEV)
    loss = ((sht.synth(a) - t) ** 2).sum()
    loss.backward()
    g = a.grad.detach().cpu().numpy().astype(np.complex128)
    ms = [0, 1, 64, 500, 1023]
    sig = B.product_sigma("tc", lmax)
    ns_, ms_ = synthetic.packed_degrees_orders(lmax)
    sel = np.isin(ms_, ms)
    for b in (0, 7, 15):
        resid = oracle.synth(lmax, lmax, nlat, nphi, a0[b]) - tgt[b]
        ref = 2 * oracle.synth_adj(lmax, lmax, nlat, nphi, resid, ms=ms)
        bnd = B.loss_grad_bounds(lmax, nlat, nphi, a0[b], resid, sig, ms, sigma_rep=B.data_sigma("tc"))
        B.check(g[b][sel], ref[sel], bnd[sel], f"config-5 gradient field {b}")
    d = synthetic.spectrum(lmax, batch=batch, seed=9).astype(np.complex64)

    def L(x):
        with torch.no_grad():
            r = sht.synth(torch.from_numpy(x).to(DEV)).double() - t.double()
            return float((r * r).sum())
    fd = (L(a0.astype(np.complex64) + d) - L(a0.astype(np.complex64) - d)) / 2.0
    an = float(np.sum(g.real * d.real + g.imag * d.imag))
    # rounding noise of either side is ~1e-5 of the signal (split-bf16 errors
    # of ~1e-5 relative summed with random signs); 1e-3 leaves a wide margin
    # while a wrong factor, sign or missing term fails
    assert abs(fd - an) < 1e-3 * abs(an), (fd, an)
