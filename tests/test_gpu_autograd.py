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
