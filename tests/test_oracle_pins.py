"""Pins of the FP64 CPU oracle against facts the paper and mathematics fix.

None of these tests re-types the oracle's own formulas: each checks it against
a library routine, a closed form, an invariant or a brute-force evaluation of
the definition, chosen so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1202_6522_gb300 import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Gauss nodes and weights (Sec. 2.3, Eq. gauss; nodes/weights cited to DLMF)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("nlat", [1, 2, 3, 7, 32, 33, 256])
def test_gauss_matches_library_leggauss(nlat):
    x, w = oracle.gauss(nlat)
    xr, wr = np.polynomial.legendre.leggauss(nlat)
    # leggauss returns ascending nodes; the oracle orders north to south
    assert np.all(np.diff(x) < 0)
    np.testing.assert_allclose(x, xr[::-1], rtol=0, atol=2e-15)
    # leggauss's own weights lose ~1e-11 relative near the poles (checked
    # against 40-digit values below), so the library comparison uses that bound
    np.testing.assert_allclose(w, wr[::-1], rtol=5e-11, atol=0)


@pytest.mark.parametrize("nlat", [17, 256, 1024])
def test_gauss_high_precision(nlat):
    """Nodes and weights against 40-digit Newton iterates (mpmath)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    x, w = oracle.gauss(nlat)
    for j in list(range(0, nlat, max(1, nlat // 5))) + [1, nlat - 1]:
        xj = mpmath.mpf(x[j])
        for _ in range(8):
            p = mpmath.legendre(nlat, xj)
            dp = nlat * (mpmath.legendre(nlat - 1, xj) - xj * p) / (1 - xj ** 2)
            xj -= p / dp
        wt = 2 * (1 - xj ** 2) / (nlat * mpmath.legendre(nlat - 1, xj)) ** 2
        assert abs(float(mpmath.mpf(x[j]) - xj)) < 1e-16
        # w depends on the node through 1 - x^2, so a node rounded to double
        # carries a relative weight error up to ~2 ulp(x) / (1 - x^2)
        bound = 5e-14 + 4.5e-16 / (1 - x[j] ** 2)
        assert abs(float((w[j] - wt) / wt)) < bound


@pytest.mark.parametrize("nlat", [4, 31, 64, 511])
def test_gauss_weights_exact_moments(nlat):
    x, w = oracle.gauss(nlat)
    assert abs(w.sum() - 2.0) < 1e-13
    np.testing.assert_allclose(w, w[::-1], rtol=1e-13)
    np.testing.assert_allclose(x, -x[::-1], atol=1e-15)
    # exact for polynomials of degree <= 2 nlat - 1 (Sec. 2.3)
    for k in range(0, 2 * nlat, 7):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13


# --------------------------------------------------------------------------
# P_n^m against its definition (Sec. 2.1), by brute force
# --------------------------------------------------------------------------
def _plm_definition(n, m, x):
    """Sec. 2.1: (-1)^m sqrt((2n+1)/4pi (n-m)!/(n+m)!) (1-x^2)^{m/2} d^m/dx^m P_n(x),
    with P_n from its power series (numpy Legendre basis), not from any recurrence."""
    dP = np.polynomial.legendre.Legendre.basis(n).deriv(m) if m else np.polynomial.legendre.Legendre.basis(n)
    norm = math.sqrt((2 * n + 1) / (4 * math.pi) * math.factorial(n - m) / math.factorial(n + m))
    return (-1) ** m * norm * (1 - x * x) ** (m / 2) * dP(x)


@pytest.mark.parametrize("x", [-0.93, -0.2, 0.0, 0.37, 0.81, 0.999])
def test_plm_matches_definition_bruteforce(x):
    lmax = 8
    p = oracle.plm(lmax, lmax, x)
    for m in range(lmax + 1):
        for n in range(m, lmax + 1):
            ref = _plm_definition(n, m, x)
            # reading: the recurrence has no Condon-Shortley phase, so multiply by (-1)^m
            got = (-1) ** m * p[oracle.lm_index(lmax, n, m)]
            assert abs(got - ref) < 1e-13 * max(1.0, abs(ref)), (n, m, x, got, ref)


def test_plm_closed_forms_from_golden():
    """Closed forms of the low-degree functions (tests/golden/plm_closed_forms.txt)."""
    rows = []
    with open(os.path.join(GOLDEN, "plm_closed_forms.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            n, m, expr = line.split(None, 2)
            rows.append((int(n), int(m), expr))
    assert len(rows) >= 6
    for x in (-0.7, 0.1, 0.55, 0.95):
        s = math.sqrt(1 - x * x)
        p = oracle.plm(3, 3, x)
        for n, m, expr in rows:
            ref = eval(expr, {"math": math, "x": x, "s": s, "pi": math.pi})
            assert abs(p[oracle.lm_index(3, n, m)] - ref) < 1e-14, (n, m)


def test_plm_mpmath_high_degree():
    """High degree against mpmath's associated Legendre function (50 digits)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    lmax = 200
    for x in (0.3, 0.9):
        p = oracle.plm(lmax, lmax, x)
        for n, m in ((200, 0), (200, 3), (150, 77), (200, 150), (120, 119)):
            ref = mpmath.legenp(n, m, x) * mpmath.sqrt(
                (2 * n + 1) / (4 * mpmath.pi) * mpmath.factorial(n - m) / mpmath.factorial(n + m))
            ref = float(ref) * (-1) ** m  # mpmath carries the Condon-Shortley phase
            got = p[oracle.lm_index(lmax, n, m)]
            assert abs(got - ref) <= 1e-12 * max(abs(ref), 1e-300), (n, m, x, got, ref)


# --------------------------------------------------------------------------
# Invariants: orthonormality (Sec. 2.1), addition theorem, mirror symmetry (Sec. 3.1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("lmax,nlat", [(31, 32), (20, 33)])
def test_orthonormality_under_quadrature(lmax, nlat):
    x, w = oracle.gauss(nlat)
    P = np.stack([oracle.plm(lmax, lmax, xj) for xj in x])  # [nlat, nlm]
    for m in range(lmax + 1):
        idx = [oracle.lm_index(lmax, n, m) for n in range(m, lmax + 1)]
        Pm = P[:, idx]
        G = 2 * math.pi * (Pm.T * w) @ Pm
        np.testing.assert_allclose(G, np.eye(len(idx)), atol=2e-14)


@pytest.mark.parametrize("lmax", [63, 1023, 2047])
def test_addition_theorem(lmax):
    for x in (0.0, 0.5, -0.97, 0.99999):
        p = oracle.plm(lmax, lmax, x)
        for n in (0, 1, lmax // 3, lmax):
            vals = np.array([p[oracle.lm_index(lmax, n, m)] for m in range(n + 1)])
            tot = vals[0] ** 2 + 2 * np.sum(vals[1:] ** 2)
            assert abs(tot - (2 * n + 1) / (4 * math.pi)) < 1e-12 * (2 * n + 1), (lmax, n, x)


def test_mirror_symmetry():
    lmax, nlat = 40, 41
    x, _ = oracle.gauss(nlat)
    for j in (0, 5, 19):
        pn = oracle.plm(lmax, lmax, x[j])
        ps = oracle.plm(lmax, lmax, x[nlat - 1 - j])
        for m in range(lmax + 1):
            for n in range(m, lmax + 1):
                i = oracle.lm_index(lmax, n, m)
                assert abs(ps[i] - (-1) ** (n + m) * pn[i]) < 1e-13 * max(1, abs(pn[i]))


def test_polar_localisation_figure1():
    """Figure 1: P_40^36 is far below P_40^33 near the pole."""
    x = math.cos(0.3)
    p = oracle.plm(40, 40, x)
    assert abs(p[oracle.lm_index(40, 40, 36)]) < 1e-2 * abs(p[oracle.lm_index(40, 40, 33)])


def test_extended_exponent_keeps_tiny_values():
    """Near the pole at high order P_m^m is far below the double range, yet the
    recurrence must still reach the correct O(1) values at higher degree."""
    lmax = 4000
    x = math.cos(0.05)
    p = oracle.plm(lmax, 300, x)
    # P_300^300(cos 0.05) ~ 0.05^300, below 1e-308: rounds to zero
    assert p[oracle.lm_index(lmax, 300, 300)] == 0.0
    # addition theorem at n = lmax restricted to m <= 300 must still hold where
    # the m > 300 terms are negligible (sin(0.05) * 4000 ~ 200 < 300)
    vals = np.array([p[oracle.lm_index(lmax, lmax, m)] for m in range(301)])
    tot = vals[0] ** 2 + 2 * np.sum(vals[1:] ** 2)
    assert abs(tot - (2 * lmax + 1) / (4 * math.pi)) < 1e-9 * (2 * lmax + 1)


# --------------------------------------------------------------------------
# Transforms against closed forms (Sec. 2.2, 2.3)
# --------------------------------------------------------------------------
def _phis(nphi):
    return 2 * math.pi * np.arange(nphi) / nphi


@pytest.mark.parametrize("cr,ci", [(1.0, 0.0), (0.3, -0.8)])
def test_synthesis_single_mode_closed_form(cr, ci):
    lmax, nlat, nphi = 5, 6, 12
    a = np.zeros(oracle.nlm(lmax), dtype=complex)
    a[oracle.lm_index(lmax, 1, 1)] = cr + 1j * ci
    a[oracle.lm_index(lmax, 1, 0)] = 0.25
    f = oracle.synth(lmax, lmax, nlat, nphi, a)
    x, _ = oracle.gauss(nlat)
    s = np.sqrt(1 - x * x)
    phi = _phis(nphi)
    # f = 0.25 Y_1^0 + (c Y_1^1 + conj(c) Y_1^{-1}) with Y_1^1 = sqrt(3/8pi) s e^{i phi}
    ref = (0.25 * math.sqrt(3 / (4 * math.pi)) * x[:, None]
           + 2 * math.sqrt(3 / (8 * math.pi)) * s[:, None] * (cr * np.cos(phi) - ci * np.sin(phi))[None, :])
    np.testing.assert_allclose(f, ref, atol=1e-15)


def test_analysis_of_closed_form_field():
    lmax, nlat, nphi = 9, 11, 24
    x, _ = oracle.gauss(nlat)
    s = np.sqrt(1 - x * x)
    phi = _phis(nphi)
    # f = 3 cos(theta) + sin(theta)^2 sin(2 phi)
    f = 3 * x[:, None] + (s * s)[:, None] * np.sin(2 * phi)[None, :]
    a = oracle.analys(lmax, lmax, nlat, nphi, f)
    ref = np.zeros_like(a)
    ref[oracle.lm_index(lmax, 1, 0)] = 3 * math.sqrt(4 * math.pi / 3)
    # s^2 e^{2i phi} = Y_2^2 / c22 with P_2^2 = c22 s^2, c22 = sqrt(15/(32 pi));
    # sin(2 phi) = Im e^{2 i phi} -> coefficient of Y_2^2 is 1/(2 i c22) = -i/(2 c22)
    c22 = math.sqrt(15 / (32 * math.pi))
    ref[oracle.lm_index(lmax, 2, 2)] = -1j / (2 * c22)
    np.testing.assert_allclose(a, ref, atol=1e-14)


@pytest.mark.parametrize("lmax,mmax,nlat,nphi", [
    (7, 7, 8, 16), (31, 31, 32, 64), (31, 31, 33, 64), (31, 20, 40, 48), (16, 16, 17, 36), (0, 0, 1, 1)])
def test_round_trip_exact(lmax, mmax, nlat, nphi):
    """Sec. 2.3: the Gauss-Legendre quadrature is exact for nlat >= N+1."""
    a = synthetic.spectrum(lmax, mmax, seed=3, uniform=True)
    f = oracle.synth(lmax, mmax, nlat, nphi, a)
    r = oracle.analys(lmax, mmax, nlat, nphi, f)
    emax, erms = oracle.eps_max_rms(r, a, lmax)
    assert emax < 1e-12 and erms < 1e-13


def test_round_trip_n255_accuracy_bound():
    """Sec. 3.5: eps_max < 1e-11 for N < 2048 (checked here at N = 255)."""
    lmax = 255
    a = synthetic.spectrum(lmax, seed=0, uniform=True)
    f = oracle.synth(lmax, lmax, 256, 512, a)
    r = oracle.analys(lmax, lmax, 256, 512, f)
    emax, erms = oracle.eps_max_rms(r, a, lmax)
    assert emax < 1e-11, emax


def test_too_few_latitudes_breaks_exactness():
    """With nlat < N+1 the quadrature is no longer exact (the validity rule)."""
    lmax = 15
    a = synthetic.spectrum(lmax, seed=4, uniform=True)
    f = oracle.synth(lmax, lmax, 12, 32, a)
    r = oracle.analys(lmax, lmax, 12, 32, f)
    assert np.abs(r - a).max() > 1e-3


def test_row_and_order_selection():
    lmax, nlat, nphi = 20, 22, 48
    a = synthetic.spectrum(lmax, seed=5)
    full = oracle.synth(lmax, lmax, nlat, nphi, a)
    part = oracle.synth(lmax, lmax, nlat, nphi, a, rows=[0, 7, 21])
    np.testing.assert_array_equal(part[[0, 7, 21]], full[[0, 7, 21]])
    assert np.all(part[1] == 0)
    g = synthetic.grid(nlat, nphi, seed=6)
    A = oracle.analys(lmax, lmax, nlat, nphi, g)
    B = oracle.analys(lmax, lmax, nlat, nphi, g, ms=[3, 11])
    for m in (3, 11):
        idx = [oracle.lm_index(lmax, n, m) for n in range(m, lmax + 1)]
        np.testing.assert_array_equal(A[idx], B[idx])


def test_error_measures_definition():
    lmax = 2
    Q = np.zeros(6, dtype=complex)
    R = Q.copy()
    R[1] = 3 + 4j
    emax, erms = oracle.eps_max_rms(R, Q, lmax)
    assert emax == 5.0
    assert abs(erms - math.sqrt(2 / 12 * 25)) < 1e-15


# --------------------------------------------------------------------------
# Vector transforms: d/dtheta, closed forms, round trip
# --------------------------------------------------------------------------
def test_dtheta_against_finite_differences():
    lmax = 12
    h = 1e-5
    for th in (0.2, 1.1, 2.5):
        d = oracle.dplm_dtheta(lmax, lmax, math.cos(th))
        pp = oracle.plm(lmax, lmax, math.cos(th + h))
        pm = oracle.plm(lmax, lmax, math.cos(th - h))
        fd = (pp - pm) / (2 * h)
        np.testing.assert_allclose(d, fd, atol=1e-8)


def test_vector_synthesis_closed_forms():
    lmax, nlat, nphi = 6, 8, 16
    x, _ = oracle.gauss(nlat)
    th = np.arccos(x)
    phi = _phis(nphi)
    k = math.sqrt(15 / (2 * math.pi))
    n = oracle.nlm(lmax)
    S = np.zeros(n, complex)
    T = np.zeros(n, complex)
    # S = Y_1^0: v_theta = -sqrt(3/4pi) sin theta, v_phi = 0
    S[oracle.lm_index(lmax, 1, 0)] = 1.0
    vt, vp = oracle.synth_vec(lmax, lmax, nlat, nphi, S, T)
    np.testing.assert_allclose(vt, -math.sqrt(3 / (4 * math.pi)) * np.sin(th)[:, None] * np.ones(nphi), atol=1e-15)
    np.testing.assert_allclose(vp, 0, atol=1e-15)
    # S with S_2^1 = 1: s = sqrt(15/2pi)(1/2) sin 2theta cos phi
    S[:] = 0
    S[oracle.lm_index(lmax, 2, 1)] = 1.0
    vt, vp = oracle.synth_vec(lmax, lmax, nlat, nphi, S, T)
    np.testing.assert_allclose(vt, k * np.cos(2 * th)[:, None] * np.cos(phi)[None], atol=1e-14)
    np.testing.assert_allclose(vp, -k * np.cos(th)[:, None] * np.sin(phi)[None], atol=1e-14)
    # toroidal T_2^1 = i: t = -sqrt(15/2pi)(1/2) sin 2theta sin phi
    S[:] = 0
    T[oracle.lm_index(lmax, 2, 1)] = 1j
    vt, vp = oracle.synth_vec(lmax, lmax, nlat, nphi, S, T)
    # v_theta = -(1/sin) dT/dphi = k cos(theta) cos(phi); v_phi = dT/dtheta = -k cos 2theta sin phi
    np.testing.assert_allclose(vt, k * np.cos(th)[:, None] * np.cos(phi)[None], atol=1e-14)
    np.testing.assert_allclose(vp, -k * np.cos(2 * th)[:, None] * np.sin(phi)[None], atol=1e-14)


def test_vector_synthesis_is_gradient_of_scalar():
    """synth_vec(S, 0) is the surface gradient of synth(S): check d/dtheta by
    central differences in colatitude using a second grid of shifted nodes."""
    lmax = 10
    S = synthetic.spectrum(lmax, seed=7)
    T = np.zeros_like(S)
    nlat, nphi = 12, 24
    vt, vp = oracle.synth_vec(lmax, lmax, nlat, nphi, S, T)
    # v_phi = (1/sin) df/dphi: differentiate the Fourier series spectrally in phi
    f = oracle.synth(lmax, lmax, nlat, nphi, S)
    F = np.fft.rfft(f, axis=1)
    kk = np.arange(F.shape[1])
    dfdphi = np.fft.irfft(1j * kk * F, n=nphi, axis=1)
    x, _ = oracle.gauss(nlat)
    np.testing.assert_allclose(vp, dfdphi / np.sqrt(1 - x * x)[:, None], atol=1e-12)
    # v_theta: finite differences of the scalar field through P at theta +- h
    h = 1e-5
    th = np.arccos(x)
    phi = _phis(nphi)
    def field_at(thetas):
        out = np.zeros((len(thetas), nphi))
        for r, t in enumerate(thetas):
            p = oracle.plm(lmax, lmax, math.cos(t))
            for m in range(lmax + 1):
                Fm = sum(S[oracle.lm_index(lmax, n, m)] * p[oracle.lm_index(lmax, n, m)] for n in range(m, lmax + 1))
                if m == 0:
                    out[r] += Fm.real
                else:
                    out[r] += 2 * (Fm * np.exp(1j * m * phi)).real
        return out
    fd = (field_at(th + h) - field_at(th - h)) / (2 * h)
    np.testing.assert_allclose(vt, fd, atol=1e-7)


@pytest.mark.parametrize("lmax,mmax,nlat,nphi", [(7, 7, 8, 16), (15, 15, 16, 32), (15, 9, 19, 24)])
def test_vector_round_trip(lmax, mmax, nlat, nphi):
    S = synthetic.spectrum(lmax, mmax, seed=8)
    T = synthetic.spectrum(lmax, mmax, seed=9)
    ns, _ = synthetic.packed_degrees_orders(lmax, mmax)
    S[ns == 0] = 0
    T[ns == 0] = 0
    vt, vp = oracle.synth_vec(lmax, mmax, nlat, nphi, S, T)
    S2, T2 = oracle.analys_vec(lmax, mmax, nlat, nphi, vt, vp)
    assert np.abs(S2 - S).max() < 1e-12
    assert np.abs(T2 - T).max() < 1e-12


def test_toroidal_field_is_divergence_free():
    """div(r x grad T) = 0: the spheroidal part of a toroidal field vanishes."""
    lmax, nlat, nphi = 12, 14, 28
    T = synthetic.spectrum(lmax, seed=10)
    S = np.zeros_like(T)
    vt, vp = oracle.synth_vec(lmax, lmax, nlat, nphi, S, T)
    S2, _ = oracle.analys_vec(lmax, lmax, nlat, nphi, vt, vp)
    assert np.abs(S2).max() < 1e-13


# --------------------------------------------------------------------------
# Adjoints: dot-product identities and dense transposes
# --------------------------------------------------------------------------
def _sdot(a, b):
    # <a, b> = sum Re(conj(a) b) over the packed set; m = 0 imaginary parts excluded
    return float(np.sum(a.real * b.real + a.imag * b.imag))


@pytest.mark.parametrize("lmax,mmax,nlat,nphi", [(7, 7, 8, 16), (11, 6, 13, 20)])
def test_scalar_adjoint_identities(lmax, mmax, nlat, nphi):
    ns, ms = synthetic.packed_degrees_orders(lmax, mmax)
    a = synthetic.spectrum(lmax, mmax, seed=11)
    g = synthetic.grid(nlat, nphi, seed=12)
    lhs = float(np.sum(oracle.synth(lmax, mmax, nlat, nphi, a) * g))
    rhs = _sdot(a, oracle.synth_adj(lmax, mmax, nlat, nphi, g))
    assert abs(lhs - rhs) < 1e-12 * max(1, abs(lhs))
    lhs = _sdot(oracle.analys(lmax, mmax, nlat, nphi, g), a)
    rhs = float(np.sum(g * oracle.analys_adj(lmax, mmax, nlat, nphi, a)))
    assert abs(lhs - rhs) < 1e-12 * max(1, abs(lhs))
    assert np.all(oracle.synth_adj(lmax, mmax, nlat, nphi, g)[ms == 0].imag == 0)


@pytest.mark.parametrize("lmax,mmax,nlat,nphi", [(7, 7, 8, 16), (11, 6, 13, 20)])
def test_vector_adjoint_identities(lmax, mmax, nlat, nphi):
    S = synthetic.spectrum(lmax, mmax, seed=13)
    T = synthetic.spectrum(lmax, mmax, seed=14)
    gt = synthetic.grid(nlat, nphi, seed=15)
    gp = synthetic.grid(nlat, nphi, seed=16)
    vt, vp = oracle.synth_vec(lmax, mmax, nlat, nphi, S, T)
    lhs = float(np.sum(vt * gt) + np.sum(vp * gp))
    S2, T2 = oracle.synth_vec_adj(lmax, mmax, nlat, nphi, gt, gp)
    rhs = _sdot(S, S2) + _sdot(T, T2)
    assert abs(lhs - rhs) < 1e-12 * max(1, abs(lhs))
    A, B = oracle.analys_vec(lmax, mmax, nlat, nphi, gt, gp)
    lhs = _sdot(A, S) + _sdot(B, T)
    ht, hp = oracle.analys_vec_adj(lmax, mmax, nlat, nphi, S, T)
    rhs = float(np.sum(gt * ht) + np.sum(gp * hp))
    assert abs(lhs - rhs) < 1e-12 * max(1, abs(lhs))


def test_dense_synthesis_matrix_transpose():
    """Columns of synth applied to unit spectra vs rows of synth_adj applied to unit grids."""
    lmax, nlat, nphi = 4, 5, 10
    n = oracle.nlm(lmax)
    _, ms = synthetic.packed_degrees_orders(lmax)
    cols = []  # real parameterisation: Re of every coefficient, Im for m > 0
    for i in range(n):
        for part in ((1.0,) if ms[i] == 0 else (1.0, 1j)):
            e = np.zeros(n, complex)
            e[i] = part
            cols.append((i, part, oracle.synth(lmax, lmax, nlat, nphi, e).ravel()))
    M = np.stack([c[2] for c in cols], axis=1)  # [nlat*nphi, ndof]
    MT = np.zeros((len(cols), nlat * nphi))
    for q in range(nlat * nphi):
        g = np.zeros(nlat * nphi)
        g[q] = 1.0
        b = oracle.synth_adj(lmax, lmax, nlat, nphi, g.reshape(nlat, nphi))
        MT[:, q] = [b[i].real if part == 1.0 else b[i].imag for i, part, _ in cols]
    np.testing.assert_allclose(MT, M.T, atol=1e-14)


def test_plm_order_is_a_column_of_plm():
    """The single-order entry point returns exactly the packed columns of plm
    and dplm_dtheta (same recurrence, same rounding)."""
    lmax = 40
    x, _ = oracle.gauss(33)
    for m in (0, 3, 40):
        idx = [oracle.lm_index(lmax, n, m) for n in range(m, lmax + 1)]
        tab = oracle.plm_order(lmax, m, x[:5])
        dtab = oracle.plm_order(lmax, m, x[:5], deriv=True)
        for j in range(5):
            assert np.array_equal(tab[j], oracle.plm(lmax, lmax, x[j])[idx])
            assert np.array_equal(dtab[j], oracle.dplm_dtheta(lmax, lmax, x[j])[idx])
