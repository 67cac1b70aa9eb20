"""Per-element error bounds of the FP32 and tensor-core paths (test code).

Every output of the transform is a sum of products, for instance a synthesis
row F_m(x_j) = sum_n a_n^m P_n^m(x_j) (Sec. 2.2) or an analysis coefficient
a_n^m = sum_j w_j P_n^m(x_j) F_m(x_j) (Sec. 2.3).  When each product carries
an independent relative rounding error of standard deviation sigma, the error
of the sum has standard deviation sigma times the root-sum-square (RSS) of the
terms.  The tests allow

    |gpu - oracle| <= LAMBDA * (sigma * RSS(terms) + sigma_fft * RSS_fft)
                      + 4 u32 |oracle|

per output element.  The terms are the exact ones, built from the oracle's
P_n^m.  The second term covers the FP32 longitude FFT: each of its log2(nphi)
butterfly levels rounds every value once in the sum and once in the twiddle
product, sigma_fft = 2 u32 sqrt(log2 nphi), applied to the RSS of the values
the FFT combines.  The third term covers the rounding of the FP32 output.
LAMBDA = 6 standard deviations.

sigma per path (data in the tests are FP32 numbers, so the rounding of the
inputs is not an error):

* Rounding to nearest with p significant bits leaves a relative error that is
  uniform over one unit in the last place.  For significands distributed
  log-uniformly on [1, 2) its mean square is (2^(1-p))^2 / 12 x E[1/s^2] with
  E[1/s^2] = (1/2 - 1/8) / ln 2 = 0.541, so its RMS is 0.425 x 2^-p.
* Split bf16 (SHT_TC_BF16X3): x = hi + lo, hi = bf16(x), lo = bf16(x - hi),
  p = 8.  The representation error of x is the rounding error of lo, relative
  to x the product of two bf16 rounding errors: RMS (0.425 x 2^-8)^2 =
  0.180 x 2^-16.  A product hi*hi + hi*lo + lo*hi carries that error from each
  factor plus the dropped lo*lo (again a product of two bf16 roundings):
  SIGMA_SPLIT = sqrt(3) x 0.180 x 2^-16.  The worst case of the same three
  terms is 3 x 2^-16; the RMS form is what lets a tenfold regression fail.
  FP32 accumulation in tensor memory over K terms adds ~ u32 sqrt(K).
  The representation error of an input coefficient is the same at every
  latitude, so where a later sum runs over latitudes it does not average:
  a round trip returns it unchanged, and the adjoint of synthesis sums its
  synthesis coherently.  Those two checks carry it as its own term, with RMS
  SIGMA_REP = 0.180 x 2^-16 (LAMBDA SIGMA_REP exceeds its worst case, 2^-16).
* FP32 recurrence restarted every 32 degrees from FP64 seeds (SHT_F32): the
  RSS over the degrees of the error of P_n^m(x_j), relative to the RSS of
  P_n^m(x_j) itself, is at most B_F32_REC for every order and node.  That
  constant is pinned on the CPU by a float32 simulation of the recurrence
  (tests/test_fp32_recurrence_cpu.py).  Products and sums add u32 (1 + sqrt(K)).
* On-the-fly P in FP32 split into bf16 (SHT_TC_OTF): both of the above.
"""
from __future__ import annotations

import functools
import math
import os

import numpy as np

import oracle
from paper_1202_6522_gb300 import synthetic

U32 = 2.0 ** -24
LAMBDA = 6.0
RN_RMS = 0.425                                  # RMS relative rounding error in units of 2^-p
SIGMA_REP = (RN_RMS * 2.0 ** -8) ** 2
SIGMA_SPLIT = math.sqrt(3.0) * SIGMA_REP
B_F32_REC = 2.0 ** -14


def product_sigma(path: str, lmax: int) -> float:
    """sigma of the docstring for a path ("tc", "otf", "f32") at truncation lmax."""
    acc = U32 * (1.0 + math.sqrt(lmax + 1.0))
    if path == "tc":
        return SIGMA_SPLIT + acc
    if path == "otf":
        return SIGMA_SPLIT + B_F32_REC + acc
    if path == "f32":
        return B_F32_REC + acc
    raise ValueError(path)


def data_sigma(path: str) -> float:
    """RMS representation error of the FP32 input coefficients in a path (the
    split paths round them to hi + lo; the FP32 path uses them as they are)."""
    return SIGMA_REP if path in ("tc", "otf") else 0.0


def fft_sigma(nphi: int) -> float:
    """sigma_fft of the docstring."""
    return 2.0 * U32 * math.sqrt(math.log2(max(nphi, 2)))


def _cm(ms):
    return np.where(ms == 0, 1.0, 2.0)


def _orders(lmax, mmax):
    return synthetic.packed_degrees_orders(lmax, mmax)


# --------------------------------------------------------------------------
# spectral -> grid (synthesis and the adjoint of analysis)
# --------------------------------------------------------------------------
def _per_order(v, ms, mmax):
    """Sums of v[..., i] over the packed entries of each order: [..., mmax+1]."""
    v2 = np.atleast_2d(v)
    out = np.zeros((v2.shape[0], mmax + 1), dtype=np.complex128)
    for b in range(v2.shape[0]):
        out[b] = (np.bincount(ms, weights=v2[b].real, minlength=mmax + 1)
                  + 1j * np.bincount(ms, weights=v2[b].imag, minlength=mmax + 1))
    return out if np.ndim(v) > 1 else out[0]


def _row_terms_bound(terms_list, ms, mmax, sigma, lg):
    """For [B, nlm] term arrays of one grid row: LAMBDA (sigma R1 + lg R2)
    per field, R1 = sqrt(sum_i c_m^2 |t_i|^2) over every product of every term
    array, R2 = sqrt(sum_m c_m^2 |F_m|^2) with F_m the per-order sums of all
    terms (what the FFT combines)."""
    c2 = _cm(ms) ** 2
    r1 = 0.0
    tot = 0.0
    for t in terms_list:
        r1 = r1 + np.sum(c2 * (t.real ** 2 + t.imag ** 2), axis=-1)
        tot = tot + t
    F = _per_order(np.asarray(tot, dtype=np.complex128), ms, mmax)
    cm = np.where(np.arange(mmax + 1) == 0, 1.0, 2.0)
    r2 = np.sum(cm ** 2 * np.abs(F) ** 2, axis=-1)
    return LAMBDA * (sigma * np.sqrt(r1) + lg * np.sqrt(r2))


def synth_row_bounds(lmax, mmax, nlat, nphi, a, sigma, rows=None, row_scale=None):
    """Bound on |gpu - oracle| for the elements of the grid rows `rows` of
    synth(a), a [B, nlm] (or [nlm]) complex: an array [B, nrows].  row_scale
    multiplies row j (the adjoint of analysis is (2 pi / nphi) w_j times the
    synthesis of b'/c_m)."""
    a = np.atleast_2d(a)
    x, _ = oracle.gauss(nlat)
    ns, ms = _orders(lmax, mmax)
    rows = list(range(nlat)) if rows is None else list(rows)
    lg = fft_sigma(nphi)
    out = np.zeros((a.shape[0], len(rows)))
    for i, j in enumerate(rows):
        P = oracle.plm(lmax, mmax, x[j])
        sc = 1.0 if row_scale is None else abs(row_scale[j])
        out[:, i] = sc * _row_terms_bound([a * P], ms, mmax, sigma, lg)
    return out


def synth_vec_row_bounds(lmax, mmax, nlat, nphi, S, T, sigma, rows=None, row_scale=None):
    """As synth_row_bounds for v_theta and v_phi of synth_vec(S, T):
    v_theta,m = sum_n [S dP - (i m / sin) T P], v_phi,m = sum_n [(i m / sin) S P + T dP]."""
    S, T = np.atleast_2d(S), np.atleast_2d(T)
    x, _ = oracle.gauss(nlat)
    ns, ms = _orders(lmax, mmax)
    rows = list(range(nlat)) if rows is None else list(rows)
    lg = fft_sigma(nphi)
    bt, bp = np.zeros((S.shape[0], len(rows))), np.zeros((S.shape[0], len(rows)))
    for i, j in enumerate(rows):
        P = oracle.plm(lmax, mmax, x[j])
        dP = oracle.dplm_dtheta(lmax, mmax, x[j])
        st = math.sqrt((1.0 - x[j]) * (1.0 + x[j]))
        imP = 1j * ms * P / st
        sc = 1.0 if row_scale is None else abs(row_scale[j])
        bt[:, i] = sc * _row_terms_bound([S * dP, -T * imP], ms, mmax, sigma, lg)
        bp[:, i] = sc * _row_terms_bound([S * imP, T * dP], ms, mmax, sigma, lg)
    return bt, bp


# --------------------------------------------------------------------------
# grid -> spectral (analysis and the adjoint of synthesis)
# --------------------------------------------------------------------------
def _row_dft(g, mmax):
    """F_m(theta_j) = sum_k g_jk e^{-i m phi_k}, m <= mmax (numpy's FFT)."""
    return np.fft.rfft(g, axis=-1)[..., : mmax + 1]


def _fold_pairs(nlat):
    npairs = (nlat + 1) // 2
    jn = np.arange(npairs)
    return npairs, jn, nlat - 1 - jn


def _folds(F, nlat, weights):
    """North/south folds of per-latitude values F[B, j, m] with per-latitude
    weights: s_p = w (F_N + F_S), d_p = w (F_N - F_S) over pairs p (the
    equator of odd nlat enters s once and d not at all)."""
    npairs, jn, js = _fold_pairs(nlat)
    wN = weights[jn][None, :, None]
    FN, FS = F[:, jn], F[:, js]
    s = wN * (FN + FS)
    d = wN * (FN - FS)
    if nlat % 2 == 1:
        s[:, -1] = wN[:, -1] * FN[:, -1]
        d[:, -1] = 0.0
    return s, d


def _fft_rss2(g, nlat, weights, scale):
    """Per pair, scale^2 w^2 (||g_N||^2 + ||g_S||^2): RSS^2 of the FFT inputs."""
    npairs, jn, js = _fold_pairs(nlat)
    rowsq = np.sum(g * g, axis=-1)
    fN, fS = rowsq[:, jn], rowsq[:, js].copy()
    if nlat % 2 == 1:
        fS[:, -1] = 0.0
    return (scale ** 2) * (weights[jn] ** 2)[None, :] * (fN + fS)


@functools.lru_cache(maxsize=4)
def _order_tables(lmax, mmax, nlat, ms_key, deriv):
    """P_n^m (or dP_n^m/dtheta) at the northern nodes for every packed entry
    of the orders ms_key (None: all): [npairs, entries of those orders]."""
    x, _ = oracle.gauss(nlat)
    npairs = (nlat + 1) // 2
    ns, ms = _orders(lmax, mmax)
    sel = np.ones(len(ms), dtype=bool) if ms_key is None else np.isin(ms, np.asarray(ms_key))
    idx = np.nonzero(sel)[0]
    out = np.zeros((npairs, len(idx)))
    mi = ms[idx]
    for m in np.unique(mi):
        cols = np.nonzero(mi == m)[0]
        tab = oracle.plm_order(lmax, int(m), x[:npairs], deriv=deriv)      # [npairs, lmax - m + 1]
        out[:, cols] = tab[:, ns[idx[cols]] - m]
    return out


def _pair_tables(lmax, mmax, nlat, ms_sel, deriv=False):
    key = None if ms_sel is None else tuple(sorted(int(m) for m in ms_sel))
    return _order_tables(lmax, mmax, nlat, key, deriv)


def analys_coeff_bounds(lmax, mmax, nlat, nphi, g, sigma, ms_sel=None, weights=None, scale=None):
    """Bound on |gpu - oracle| for the packed coefficients of analys(g), g
    [B, nlat, nphi] (or one grid), at the orders ms_sel (default all; the other
    entries are 0): an array [B, nlm].  weights: per-latitude factors (default
    the Gauss weights); scale: the factor of the longitude sum (default
    2 pi / nphi)."""
    g = np.asarray(g, dtype=np.float64)
    g = g[None] if g.ndim == 2 else g
    x, w = oracle.gauss(nlat)
    weights = w if weights is None else weights
    scale = 2.0 * math.pi / nphi if scale is None else scale
    ns, ms = _orders(lmax, mmax)
    F = scale * _row_dft(g, mmax)                           # [B, nlat, mmax+1]
    s, d = _folds(F, nlat, weights)
    fftsq = _fft_rss2(g, nlat, weights, scale)              # [B, npairs]
    sel = np.ones(len(ms), dtype=bool) if ms_sel is None else np.isin(ms, np.asarray(ms_sel))
    idx = np.nonzero(sel)[0]
    P = _pair_tables(lmax, mmax, nlat, ms_sel)             # [npairs, nsel]
    mi, par = ms[idx], (ns[idx] - ms[idx]) % 2
    out = np.zeros((g.shape[0], len(ms)))
    lg = fft_sigma(nphi)
    for b in range(g.shape[0]):
        v = np.where(par[None, :] == 0, s[b][:, mi], d[b][:, mi])    # fold of the matching parity
        r1 = np.sqrt(np.sum(P ** 2 * np.abs(v) ** 2, axis=0))
        r2 = np.sqrt(np.sum(P ** 2 * fftsq[b][:, None], axis=0))
        out[b, idx] = LAMBDA * (sigma * r1 + lg * r2)
    return out


def synth_adj_coeff_bounds(lmax, mmax, nlat, nphi, g, sigma, ms_sel=None):
    """Bounds for synth_adj(g)_n^m = c_m sum_j P_n^m(x_j) sum_k g_jk e^{-i m phi_k}."""
    ns, ms = _orders(lmax, mmax)
    out = analys_coeff_bounds(lmax, mmax, nlat, nphi, g, sigma, ms_sel=ms_sel, weights=np.ones(nlat), scale=1.0)
    return out * _cm(ms)[None, :]


def analys_vec_coeff_bounds(lmax, mmax, nlat, nphi, gt, gp, sigma, ms_sel=None, adjoint=False):
    """Bounds for (S, T) = analys_vec(gt, gp): per coefficient the RSS of the
    products dP V and m P V / sin of both components, over n(n+1).  With
    adjoint=True, for synth_vec_adj(gt, gp): no Gauss weights, no 2 pi / nphi,
    and c_m in place of 1 / (n(n+1))."""
    gt = np.asarray(gt, dtype=np.float64)
    gp = np.asarray(gp, dtype=np.float64)
    gt = gt[None] if gt.ndim == 2 else gt
    gp = gp[None] if gp.ndim == 2 else gp
    x, w = oracle.gauss(nlat)
    ns, ms = _orders(lmax, mmax)
    scale = 1.0 if adjoint else 2.0 * math.pi / nphi
    wt = (1.0 if adjoint else w) / np.sqrt((1.0 - x) * (1.0 + x))
    ts, td = _folds(scale * _row_dft(gt, mmax), nlat, wt)
    ps, pd = _folds(scale * _row_dft(gp, mmax), nlat, wt)
    fftsq = _fft_rss2(gt, nlat, wt, scale) + _fft_rss2(gp, nlat, wt, scale)
    sel = np.ones(len(ms), dtype=bool) if ms_sel is None else np.isin(ms, np.asarray(ms_sel))
    idx = np.nonzero(sel)[0]
    P = _pair_tables(lmax, mmax, nlat, ms_sel)
    dP = _pair_tables(lmax, mmax, nlat, ms_sel, deriv=True)
    mi, par = ms[idx], (ns[idx] - ms[idx]) % 2
    mP2 = (mi[None, :] * P) ** 2
    n = ns[idx].astype(np.float64)
    inv = np.where(n > 0, 1.0 / np.maximum(n * (n + 1.0), 1.0), 0.0)
    if adjoint:
        inv = _cm(mi)
    lg = fft_sigma(nphi)
    out = np.zeros((gt.shape[0], len(ms)))
    for b in range(gt.shape[0]):
        # P has the parity of n - m, dP the opposite one
        even = par[None, :] == 0
        vt_P = np.where(even, ts[b][:, mi], td[b][:, mi])
        vp_P = np.where(even, ps[b][:, mi], pd[b][:, mi])
        vt_dP = np.where(even, td[b][:, mi], ts[b][:, mi])
        vp_dP = np.where(even, pd[b][:, mi], ps[b][:, mi])
        r1 = np.sqrt(np.sum(dP ** 2 * (np.abs(vt_dP) ** 2 + np.abs(vp_dP) ** 2)
                            + mP2 * (np.abs(vt_P) ** 2 + np.abs(vp_P) ** 2), axis=0))
        r2 = np.sqrt(np.sum((dP ** 2 + mP2) * fftsq[b][:, None], axis=0))
        out[b, idx] = inv * LAMBDA * (sigma * r1 + lg * r2)
    return out


# --------------------------------------------------------------------------
# checks
# --------------------------------------------------------------------------
def check(got, ref, bound, what=""):
    """Asserts |got - ref| <= bound + 4 u32 |ref| element by element (bound
    broadcast against the arrays) and returns the largest ratio of the error
    to that allowance (at most 1)."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    allow = np.asarray(bound) + 4.0 * U32 * np.abs(ref) + 1e-300
    err = np.abs(got - ref)
    ratio = err / allow
    worst = float(ratio.max()) if ratio.size else 0.0
    log = os.environ.get("SHT_BOUND_LOG")
    if log:
        with open(log, "a") as fh:
            fh.write(f"{what}\t{worst:.4f}\t{float(err.max()):.3e}\n")
    assert worst <= 1.0, (f"{what}: error exceeds the derived bound {worst:.2f}x (max error "
                          f"{float(err.max()):.3e} at {np.unravel_index(int(ratio.argmax()), ratio.shape)})")
    return worst


def assert_synth(got, a, lmax, mmax, nlat, nphi, path, rows=None, ref=None, what="synthesis"):
    """got [B, nlat, nphi] against oracle.synth(a) on `rows` (default all)."""
    a = np.atleast_2d(a)
    got = np.asarray(got).reshape(a.shape[0], nlat, nphi)
    rr = list(range(nlat)) if rows is None else list(rows)
    if ref is None:
        ref = oracle.synth(lmax, mmax, nlat, nphi, a, rows=rows)
    ref = np.asarray(ref).reshape(a.shape[0], nlat, nphi)
    bnd = synth_row_bounds(lmax, mmax, nlat, nphi, a, product_sigma(path, lmax), rows=rr)
    return check(got[:, rr], ref[:, rr], bnd[:, :, None], what)


def assert_analys(got, g, lmax, mmax, nlat, nphi, path, ms_sel=None, ref=None, what="analysis"):
    """got [B, nlm] against oracle.analys(g) at the orders ms_sel (default all)."""
    g = np.asarray(g, dtype=np.float64)
    g = g[None] if g.ndim == 2 else g
    got = np.asarray(got).reshape(g.shape[0], -1)
    if ref is None:
        ref = oracle.analys(lmax, mmax, nlat, nphi, g, ms=ms_sel)
    ref = np.asarray(ref).reshape(g.shape[0], -1)
    ns, ms = _orders(lmax, mmax)
    sel = np.ones(len(ms), dtype=bool) if ms_sel is None else np.isin(ms, np.asarray(ms_sel))
    bnd = analys_coeff_bounds(lmax, mmax, nlat, nphi, g, product_sigma(path, lmax), ms_sel=ms_sel)
    return check(got[:, sel], ref[:, sel], bnd[:, sel], what)


LAMBDA_RT = 10.0


def round_trip_bounds(lmax, nlat, nphi, Q, sigma_s, sigma_a, ms_sel, sigma_rep=0.0):
    """Bound on |analys(synth(Q)) - Q| (Sec. 3.5) for the coefficients of the
    orders ms_sel (one field, lmax = mmax; the other entries 0).  The synthesis
    errors of row x_j, RSS sigma_s sqrt(sum_n |Q_n^m|^2 P_n^m(x_j)^2) for order m,
    pass through the analysis sum sum_j w_j P_n^m(x_j); the analysis adds its own
    products P_n^m(x_p) times the folds 2 w_p E_m(x_p) or 2 w_p O_m(x_p); the FFTs
    add sigma_fft on the rows of the grid; the representation error of Q_n^m
    itself (sigma_rep, the same at every latitude) comes back unchanged.

    These sources are not independent here: synthesis and analysis multiply
    by the same stored P_n^m, and near the poles at low order P_n^m varies so
    slowly from node to node that the representation errors of neighbouring
    nodes share their sign (a CPU emulation of the split-bf16 products at
    N = 1023 shows means of up to 0.14 of the RMS over the nodes of one
    degree).  So the standard deviations of the sources are added, not their
    variances, LAMBDA_RT = 10 of them are allowed, and P_0^0 -- a constant,
    represented with the same error at every node -- contributes its worst
    case 2^-16 |Q_0^0| once per direction."""
    x, w = oracle.gauss(nlat)
    ns, ms = _orders(lmax, lmax)
    npairs = (nlat + 1) // 2
    sel = np.isin(ms, np.asarray(ms_sel))
    idx = np.nonzero(sel)[0]
    P = _pair_tables(lmax, lmax, nlat, ms_sel)              # [npairs, nsel]
    wp = w[:npairs]
    Qs = Q[idx]
    mi, par = ms[idx], (ns[idx] - ms[idx]) % 2
    # the grid rows' RSS for the FFT term: ||g_j||^2 = nphi (|F_0|^2 + 2 sum_m |F_m|^2)
    rowsq = np.zeros(npairs)
    for p in range(npairs):
        Pall = oracle.plm(lmax, lmax, x[p])
        F = _per_order(Q * Pall, ms, lmax)
        FS = _per_order(Q * Pall * np.where((ns - ms) % 2 == 0, 1.0, -1.0), ms, lmax)
        cm = np.where(np.arange(lmax + 1) == 0, 1.0, 2.0)
        rowsq[p] = nphi * (np.sum(cm * np.abs(F) ** 2) + np.sum(cm * np.abs(FS) ** 2))
    out = np.zeros(len(ms))
    scale = 2.0 * math.pi / nphi
    for m in np.unique(mi):
        cols = np.nonzero(mi == m)[0]
        Pm, Qm, pm = P[:, cols], Qs[cols], par[cols]
        Bp = np.sum(np.abs(Qm)[None, :] ** 2 * Pm ** 2, axis=1)          # [npairs]
        E = Pm[:, pm == 0] @ Qm[pm == 0]
        O = Pm[:, pm == 1] @ Qm[pm == 1]
        fold = np.where(pm[None, :] == 0, np.abs(2 * wp * E)[:, None], np.abs(2 * wp * O)[:, None])
        sd_syn = sigma_s * np.sqrt(2.0 * np.sum(Pm ** 2 * (wp ** 2 * Bp)[:, None], axis=0))
        sd_ana = sigma_a * np.sqrt(np.sum(Pm ** 2 * fold ** 2, axis=0))
        sd_fft = fft_sigma(nphi) * np.sqrt(2.0 * np.sum(Pm ** 2 * (scale ** 2 * wp ** 2 * rowsq)[:, None], axis=0))
        sd_rep = sigma_rep * np.abs(Qm)
        out[idx[cols]] = LAMBDA_RT * (sd_syn + sd_ana + sd_fft + sd_rep)
    if 0 in set(int(v) for v in ms_sel) and sigma_rep > 0:
        out[0] += 2.0 * 2.0 ** -16 * abs(Q[0])
    return out


def loss_grad_bounds(lmax, nlat, nphi, a, resid, sigma, ms_sel, sigma_rep=0.0):
    """Bound on the error of grad = 2 synth^T(synth(a) - target) (one field,
    lmax = mmax) at the orders ms_sel: the adjoint's own products on the
    residual r (synth_adj_coeff_bounds), and the synthesis error of r carried
    through synth^T.  For m > 0, sum_k dr_jk e^{-i m phi_k} = nphi dF_m(x_j)
    when dr is the synthesis of per-order errors dF_m, so that part is
    c_m nphi sum_j P_n^m(x_j) dF_m(x_j), whose variance is
    (c_m nphi sigma)^2 sum_j P_n^m(x_j)^2 sum_n' |a_n'^m|^2 P_n'^m(x_j)^2.  The
    representation errors of the coefficients, da_n' (sigma_rep), are the same
    at every latitude: they enter as c_m nphi sum_n' M_nn' da_n' with the
    unweighted Gram matrix M_nn' = sum_j P_n^m(x_j) P_n'^m(x_j) (nlat even:
    twice the northern sum when n - n' is even, else 0)."""
    own = synth_adj_coeff_bounds(lmax, lmax, nlat, nphi, resid, sigma, ms_sel=ms_sel)[0]
    ns, ms = _orders(lmax, lmax)
    sel = np.isin(ms, np.asarray(ms_sel))
    idx = np.nonzero(sel)[0]
    P = _pair_tables(lmax, lmax, nlat, ms_sel)               # [npairs, nsel], |P(-x)| = |P(x)|
    mi = ms[idx]
    prop = np.zeros(len(ms))
    for m in np.unique(mi):
        cols = np.nonzero(mi == m)[0]
        Pm = P[:, cols]
        Bm = np.sum(np.abs(a[idx[cols]])[None, :] ** 2 * Pm ** 2, axis=1)
        cm = 1.0 if m == 0 else 2.0
        v = 2.0 * sigma ** 2 * np.sum(Pm ** 2 * Bm[:, None], axis=0)
        if sigma_rep > 0:
            nn = ns[idx[cols]]
            M = 2.0 * (Pm.T @ Pm) * ((nn[:, None] - nn[None, :]) % 2 == 0)
            v = v + sigma_rep ** 2 * (M ** 2 @ np.abs(a[idx[cols]]) ** 2)
        prop[idx[cols]] = LAMBDA * cm * nphi * np.sqrt(v)
    return 2.0 * np.sqrt(own ** 2 + prop ** 2)


# --------------------------------------------------------------------------
# composite checks used by several test files
# --------------------------------------------------------------------------
def check_scalar_adjoints(got_sa, got_aa, g, a, lmax, mmax, nlat, nphi, path, what, rows=None, ms_sel=None):
    """synth_adj(g) (orders ms_sel) and analys_adj(a) (grid rows `rows`) of a
    path against the oracle under the per-element bounds: synth^T is an
    unweighted analysis times c_m, analys^T the synthesis of a / c_m
    (imaginary part of order 0 dropped) times (2 pi / nphi) w_j on row j."""
    sig = product_sigma(path, lmax)
    g = np.asarray(g, dtype=np.float64)
    g = g[None] if g.ndim == 2 else g
    nb = g.shape[0]
    ns, ms = _orders(lmax, mmax)
    sel = np.ones(len(ms), dtype=bool) if ms_sel is None else np.isin(ms, np.asarray(ms_sel))
    ref = oracle.synth_adj(lmax, mmax, nlat, nphi, g, ms=ms_sel).reshape(nb, -1)
    bnd = synth_adj_coeff_bounds(lmax, mmax, nlat, nphi, g, sig, ms_sel=ms_sel)
    r1 = check(np.asarray(got_sa).reshape(nb, -1)[:, sel], ref[:, sel], bnd[:, sel], f"{what} synth_adj N{lmax}")
    a2 = np.atleast_2d(a)
    ap = np.where(ms == 0, a2.real, a2) / _cm(ms)
    _, w = oracle.gauss(nlat)
    rr = list(range(nlat)) if rows is None else list(rows)
    ref = oracle.analys_adj(lmax, mmax, nlat, nphi, a2, rows=rows).reshape(nb, nlat, nphi)
    bnd = synth_row_bounds(lmax, mmax, nlat, nphi, ap, sig, rows=rr, row_scale=2 * np.pi / nphi * w)
    r2 = check(np.asarray(got_aa).reshape(nb, nlat, nphi)[:, rr], ref[:, rr], bnd[:, :, None],
               f"{what} analys_adj N{lmax}")
    return max(r1, r2)


def check_vector(vt, vp, rt, rp, S, T, S2, T2, rS, rT, gt, gp, lmax, mmax, nlat, nphi, path, what, rows=None,
                 ms_sel=None):
    """Vector synthesis (rows) and analysis (orders ms_sel) of a path against
    the oracle under the per-element bounds."""
    sig = product_sigma(path, lmax)
    S, T = np.atleast_2d(S), np.atleast_2d(T)
    nb = S.shape[0]
    rr = list(range(nlat)) if rows is None else list(rows)
    bt, bp = synth_vec_row_bounds(lmax, mmax, nlat, nphi, S, T, sig, rows=rr)
    shp = (nb, nlat, nphi)
    check(np.asarray(vt).reshape(shp)[:, rr], np.asarray(rt).reshape(shp)[:, rr], bt[:, :, None],
          f"{what} synth_vec theta N{lmax}")
    check(np.asarray(vp).reshape(shp)[:, rr], np.asarray(rp).reshape(shp)[:, rr], bp[:, :, None],
          f"{what} synth_vec phi N{lmax}")
    bnd = analys_vec_coeff_bounds(lmax, mmax, nlat, nphi, gt, gp, sig, ms_sel=ms_sel)
    ns, ms = _orders(lmax, mmax)
    sel = np.ones(len(ms), dtype=bool) if ms_sel is None else np.isin(ms, ms_sel)
    check(np.asarray(S2).reshape(nb, -1)[:, sel], np.asarray(rS).reshape(nb, -1)[:, sel], bnd[:, sel],
          f"{what} analys_vec S N{lmax}")
    check(np.asarray(T2).reshape(nb, -1)[:, sel], np.asarray(rT).reshape(nb, -1)[:, sel], bnd[:, sel],
          f"{what} analys_vec T N{lmax}")


def check_vector_adjoints(S, T, rS, rT, gt, gp, ht, hp, rt, rp, A, Bs, lmax, mmax, nlat, nphi, path, what):
    """synth_vec_adj (a weight-free vector analysis times c_m) and
    analys_vec_adj (the vector synthesis of A, B over c_m n(n+1), times
    (2 pi / nphi) w_j on row j) under the per-element bounds."""
    sig = product_sigma(path, lmax)
    bnd = analys_vec_coeff_bounds(lmax, mmax, nlat, nphi, gt, gp, sig, adjoint=True)
    nb = bnd.shape[0]
    check(np.asarray(S).reshape(nb, -1), np.asarray(rS).reshape(nb, -1), bnd, f"{what} synth_vec_adj S N{lmax}")
    check(np.asarray(T).reshape(nb, -1), np.asarray(rT).reshape(nb, -1), bnd, f"{what} synth_vec_adj T N{lmax}")
    ns, ms = _orders(lmax, mmax)
    cm = _cm(ms)
    nn = ns.astype(np.float64)
    f = np.where(ns > 0, 1.0 / (cm * np.maximum(nn * (nn + 1), 1.0)), 0.0)
    A2 = np.where(ms == 0, np.atleast_2d(A).real, np.atleast_2d(A)) * f
    B2 = np.where(ms == 0, np.atleast_2d(Bs).real, np.atleast_2d(Bs)) * f
    _, w = oracle.gauss(nlat)
    bt, bp = synth_vec_row_bounds(lmax, mmax, nlat, nphi, A2, B2, sig, row_scale=2 * np.pi / nphi * w)
    shp = (nb, nlat, nphi)
    check(np.asarray(ht).reshape(shp), np.asarray(rt).reshape(shp), bt[:, :, None],
          f"{what} analys_vec_adj theta N{lmax}")
    check(np.asarray(hp).reshape(shp), np.asarray(rp).reshape(shp), bp[:, :, None],
          f"{what} analys_vec_adj phi N{lmax}")
