/*
 * sht_oracle.c -- plain FP64 CPU oracle for the Gauss-Legendre spherical
 * harmonic transform of Schaeffer, "Efficient Spherical Harmonic Transforms
 * aimed at pseudo-spectral numerical simulations" (arXiv:1202.6522).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product library never calls, links or includes it, and it shares no code,
 * table or helper with the CUDA path.
 *
 * What it computes, and where each step comes from:
 *   - Gauss nodes x_j (roots of P_nlat) and weights w_j by Newton iteration on
 *     the Legendre recurrence of Sec. 2.1; nodes sorted north to south.
 *   - P_n^m(x) by the recurrence of Sec. 3.2 (P_m^m, P_{m+1}^m, three-term
 *     relation with a_n^m, b_n^m).  Every value is carried as y*2^e with an
 *     integer exponent e, so nothing underflows at any degree; the value is
 *     rounded to a double only when it enters a sum.  No term is ever dropped.
 *   - Synthesis f(theta_j, phi_k) = sum_m c_m Re(F_m(theta_j) e^{i m phi_k}),
 *     F_m = sum_n f_n^m P_n^m (Sec. 2.2, the m<0 half given by the Hermitian
 *     symmetry of Sec. 3.1, so c_0 = 1, c_m = 2), evaluated as a direct
 *     (slow) Fourier sum, not an FFT.
 *   - Analysis f_n^m = sum_j w_j P_n^m(x_j) F_m(theta_j) with the rectangle rule
 *     F_m = (2 pi / nphi) sum_k f_jk e^{-i m phi_k} (Sec. 2.3, Gauss-Legendre sum).
 *   - Spheroidal/toroidal vector transforms and all adjoints, written as the
 *     plain sums that define them (conventions below).
 *   - No north/south folding, no polar skipping: every latitude is evaluated.
 *
 * Readings where the paper is silent or ambiguous:
 *   - Sign: the recurrence's P_m^m is positive (no (-1)^m Condon-Shortley
 *     factor); the definition in Sec. 2.1 differs by (-1)^m only.
 *   - Im f_n^0 is ignored on input and written as 0 on output.
 *   - Vector fields: v = grad_H S + r x grad_H T, i.e.
 *       v_theta = dS/dtheta - (1/sin) dT/dphi,  v_phi = (1/sin) dS/dphi + dT/dtheta,
 *     analysis divides by n(n+1) and returns 0 at n = 0.
 *   - sin(theta) dP_n^m/dtheta = n x P_n^m - sqrt((2n+1)(n^2-m^2)/(2n-1)) P_{n-1}^m,
 *     which follows from the definition in Sec. 2.1.
 *   - Adjoints use <a,b>_spec = sum over packed m>=0 of Re(conj(a) b) (Im at
 *     m = 0 excluded) and <f,g>_grid = sum f g.
 *
 * Layouts shared with the library's C ABI (layout only, no arithmetic):
 *   spectral: packed m-major, idx(n,m) = m(2 lmax + 3 - m)/2 + (n - m),
 *             interleaved complex (re, im) doubles;
 *   grid:     [nlat][nphi] real doubles, row j at node x_j (descending),
 *             phi_k = 2 pi k / nphi.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double PI = 3.14159265358979323846264338327950288;

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static long lm_index(int lmax, int n, int m)
{
    return (long)m * (2 * lmax + 3 - m) / 2 + (n - m);
}

long oracle_nlm(int lmax, int mmax)
{
    return lm_index(lmax, lmax, mmax) + 1;
}

/* ---------------------------------------------------------------------------
 * Gauss-Legendre nodes and weights (Sec. 2.3, Eq. "gauss").
 * P_n(x) by the recurrence of Sec. 2.1:  P_0 = 1, P_1 = x,
 *   n P_n = (2n-1) x P_{n-1} - (n-1) P_{n-2};
 * the derivative from (1 - x^2) P_n' = n (P_{n-1} - x P_n).
 * ------------------------------------------------------------------------- */
static void legendre_poly(int n, double x, double *pn, double *pnm1)
{
    double p0 = 1.0, p1 = x;
    if (n == 0) { *pn = 1.0; *pnm1 = 0.0; return; }
    for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *pnm1 = p0;
}

int oracle_gauss(int nlat, double *x, double *w)
{
    if (nlat < 1) return -1;
    for (int j = 0; j < nlat; ++j) {
        /* starting guess: the usual asymptotic cosine estimate of the j-th root */
        double xj = cos(PI * (j + 0.75) / (nlat + 0.5));
        double pn, pnm1, dp;
        for (int it = 0; it < 100; ++it) {
            legendre_poly(nlat, xj, &pn, &pnm1);
            dp = nlat * (pnm1 - xj * pn) / ((1.0 - xj) * (1.0 + xj));
            double dx = pn / dp;
            xj -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        /* one more step at the converged point */
        legendre_poly(nlat, xj, &pn, &pnm1);
        dp = nlat * (pnm1 - xj * pn) / ((1.0 - xj) * (1.0 + xj));
        xj -= pn / dp;
        legendre_poly(nlat, xj, &pn, &pnm1);
        dp = nlat * (pnm1 - xj * pn) / ((1.0 - xj) * (1.0 + xj));
        x[j] = xj;
        w[j] = 2.0 / ((1.0 - xj) * (1.0 + xj) * dp * dp);
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Associated Legendre functions, one order m at one point x (Sec. 3.2):
 *   P_m^m     = a_m^m (1 - x^2)^{m/2},  a_m^m = sqrt( (1/4pi) prod_{k=1}^{m} (2k+1)/(2k) )
 *   P_{m+1}^m = a_{m+1}^m x P_m^m       (a_{m+1}^m = sqrt(2m+3))
 *   P_n^m     = a_n^m x P_{n-1}^m + b_n^m P_{n-2}^m,
 *   a_n^m = sqrt((4n^2 - 1)/(n^2 - m^2)),
 *   b_n^m = -sqrt( (2n+1)/(2n-3) * ((n-1)^2 - m^2)/(n^2 - m^2) ).
 * out[n - m] = P_n^m(x) for n = m..lmax.  Values are carried as y * 2^e with a
 * common integer exponent e (exact power-of-two rescaling), so the result is
 * the recurrence's value rounded once to a double.
 * ------------------------------------------------------------------------- */
static void plm_order(int lmax, int m, double x, double *out)
{
    double s = sqrt((1.0 - x) * (1.0 + x));
    int e = 0, ee;
    double y = sqrt(1.0 / (4.0 * PI));
    for (int k = 1; k <= m; ++k) {
        y *= sqrt((2.0 * k + 1.0) / (2.0 * k)) * s;
        y = frexp(y, &ee);
        e += ee;
    }
    out[0] = ldexp(y, e);
    if (lmax == m) return;
    double y_nm2 = y;                                   /* P_m^m     */
    double y_nm1 = sqrt(2.0 * m + 3.0) * x * y;         /* P_{m+1}^m */
    out[1] = ldexp(y_nm1, e);
    for (int n = m + 2; n <= lmax; ++n) {
        double dn = n, dm = m;
        double a = sqrt((4.0 * dn * dn - 1.0) / (dn * dn - dm * dm));
        double b = -sqrt((2.0 * dn + 1.0) / (2.0 * dn - 3.0)
                         * ((dn - 1.0) * (dn - 1.0) - dm * dm) / (dn * dn - dm * dm));
        double y_n = a * x * y_nm1 + b * y_nm2;
        y_nm2 = y_nm1;
        y_nm1 = y_n;
        double big = fmax(fabs(y_nm1), fabs(y_nm2));
        if (big > 0x1p256) {
            y_nm1 = ldexp(y_nm1, -256); y_nm2 = ldexp(y_nm2, -256); e += 256;
        } else if (big < 0x1p-256 && big > 0.0) {
            y_nm1 = ldexp(y_nm1, 256); y_nm2 = ldexp(y_nm2, 256); e -= 256;
        }
        out[n - m] = ldexp(y_nm1, e);   /* y_nm1 now holds P_n^m * 2^-e */
    }
}

/* dtheta[n - m] = dP_n^m(cos theta)/dtheta from
 *   sin(theta) dP_n^m/dtheta = n x P_n^m - sqrt((2n+1)(n^2-m^2)/(2n-1)) P_{n-1}^m,
 * with P_{m-1}^m = 0.  p[] holds P_n^m, n = m..lmax. */
static void dtheta_order(int lmax, int m, double x, const double *p, double *dtheta)
{
    double s = sqrt((1.0 - x) * (1.0 + x));
    for (int n = m; n <= lmax; ++n) {
        double dn = n, dm = m;
        double prev = (n > m) ? p[n - m - 1] : 0.0;
        double c = (n > m) ? sqrt((2.0 * dn + 1.0) * (dn * dn - dm * dm) / (2.0 * dn - 1.0)) : 0.0;
        dtheta[n - m] = (dn * x * p[n - m] - c * prev) / s;
    }
}

/* Public: P_n^m(x) for all (n, m <= mmax) into the packed layout. */
void oracle_plm(int lmax, int mmax, double x, double *out)
{
    double *col = (double *)malloc(sizeof(double) * (lmax + 1));
    for (int m = 0; m <= mmax; ++m) {
        plm_order(lmax, m, x, col);
        for (int n = m; n <= lmax; ++n) out[lm_index(lmax, n, m)] = col[n - m];
    }
    free(col);
}

/* Public: P_n^m(x) and dP_n^m/dtheta at x of one order m, n = m..lmax, into
 * p[n - m] and (if not NULL) dtheta[n - m] -- the columns oracle_plm and
 * oracle_dplm pack, for callers that need one order at many nodes. */
void oracle_plm_order(int lmax, int m, double x, double *p, double *dtheta)
{
    plm_order(lmax, m, x, p);
    if (dtheta) dtheta_order(lmax, m, x, p, dtheta);
}

/* Public: dP_n^m/dtheta at x for all (n, m <= mmax), packed. */
void oracle_dplm(int lmax, int mmax, double x, double *out)
{
    double *col = (double *)malloc(sizeof(double) * (lmax + 1));
    double *dcol = (double *)malloc(sizeof(double) * (lmax + 1));
    for (int m = 0; m <= mmax; ++m) {
        plm_order(lmax, m, x, col);
        dtheta_order(lmax, m, x, col, dcol);
        for (int n = m; n <= lmax; ++n) out[lm_index(lmax, n, m)] = dcol[n - m];
    }
    free(col);
    free(dcol);
}

/* ---------------------------------------------------------------------------
 * Longitude sums, written as direct Fourier sums (no FFT).
 * cos/sin(m phi_k) = cos/sin(2 pi q / nphi) with q = m k mod nphi.
 * ------------------------------------------------------------------------- */
typedef struct { double *c, *s; int nphi; } trig_table;

static trig_table trig_make(int nphi)
{
    trig_table t;
    t.nphi = nphi;
    t.c = (double *)malloc(sizeof(double) * nphi);
    t.s = (double *)malloc(sizeof(double) * nphi);
    for (int q = 0; q < nphi; ++q) {
        t.c[q] = cos(2.0 * PI * q / nphi);
        t.s[q] = sin(2.0 * PI * q / nphi);
    }
    return t;
}

static void trig_free(trig_table *t) { free(t->c); free(t->s); }

/* row[k] = scale * sum_{m=0}^{mmax} cm(m) Re(F[m] e^{i m phi_k}); F interleaved complex.
 * cm(0) = c0, cm(m>0) = cpos.  Only Re F[0] enters. */
static void fourier_synth_row(const trig_table *t, int mmax, const double *F,
                              double c0, double cpos, double scale, double *row)
{
    int nphi = t->nphi;
    for (int k = 0; k < nphi; ++k) {
        double acc = c0 * F[0];
        for (int m = 1; m <= mmax; ++m) {
            int q = (int)(((long)m * k) % nphi);
            acc += cpos * (F[2 * m] * t->c[q] - F[2 * m + 1] * t->s[q]);
        }
        row[k] = scale * acc;
    }
}

/* ---------------------------------------------------------------------------
 * Scalar synthesis (Sec. 2.2): F_m(theta_j) = sum_{n=m}^{lmax} f_n^m P_n^m(x_j),
 * f(theta_j, phi_k) = sum_m c_m Re(F_m e^{i m phi_k}).
 *
 * rows == NULL: all nlat rows of grid[nlat][nphi] are written; otherwise only
 * the nrows listed rows (others untouched).
 * adjoint of analysis (analys_adj): same sum with c_m = 1 for all m and row
 * weight (2 pi / nphi) w_j.
 * ------------------------------------------------------------------------- */
static void scalar_synth_core(int lmax, int mmax, int nlat, int nphi, const double *spec,
                              double *grid, const int *rows, int nrows, int adjoint_of_analysis)
{
    double *x = (double *)malloc(sizeof(double) * nlat);
    double *w = (double *)malloc(sizeof(double) * nlat);
    oracle_gauss(nlat, x, w);
    int nr = rows ? nrows : nlat;
    /* F[r][m] complex for each selected row r */
    double *F = (double *)calloc((size_t)nr * (mmax + 1) * 2, sizeof(double));
    /* Legendre stage: OpenMP over m, cyclic assignment (Sec. 3.3) */
#pragma omp parallel
    {
        double *col = (double *)malloc(sizeof(double) * (lmax + 1));
#pragma omp for schedule(static, 1)
        for (int m = 0; m <= mmax; ++m) {
            for (int r = 0; r < nr; ++r) {
                int j = rows ? rows[r] : r;
                plm_order(lmax, m, x[j], col);
                double re = 0.0, im = 0.0;
                for (int n = m; n <= lmax; ++n) {
                    long i = lm_index(lmax, n, m);
                    re += spec[2 * i] * col[n - m];
                    im += spec[2 * i + 1] * col[n - m];
                }
                F[((size_t)r * (mmax + 1) + m) * 2] = re;
                F[((size_t)r * (mmax + 1) + m) * 2 + 1] = (m == 0) ? 0.0 : im;
            }
        }
        free(col);
    }
    trig_table t = trig_make(nphi);
#pragma omp parallel for schedule(static, 1)
    for (int r = 0; r < nr; ++r) {
        int j = rows ? rows[r] : r;
        double scale = adjoint_of_analysis ? (2.0 * PI / nphi) * w[j] : 1.0;
        double cpos = adjoint_of_analysis ? 1.0 : 2.0;
        fourier_synth_row(&t, mmax, F + (size_t)r * (mmax + 1) * 2, 1.0, cpos, scale,
                          grid + (size_t)j * nphi);
    }
    trig_free(&t);
    free(F);
    free(x);
    free(w);
}

/* ---------------------------------------------------------------------------
 * Scalar analysis (Sec. 2.3): F_m(theta_j) = (2 pi/nphi) sum_k f_jk e^{-i m phi_k},
 * f_n^m = sum_j w_j P_n^m(x_j) F_m(theta_j).
 * ms == NULL: all orders; otherwise only the listed orders of spec are written.
 * adjoint of synthesis (synth_adj): no weights, no 2 pi/nphi, factor c_m.
 * ------------------------------------------------------------------------- */
static void scalar_analys_core(int lmax, int mmax, int nlat, int nphi, const double *grid,
                               double *spec, const int *ms, int nms, int adjoint_of_synthesis)
{
    double *x = (double *)malloc(sizeof(double) * nlat);
    double *w = (double *)malloc(sizeof(double) * nlat);
    oracle_gauss(nlat, x, w);
    int nm = ms ? nms : mmax + 1;
    trig_table t = trig_make(nphi);
    double fscale = adjoint_of_synthesis ? 1.0 : 2.0 * PI / nphi;
    /* Legendre stage: OpenMP over the orders, cyclic assignment (Sec. 3.3) */
#pragma omp parallel
    {
        double *col = (double *)malloc(sizeof(double) * (lmax + 1));
        double *acc = (double *)malloc(sizeof(double) * 2 * (lmax + 1));
        double *F = (double *)malloc(sizeof(double) * 2 * (size_t)nlat);
#pragma omp for schedule(static, 1)
        for (int q = 0; q < nm; ++q) {
            int m = ms ? ms[q] : q;
            /* F_m(theta_j) = fscale sum_k f_jk e^{-i m phi_k} for this order */
            for (int j = 0; j < nlat; ++j) {
                const double *row = grid + (size_t)j * nphi;
                double re = 0.0, im = 0.0;
                for (int k = 0; k < nphi; ++k) {
                    int qq = (int)(((long)m * k) % nphi);
                    re += row[k] * t.c[qq];
                    im -= row[k] * t.s[qq];
                }
                F[2 * j] = fscale * re;
                F[2 * j + 1] = fscale * im;
            }
            memset(acc, 0, sizeof(double) * 2 * (lmax + 1));
            for (int j = 0; j < nlat; ++j) {
                plm_order(lmax, m, x[j], col);
                double wj = adjoint_of_synthesis ? 1.0 : w[j];
                for (int n = m; n <= lmax; ++n) {
                    acc[2 * (n - m)] += wj * col[n - m] * F[2 * j];
                    acc[2 * (n - m) + 1] += wj * col[n - m] * F[2 * j + 1];
                }
            }
            double cm = adjoint_of_synthesis ? (m == 0 ? 1.0 : 2.0) : 1.0;
            for (int n = m; n <= lmax; ++n) {
                long i = lm_index(lmax, n, m);
                spec[2 * i] = cm * acc[2 * (n - m)];
                spec[2 * i + 1] = (m == 0) ? 0.0 : cm * acc[2 * (n - m) + 1];
            }
        }
        free(col);
        free(acc);
        free(F);
    }
    trig_free(&t);
    free(x);
    free(w);
}

void oracle_synth(int lmax, int mmax, int nlat, int nphi, const double *spec, double *grid,
                  const int *rows, int nrows)
{
    scalar_synth_core(lmax, mmax, nlat, nphi, spec, grid, rows, nrows, 0);
}

void oracle_analys(int lmax, int mmax, int nlat, int nphi, const double *grid, double *spec,
                   const int *ms, int nms)
{
    scalar_analys_core(lmax, mmax, nlat, nphi, grid, spec, ms, nms, 0);
}

/* Adjoint of synthesis: b_n^m = c_m sum_j P_n^m(x_j) sum_k g_jk e^{-i m phi_k}. */
void oracle_synth_adj(int lmax, int mmax, int nlat, int nphi, const double *grid, double *spec,
                      const int *ms, int nms)
{
    scalar_analys_core(lmax, mmax, nlat, nphi, grid, spec, ms, nms, 1);
}

/* Adjoint of analysis: g_jk = (2 pi/nphi) w_j sum_{m>=0} Re(e^{i m phi_k} sum_n P_n^m b_n^m). */
void oracle_analys_adj(int lmax, int mmax, int nlat, int nphi, const double *spec, double *grid,
                       const int *rows, int nrows)
{
    scalar_synth_core(lmax, mmax, nlat, nphi, spec, grid, rows, nrows, 1);
}

/* ---------------------------------------------------------------------------
 * Vector synthesis: per order m and latitude j
 *   V_theta,m = sum_n [ S_n^m dP_n^m/dtheta - (i m / sin) T_n^m P_n^m ]
 *   V_phi,m   = sum_n [ (i m / sin) S_n^m P_n^m + T_n^m dP_n^m/dtheta ]
 * then v = sum_m c_m Re(V_m e^{i m phi}).
 * adjoint of analysis (analys_vec_adj): coefficients divided by n(n+1) (n = 0
 * dropped), c_m = 1 and row weight (2 pi/nphi) w_j.
 * ------------------------------------------------------------------------- */
static void vector_synth_core(int lmax, int mmax, int nlat, int nphi, const double *S,
                              const double *T, double *vt, double *vp, const int *rows,
                              int nrows, int adjoint_of_analysis)
{
    double *x = (double *)malloc(sizeof(double) * nlat);
    double *w = (double *)malloc(sizeof(double) * nlat);
    oracle_gauss(nlat, x, w);
    int nr = rows ? nrows : nlat;
    size_t fsz = (size_t)nr * (mmax + 1) * 2;
    double *Ft = (double *)calloc(fsz, sizeof(double));
    double *Fp = (double *)calloc(fsz, sizeof(double));
#pragma omp parallel
    {
        double *col = (double *)malloc(sizeof(double) * (lmax + 1));
        double *dcol = (double *)malloc(sizeof(double) * (lmax + 1));
#pragma omp for schedule(static, 1)
        for (int m = 0; m <= mmax; ++m) {
            for (int r = 0; r < nr; ++r) {
                int j = rows ? rows[r] : r;
                double s = sqrt((1.0 - x[j]) * (1.0 + x[j]));
                plm_order(lmax, m, x[j], col);
                dtheta_order(lmax, m, x[j], col, dcol);
                double tr = 0, ti = 0, pr = 0, pi_ = 0;
                for (int n = m; n <= lmax; ++n) {
                    long i = lm_index(lmax, n, m);
                    double f = 1.0;
                    if (adjoint_of_analysis) f = (n == 0) ? 0.0 : 1.0 / ((double)n * (n + 1));
                    double Sr = f * S[2 * i], Si = f * S[2 * i + 1];
                    double Tr = f * T[2 * i], Ti = f * T[2 * i + 1];
                    double P = col[n - m], dP = dcol[n - m];
                    double ms = (double)m / s;
                    /* V_theta += S dP - i (m/s) T P */
                    tr += Sr * dP + ms * Ti * P;
                    ti += Si * dP - ms * Tr * P;
                    /* V_phi += i (m/s) S P + T dP */
                    pr += -ms * Si * P + Tr * dP;
                    pi_ += ms * Sr * P + Ti * dP;
                }
                size_t o = ((size_t)r * (mmax + 1) + m) * 2;
                Ft[o] = tr; Ft[o + 1] = (m == 0) ? 0.0 : ti;
                Fp[o] = pr; Fp[o + 1] = (m == 0) ? 0.0 : pi_;
            }
        }
        free(col);
        free(dcol);
    }
    trig_table t = trig_make(nphi);
#pragma omp parallel for schedule(static, 1)
    for (int r = 0; r < nr; ++r) {
        int j = rows ? rows[r] : r;
        double scale = adjoint_of_analysis ? (2.0 * PI / nphi) * w[j] : 1.0;
        double cpos = adjoint_of_analysis ? 1.0 : 2.0;
        fourier_synth_row(&t, mmax, Ft + (size_t)r * (mmax + 1) * 2, 1.0, cpos, scale, vt + (size_t)j * nphi);
        fourier_synth_row(&t, mmax, Fp + (size_t)r * (mmax + 1) * 2, 1.0, cpos, scale, vp + (size_t)j * nphi);
    }
    trig_free(&t);
    free(Ft);
    free(Fp);
    free(x);
    free(w);
}

/* ---------------------------------------------------------------------------
 * Vector analysis: V_m = (2 pi/nphi) sum_k v_jk e^{-i m phi_k},
 *   S_n^m = [n(n+1)]^-1 sum_j w_j [ V_theta dP/dtheta - (i m/sin) V_phi P ]
 *   T_n^m = [n(n+1)]^-1 sum_j w_j [ (i m/sin) V_theta P + V_phi dP/dtheta ]
 * n = 0 gives 0.
 * adjoint of synthesis (synth_vec_adj): no weights, no 2 pi/nphi, factor c_m
 * in place of 1/(n(n+1)).
 * ------------------------------------------------------------------------- */
static void vector_analys_core(int lmax, int mmax, int nlat, int nphi, const double *vt,
                               const double *vp, double *S, double *T, const int *ms, int nms,
                               int adjoint_of_synthesis)
{
    double *x = (double *)malloc(sizeof(double) * nlat);
    double *w = (double *)malloc(sizeof(double) * nlat);
    oracle_gauss(nlat, x, w);
    int nm = ms ? nms : mmax + 1;
    trig_table t = trig_make(nphi);
    double fscale = adjoint_of_synthesis ? 1.0 : 2.0 * PI / nphi;
#pragma omp parallel
    {
        double *col = (double *)malloc(sizeof(double) * (lmax + 1));
        double *dcol = (double *)malloc(sizeof(double) * (lmax + 1));
        double *acc = (double *)malloc(sizeof(double) * 4 * (lmax + 1));
        double *Ft = (double *)malloc(sizeof(double) * 2 * (size_t)nlat);
        double *Fp = (double *)malloc(sizeof(double) * 2 * (size_t)nlat);
#pragma omp for schedule(static, 1)
        for (int q = 0; q < nm; ++q) {
            int m = ms ? ms[q] : q;
            for (int j = 0; j < nlat; ++j) {
                const double *rt = vt + (size_t)j * nphi, *rp = vp + (size_t)j * nphi;
                double tr = 0.0, ti = 0.0, pr = 0.0, pim = 0.0;
                for (int k = 0; k < nphi; ++k) {
                    int qq = (int)(((long)m * k) % nphi);
                    tr += rt[k] * t.c[qq];
                    ti -= rt[k] * t.s[qq];
                    pr += rp[k] * t.c[qq];
                    pim -= rp[k] * t.s[qq];
                }
                Ft[2 * j] = fscale * tr; Ft[2 * j + 1] = fscale * ti;
                Fp[2 * j] = fscale * pr; Fp[2 * j + 1] = fscale * pim;
            }
            memset(acc, 0, sizeof(double) * 4 * (lmax + 1));
            for (int j = 0; j < nlat; ++j) {
                double s = sqrt((1.0 - x[j]) * (1.0 + x[j]));
                plm_order(lmax, m, x[j], col);
                dtheta_order(lmax, m, x[j], col, dcol);
                double wj = adjoint_of_synthesis ? 1.0 : w[j];
                double Vtr = Ft[2 * j], Vti = Ft[2 * j + 1], Vpr = Fp[2 * j], Vpi = Fp[2 * j + 1];
                double msj = (double)m / s;
                for (int n = m; n <= lmax; ++n) {
                    double P = col[n - m], dP = dcol[n - m];
                    /* S += w [V_theta dP - i (m/s) V_phi P] */
                    acc[4 * (n - m) + 0] += wj * (Vtr * dP + msj * Vpi * P);
                    acc[4 * (n - m) + 1] += wj * (Vti * dP - msj * Vpr * P);
                    /* T += w [i (m/s) V_theta P + V_phi dP] */
                    acc[4 * (n - m) + 2] += wj * (-msj * Vti * P + Vpr * dP);
                    acc[4 * (n - m) + 3] += wj * (msj * Vtr * P + Vpi * dP);
                }
            }
            for (int n = m; n <= lmax; ++n) {
                long i = lm_index(lmax, n, m);
                double f;
                if (adjoint_of_synthesis) f = (m == 0) ? 1.0 : 2.0;
                else f = (n == 0) ? 0.0 : 1.0 / ((double)n * (n + 1));
                S[2 * i] = f * acc[4 * (n - m) + 0];
                S[2 * i + 1] = (m == 0) ? 0.0 : f * acc[4 * (n - m) + 1];
                T[2 * i] = f * acc[4 * (n - m) + 2];
                T[2 * i + 1] = (m == 0) ? 0.0 : f * acc[4 * (n - m) + 3];
            }
        }
        free(col);
        free(dcol);
        free(acc);
        free(Ft);
        free(Fp);
    }
    trig_free(&t);
    free(x);
    free(w);
}

void oracle_synth_vec(int lmax, int mmax, int nlat, int nphi, const double *S, const double *T,
                      double *vt, double *vp, const int *rows, int nrows)
{
    vector_synth_core(lmax, mmax, nlat, nphi, S, T, vt, vp, rows, nrows, 0);
}

void oracle_analys_vec(int lmax, int mmax, int nlat, int nphi, const double *vt, const double *vp,
                       double *S, double *T, const int *ms, int nms)
{
    vector_analys_core(lmax, mmax, nlat, nphi, vt, vp, S, T, ms, nms, 0);
}

/* Adjoint of vector synthesis:
 *   S'_n^m = c_m sum_j [ dP/dtheta G_theta,m - (i m/sin) P G_phi,m ],
 *   T'_n^m = c_m sum_j [ (i m/sin) P G_theta,m + dP/dtheta G_phi,m ],
 *   G_m = sum_k g_jk e^{-i m phi_k}. */
void oracle_synth_vec_adj(int lmax, int mmax, int nlat, int nphi, const double *gt,
                          const double *gp, double *S, double *T, const int *ms, int nms)
{
    vector_analys_core(lmax, mmax, nlat, nphi, gt, gp, S, T, ms, nms, 1);
}

/* Adjoint of vector analysis: the weighted vector synthesis of b / n(n+1)
 * with c_m = 1 and row weight (2 pi/nphi) w_j. */
void oracle_analys_vec_adj(int lmax, int mmax, int nlat, int nphi, const double *S,
                           const double *T, double *gt, double *gp, const int *rows, int nrows)
{
    vector_synth_core(lmax, mmax, nlat, nphi, S, T, gt, gp, rows, nrows, 1);
}
