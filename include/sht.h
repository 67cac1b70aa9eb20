/*
 * sht.h -- C ABI of libsht, a Gauss-Legendre spherical harmonic transform for
 * NVIDIA GB300 (sm_103a).
 *
 * The method is the one of Schaeffer, "Efficient Spherical Harmonic Transforms
 * aimed at pseudo-spectral numerical simulations" (arXiv:1202.6522):
 *   synthesis  f(theta, phi) = sum_m ( sum_n f_n^m P_n^m(cos theta) ) e^{i m phi}
 *              (Sec. 2.2, Eq. synth_direct, then a real FFT in longitude),
 *   analysis   f_n^m = sum_j w_j P_n^m(cos theta_j) f_m(theta_j)
 *              (Sec. 2.3, Eq. gauss, after a real FFT in longitude),
 * with P_n^m generated on the fly by the recurrence of Sec. 3.2, north/south
 * folding by the mirror symmetry of Sec. 3.1 and the underflow rescaling of
 * Sec. 3.5.
 *
 * Conventions
 *   - Orthonormal P_n^m as produced by the recurrence of Sec. 3.2: P_m^m > 0,
 *     i.e. no (-1)^m Condon-Shortley factor.
 *   - Real fields: only m >= 0 is stored (Hermitian symmetry, Sec. 3.1).
 *     Im f_n^0 is ignored on input and written as 0 on output.
 *   - Spectral layout: packed m-major, idx(n, m) = m (2 lmax + 3 - m) / 2 + (n - m)
 *     for 0 <= m <= mmax, m <= n <= lmax; interleaved complex (re, im).
 *     nlm = sht_nlm(h) coefficients per field.
 *   - Grid layout: [nlat][nphi] reals per field, row j at the Gauss node x_j
 *     (x descending: north to south), column k at phi_k = 2 pi k / nphi.
 *   - Batches are contiguous: field b of a spectral array starts at b * nlm
 *     complex values, of a grid at b * nlat * nphi reals.
 *   - Vector fields: v = grad_H S + r x grad_H T, that is
 *       v_theta = dS/dtheta - (1/sin theta) dT/dphi,
 *       v_phi   = (1/sin theta) dS/dphi + dT/dtheta;
 *     vector analysis divides by n(n+1) and returns 0 at n = 0.
 *   - Adjoints are taken for <a, b> = sum_packed Re(conj(a) b) (m = 0
 *     imaginary parts excluded) and <f, g> = sum f g.
 *
 * Memory and streams
 *   - Every data pointer is a DEVICE pointer owned by the caller, contiguous,
 *     aligned to at least 16 bytes.  Element type follows `mode`:
 *       SHT_F64: double (spectral arrays: pairs of doubles);
 *       SHT_F32: float.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls only
 *     enqueue work; they do not synchronise.  Input and output must not alias.
 *   - The handle owns its tables and a scratch buffer that grows on demand
 *     (the first call at a larger batch allocates; sht_reserve allocates ahead).
 *     Calls on one handle must not run concurrently on different streams.
 *
 * Errors
 *   Every int-returning function returns SHT_OK (0) or a negative code;
 *   sht_last_error() gives a message for the calling thread.  Argument errors
 *   are detected on the host before anything is enqueued.
 */
#ifndef SHT_H
#define SHT_H

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SHT_API __attribute__((visibility("default")))
#else
#define SHT_API
#endif

typedef struct sht_plan *sht_handle;

enum {
    SHT_OK = 0,
    SHT_EINVAL = -1,       /* bad argument (sizes, null pointer, mode)           */
    SHT_ENOMEM = -2,       /* device or host allocation failed                   */
    SHT_ECUDA = -3,        /* a CUDA runtime call failed                         */
    SHT_ETIMEOUT = -4,     /* a bounded device-side wait gave up                 */
    SHT_EUNSUPPORTED = -5  /* valid but not supported (e.g. nphi not a power of 2) */
};

enum {
    SHT_F64 = 0,       /* FP64 throughout: the plain path.  Scalar transforms restart
                        * the recurrence at every 32-degree segment they run, from
                        * states the FP64 recurrence computes once per plan together
                        * with the table of the static polar optimisation (built by
                        * the first scalar call in this mode or by sht_reserve: 20 B
                        * per latitude pair and 32 degrees, 175 MB at lmax = 1023). */
    SHT_F32 = 1,       /* FP32 data and recurrence with the explicit exponent scale of
                        * Sec. 3.5, restarted every 32 degrees from states the FP64
                        * recurrence computes once per plan (built by the first call
                        * in this mode or by sht_reserve: 16 B per latitude pair and
                        * 32 degrees, (lmax+1)^2 ceil(nlat/2) / 4 bytes, 138 MB at
                        * lmax = 1023), so that FP32 rounding errors grow over at most
                        * 32 steps instead of lmax. */
    SHT_TC_BF16X3 = 2, /* FP32 data; the per-order Legendre contraction on the tensor
                        * cores against P_n^m panels built once by the FP64 recurrence
                        * (the precomputed-P_n^m variant of Sec. 3.1), each operand split
                        * into bf16 hi + lo and multiplied as hi*hi + hi*lo + lo*hi with
                        * FP32 accumulation.  Scalar and vector transforms and their
                        * adjoints; vector calls add panels of sin(theta) dP/dtheta.
                        * The panels take about 2 (lmax+1)^3 bytes (2.2 GB at
                        * lmax = 1023; twice that once a vector call was made) and
                        * are built by the first call in this mode or by sht_reserve. */
    SHT_F32_AUTO = 3,  /* FP32 data: whichever of SHT_F32, SHT_TC_BF16X3 and SHT_TC_OTF
                        * sht_tune measured fastest for this batch size (SHT_F32 if
                        * untuned); vector transforms take SHT_F32. */
    SHT_TC_OTF = 4,    /* FP32 data; the same tensor-core contraction, but P_n^m is
                        * generated on the fly (the variant of Sec. 3.1 the paper
                        * favours) by CUDA-core warps inside the contraction kernel:
                        * the FP32 recurrence of Sec. 3.2, restarted every 32 degrees
                        * from seeds computed once by the FP64 recurrence with the
                        * rescaling of Sec. 3.5, so rounding errors grow over at most
                        * 32 steps.  Seeds take 16 (lmax+1)^2 ceil(nlat/2) / 64 bytes
                        * (138 MB at lmax = 1023) instead of the panels' ~(lmax+1)^3.
                        * Scalar transforms and adjoints; vector calls run
                        * SHT_TC_BF16X3.  SHT_EUNSUPPORTED if a segment of the
                        * recurrence would leave the FP32 range (large lmax). */
    SHT_TC_F64 = 5     /* FP64 data; the per-order Legendre contraction on the bf16
                        * tensor cores to FP64 accuracy: P_n^m (per row) and the data
                        * (per field) are scaled by powers of two and split into
                        * signed 7-bit digit slices (7 for P: 49 bits of the row
                        * maximum; 8 for the data: 56 bits of the field maximum); the
                        * tensor core sums the integer products of each level exactly
                        * in FP32, and the epilogue combines the 8 leading levels in
                        * 128-bit integers.  FFTs in double-float arithmetic (pairs of
                        * FP32 numbers, ~2^-48 per operation) with a power-of-two scale
                        * per latitude pair.  Scalar transforms and adjoints, up to 16
                        * fields per launch (larger batches run in groups of 16).
                        * Requires lmax <= 1023 and nlat <= 1024 (so that every
                        * level's sum stays below 2^24), else SHT_EUNSUPPORTED.  The
                        * digit panels take about 8 (lmax+1)^3 bytes (8.6 GB at
                        * lmax = 1023) and are built by the first call in this mode
                        * or by sht_reserve. */
};

/* Build a plan (Sec. 2.3 nodes/weights, Sec. 3.2 recurrence tables, FFT
 * twiddles) on the host and copy it to the current CUDA device.
 * Requires 0 <= mmax <= lmax, nlat >= lmax + 1 (exactness of the quadrature,
 * Sec. 2.3), nphi >= 2 mmax + 1 and nphi = 2 x 2^a 3^b 5^c <= 8192
 * (SHT_EUNSUPPORTED otherwise; the longitude FFT of length nphi / 2 runs in
 * radix-16/8/4/2, 3 and 5 passes, and power-of-two lengths up to 1024 in FP32
 * take the faster one-warp-per-row kernel).  On success *out receives the
 * handle; on failure *out is NULL. */
SHT_API int sht_create(int lmax, int mmax, int nlat, int nphi, sht_handle *out);

/* Plan for the orders m = k mres, k = 0 .. mmax (mmax mres <= lmax): fields
 * whose longitude period is 2 pi / mres, sampled on one sector of the circle,
 * phi_j = 2 pi j / (nphi mres), j < nphi (the m-stride variant; needs
 * nphi >= 2 mmax + 1).  The spectral layout packs the orders present:
 * order index k holds degrees n = k mres .. lmax, from index
 * k (lmax + 1) - mres k (k - 1) / 2 (sht_lm_index takes the order m itself).
 * The longitude quadrature is the rectangle rule on the sector, equal to the
 * full circle's for these orders.  Every mode takes such plans: the
 * tensor-core panels, recurrence seeds and digit tables hold the strided
 * orders only.  sht_create(...) is sht_create_mres(lmax, mmax, 1, ...). */
SHT_API int sht_create_mres(int lmax, int mmax, int mres, int nlat, int nphi, sht_handle *out);

/* Free the plan and everything it owns.  NULL is ignored.  The caller must
 * make sure no work using the handle is still running. */
SHT_API void sht_destroy(sht_handle h);

/* Pre-allocate scratch for transforms of up to `batch` fields in `mode`, so
 * that later calls at that size allocate nothing (SHT_TC_BF16X3: scalar and
 * vector transforms, including the vector panels). */
SHT_API int sht_reserve(sht_handle h, int batch, int mode);

/* Scalar synthesis, Sec. 2.2: spec [batch][nlm] complex -> grid [batch][nlat][nphi]. */
SHT_API int sht_synth(sht_handle h, const void *spec, void *grid, int batch, int mode, void *stream);

/* Scalar analysis, Sec. 2.3 (Gauss-Legendre quadrature):
 * grid [batch][nlat][nphi] -> spec [batch][nlm] complex. */
SHT_API int sht_analys(sht_handle h, const void *grid, void *spec, int batch, int mode, void *stream);

/* Spheroidal/toroidal synthesis (vector transform named in Sec. 4):
 * S, T [batch][nlm] complex -> v_theta, v_phi [batch][nlat][nphi]. */
SHT_API int sht_synth_vec(sht_handle h, const void *S, const void *T, void *vt, void *vp,
                  int batch, int mode, void *stream);

/* Spheroidal/toroidal analysis: v_theta, v_phi -> S, T (divided by n(n+1)). */
SHT_API int sht_analys_vec(sht_handle h, const void *vt, const void *vp, void *S, void *T,
                   int batch, int mode, void *stream);

/* Adjoint of sht_synth: grid -> spec,
 *   b_n^m = c_m sum_j P_n^m(x_j) sum_k g_jk e^{-i m phi_k},  c_0 = 1, c_m = 2. */
SHT_API int sht_synth_adj(sht_handle h, const void *grid, void *spec, int batch, int mode, void *stream);

/* Adjoint of sht_analys: spec -> grid,
 *   g_jk = (2 pi / nphi) w_j sum_{m>=0} Re(e^{i m phi_k} sum_n P_n^m b_n^m). */
SHT_API int sht_analys_adj(sht_handle h, const void *spec, void *grid, int batch, int mode, void *stream);

/* Adjoint of sht_synth_vec: (g_theta, g_phi) -> (S', T'). */
SHT_API int sht_synth_vec_adj(sht_handle h, const void *gt, const void *gp, void *S, void *T,
                      int batch, int mode, void *stream);

/* Adjoint of sht_analys_vec: (S', T') -> (g_theta, g_phi). */
SHT_API int sht_analys_vec_adj(sht_handle h, const void *S, const void *T, void *gt, void *gp,
                       int batch, int mode, void *stream);

/* Layout helpers: number of packed coefficients, and idx(n, m) (-1 if out of range). */
SHT_API int sht_nlm(sht_handle h);
SHT_API int sht_lm_index(sht_handle h, int n, int m);

/* Host copies of the Gauss nodes x_j = cos(theta_j) (descending) and weights
 * w_j, each an array of nlat doubles owned by the caller. */
SHT_API int sht_gauss(sht_handle h, double *x, double *w);

/* Synchronise `stream` and report any CUDA error raised by work enqueued by
 * this library (SHT_ECUDA), a tensor-core kernel whose bounded wait for its
 * own copies or MMAs gave up (SHT_ETIMEOUT; the kernel then skipped its
 * output and returned), or SHT_OK.  Reading the status clears it. */
SHT_API int sht_sync_status(sht_handle h, void *stream);

/* Scalar synthesis that allocates nothing (no counterpart in the paper; an
 * interface addition).  Same inputs, outputs and result as sht_synth, but its
 * intermediate buffer is a fixed array compiled into this library instead of
 * the handle's scratch, so the call never asks the CUDA runtime for memory.
 * It is meant for callers that must not allocate device memory at call time:
 * code that runs under a fixed device-memory budget owned by a host framework
 * or a custom pool, and loops where the implicit device synchronisation of
 * cudaMalloc/cudaFree is not acceptable.  The handle itself must have been
 * created beforehand (sht_create allocates the plan tables).
 *   - Modes SHT_F64 and SHT_F32 (SHT_F32_AUTO runs SHT_F32 here), any plan
 *     including m-stride ones; SHT_TC_BF16X3, SHT_TC_OTF and SHT_TC_F64 return
 *     SHT_EUNSUPPORTED, their panels or seeds being allocated.  Both modes
 *     need the plan's recurrence restart states of their precision (and the
 *     polar table), which the first scalar call in that mode or
 *     sht_reserve(h, batch, mode) builds; without them the call returns
 *     SHT_EUNSUPPORTED and enqueues nothing.
 *   - The fixed array holds SHT_STATIC_SCRATCH_BYTES (16 MiB) on every GPU that
 *     loads this library, until the process exits.  A call needs
 *     batch * (mmax+1) * ceil(nlat/2) * 4 * sizeof(element) bytes (N = 1023 in
 *     FP64 fits one field, in FP32 two); larger calls return SHT_EINVAL and
 *     enqueue nothing.
 *   - The array's device address is looked up (cudaGetSymbolAddress) by
 *     sht_create, with the plan's device current, and kept per device; this
 *     call only reads it.  cudaDeviceReset invalidates every handle; a handle
 *     created after a reset stores the address of the reloaded module.
 *   - All calls, from any handle, share the one array: calls whose work can
 *     overlap on the GPU (different streams without ordering) race on it.
 *     Nothing in it needs to start at zero: each call overwrites the part it
 *     reads before reading it. */
#define SHT_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)
SHT_API int sht_synth_static(sht_handle h, const void *spec, void *grid, int batch, int mode, void *stream);

/* Runtime tuning, after the paper's runtime tuning (Sec. 3.2): time the
 * candidate kernel shapes of the Legendre stage (latitude pairs per thread x
 * fields per CTA) for `batch` fields in `mode` (SHT_F64 or SHT_F32) and keep
 * the fastest for later calls with that batch size.  With SHT_F32_AUTO it also
 * times full round trips of the FP32 CUDA-core path, the tensor-core path with
 * precomputed panels and the tensor-core path with on-the-fly P_n^m (the
 * paper's precomputed and on-the-fly variants) and records the fastest for
 * SHT_F32_AUTO calls at that batch.
 * report (may be NULL, else 3 doubles): report[0], report[1] = best synthesis
 * and analysis Legendre times in ms (SHT_F64/SHT_F32; report[2] = -1), or the
 * round-trip times in ms of SHT_F32, SHT_TC_BF16X3 and SHT_TC_OTF (SHT_F32_AUTO;
 * -1 for a path that could not run).  Allocates temporary buffers, synchronises the
 * stream, and takes from milliseconds to a few seconds. */
SHT_API int sht_tune(sht_handle h, int batch, int mode, double *report, void *stream);

/* Uneven batches: many scalar FP32 fields, each with its own truncation
 * (mmax = lmax), transformed by one launch.  The plan groups fields of equal
 * shape, builds one tile list per stage over all fields, sorted longest first,
 * and runs each stage as one persistent kernel whose CTAs take tiles from an
 * atomic counter (no CTA waits on another).  With use_graph != 0 the whole
 * sequence (pointer-table copy, counter reset, Legendre and FFT kernels) is
 * captured into a CUDA graph by the first call of each direction and replayed
 * afterwards; the capture happens on a private stream.
 * Limits: nphi = 2 x 2^a 3^b 5^c in [2, 4096], nlat <= 1024.
 * spec[f] / grid[f]: device pointers of field f ([nlm_f] complex floats and
 * [nlat_f][nphi_f] floats).  A call waits on the host until the previous call
 * on this batch plan has started its pointer-table copy. */
typedef struct sht_batch_plan *sht_batch;
SHT_API int sht_batch_create(int nfields, const int *lmax, const int *nlat, const int *nphi, sht_batch *out);
/* The same with a choice of path (Sec. 3.2's runtime choice, for batches):
 * SHT_F32 the persistent CUDA-core kernels above; SHT_TC_BF16X3 the Legendre
 * stage of each group of equal shape as one batched tensor-core contraction
 * against that shape's P panels (built here, ~(N+1)^3 bytes per direction per
 * shape), the group's spectra gathered into (synthesis) or scattered from
 * (analysis) a contiguous buffer by one copy kernel, the FFTs one persistent
 * kernel over all fields -- the graph then holds the copies, one contraction
 * per group and the FFT; SHT_F32_AUTO times a round trip of both on zero
 * fields here (a few launches, synchronising) and keeps the faster.  Errors as
 * sht_batch_create, SHT_EINVAL for another mode, and the tensor-core
 * preparation's (SHT_ENOMEM) for SHT_TC_BF16X3. */
SHT_API int sht_batch_create_mode(int nfields, const int *lmax, const int *nlat, const int *nphi, int mode,
                                  sht_batch *out);
/* The path a batch plan runs (SHT_F32 or SHT_TC_BF16X3); for SHT_F32_AUTO
 * plans also the round-trip times it measured (ms, 0 when not timed) of the
 * CUDA-core and tensor-core paths, into *ms_f32 and *ms_tc (either may be
 * NULL).  Negative SHT error for a NULL handle. */
SHT_API int sht_batch_mode(sht_batch b, float *ms_f32, float *ms_tc);
SHT_API void sht_batch_destroy(sht_batch b);
SHT_API int sht_batch_synth(sht_batch b, void *const *spec, void *const *grid, int use_graph, void *stream);
SHT_API int sht_batch_analys(sht_batch b, void *const *grid, void *const *spec, int use_graph, void *stream);

/* Per-kernel timing, for measurement (no counterpart in the paper).  While
 * enabled, every kernel the handle launches is bracketed by CUDA events on the
 * call's stream.  sht_profile_read synchronises those events and writes, for
 * each kernel kind k < min(cap, SHT_NKERNELS), the summed duration in
 * milliseconds into ms[k] and the number of launches into count[k], then
 * clears the record.  Kind names: sht_kernel_name(k). */
enum {
    SHT_K_LEGENDRE_SYNTH = 0,
    SHT_K_LEGENDRE_ANALYS = 1,
    SHT_K_LEGENDRE_SYNTH_VEC = 2,
    SHT_K_LEGENDRE_ANALYS_VEC = 3,
    SHT_K_FFT_SYNTH = 4,
    SHT_K_FFT_ANALYS = 5,
    SHT_K_TC_SYNTH = 6,      /* data prep + tensor-core contraction */
    SHT_K_TC_ANALYS = 7,
    SHT_K_TC_SYNTH_VEC = 8,
    SHT_K_TC_ANALYS_VEC = 9,
    SHT_NKERNELS = 10
};
SHT_API int sht_profile(sht_handle h, int enable);
SHT_API int sht_profile_read(sht_handle h, double *ms, int *count, int cap);
SHT_API const char *sht_kernel_name(int kind);

/* Static polar optimisation of the tensor-core mode (Sec. 3.1): panel chunks
 * whose values are all below 2^-40 (near the poles at high order) are neither
 * loaded nor multiplied (SHT_TC_OTF: neither generated nor multiplied).
 * Fractions of the synthesis and analysis chunks skipped -- of the panels if
 * built, else of the on-the-fly mode's tables, else of the SHT_TC_F64 digit
 * panels (per chunk, the 8-row groups below its first group with a nonzero
 * digit, which the contraction does not read) -- or -1 if none is built. */
SHT_API int sht_tc_polar_skip(sht_handle h, double *synth_frac, double *analys_frac);

/* Threshold of the static polar optimisation (Sec. 3.1; the paper leaves its
 * value open).  Tensor-core modes: a panel chunk is skipped while all its
 * |P_n^m| (and, for the vector transforms, |sin(theta) dP/dtheta|) are below
 * it; default 2^-40.  CUDA-core scalar transforms (SHT_F64, SHT_F32): per
 * order and latitude pair the 32-degree segments before the first one that
 * holds a |P_n^m| at or above it run neither the recurrence nor the sums
 * (whole warps skip them); defaults 2^-64 (SHT_F64) and 2^-40 (SHT_F32) until
 * the threshold is set, then the set value for both.  0 skips nothing.  Must
 * be in [0, 1]; waits for the device to be idle, then recomputes the skip
 * tables that exist. */
SHT_API int sht_set_polar_threshold(sht_handle h, double threshold);

/* Share of the (order, latitude pair, degree) terms of the CUDA-core scalar
 * transforms in `mode` (SHT_F64 or SHT_F32) that lie before their pair's
 * first live 32-degree segment under the current threshold (the terms the
 * static polar optimisation may skip; a warp skips a segment only when all
 * its pairs do), or -1 if the table was not built yet. */
SHT_API int sht_cc_polar_skip(sht_handle h, int mode, double *frac);

/* Failure-detection self-test (no counterpart in the paper): enqueue a kernel
 * that waits, with a bound of timeout_us microseconds, on a barrier that
 * nothing completes -- the same bounded wait the tensor-core kernels use --
 * so that the next sht_sync_status on that stream reports SHT_ETIMEOUT.  The
 * kernel never faults or hangs, and the handle stays usable afterwards. */
SHT_API int sht_selftest_timeout(sht_handle h, int timeout_us, void *stream);

/* Measured FMA throughput of the current device (no counterpart in the paper;
 * the denominators of the ALU rooflines of the on-the-fly Legendre kernels):
 * 8 independent FMA chains per thread, 8 CTAs of 256 threads per SM, timed
 * with CUDA events on `stream` (which it synchronises).  Writes FP32 and FP64
 * TFLOP/s (an FMA counts 2 flops) at the clock the GPU runs at. */
SHT_API int sht_alu_peaks(double *fp32_tflops, double *fp64_tflops, void *stream);

/* Message for the last error raised in the calling thread ("" if none). */
SHT_API const char *sht_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SHT_H */
