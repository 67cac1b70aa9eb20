// sht_internal.h -- plan structure and kernel launchers shared by the
// translation units of libsht.  Not part of the public ABI (see include/sht.h).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "sht.h"

namespace sht {

// Exponent step of the underflow rescaling (Sec. 3.5): a value is carried as
// y * 2^(-S k) with an integer k >= 0.  While k > 0 the true value is below
// 2^-S: it is left out of the Legendre sums but still advanced by the
// recurrence.  Dropped terms are < 2^-240 (FP64) or 2^-64 (FP32).
template <typename T> struct Scale;
template <> struct Scale<double> { static constexpr int S = 240; };
template <> struct Scale<float> { static constexpr int S = 64; };

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

// Device tables of one precision.
template <typename T>
struct Tables {
    using T2 = typename Vec2<T>::type;
    T2 *ab = nullptr;    // [nlm] (a_n^m, b_n^m); (0, 1) at n = m, (sqrt(2m+3), 0) at n = m+1
    T *dc = nullptr;     // [nlm] sqrt((2n+1)(n^2-m^2)/(2n-1)); 0 at n = m
    T *x = nullptr;      // [npairs] cos(theta) of the northern node of each pair (>= 0)
    T *st = nullptr;     // [npairs] sin(theta)
    T *wq = nullptr;     // [npairs] Gauss weight of that node
    T *pmm = nullptr;    // [mmax+1][npairs] P_m^m(x_p) * 2^(S k) (mantissa)
    int *pmmk = nullptr; // [mmax+1][npairs] k (number of 2^S steps)
    T2 *tw = nullptr;    // [nphi/2] e^{2 pi i k / nphi}
    T2 *rtw = nullptr;   // [H] four-step FFT twiddles: rtw[k1 N2 + n2] = e^{2 pi i n2 k1 / H}
};

// Four-step split of an FFT of length H = 2^logH = N1 N2 (fft.cu):
// N1 = 2^ceil(logH / 2), N2 = H / N1.
inline int fft_n1(int logH) { return 1 << ((logH + 1) / 2); }

// Kernel-side view of a plan in precision T.
template <typename T>
struct PlanView {
    using T2 = typename Vec2<T>::type;
    int lmax, mmax, nlat, nphi, npairs, nlm;
    const T2 *ab;
    const T *dc;
    const T *x;
    const T *st;
    const T *wq;
    const T *pmm;
    const int *pmmk;
    const T2 *tw;
    const T2 *rtw;
    unsigned long long fftplan;   // radices of the FFT of length nphi/2 (fft_plan_of)
    int mres;                     // order stride: order index k is the order m = k mres
    const float4 *twdf;           // FP64 plans: tw as double-float pairs (re.hi, re.lo, im.hi, im.lo)
    // FP32 plans: restart states of the recurrence (see kSeedSeg), [segment][npairs]
    // float4 (y1, y2, k as int bits, 0), segments of order index m from segoff[m].
    const float4 *seeds;
    const unsigned long long *segoff;
    // FP64 plans: the same states as (y1, y2) and k, [segment][npairs].
    const double2 *seeds64;
    const int *seeds64k;
    // Static polar optimisation (Sec. 3.1): per (order index m, pair) the
    // first kSeedSeg-degree segment holding a |P_n^m| at or above the
    // threshold (the segment count when none does), [mmax+1][npairs].
    const unsigned short *live;
};

// The FP32 Legendre kernels restart the recurrence of Sec. 3.2 every kSeedSeg
// degrees from the state (P_{n0-1}, P_{n0-2}) computed by the FP64 recurrence,
// carried in the exponent-scaled form of Sec. 3.5 (y * 2^(-64 k)), so that
// FP32 rounding errors accumulate over at most kSeedSeg steps.
constexpr int kSeedSeg = 32;
// Analysis shape code (TunedShape::analys_lpt) of the FP64 warp-per-segment kernel.
constexpr int kAnalysSeg = 32;

// First packed index of order index k (order m = k mres): the degrees of the
// orders before it, sum_{k' < k} (lmax - k' mres + 1).
__host__ __device__ inline long col_of_mres(int lmax, int k, int mres)
{
    return (long)k * (lmax + 1) - (long)mres * k * (k - 1) / 2;
}

// Pass plan of a mixed-radix FFT of length H = 2^a 3^b 5^c: bits 0-3 the
// number of passes (none for H = 1), then 5 bits per pass radix (2, 4, 8, 16,
// 3 or 5), the power-of-two part first.  kFftPlanBad if H has another prime
// factor or needs more than 12 passes.
constexpr unsigned long long kFftPlanBad = ~0ull;
inline unsigned long long fft_plan_of(int H)
{
    if (H < 1) return kFftPlanBad;
    int a = 0, b = 0, c = 0, h = H;
    while (h % 2 == 0) { h /= 2; ++a; }
    while (h % 3 == 0) { h /= 3; ++b; }
    while (h % 5 == 0) { h /= 5; ++c; }
    if (h != 1) return kFftPlanBad;
    int rad[16], n = 0;
    if (a % 4) rad[n++] = 1 << (a % 4);
    for (int i = 0; i < a / 4; ++i) rad[n++] = 16;
    for (int i = 0; i < b; ++i) rad[n++] = 3;
    for (int i = 0; i < c; ++i) rad[n++] = 5;
    if (n > 12) return kFftPlanBad;
    unsigned long long p = (unsigned long long)n;
    for (int i = 0; i < n; ++i) p |= (unsigned long long)rad[i] << (4 + 5 * i);
    return p;
}
__host__ __device__ inline int fft_plan_npass(unsigned long long p) { return (int)(p & 15u); }
__host__ __device__ inline int fft_plan_radix(unsigned long long p, int i) { return (int)((p >> (4 + 5 * i)) & 31u); }

// What a Legendre or FFT launch computes; selects the scale factors.
enum Op {
    OP_SYNTH = 0,       // forward synthesis
    OP_ANALYS = 1,      // forward analysis
    OP_SYNTH_ADJ = 2,   // adjoint of synthesis (an unweighted analysis times c_m)
    OP_ANALYS_ADJ = 3   // adjoint of analysis (a weighted synthesis of b / c_m)
};

// Kernel shapes chosen by sht_tune for one (precision, batch).
struct TunedShape {
    int synth_lpt = 0, synth_bc = 0, analys_lpt = 0, analys_bc = 0;
    int auto_mode = 1;           // SHT_F32_AUTO: the fastest of SHT_F32, SHT_TC_BF16X3, SHT_TC_OTF
};

// Event pairs recorded around kernel launches while profiling is enabled.
struct KernelTimer {
    bool enabled = false;
    std::vector<cudaEvent_t> pool;   // created on demand, reused
    std::vector<int> kinds;          // kind of each recorded pair
    size_t used = 0;                 // events in use (2 per launch)
};

struct Plan {
    int lmax, mmax, nlat, nphi, npairs, nlm;
    int mres = 1;                    // order stride (orders 0, mres, .., mmax mres)
    std::vector<double> x, w;        // host nodes (descending) and weights, all nlat
    Tables<double> t64;
    Tables<float> t32;
    void *tables_base = nullptr;     // single device allocation holding t64 and t32
    float4 *twdf = nullptr;          // [nphi/2] e^{2 pi i k / nphi} as double-float pairs
    int *d_err = nullptr;            // device error word written by bounded waits
    unsigned char *panel_s = nullptr, *panel_a = nullptr;   // tensor-core P panels
    unsigned long long *d_off_s = nullptr, *d_off_a = nullptr, *d_dchunk = nullptr;
    size_t tc_nchunk_s = 0;                     // synthesis data chunks over all orders
    int *d_c0_s = nullptr, *d_c0_a = nullptr;   // first live chunk per (m, tile)
    unsigned short *d_gf_s = nullptr, *d_gf_a = nullptr;  // ... per 8-row group of (m, tile)
    double polar_skip_s = 0, polar_skip_a = 0;  // fraction of panel bytes skipped
    float polar_thr = 0x1p-40f;                 // polar threshold (sht_set_polar_threshold)
    unsigned char *dpanel_s = nullptr, *dpanel_a = nullptr; // sin(theta) dP/dtheta panels (vector)
    int *d_c0v_s = nullptr, *d_c0v_a = nullptr; // first chunk live in P or dP
    unsigned char *p64_s = nullptr, *p64_a = nullptr;     // SHT_TC_F64: digit-slice panels
    unsigned long long *d_off64_s = nullptr, *d_off64_a = nullptr, *d_dchunk64 = nullptr;
    size_t nchunk64_s = 0;                                // ... synthesis data chunks over all orders
    int *d_e64_s = nullptr, *d_e64_a = nullptr;           // ... row exponents
    int *d_c064_s = nullptr, *d_c064_a = nullptr;         // ... first nonzero chunk per (m, tile)
    unsigned short *d_gf64_s = nullptr, *d_gf64_a = nullptr;  // ... and per (m, tile, parity, 8-row group)
    unsigned char *d_zero64 = nullptr;                    // ... zeros for the stage rows it does not read
    int *d_sched64_s = nullptr, *d_sched64_a = nullptr;   // ... work lists of the persistent contraction
    int sched64_ctas = 0;                                 // ... and their CTA count
    int *d_schedv_s[2] = {nullptr, nullptr};              // vector contraction work lists (1 | 2 field halves)
    int *d_schedv_a[2] = {nullptr, nullptr};
    int schedv_ctas = 0;
    int *d_fcol = nullptr;                                // ... field exponents of a launch
    double skip64_s = -1, skip64_a = -1;                  // ... fractions of the panel bytes not read
    float4 *otf_seeds = nullptr;                // on-the-fly mode: recurrence seeds
    unsigned long long *d_segoff = nullptr;     // first segment of each order
    int *d_c0o_s = nullptr, *d_c0o_a = nullptr; // on-the-fly mode: first live chunk per (m, tile)
    int otf_state = 0;                          // 0 not built, 1 built, -1 not supported for this plan
    float4 *seeds32 = nullptr;                  // FP32 recurrence restart states (kSeedSeg), built on first use
    unsigned long long *d_seg32 = nullptr;      // first kSeedSeg segment of each order index (both precisions)
    double2 *seeds64 = nullptr;                 // FP64 restart states (y1, y2) ...
    int *seeds64k = nullptr;                    // ... and their exponent counters
    unsigned short *live32 = nullptr, *live64 = nullptr;   // first live segment per (m, pair), per precision
    bool polar_thr_set = false;                 // sht_set_polar_threshold was called
    // thresholds of the static polar optimisation of the CUDA-core kernels:
    // the set value, else 2^-40 (FP32) and 2^-64 (FP64, below the rounding of its sums)
    float thr_cc32() const { return polar_thr_set ? polar_thr : 0x1p-40f; }
    float thr_cc64() const { return polar_thr_set ? polar_thr : 0x1p-64f; }
    double otf_skip_s = 0, otf_skip_a = 0;      // on-the-fly mode: fraction of chunks skipped
    void *work = nullptr;            // scratch (grown on demand)
    size_t work_bytes = 0;
    int device = 0;
    KernelTimer timer;
    std::vector<std::pair<long long, TunedShape>> tuned;   // key: mode * 2^32 + batch

    PlanView<double> view64() const;
    PlanView<float> view32() const;
};

// Host plan construction (plan.cpp).
int plan_build(Plan &p, std::string &err);
void plan_free(Plan &p);
// Frees the FP64-accurate tensor-core mode's tables (digit panels, exponents, work lists).
void plan_free_tc64(Plan &p);
// Builds the recurrence restart states of a plan once, with the first-live
// table of the static polar optimisation: FP32 (16 B per pair and kSeedSeg
// degrees, (lmax+1)^2 npairs / 4 bytes, 138 MB at lmax = 1023) or FP64
// (20 B, 175 MB at lmax = 1023).  SHT status, message in err.
int plan_seeds32(Plan &p, std::string &err);
int plan_seeds64(Plan &p, std::string &err);
// Recomputes the first-live tables that exist (threshold change).
int plan_relive(Plan &p, std::string &err);
// Segment offsets of kSeedSeg degrees per order index; returns the total.
size_t seed_segment_offsets(int lmax, int mmax, int mres, std::vector<unsigned long long> &segoff);
// One thread per (m, pair): FP32 states (seeds32) or FP64 states (seeds64,
// seeds64k), and the first segment holding |P| >= thr (thr <= 0: segment 0).
cudaError_t launch_build_restarts(const PlanView<double> &pv, const unsigned long long *segoff, float4 *seeds32,
                                  double2 *seeds64, int *seeds64k, unsigned short *live, double thr, cudaStream_t st);

// Launchers (legendre.cu, fft.cu).  `eo` / `sd` are intermediate buffers of
// [batch][mmax+1][npairs][2] complex values of precision T.
template <typename T>
cudaError_t launch_legendre_synth(const PlanView<T> &pv, const T *spec, T *eo, int batch, Op op,
                                  cudaStream_t s);
template <typename T>
cudaError_t launch_legendre_analys(const PlanView<T> &pv, const T *sd, T *spec, int batch, Op op,
                                   cudaStream_t s);
// Explicit kernel shapes (lpt pairs per thread, bc fields per CTA; 0 = default).
// Synthesis: lpt in {1,2,4}, bc in {1,2,4}; analysis: lpt in {2,4,8}, bc in {1,2}.
template <typename T>
cudaError_t launch_legendre_synth_cfg(const PlanView<T> &pv, const T *spec, T *eo, int batch, Op op, int lpt,
                                      int bc, cudaStream_t s);
template <typename T>
cudaError_t launch_legendre_analys_cfg(const PlanView<T> &pv, const T *sd, T *spec, int batch, Op op, int lpt,
                                       int bc, cudaStream_t s);

template <typename T>
cudaError_t launch_legendre_synth_vec(const PlanView<T> &pv, const T *S, const T *Tc, T *eot,
                                      T *eop, int batch, Op op, cudaStream_t s);
template <typename T>
cudaError_t launch_legendre_analys_vec(const PlanView<T> &pv, const T *sdt, const T *sdp, T *S,
                                       T *Tc, int batch, Op op, cudaStream_t s);
template <typename T>
cudaError_t launch_fft_synth(const PlanView<T> &pv, const T *eo, T *grid, int batch, Op op,
                             cudaStream_t s);
template <typename T>
cudaError_t launch_fft_analys(const PlanView<T> &pv, const T *grid, T *sd, int batch, Op op,
                              bool vector, cudaStream_t s);
// The same transforms of FP64 data in double-float arithmetic (pairs of FP32
// numbers, ~2^-48 relative error per operation), for the FP64-accurate
// tensor-core mode; needs the plan's double-float twiddles (pv.twdf).  With
// fmax, the analysis also raises fmax[b] to the frexp exponent of every fold
// of field b it writes (fmax initialised by the caller).
cudaError_t launch_fft_synth_df(const PlanView<double> &pv, const double *eo, double *grid, int batch, Op op,
                                cudaStream_t s);
cudaError_t launch_fft_analys_df(const PlanView<double> &pv, const double *grid, double *sd, int batch, Op op,
                                 bool vector, cudaStream_t s, int *fmax = nullptr);



// Uneven batches (batch.cu): one field of an uneven batch, as the persistent
// kernels see it.  FP32 data.
struct BatchField {
    PlanView<float> pv;
    const float *in;   // spectra (synthesis) or grid (analysis)
    float *out;        // grid (synthesis) or spectra (analysis)
    float *inter;      // E/O (synthesis) or s/d folds (analysis) of this field
    int logH, G;       // log2(nphi/2) (kRowLogMax + 1 or more when not a power of two) and pairs per FFT tile
};

// Persistent kernels over a tile list: each CTA takes the next tile from
// *counter (atomicAdd) until the list is exhausted; tiles are int4
// (field, m or p0, pair block, 0) sorted longest first.
cudaError_t launch_batch_legendre(bool synth, const BatchField *fields, const int4 *tiles, int ntiles, int *counter,
                                  int ctas, cudaStream_t s);
cudaError_t launch_batch_fft(bool synth, const BatchField *fields, const int4 *tiles, int ntiles, int *counter,
                             int ctas, size_t smem, cudaStream_t s);
size_t batch_fft_smem(int H, int G);
cudaError_t batch_fft_prepare(size_t smem);   // once, outside any stream capture

// Uneven batches on the tensor cores (capi.cu): panels + operand scratch of a
// plan for up to `batch` fields (SHT status), and the contraction alone over a
// contiguous group of fields (E/O or folds in [batch][mmax+1][npairs][4]).
int tc_batch_prepare(Plan &p, int batch);
cudaError_t tc_batch_legendre(Plan &p, bool synth, const float *in, float *out, int batch, cudaStream_t s);

// Records an error message for sht_last_error and returns `code`.
int set_error(int code, const std::string &msg);
int batch_fft_group(int H, int npairs);
constexpr int kBatchSynthPairs = 256;   // pairs per synthesis tile (128 threads x 2)
constexpr int kBatchMaxPairs = 512;     // analysis CTA (256 threads x 2 pairs) limit

// Tensor-core path (tc.cu).  `mres` is the plan's order stride everywhere:
// order index m (0 .. mmax) is the order m mres.
// Panel byte offsets per order (synthesis and analysis layouts), their total
// sizes, and the first synthesis data chunk of each order.
void tc_panel_layout(int lmax, int mmax, int mres, int npairs, std::vector<unsigned long long> &off_s,
                     std::vector<unsigned long long> &off_a, size_t &bytes_s, size_t &bytes_a,
                     std::vector<unsigned long long> &dchunk, size_t &nchunk_s);
// Bytes of the blocked data operand (either layout) for `batch` fields.
size_t tc_data_bytes(int mmax, int npairs, size_t nchunk_s, int batch, bool vec);
// deriv: build sin(theta) dP/dtheta instead of P.
cudaError_t launch_build_panels(const PlanView<double> &pv, const unsigned long long *off_s,
                                const unsigned long long *off_a, unsigned char *ps, unsigned char *pa, bool deriv,
                                cudaStream_t st);
// Scalar contraction of <= tc_max_batch() fields: prep kernel (FP32 -> blocked
// bf16 hi/lo in `data`; skipped when `prepped`, i.e. `data` already holds
// this operand) then the tcgen05 kernel.  Synthesis: spectra -> E/O;
// analysis: s/d folds -> spectra.
cudaError_t launch_tc_legendre(bool synth, int lmax, int mmax, int mres, int npairs, int nlm, const unsigned char *panel,
                               const unsigned long long *off, const int *c0, const unsigned short *gfirst,
                               const unsigned long long *dchunk,
                               unsigned char *data, const float *in, float *out, int batch, Op op, int *err,
                               bool prepped, cudaStream_t st);
// Vector contraction of <= tc_vec_max_batch() fields.  Synthesis: (S, T) ->
// (theta E/O, phi E/O); analysis: (theta, phi) folds -> (S, T).
cudaError_t launch_tc_vec(bool synth, int lmax, int mmax, int mres, int npairs, int nlm, const unsigned char *panel,
                          const unsigned char *dpanel, const unsigned long long *off, const int *c0,
                          const int *const sched[2], int nctas,
                          const unsigned long long *dchunk, unsigned char *data, const float *in0, const float *in1,
                          float *out0, float *out1, const float *st_pairs, int batch, Op op, int *err, bool prepped,
                          cudaStream_t st);
cudaError_t launch_min_int(const int *a, const int *b, int *out, int n, cudaStream_t st);
int tc_vec_max_batch();
int tc_otf_max_batch();
// Rows of the data operand for `batch` fields: 32 ceil(2 batch / 32), twice that for vectors.
inline int tc_rows(int batch, bool vec) { return (vec ? 2 : 1) * (((2 * batch + 31) / 32) * 32); }
// Static polar optimisation: per (m, tile) first chunk with a panel value >=
// thr; with `gfirst`, also per 8-row group of the tile ([m][tile][16]).
cudaError_t launch_panel_first_live(bool synth, int lmax, int mmax, int mres, int npairs, const unsigned long long *off,
                                    const unsigned char *panel, float thr, int *c0, int &ntiles, cudaStream_t st,
                                    unsigned short *gfirst = nullptr);
void tc_tile_counts(int lmax, int npairs, int &ntiles_s, int &ntiles_a);
// Fractions of panel bytes skipped: per 8-row group when the group tables are
// given, else per whole chunk.
cudaError_t tc_polar_stats(int lmax, int mmax, int mres, int npairs, const int *d_c0_s, const int *d_c0_a, double &frac_s,
                           double &frac_a, const unsigned short *d_gf_s = nullptr,
                           const unsigned short *d_gf_a = nullptr);
int tc_max_batch();
// FP64-accurate contraction (tc64.cu): digit-slice panels and row exponents,
// built once; per launch the field exponents, the data digits and the
// contraction.  Synthesis: FP64 spectra -> E/O (double4 [b][m][pair]);
// analysis: FP64 s/d folds -> spectra.
int tc64_max_batch();
int tc64_ctas_per_sm();   // resident CTAs per SM of the persistent contraction
// Byte offsets of each order's digit-slice panel chunks (synthesis, analysis),
// total bytes, and the first synthesis data chunk of each order.
void tc64_panel_layout(int lmax, int mmax, int mres, int npairs, std::vector<unsigned long long> &off_s,
                       std::vector<unsigned long long> &off_a, size_t &bytes_s, size_t &bytes_a,
                       std::vector<unsigned long long> &dchunk, size_t &nchunk_s);
size_t tc64_data_bytes(int mmax, int npairs, size_t nchunk_s);
cudaError_t tc64_build(const PlanView<double> &pv, const unsigned long long *off_s, const unsigned long long *off_a,
                       unsigned char *ps, unsigned char *pa, int *es, int *ea, int *c0_s, int *c0_a,
                       unsigned short *gf_s, unsigned short *gf_a, cudaStream_t st);
// Bytes of the zero buffer the FP64-accurate contraction copies from.
size_t tc64_zero_bytes();
void tc64_skip_stats(int lmax, int mmax, int mres, int npairs, const std::vector<int> &c0s,
                     const std::vector<int> &c0a, const std::vector<unsigned short> &gfs,
                     const std::vector<unsigned short> &gfa, double &frac_s, double &frac_a);
// fcol_ready: fcol already holds the field exponents of `in` (else this
// computes them first).
// Work lists of persistent CTAs, longest processing time first: the items
// with cost >= 0 form groups (items of one group id go to one CTA, in
// ascending order, so that the data they share is still in L2); groups are
// taken heaviest first, each to the CTA with the least work so far.
// sched = [nctas + 1 offsets | items].
void schedule_lpt(const std::vector<int> &cost, const std::vector<int> &group, int nctas, std::vector<int> &sched);
// Item costs and groups of the persistent FP64-accurate contraction (item =
// 2 (m tiles + tile) + parity; group = (m, parity), whose tiles read the same
// data digits) from the first nonzero chunks c0 [mmax+1][tiles] and gf
// [mmax+1][tiles][parity][16 groups]: the panel groups each item reads.
void tc64_costs(int lmax, int mmax, int mres, int npairs, bool synth, const std::vector<int> &c0,
                const std::vector<unsigned short> &gf, std::vector<int> &cost, std::vector<int> &group);
// Item costs and groups of the persistent vector contraction (item =
// (m tiles + tile) halves + half; group = m: the halves of a tile share its
// panel chunks, the tiles share the data) from its first live chunks c0.
void tc_vec_costs(int lmax, int mmax, int mres, int npairs, bool synth, int halves, const std::vector<int> &c0,
                  std::vector<int> &cost, std::vector<int> &group);
cudaError_t launch_tc64(bool synth, int lmax, int mmax, int mres, int npairs, int nlm, const unsigned char *panel,
                        const unsigned long long *off, const int *c0, const unsigned short *gf,
                        const unsigned char *zero, const int *sched, int nctas, const int *erow,
                        const unsigned long long *dchunk, int *fcol, unsigned char *data, const double *in,
                        double *out, int batch, Op op, int *err, cudaStream_t st, bool fcol_ready = false);
// Sets fcol[0 .. batch) to "no value yet" before a producer raises it.
cudaError_t tc64_reset_fcol(int *fcol, int batch, cudaStream_t st);
cudaError_t launch_selftest_timeout(int *err, unsigned long long max_ns, cudaStream_t st);

// On-the-fly mode (tc.cu): FP32 recurrence reseeded every 32 degrees.
// Segment offsets per order (= synthesis data chunk numbering); returns the
// total number of segments.
size_t otf_segment_offsets(int lmax, int mmax, int mres, std::vector<unsigned long long> &segoff);
// Seeds [segments][npairs] float4 and the polar-skip tables (first live chunk
// per (m, synthesis tile) and per (m, analysis tile)); *flag set if some
// segment would exceed the FP32 range.
cudaError_t launch_build_seeds(const PlanView<double> &pv, const unsigned long long *segoff, float4 *seeds,
                               float thr, int *c0s, int *c0a, int *flag, cudaStream_t st);
// Scalar contraction (prep + on-the-fly kernel) of <= tc_max_batch() fields.
cudaError_t launch_tc_otf(bool synth, int lmax, int mmax, int mres, int npairs, int nlm, const float4 *seeds,
                          const unsigned long long *segoff, const int *c0, const float2 *ab32, const float *x32,
                          unsigned char *data, const float *in, float *out, int batch, Op op, int *err,
                          cudaStream_t st);

}  // namespace sht
