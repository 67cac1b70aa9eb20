// tc64.cu -- the per-order Legendre contraction to FP64 accuracy on the bf16
// tensor cores (mode SHT_TC_F64): the same GEMMs as tc.cu (Sec. 3.1, Eq.
// synth_direct and Eq. gauss per order m and parity of n - m), with both
// operands split into fixed-point digit slices whose products the tensor
// core adds exactly.
//
// Splitting (an Ozaki-style scheme).  A row of P (a latitude pair for
// synthesis, a degree for analysis) is scaled by 2^-e with 2^e above its
// largest |P|, and a data column (one field) by 2^-f likewise; then
//     P 2^(6 - e) = sum_i d_i 2^(-7 i),   a 2^(6 - f) = sum_j c_j 2^(-7 j),
// i < kSA = 7 panel digits, j < kSB = 8 data digits, all signed with
// |d_i|, |c_j| <= 64 (exact in bf16): 49 bits of P relative to its row
// maximum and 56 of the data relative to the field maximum, so that the
// small coefficients of a decaying spectrum keep FP64-level absolute error.
// The digits of level t = i + j all carry the scale 2^(e + f - 12 - 7 t), so
//     sum_n P a = 2^(e + f - 12) sum_t 2^(-7 t) L_t,  L_t = sum_{i+j=t} sum_n d_i c_j,
// and the tensor core forms each L_t as a sum of integer products: at most
// kSA x 512 products of magnitude <= 2^12, below 2^24, so the FP32
// accumulation in tensor memory is exact.  Levels t < kL = 8 are kept (the
// dropped ones are below 2^-56 of the leading level); the epilogue combines
// them in 64-bit integers and scales in FP64.
//
// For A slice i, one MMA multiplies it by the data slices j = 0 .. kL-1-i,
// stacked along N, whose products land on levels i .. kL-1: the accumulator
// columns of the levels are contiguous, so the MMA's D starts at level i.
// That is kSA MMAs per parity and chunk (N = 32 (kL - i)), 14 per chunk.
// The accumulators are zeroed once and every MMA accumulates.
//
// Work item: one (order m, 128-row tile, parity of n - m).  Two persistent
// CTAs per SM walk balanced lists of items with 192 threads: warps 0-3 run the
// epilogue, warp 4 lane 0 issues the MMAs, warp 5 lane 0 streams the parity's
// share of each panel chunk (up to 28 KB: from the chunk's first 8-row group
// with a nonzero digit on, the polar optimisation of Sec. 3.1 at the digits'
// own precision) and its 6 KB of data by bulk copy into a ring of 3 stages that
// runs on across items.  Tensor memory: kL levels x 32 columns (16
// fields x re/im) = 256 per CTA.  Every wait is bounded; a kernel whose wait
// gave up records SHT_ETIMEOUT and skips the rest of its output.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <vector>

#include "sht_internal.h"
#include "tc_common.cuh"
#include "tc_layout.cuh"
#include "tc_ptx.cuh"

namespace sht {
namespace {

using sht::col_of_mres;
using tcc::raise_err;
using tcc::wait_or_abort;

constexpr int kR = 128;                        // MMA M
constexpr int kSA = 7;                         // digit slices of P
constexpr int kSB = 8;                         // digit slices of the data
constexpr int kNC = 32;                        // data rows per slice: 16 fields x (re, im)
constexpr int kBatch64 = kNC / 2;              // fields per launch
constexpr int kPBlk = kR * kKc * 2;            // one slice of one parity: [128 x 16] bf16 = 4 KB
constexpr int kPPar = kSA * kPBlk;             // one parity's slices: 28 KB
constexpr int kPChunk = 2 * kPPar;             // panel chunk: [parity][slice] blocks = 56 KB
constexpr int kDRows = kSB * kNC;              // data rows per class: slices stacked along N
constexpr int kDBlk = kDRows * kKc * 2;        // 6 KB
constexpr int kDChunk = 2 * kDBlk;             // data chunk: [class] blocks = 12 KB
constexpr int kStage = kPPar + kDBlk;          // one parity: 36 KB
constexpr int kStages = 3;                     // two CTAs per SM: 2 x 108 KB of ring
constexpr int kCtasPerSm = 2;                  // two MMA chains per SM (each MMA of a chunk accumulates
                                               // onto the previous one's columns, so one chain waits out
                                               // every MMA's latency)
constexpr int kThreads = 192;
constexpr int kL = kSB;                        // accumulated levels t = i + j < kL
constexpr int kLevelCols = kNC;                // accumulator columns per level
constexpr int kParCols = kL * kLevelCols;      // accumulator columns of a CTA: 256
constexpr uint32_t kTmemCols = kParCols;       // one accumulator per CTA: half of tensor memory
constexpr int kExpNone = INT_MIN / 2;          // exponent of an all-zero row or column

// Panel chunk layout: per parity (kPPar bytes), 8-row group g of slice i at
// g kGS + i kSbo, a [8 x kKc] bf16 pair of core matrices -- the seven slices of
// a group side by side, so that groups [g0, g1) of every slice are one
// contiguous range (one bulk copy).  The MMA operand of slice i starts at
// i kSbo with 8-row group stride kGS.
constexpr uint32_t kGS = (uint32_t)kSA * kSbo;
__host__ __device__ __forceinline__ uint32_t pofs(int i, int par, int row, int k)
{
    return (uint32_t)(par * kPPar) + (uint32_t)(row >> 3) * kGS + (uint32_t)i * kSbo + (uint32_t)(k >> 3) * kLbo +
           (uint32_t)((row & 7) * 16 + (k & 7) * 2);
}

// Z 2^k as a double, for a 128-bit integer Z, with integer operations only
// (the FP64 pipe is the scarce one): normalise, round the 53-bit mantissa to
// nearest (ties away from zero), and assemble the exponent.  Results below
// the normal range are flushed to zero: they are under 2^-1022, far below the
// FP64 rounding of the sums this kernel forms.
__device__ __forceinline__ double i128_ldexp(__int128 Z, int k)
{
    if (Z == 0) return 0.0;
    const bool neg = Z < 0;
    const unsigned __int128 u = neg ? (unsigned __int128)(-Z) : (unsigned __int128)Z;
    const unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
    int msb = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
    unsigned long long mant;
    if (msb > 52) {
        mant = (unsigned long long)(u >> (msb - 53));   // 54 bits: one rounding bit
        mant = (mant + 1) >> 1;
        if (mant >> 53) {
            mant >>= 1;
            msb += 1;
        }
    } else {
        mant = lo << (52 - msb);
    }
    const int e = msb + k + 1023;
    if (e <= 0) return 0.0;
    const unsigned long long bits =
        ((unsigned long long)e << 52) | (mant & 0xFFFFFFFFFFFFFull) | (neg ? 0x8000000000000000ull : 0ull);
    return __longlong_as_double((long long)bits);
}

// Exponent e with |v| < 2^e for every |v| <= max (frexp convention).
__device__ __forceinline__ int exp_above(double max_abs)
{
    int e;
    (void)frexp(max_abs, &e);
    return e;
}

// Digits of a panel value (FP64 arithmetic; the panels are built once):
// v 2^(6 - e) = sum_i d[i] 2^(-7 i), rounding each digit to nearest.
__device__ __forceinline__ void digits_fp64(double v, int e, int (&d)[kSA])
{
    double X = ldexp(v, 6 - e);
#pragma unroll
    for (int i = 0; i < kSA; ++i) {
        const double r = rint(X);
        d[i] = (int)r;
        X = (X - r) * 128.0;
    }
}

// Digits of a data value with integer operations only (no FP64 pipe):
// Y = round(v 2^(55 - e)) from the bit pattern (|Y| < 2^55), then signed
// base-2^7 digits from the top, Y = sum_i d[i] 2^(7 (kSB - 1 - i)).
// Requires |v| < 2^e.
__device__ __forceinline__ void digits_int(double v, int e, int (&d)[kSB])
{
    const long long bits = __double_as_longlong(v);
    const int ex = (int)((bits >> 52) & 0x7ff);
    long long Y = 0;
    if (ex != 0 && e != kExpNone) {
        const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
        const int sh = ex - 1075 + 7 * (kSB - 1) + 6 - e;   // |v| 2^(55 - e) = mant 2^sh, sh <= 2
        if (sh >= 0) Y = mant << sh;
        else if (sh > -63) Y = (mant + (1LL << (-sh - 1))) >> (-sh);
        if (bits < 0) Y = -Y;
    }
#pragma unroll
    for (int i = 0; i < kSB - 1; ++i) {
        const int s = 7 * (kSB - 1 - i);
        const long long q = (Y + (1LL << (s - 1))) >> s;
        d[i] = (int)q;
        Y -= q << s;
    }
    d[kSB - 1] = (int)Y;
}

// The Sec. 3.2 recurrence for (order index m, pair p) as in the panel builder
// of tc.cu, calling f(nn, P) for every degree n = m mres + nn with P != 0
// (k = 0 region).
template <typename F>
__device__ __forceinline__ void recur_pair(const PlanView<double> &pv, int m, int p, F &&f)
{
    const int npairs = pv.npairs, lmax = pv.lmax;
    const int L = lmax - m * pv.mres + 1;
    const long col = col_of_mres(lmax, m, pv.mres);
    const double x = pv.x[p];
    double y2 = pv.pmm[(size_t)m * npairs + p], y1 = 0.0;
    int k = pv.pmmk[(size_t)m * npairs + p];
    for (int nn = 0; nn < L; ++nn) {
        const double2 ab = pv.ab[col + nn];
        const double yn = fma(ab.x * x, y1, ab.y * y2);
        y2 = y1;
        y1 = yn;
        if (k > 0 && fabs(yn) >= 1.0) {
            y1 *= 0x1p-240;
            y2 *= 0x1p-240;
            k -= 1;
        }
        if (k != 0 || y1 == 0.0) continue;
        f(nn, y1);
    }
}

// Row exponents: es[m][p] over the degrees of (m, p) (synthesis rows), and
// ea[col(m) + nn] over the pairs (analysis rows; initialised to kExpNone).
__global__ void k_p64_scales(PlanView<double> pv, int *__restrict__ es, int *__restrict__ ea)
{
    const int m = blockIdx.y, p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= pv.npairs) return;
    const long col = col_of_mres(pv.lmax, m, pv.mres);
    double mx = 0.0;
    recur_pair(pv, m, p, [&](int nn, double P) {
        mx = fmax(mx, fabs(P));
        atomicMax(&ea[col + nn], exp_above(fabs(P)));
    });
    es[(size_t)m * pv.npairs + p] = mx > 0.0 ? exp_above(mx) : kExpNone;
}

// Digit-slice panels, in the operand layout of the contraction.  Synthesis
// chunk (m, tile t, c): rows = pairs of the tile, K = the kKc degree indices
// kk = (n - m) / 2 of chunk c, one block per (slice, parity of n - m).
// Analysis chunk (m, degree tile mt, pair chunk kc): rows = kk, K = pairs.
__global__ void k_p64_build(PlanView<double> pv, const int *__restrict__ es, const int *__restrict__ ea,
                            const unsigned long long *__restrict__ off_s, const unsigned long long *__restrict__ off_a,
                            unsigned char *__restrict__ ps, unsigned char *__restrict__ pa)
{
    const int m = blockIdx.y, p = blockIdx.x * blockDim.x + threadIdx.x;
    const int npairs = pv.npairs;
    if (p >= npairs) return;
    const int L = pv.lmax - m * pv.mres + 1, Le = (L + 1) / 2;
    const int nch = (Le + kKc - 1) / kKc, kch = (npairs + kKc - 1) / kKc;
    const long col = col_of_mres(pv.lmax, m, pv.mres);
    const int t = p / kR, row = p % kR, kc = p / kKc, pc = p % kKc;
    const int e_row = es[(size_t)m * npairs + p];
    unsigned char *sbase = ps + off_s[m] + (size_t)t * nch * kPChunk;
    unsigned char *abase = pa + off_a[m];
    recur_pair(pv, m, p, [&](int nn, double P) {
        const int par = nn & 1, kk = nn >> 1;
        int d[kSA];
        digits_fp64(P, e_row, d);
        unsigned char *b = sbase + (size_t)(kk / kKc) * kPChunk;
#pragma unroll
        for (int i = 0; i < kSA; ++i)
            *reinterpret_cast<__nv_bfloat16 *>(b + pofs(i, par, row, kk % kKc)) = __int2bfloat16_rn(d[i]);
        digits_fp64(P, ea[col + nn], d);
        const int mt = kk / kR, r = kk % kR;
        unsigned char *ba = abase + ((size_t)mt * kch + kc) * kPChunk;
#pragma unroll
        for (int i = 0; i < kSA; ++i)
            *reinterpret_cast<__nv_bfloat16 *>(ba + pofs(i, par, r, pc)) = __int2bfloat16_rn(d[i]);
    });
}

// First chunk of each (m, tile) holding a nonzero digit (all-zero chunks,
// high orders near the poles, add nothing: the polar optimisation of
// Sec. 3.1 without a threshold).
__global__ void k_p64_first_live(int synth, int lmax, int mres, int npairs, int ntiles,
                                 const unsigned long long *__restrict__ off, const unsigned char *__restrict__ panel,
                                 int *__restrict__ c0)
{
    const int m = blockIdx.y, tile = blockIdx.x;   // order index m, order m mres
    const int L = lmax - m * mres + 1, Le = (L + 1) / 2;
    const int nchunks = synth ? (Le + kKc - 1) / kKc : (npairs + kKc - 1) / kKc;
    const bool valid = synth || tile * kR < Le;
    __shared__ int s_live;
    int first = nchunks;
    if (valid) {
        const uint4 *base =
            reinterpret_cast<const uint4 *>(panel + off[m] + (size_t)tile * nchunks * kPChunk);
        for (int c = 0; c < nchunks; ++c) {
            if (threadIdx.x == 0) s_live = 0;
            __syncthreads();
            bool live = false;
            for (int i = threadIdx.x; i < kPChunk / 16; i += blockDim.x) {
                const uint4 v = base[(size_t)c * (kPChunk / 16) + i];
                live |= (v.x | v.y | v.z | v.w) != 0u;
            }
            if (live) s_live = 1;
            __syncthreads();
            const int any = s_live;
            __syncthreads();
            if (any) { first = c; break; }
        }
    }
    if (threadIdx.x == 0) c0[m * ntiles + tile] = first;
}

// First chunk with a nonzero digit of each (parity, 8-row group) of a tile,
// nchunks if none: gfirst[((m ntiles + tile) 2 + par) 16 + g].  The rows of a
// group below its first live chunk hold only zero digits (their P lies 2^-48
// or more below the row's largest), so the contraction need not read them.
// Thread t: (parity, group) t / 8, one eighth of the group's kGS bytes.
__global__ void k_p64_group_first(int synth, int lmax, int mres, int npairs, int ntiles,
                                  const unsigned long long *__restrict__ off,
                                  const unsigned char *__restrict__ panel, unsigned short *__restrict__ gfirst)
{
    const int m = blockIdx.y, tile = blockIdx.x;   // order index m, order m mres
    const int L = lmax - m * mres + 1, Le = (L + 1) / 2;
    const int nchunks = synth ? (Le + kKc - 1) / kKc : (npairs + kKc - 1) / kKc;
    const bool valid = synth || tile * kR < Le;
    const int pg = threadIdx.x >> 3, part = threadIdx.x & 7, par = pg >> 4, g = pg & 15;
    constexpr int kV = (int)(kGS / 16);              // 16-byte words of one 8-row group (all slices)
    const unsigned gmask = 0xffu << (threadIdx.x & 24);
    int first = nchunks;
    if (valid) {
        const unsigned char *base = panel + off[m] + (size_t)tile * nchunks * kPChunk;
        for (int c = 0; c < nchunks; ++c) {
            bool nz = false;
            if (first == nchunks) {
                for (int v = part; v < kV; v += 8) {
                    const uint4 x = *reinterpret_cast<const uint4 *>(base + (size_t)c * kPChunk + (size_t)par * kPPar +
                                                                     (size_t)g * kGS + (size_t)v * 16);
                    nz |= (x.x | x.y | x.z | x.w) != 0u;
                }
            }
            nz = __any_sync(gmask, nz);   // the 8 threads of (parity, group)
            if (nz && first == nchunks) first = c;
            if (__syncthreads_and(first != nchunks)) break;
        }
    }
    if (part == 0) gfirst[(((size_t)m * ntiles + tile) * 2 + par) * 16 + g] = (unsigned short)min(first, 65535);
}

// First live 8-row group of a chunk: the smallest g < hi whose first live
// chunk is at or before c (hi if none).  Rows of the tile below it are all-zero
// digits in chunk c; from it on they are copied (any dead group among them
// holds zeros in the panel too).
__host__ __device__ __forceinline__ int first_live_group(const unsigned short *f, int c, int hi)
{
    for (int g = 0; g < hi; ++g)
        if ((int)f[g] <= c) return g;
    return hi;
}

// Column exponents: f[b] with |x| < 2^f[b] for every value of field b
// (initialised to kExpNone by the caller).
__global__ void k_colscale(const double *__restrict__ x, size_t per_field, int *__restrict__ f)
{
    const int b = blockIdx.y;
    // the bit patterns of non-negative doubles order like the values: the
    // maximum |x| is an integer maximum, off the FP64 pipe
    constexpr unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull;
    const unsigned long long *xb = reinterpret_cast<const unsigned long long *>(x) + (size_t)b * per_field;
    const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    unsigned long long mx = 0;
    if ((per_field & 1) == 0 && (reinterpret_cast<uintptr_t>(xb) & 15) == 0) {
        // 16-byte loads when the field starts on a 16-byte boundary, four in
        // flight per thread
        const ulonglong2 *x2 = reinterpret_cast<const ulonglong2 *>(xb);
        const size_t n2 = per_field / 2;
        size_t i = i0;
        for (; i + 3 * stride < n2; i += 4 * stride) {
            ulonglong2 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = x2[i + u * stride];
#pragma unroll
            for (int u = 0; u < 4; ++u) mx = max(mx, max(v[u].x & kAbs, v[u].y & kAbs));
        }
        for (; i < n2; i += stride) {
            const ulonglong2 v = x2[i];
            mx = max(mx, max(v.x & kAbs, v.y & kAbs));
        }
    } else {
        for (size_t i = i0; i < per_field; i += stride) mx = max(mx, xb[i] & kAbs);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx != 0) atomicMax(&f[b], exp_above(__longlong_as_double((long long)mx)));
}

__global__ void k_fill_int(int *__restrict__ a, int v, size_t n)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

// Data digits in the blocked operand layout: chunk [class][kDRows x kKc],
// row = 32 slice + 2 field + (re|im).  Synthesis chunk (m, c) = degrees
// n - m in [2 kKc c, 2 kKc (c + 1)), class = parity of n - m, numbered from
// dchunk[m]; analysis chunk (m, kc) = pairs [kKc kc, kKc (kc + 1)), class
// 0 = s fold, 1 = d fold, numbered m kch + kc.  One thread per (chunk, class,
// field, re|im, half of the K positions): it splits 8 values and writes each
// slice's 8 digits as one 16-byte core-matrix row.
__global__ void k_prep64(int synth, int lmax, int mmax, int mres, int npairs, int nlm, int batch, int op,
                         const double *__restrict__ in, const int *__restrict__ f,
                         const unsigned long long *__restrict__ dchunk, unsigned char *__restrict__ data)
{
    const int m = blockIdx.y;   // order index: the order is m mres
    const int L = lmax - m * mres + 1, Le = (L + 1) / 2;
    const int nchunks = synth ? (Le + kKc - 1) / kKc : (npairs + kKc - 1) / kKc;
    const long item = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int per = 8 * batch;                                // items per chunk
    if (item >= (long)nchunks * per) return;
    const int c = (int)(item / per);
    int r = (int)(item - (long)c * per);
    const int kh = r & 1, q = (r >> 1) & 1;                   // K half, re|im
    r >>= 2;
    const int b = r % batch, cls = r / batch;
    const int e = f[b];
    double v[8];
    if (synth) {
        const long col = col_of_mres(lmax, m, mres);
        const double sc = (op == OP_ANALYS_ADJ && m > 0) ? 0.5 : 1.0;   // adjoint factor 1/2
        const double2 *spec = reinterpret_cast<const double2 *>(in) + (size_t)b * nlm + col;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int nn = 2 * kKc * c + 2 * (8 * kh + i) + cls;
            double x = 0.0;
            if (nn < L && !(q == 1 && m == 0)) x = q ? spec[nn].y : spec[nn].x;
            v[i] = sc == 1.0 ? x : x * sc;
        }
    } else {
        const double *folds = in + (((size_t)b * (mmax + 1) + m) * npairs) * 4 + 2 * cls + q;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int p = kKc * c + 8 * kh + i;
            v[i] = p < npairs ? folds[(size_t)p * 4] : 0.0;
        }
    }
    uint32_t w[kSB][4];
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
        int d0[kSB], d1[kSB];
        digits_int(v[i], e, d0);
        digits_int(v[i + 1], e, d1);
#pragma unroll
        for (int s = 0; s < kSB; ++s)
            w[s][i / 2] = (uint32_t)__bfloat16_as_ushort(__int2bfloat16_rn(d0[s])) |
                          ((uint32_t)__bfloat16_as_ushort(__int2bfloat16_rn(d1[s])) << 16);
    }
    unsigned char *chunk = data +
                           (synth ? (size_t)(dchunk[m] + c) : (size_t)m * nchunks + c) * kDChunk +
                           (size_t)cls * kDBlk;
#pragma unroll
    for (int s = 0; s < kSB; ++s)
        *reinterpret_cast<uint4 *>(chunk + blk_off(kNC * s + 2 * b + q, 8 * kh)) =
            make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
}

struct Tc64Args {
    int lmax, mmax, npairs, nlm, batch, ntiles, op;
    int mres;                              // order stride: order index m is the order m mres
    const unsigned char *panel;
    const unsigned long long *off;         // per-order panel byte offsets
    const int *c0;                         // per (m, tile): first chunk with a nonzero digit
    const unsigned short *gf;              // per (m, tile, parity, 8-row group): first chunk with a nonzero digit
    const unsigned char *zero;             // kPPar zero bytes, copied into the stage rows not read
    const int *erow;                       // row exponents (synthesis [m][pair], analysis packed [nlm])
    const int *fcol;                       // field exponents
    const unsigned char *data;             // blocked data digits
    const unsigned long long *dchunk;      // synthesis: first data chunk of each order
    double *out;                           // synthesis: E/O [b][m][pair] (double4); analysis: spectra
    int *err;
};

// Work item w of a launch (heaviest first): parity w & 1, then order index
// and 128-row tile.  Every role of a CTA walks the same items.
struct Item64 {
    int m, tile, par, L, Le, nchunks, cstart, nlive;
    long col;
    bool valid;
};

template <bool SYNTH>
__device__ __forceinline__ Item64 item64(const Tc64Args &a, int w)
{
    Item64 it;
    it.par = w & 1;
    it.m = (w >> 1) / a.ntiles;
    it.tile = (w >> 1) - it.m * a.ntiles;
    it.L = a.lmax - it.m * a.mres + 1;   // m is the order index
    it.Le = (it.L + 1) / 2;
    it.col = col_of_mres(a.lmax, it.m, a.mres);
    it.valid = SYNTH || it.tile * kR < it.Le;
    it.nchunks = SYNTH ? (it.Le + kKc - 1) / kKc : (a.npairs + kKc - 1) / kKc;
    it.cstart = it.valid ? a.c0[it.m * a.ntiles + it.tile] : 0;
    it.nlive = it.valid ? it.nchunks - it.cstart : 0;
    return it;
}

// Persistent contraction: kCtasPerSm CTAs per SM, each walking its list of
// work items, the entries sched[gridDim.x + 1 + k] for k in
// [sched[blockIdx.x], sched[blockIdx.x + 1]) (schedule_lpt).  The producer's
// ring of kStages stages runs on across items, so the next item's first
// chunks load while the epilogue reads the accumulator; the MMAs of item j + 1
// start once it has.  Barriers: bar_load / bar_mma per stage (full / free),
// bar_full / bar_free for the accumulator, bar_done for the drain.
template <bool SYNTH>
__global__ void __launch_bounds__(kThreads, kCtasPerSm) k_tc64(Tc64Args a, const int *__restrict__ sched)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    uint64_t *bar_load = reinterpret_cast<uint64_t *>(smem + (size_t)kStages * kStage);
    uint64_t *bar_mma = bar_load + kStages;
    uint64_t *bar_full = bar_mma + kStages;
    uint64_t *bar_free = bar_full + 1;
    uint64_t *bar_done = bar_free + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_done + 1);
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int k0 = sched[blockIdx.x], k1 = sched[blockIdx.x + 1];
    const int *items = sched + gridDim.x + 1;

    if (tid == 0) {
        for (int q = 0; q < kStages; ++q) {
            tc::mbar_init(&bar_load[q], 1);
            tc::mbar_init(&bar_mma[q], 1);
        }
        tc::mbar_init(bar_full, 1);
        tc::mbar_init(bar_free, 4);   // one arrival per epilogue warp
        tc::mbar_init(bar_done, 1);
        tc::mbar_fence_init();
        s_abort = 0;
    }
    if (warp == 0) tc::tmem_alloc(tslot, kTmemCols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 4) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            uint64_t da[kSA], db;
            uint32_t idesc[kSA];
#pragma unroll
            for (int i = 0; i < kSA; ++i) {
                idesc[i] = tc::idesc_bf16_f32(kR, (kL - i) * kNC);
                da[i] = tc::smem_desc(smem + (size_t)i * kSbo, kLbo, kGS);
            }
            db = tc::smem_desc(smem + kPPar, kLbo, kSbo);
            const uint64_t sstep = (uint64_t)kStage >> 4;
            bool ok = true;
            unsigned u = 0, j = 0;
            for (int kk = k0; ok && kk < k1; ++kk) {
                const Item64 it = item64<SYNTH>(a, items[kk]);
                if (!it.valid) continue;
                if (j >= 1 && !wait_or_abort(bar_free, (j - 1) & 1, &s_abort)) { ok = false; break; }
                tc::tc_fence_after();
                const uint32_t acc = tmem;
                for (int c = 0; c < it.nlive; ++c, ++u) {
                    const unsigned q = u % kStages;
                    if (!wait_or_abort(&bar_load[q], (u / kStages) & 1, &s_abort)) { ok = false; break; }
                    tc::tc_fence_after();
                    const uint64_t so = sstep * (uint64_t)q;
                    // slice 0 spans every level: its first MMA of the item overwrites them
#pragma unroll
                    for (int i = 0; i < kSA; ++i)
                        tc::mma_bf16(acc + (uint32_t)(i * kLevelCols), da[i] + so, db + so, idesc[i], c > 0 || i > 0);
                    tc::mma_commit(&bar_mma[q]);
                }
                if (!ok) break;
                tc::mma_commit(bar_full);
                ++j;
            }
            if (!ok) raise_err(a.err, SHT_ETIMEOUT);
            // drain: no MMA may still write tensor memory when it is freed
            tc::mma_commit(bar_done);
            (void)tc::mbar_wait_bounded(bar_done, 0, 100000000ull);
        }
    } else if (warp == 5) {
        if (lane == 0) {
            // ---------------- producer ----------------
            bool ok = true;
            unsigned u = 0;
            int zl[kStages];   // leading 8-row groups of each stage known to hold zeros
#pragma unroll
            for (int q = 0; q < kStages; ++q) zl[q] = 0;
            for (int kk = k0; ok && kk < k1; ++kk) {
                const Item64 it = item64<SYNTH>(a, items[kk]);
                if (!it.valid) continue;
                const unsigned char *panel =
                    a.panel + a.off[it.m] + (size_t)it.tile * it.nchunks * kPChunk + (size_t)it.par * kPPar;
                const unsigned char *data =
                    a.data + (SYNTH ? a.dchunk[it.m] : (unsigned long long)it.m * it.nchunks) *
                                 (unsigned long long)kDChunk + (size_t)it.par * kDBlk;
                // rows of the tile that hold a pair (synthesis) or a degree (analysis):
                // 8-row groups [0, hi).  Of those, the groups below the chunk's
                // first live one, g0, are all-zero digits: they are not read, and
                // the stage must hold zeros there for the MMAs.  zl[q] counts the
                // leading groups of stage q known to be zero; groups [zl, g0) are
                // zeroed from a zero buffer (in L2) when g0 is above it, which
                // happens at an item's first chunks only, since g0 never grows
                // with c.  Groups from hi on keep whatever the stage held: they
                // reach only accumulator rows the epilogue does not write.
                const int live_rows = min(kR, (SYNTH ? a.npairs : it.Le) - it.tile * kR);
                const int hi = (live_rows + 7) / 8;
                uint4 fv[2];   // the item's 16 first live chunks, one per 8-row group
                {
                    const uint4 *fp = reinterpret_cast<const uint4 *>(
                        a.gf + (((size_t)it.m * a.ntiles + it.tile) * 2 + it.par) * 16);
                    fv[0] = fp[0];
                    fv[1] = fp[1];
                }
                const unsigned short *f = reinterpret_cast<const unsigned short *>(fv);
                for (int c = it.cstart; c < it.nchunks; ++c, ++u) {
                    const unsigned q = u % kStages;
                    if (u >= kStages && !wait_or_abort(&bar_mma[q], (u / kStages - 1) & 1, &s_abort)) {
                        ok = false;
                        break;
                    }
                    unsigned char *st = smem + (size_t)q * kStage;
                    const unsigned char *src = panel + (size_t)c * kPChunk;
                    const int g0 = first_live_group(f, c, hi), z0 = zl[q];
                    const int nzero = g0 > z0 ? g0 - z0 : 0;
                    tc::mbar_arrive_expect_tx(&bar_load[q], (uint32_t)(hi - g0 + nzero) * kGS + (uint32_t)kDBlk);
                    if (g0 < hi)
                        tc::bulk_g2s_stream(st + (size_t)g0 * kGS, src + (size_t)g0 * kGS, (uint32_t)(hi - g0) * kGS,
                                            &bar_load[q]);
                    if (nzero > 0) tc::bulk_g2s(st + (size_t)z0 * kGS, a.zero, (uint32_t)nzero * kGS, &bar_load[q]);
                    zl[q] = g0;
                    tc::bulk_g2s(st + kPPar, data + (size_t)c * kDChunk, (uint32_t)kDBlk, &bar_load[q]);
                }
            }
            if (!ok) {
                raise_err(a.err, SHT_ETIMEOUT);
                // wait (bounded) for the copies still in flight
                for (unsigned v = u > kStages ? u - kStages : 0; v < u; ++v)
                    (void)tc::mbar_wait_bounded(&bar_load[v % kStages], (v / kStages) & 1, 100000000ull);
            }
        }
    } else {
        // ---------------- epilogue (warps 0-3: TMEM lanes 32 warp ..) ----------------
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        unsigned j = 0;
        for (int kk = k0; kk < k1; ++kk) {
            const Item64 it = item64<SYNTH>(a, items[kk]);
            if (!it.valid) continue;
            if (!wait_or_abort(bar_full, j & 1, &s_abort)) {
                raise_err(a.err, SHT_ETIMEOUT);
                break;
            }
            tc::tc_fence_after();
            ++j;
            const int row = it.tile * kR + warp * 32 + lane;
            const int sc_log2 = (!SYNTH && a.op == OP_SYNTH_ADJ && it.m > 0) ? 1 : 0;   // adjoint factor 2
            // row exponent: synthesis per (m, pair), analysis per (m, n)
            const int nn = 2 * row + it.par;
            int e_row = kExpNone;
            if (SYNTH) {
                if (row < a.npairs) e_row = a.erow[(size_t)it.m * a.npairs + row];
            } else {
                if (nn < it.L) e_row = a.erow[it.col + nn];
            }
#pragma unroll 1
            for (int h = 0; h < kNC / 16; ++h) {
                // Z = sum_t L_t 2^(7 (kL - 1 - t)) = Zh 2^28 + Zl per column, levels
                // split so that both parts stay exact in 64-bit integers (< 2^48)
                long long Zh[16], Zl[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) Zh[k] = Zl[k] = 0;
                if (it.nlive > 0) {
#pragma unroll
                    for (int t = 0; t < kL; ++t) {
                        float v[16];
                        tc::tmem_ld16(lane_base + (uint32_t)(t * kLevelCols + 16 * h), v);
#pragma unroll
                        for (int k = 0; k < 16; ++k) {
                            const long long L = __float2int_rn(v[k]);   // an integer below 2^24
                            if (t < kL / 2) Zh[k] += L << (7 * (kL / 2 - 1 - t));
                            else Zl[k] += L << (7 * (kL - 1 - t));
                        }
                    }
                }
                if (h == kNC / 16 - 1) {
                    // the accumulator is read: the next item's MMAs may overwrite it
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(bar_free);
                }
#pragma unroll
                for (int k = 0; k < 16; k += 2) {
                    const int b = (16 * h + k) >> 1;
                    if (b >= a.batch) break;
                    // sum = 2^(e + f - 12 - 7 (kL - 1)) Z; zero for a row whose P are all
                    // zero (or outside the order) and for an all-zero field
                    const bool zero = e_row == kExpNone || a.fcol[b] == kExpNone;
                    const int sh = zero ? 0 : e_row + a.fcol[b] - 12 - 7 * (kL - 1) + sc_log2;
                    const __int128 zr = ((__int128)Zh[k] << (7 * (kL / 2))) + Zl[k];
                    const __int128 zi = ((__int128)Zh[k + 1] << (7 * (kL / 2))) + Zl[k + 1];
                    const double re = zero ? 0.0 : i128_ldexp(zr, sh);
                    double im = zero ? 0.0 : i128_ldexp(zi, sh);
                    if (SYNTH) {
                        if (row < a.npairs) {
                            double2 *eo = reinterpret_cast<double2 *>(a.out);
                            eo[(((size_t)b * (a.mmax + 1) + it.m) * a.npairs + row) * 2 + it.par] =
                                make_double2(re, im);
                        }
                    } else {
                        if (it.m == 0) im = 0.0;
                        if (nn < it.L)
                            reinterpret_cast<double2 *>(a.out)[(size_t)b * a.nlm + it.col + nn] = make_double2(re, im);
                    }
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

int tc64_max_batch() { return kBatch64; }
int tc64_ctas_per_sm() { return kCtasPerSm; }

// Work items of the persistent contraction, (order index, tile) x parity,
// costed as their nonzero chunks plus two for the epilogue (-1: no rows),
// grouped by (order index, parity).
void tc64_costs(int lmax, int mmax, int mres, int npairs, bool synth, const std::vector<int> &c0,
                const std::vector<unsigned short> &gf, std::vector<int> &cost, std::vector<int> &group)
{
    int ts, ta;
    tc_tile_counts(lmax, npairs, ts, ta);
    const int ntiles = synth ? ts : ta;
    cost.assign((size_t)2 * (mmax + 1) * ntiles, -1);
    group.assign(cost.size(), 0);
    for (int w = 0; w < 2 * (mmax + 1) * ntiles; ++w) {
        const int m = (w >> 1) / ntiles, tile = (w >> 1) - m * ntiles;
        group[w] = 2 * m + (w & 1);
        const int L = lmax - m * mres + 1, Le = (L + 1) / 2;
        if (!synth && tile * kR >= Le) continue;
        const int nchunks = synth ? (Le + kKc - 1) / kKc : (npairs + kKc - 1) / kKc;
        const int hi = (std::min(kR, (synth ? npairs : Le) - tile * kR) + 7) / 8;
        const unsigned short *f = gf.data() + ((size_t)(w >> 1) * 2 + (w & 1)) * 16;
        // in 8-row groups of panel (kGS bytes each): the groups read, 8 per
        // chunk for the data copy and the MMAs, 32 for the epilogue
        int units = 32;
        for (int c = c0[(size_t)m * ntiles + tile]; c < nchunks; ++c)
            units += hi - first_live_group(f, c, hi) + 8;
        cost[w] = units;
    }
}

// Fractions of the digit panels' bytes the contraction does not read: the
// chunks before the tile's first live chunk and the 8-row groups of each
// (m, tile, parity) and chunk below the chunk's first live group.
void tc64_skip_stats(int lmax, int mmax, int mres, int npairs, const std::vector<int> &c0s,
                     const std::vector<int> &c0a, const std::vector<unsigned short> &gfs,
                     const std::vector<unsigned short> &gfa, double &frac_s, double &frac_a)
{
    int ts, ta;
    tc_tile_counts(lmax, npairs, ts, ta);
    for (int dir = 0; dir < 2; ++dir) {
        const bool synth = dir == 0;
        const int ntiles = synth ? ts : ta;
        const std::vector<int> &c0 = synth ? c0s : c0a;
        const std::vector<unsigned short> &gf = synth ? gfs : gfa;
        double read = 0, tot = 0;
        for (int m = 0; m <= mmax; ++m) {
            const int Le = (lmax - m * mres + 2) / 2;
            const int nchunks = synth ? (Le + kKc - 1) / kKc : (npairs + kKc - 1) / kKc;
            for (int t = 0; t < ntiles; ++t) {
                if (!synth && t * kR >= Le) continue;
                const int hi = (std::min(kR, (synth ? npairs : Le) - t * kR) + 7) / 8;
                for (int par = 0; par < 2; ++par) {
                    const unsigned short *f = gf.data() + (((size_t)m * ntiles + t) * 2 + par) * 16;
                    tot += (double)nchunks * hi;
                    for (int c = c0[(size_t)m * ntiles + t]; c < nchunks; ++c)
                        read += hi - first_live_group(f, c, hi);
                }
            }
        }
        (synth ? frac_s : frac_a) = tot > 0 ? 1.0 - read / tot : 0.0;
    }
}

size_t tc64_zero_bytes() { return (size_t)kPPar; }

cudaError_t tc64_reset_fcol(int *fcol, int batch, cudaStream_t st)
{
    k_fill_int<<<1, 32, 0, st>>>(fcol, kExpNone, (size_t)batch);
    return cudaGetLastError();
}

void tc64_panel_layout(int lmax, int mmax, int mres, int npairs, std::vector<unsigned long long> &off_s,
                       std::vector<unsigned long long> &off_a, size_t &bytes_s, size_t &bytes_a,
                       std::vector<unsigned long long> &dchunk, size_t &nchunk_s)
{
    off_s.assign(mmax + 1, 0);
    off_a.assign(mmax + 1, 0);
    dchunk.assign(mmax + 1, 0);
    const int T = (npairs + kR - 1) / kR;
    const int kch = (npairs + kKc - 1) / kKc;
    unsigned long long s = 0, q = 0, ch = 0;
    for (int m = 0; m <= mmax; ++m) {
        const int L = lmax - m * mres + 1, Le = (L + 1) / 2;
        const int nch = (Le + kKc - 1) / kKc;
        const int Mt = (Le + kR - 1) / kR;
        off_s[m] = s;
        off_a[m] = q;
        dchunk[m] = ch;
        s += (unsigned long long)T * nch * kPChunk;
        q += (unsigned long long)Mt * kch * kPChunk;
        ch += (unsigned long long)nch;
    }
    bytes_s = s;
    bytes_a = q;
    nchunk_s = (size_t)ch;
}

size_t tc64_data_bytes(int mmax, int npairs, size_t nchunk_s)
{
    const size_t kch = (size_t)(npairs + kKc - 1) / kKc;
    const size_t an = (size_t)(mmax + 1) * kch;
    return (nchunk_s > an ? nchunk_s : an) * kDChunk;
}

cudaError_t tc64_build(const PlanView<double> &pv, const unsigned long long *off_s, const unsigned long long *off_a,
                       unsigned char *ps, unsigned char *pa, int *es, int *ea, int *c0_s, int *c0_a,
                       unsigned short *gf_s, unsigned short *gf_a, cudaStream_t st)
{
    const int nlm = pv.nlm;
    k_fill_int<<<(unsigned)((nlm + 255) / 256), 256, 0, st>>>(ea, kExpNone, (size_t)nlm);
    dim3 g((unsigned)((pv.npairs + 127) / 128), (unsigned)(pv.mmax + 1));
    k_p64_scales<<<g, 128, 0, st>>>(pv, es, ea);
    k_p64_build<<<g, 128, 0, st>>>(pv, es, ea, off_s, off_a, ps, pa);
    int ts, ta;
    tc_tile_counts(pv.lmax, pv.npairs, ts, ta);
    k_p64_first_live<<<dim3((unsigned)ts, (unsigned)(pv.mmax + 1)), 256, 0, st>>>(1, pv.lmax, pv.mres, pv.npairs, ts, off_s,
                                                                                 ps, c0_s);
    k_p64_first_live<<<dim3((unsigned)ta, (unsigned)(pv.mmax + 1)), 256, 0, st>>>(0, pv.lmax, pv.mres, pv.npairs, ta, off_a,
                                                                                 pa, c0_a);
    k_p64_group_first<<<dim3((unsigned)ts, (unsigned)(pv.mmax + 1)), 256, 0, st>>>(1, pv.lmax, pv.mres, pv.npairs, ts,
                                                                                  off_s, ps, gf_s);
    k_p64_group_first<<<dim3((unsigned)ta, (unsigned)(pv.mmax + 1)), 256, 0, st>>>(0, pv.lmax, pv.mres, pv.npairs, ta,
                                                                                  off_a, pa, gf_a);
    return cudaGetLastError();
}

cudaError_t launch_tc64(bool synth, int lmax, int mmax, int mres, int npairs, int nlm, const unsigned char *panel,
                        const unsigned long long *off, const int *c0, const unsigned short *gf,
                        const unsigned char *zero, const int *sched, int nctas, const int *erow,
                        const unsigned long long *dchunk, int *fcol, unsigned char *data, const double *in,
                        double *out, int batch, Op op, int *err, cudaStream_t st, bool fcol_ready)
{
    if (batch < 1 || batch > kBatch64) return cudaErrorInvalidValue;
    if (!fcol_ready) {
        // field exponents of the data
        k_fill_int<<<1, 32, 0, st>>>(fcol, kExpNone, (size_t)batch);
        const size_t per_field = synth ? (size_t)2 * nlm : (size_t)(mmax + 1) * npairs * 4;
        k_colscale<<<dim3(64, (unsigned)batch), 256, 0, st>>>(in, per_field, fcol);
    }
    // data digits
    const int Le0 = (lmax + 2) / 2;
    const int maxch = synth ? (Le0 + kKc - 1) / kKc : (npairs + kKc - 1) / kKc;
    const long items = (long)maxch * batch * 8;
    k_prep64<<<dim3((unsigned)((items + 127) / 128), (unsigned)(mmax + 1)), 128, 0, st>>>(
        synth ? 1 : 0, lmax, mmax, mres, npairs, nlm, batch, (int)op, in, fcol, dchunk, data);
    Tc64Args a{};
    a.lmax = lmax;
    a.mmax = mmax;
    a.mres = mres;
    a.npairs = npairs;
    a.nlm = nlm;
    a.batch = batch;
    a.op = (int)op;
    a.panel = panel;
    a.off = off;
    a.c0 = c0;
    a.gf = gf;
    a.zero = zero;
    a.erow = erow;
    a.fcol = fcol;
    a.data = data;
    a.dchunk = dchunk;
    a.out = out;
    a.err = err;
    int ts, ta;
    tc_tile_counts(lmax, npairs, ts, ta);
    a.ntiles = synth ? ts : ta;
    // ring, barriers (2 per stage, 2 for the accumulator, the drain) and the TMEM slot
    const size_t smem = 128 + (size_t)kStages * kStage + 8 * (2 * kStages + 3) + 16;
    if (!sched || nctas < 1 || !gf || !zero) return cudaErrorInvalidValue;
    cudaError_t e;
    if (synth) {
        e = cudaFuncSetAttribute(k_tc64<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_tc64<true><<<(unsigned)nctas, kThreads, smem, st>>>(a, sched);
    } else {
        e = cudaFuncSetAttribute(k_tc64<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_tc64<false><<<(unsigned)nctas, kThreads, smem, st>>>(a, sched);
    }
    return cudaGetLastError();
}

}  // namespace sht
