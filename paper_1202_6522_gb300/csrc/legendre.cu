// legendre.cu -- the per-order Legendre stage of the Gauss-Legendre SHT.
//
// Synthesis (Sec. 2.2, Eq. synth_direct): for each order m and each latitude
// pair (x, -x), sum over n the spectral coefficients times P_n^m, split by the
// parity of n - m (mirror symmetry, Sec. 3.1):
//   E = sum_{n-m even} f_n^m P_n^m(x),  O = sum_{n-m odd} f_n^m P_n^m(x),
//   f_m(x) = E + O,  f_m(-x) = E - O   (the fold is applied by the FFT kernel).
// Analysis (Sec. 2.3, Eq. gauss): with s = w (F(x) + F(-x)), d = w (F(x) - F(-x))
// prepared by the FFT kernel, f_n^m = sum_pairs P_n^m(x) (s if n-m even else d).
//
// P_n^m is generated on the fly by the recurrence of Sec. 3.2, held in
// registers, one thread per latitude pair (LPT pairs per thread); the
// coefficients (a_n^m, b_n^m) and the spectral values are staged through
// shared memory and read as broadcasts.  Underflow is handled as in Sec. 3.5:
// a value is y * 2^(-S k); while k > 0 it is left out of the sums and the
// recurrence rescales y by 2^-S when it exceeds 1.  Warps in which every pair
// is still scaled skip the accumulation (the dynamic polar optimisation).
//
// Analysis reduces over latitudes without atomics: each thread sums its own
// pairs in registers for K consecutive degrees, a warp-level transposing
// butterfly leaves one partial per lane, and the warps' partials are added in
// shared memory in a fixed order, so results are bitwise reproducible.
#include <cuda_runtime.h>

#include "sht_internal.h"

namespace sht {
namespace {

constexpr unsigned kFull = 0xffffffffu;

template <typename T> __device__ __forceinline__ bool abs_ge_one(T y);
template <> __device__ __forceinline__ bool abs_ge_one<double>(double y)
{
    return (__double2hiint(y) & 0x7fffffff) >= 0x3ff00000;
}
template <> __device__ __forceinline__ bool abs_ge_one<float>(float y)
{
    return (__float_as_int(y) & 0x7fffffff) >= 0x3f800000;
}

template <typename T> __device__ __forceinline__ T down_scale();
template <> __device__ __forceinline__ double down_scale<double>() { return 0x1p-240; }
template <> __device__ __forceinline__ float down_scale<float>() { return 0x1p-64f; }

// One step of P_n = a x P_{n-1} + b P_{n-2} for LPT pairs.  With CHECK the
// rescaling of Sec. 3.5 is applied and c[] receives the value entering the
// sums (0 while k > 0); without it c[] is the value itself.  Pairs i whose
// bit in `live` (warp-uniform) is clear are left as they are, with c[i] = 0.
template <typename T, int LPT, bool CHECK>
__device__ __forceinline__ void rec_step(T a, T b, const T (&x)[LPT], T (&y1)[LPT], T (&y2)[LPT],
                                         int (&k)[LPT], T (&c)[LPT], unsigned live = ~0u)
{
#pragma unroll
    for (int i = 0; i < LPT; ++i) {
        if (!((live >> i) & 1)) {
            c[i] = T(0);
            continue;
        }
        T yn = fma(a * x[i], y1[i], b * y2[i]);
        y2[i] = y1[i];
        y1[i] = yn;
        if (CHECK) {
            if (k[i] > 0 && abs_ge_one(yn)) {
                y1[i] *= down_scale<T>();
                y2[i] *= down_scale<T>();
                k[i] -= 1;
            }
            c[i] = (k[i] == 0) ? y1[i] : T(0);
        } else {
            c[i] = yn;
        }
    }
}

template <typename T, int LPT>
__device__ __forceinline__ int kmax_of(const int (&k)[LPT])
{
    int r = 0;
#pragma unroll
    for (int i = 0; i < LPT; ++i) r = max(r, k[i]);
    return r;
}

template <typename T, int LPT>
__device__ __forceinline__ int kmin_of(const int (&k)[LPT])
{
    int r = k[0];
#pragma unroll
    for (int i = 1; i < LPT; ++i) r = min(r, k[i]);
    return r;
}

// Restart the recurrence of the LPT pairs p[] at segment `seg` (degrees
// n - m in [kSeedSeg seg, kSeedSeg (seg + 1))) of order index m from the
// state the FP64 recurrence computed once per plan: y1 = P_{n0-1},
// y2 = P_{n0-2} and the exponent counter k of Sec. 3.5, in the precision's
// own scaled form.  FP32 kernels restart every segment (the FP32 recurrence
// alone loses accuracy with n); FP64 kernels restart where they skip dead
// segments (the static polar optimisation).
template <typename T, int LPT>
__device__ __forceinline__ void reseed(const PlanView<T> &pv, int m, int seg, const int (&p)[LPT], T (&y1)[LPT],
                                       T (&y2)[LPT], int (&k)[LPT])
{
    const size_t base = (size_t)(pv.segoff[m] + seg) * pv.npairs;
#pragma unroll
    for (int i = 0; i < LPT; ++i) {
        if (p[i] < pv.npairs) {
            if constexpr (sizeof(T) == sizeof(float)) {
                const float4 v = __ldg(pv.seeds + base + p[i]);
                y1[i] = v.x;
                y2[i] = v.y;
                k[i] = __float_as_int(v.z);
            } else {
                const double2 v = __ldg(pv.seeds64 + base + p[i]);
                y1[i] = v.x;
                y2[i] = v.y;
                k[i] = __ldg(pv.seeds64k + base + p[i]);
            }
        }
    }
}

// First live segment of each group i of 32 pairs (the warp's lanes' p[i];
// no pair: past every segment), warp-uniform; returns the smallest.
template <typename T, int LPT>
__device__ __forceinline__ int group_first_live(const PlanView<T> &pv, int m, const int (&p)[LPT], int (&gf)[LPT])
{
    int r = 0xffff;
#pragma unroll
    for (int i = 0; i < LPT; ++i) {
        const int f = p[i] < pv.npairs ? (int)__ldg(pv.live + (size_t)m * pv.npairs + p[i]) : 0xffff;
        gf[i] = __reduce_min_sync(kFull, f);
        r = min(r, gf[i]);
    }
    return r;
}

// Bit i set when group i has a live pair in segment seg.
template <int LPT>
__device__ __forceinline__ unsigned live_groups(const int (&gf)[LPT], int seg)
{
    unsigned r = 0;
#pragma unroll
    for (int i = 0; i < LPT; ++i)
        if (seg >= gf[i]) r |= 1u << i;
    return r;
}

// The scalar kernels need the restart states and the first-live table (both
// precisions); the vector kernels need the restart states in FP32 only.  A
// plan without them is refused rather than run on other arithmetic.
template <typename T> bool seeds_ok(const PlanView<T> &pv, bool scalar)
{
    if (sizeof(T) == sizeof(float))
        return pv.segoff != nullptr && pv.seeds != nullptr && (!scalar || pv.live != nullptr);
    return !scalar || (pv.segoff != nullptr && pv.seeds64 != nullptr && pv.seeds64k != nullptr && pv.live != nullptr);
}

// Warp butterfly that sums V values (V a multiple of 32) over the 32 lanes and
// leaves lane l holding the sums of values [l*V/32, (l+1)*V/32) in v[0..V/32).
template <typename T, int V>
__device__ __forceinline__ void warp_transpose_reduce(T (&v)[V], int lane)
{
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int o = 16 >> s;
        const int h = V >> (s + 1);
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int q = 0; q < h; ++q) {
            T send = up ? v[q] : v[q + h];
            T keep = up ? v[q + h] : v[q];
            v[q] = keep + __shfl_xor_sync(kFull, send, o);
        }
    }
}

// ---------------------------------------------------------------------------
// Scalar synthesis.  grid.x = (m, pair block), heaviest m first; grid.y = field chunk.
// ---------------------------------------------------------------------------
constexpr int kSynthNch = 128;  // degrees staged per chunk (scalar synthesis)
static_assert(kSynthNch % kSeedSeg == 0, "restart segments must not straddle staged chunks");

// One (order m, pair block pb, field chunk b0) tile of the scalar synthesis,
// run by a whole CTA of NT threads; s_ab[kSynthNch], s_f[kSynthNch * BC] are
// the CTA's staging buffers, *s_first a shared word.
//
// Static polar optimisation (Sec. 3.1): the CTA starts at the first segment
// in which one of its pairs is live; within a warp, a group of 32 pairs (one
// p[i] per lane) runs neither the recurrence nor the sums over a segment in
// which none of its pairs is live.  Each segment a warp runs restarts the
// recurrence from the stored state.
template <typename T, int LPT, int BC, int NT>
__device__ __forceinline__ void synth_tile(const PlanView<T> &pv, const T *__restrict__ spec, T *__restrict__ eo,
                                           int batch, int m, int pb, int b0, int op, typename Vec2<T>::type *s_ab,
                                           typename Vec2<T>::type *s_f, int *s_first)
{
    using T2 = typename Vec2<T>::type;
    constexpr int NCH = kSynthNch;
    const int lmax = pv.lmax, npairs = pv.npairs;
    const int L = lmax - m * pv.mres + 1;   // order index m is the order m mres
    const long col = col_of_mres(lmax, m, pv.mres);

    T x[LPT], y1[LPT], y2[LPT], c[LPT];
    int k[LPT], p[LPT];
#pragma unroll
    for (int i = 0; i < LPT; ++i) {
        p[i] = pb * NT * LPT + i * NT + threadIdx.x;
        const bool v = p[i] < npairs;
        const size_t o = (size_t)m * npairs + p[i];
        x[i] = v ? pv.x[p[i]] : T(0);
        y2[i] = v ? pv.pmm[o] : T(0);
        k[i] = v ? pv.pmmk[o] : 0;
        y1[i] = T(0);
    }
    T er[LPT][BC], ei[LPT][BC], orr[LPT][BC], oi[LPT][BC];
#pragma unroll
    for (int i = 0; i < LPT; ++i)
#pragma unroll
        for (int b = 0; b < BC; ++b) er[i][b] = ei[i][b] = orr[i][b] = oi[i][b] = T(0);

    // adjoint of analysis: synthesis of b / c_m
    const T insc = (op == OP_ANALYS_ADJ && m > 0) ? T(0.5) : T(1);
    const T2 *spec2 = reinterpret_cast<const T2 *>(spec);

    int gf[LPT];
    const int wfirst = group_first_live<T, LPT>(pv, m, p, gf);
    if (threadIdx.x == 0) *s_first = 0xffff;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicMin(s_first, wfirst);
    __syncthreads();
    const int start = min(*s_first * kSeedSeg, L);

    for (int n0 = start; n0 < L; n0 += NCH) {
        const int cnt = min(NCH, L - n0);
        __syncthreads();
        for (int t = threadIdx.x; t < NCH; t += NT) {
            T2 ab;
            ab.x = T(0); ab.y = T(0);
            if (t < cnt) ab = pv.ab[col + n0 + t];
            s_ab[t] = ab;
#pragma unroll
            for (int b = 0; b < BC; ++b) {
                T2 f;
                f.x = T(0); f.y = T(0);
                if (t < cnt && b0 + b < batch) {
                    f = spec2[(size_t)(b0 + b) * pv.nlm + col + n0 + t];
                    f.x *= insc;
                    f.y = (m == 0) ? T(0) : f.y * insc;
                }
                s_f[t * BC + b] = f;
            }
        }
        __syncthreads();
        for (int s0 = 0; s0 < cnt; s0 += kSeedSeg) {
            const unsigned gl = live_groups<LPT>(gf, (n0 + s0) / kSeedSeg);
            if (gl == 0) continue;   // no live pair in this warp yet
            reseed<T, LPT>(pv, m, (n0 + s0) / kSeedSeg, p, y1, y2, k);
            const int s1 = min(cnt, s0 + kSeedSeg);
            const bool scaled = __any_sync(kFull, kmax_of<T, LPT>(k) > 0);
            if (!scaled) {
                for (int t = s0; t < s1; t += 2) {
                    T2 ab = s_ab[t];
                    rec_step<T, LPT, false>(ab.x, ab.y, x, y1, y2, k, c, gl);
#pragma unroll
                    for (int b = 0; b < BC; ++b) {
                        const T2 f = s_f[t * BC + b];
#pragma unroll
                        for (int i = 0; i < LPT; ++i) {
                            if (!((gl >> i) & 1)) continue;
                            er[i][b] = fma(f.x, c[i], er[i][b]);
                            ei[i][b] = fma(f.y, c[i], ei[i][b]);
                        }
                    }
                    ab = s_ab[t + 1];
                    rec_step<T, LPT, false>(ab.x, ab.y, x, y1, y2, k, c, gl);
#pragma unroll
                    for (int b = 0; b < BC; ++b) {
                        const T2 f = s_f[(t + 1) * BC + b];
#pragma unroll
                        for (int i = 0; i < LPT; ++i) {
                            if (!((gl >> i) & 1)) continue;
                            orr[i][b] = fma(f.x, c[i], orr[i][b]);
                            oi[i][b] = fma(f.y, c[i], oi[i][b]);
                        }
                    }
                }
            } else {
                for (int t = s0; t < s1; t += 2) {
                    T2 ab = s_ab[t];
                    rec_step<T, LPT, true>(ab.x, ab.y, x, y1, y2, k, c, gl);
                    if (__any_sync(kFull, kmin_of<T, LPT>(k) == 0)) {
#pragma unroll
                        for (int b = 0; b < BC; ++b) {
                            const T2 f = s_f[t * BC + b];
#pragma unroll
                            for (int i = 0; i < LPT; ++i) {
                                if (!((gl >> i) & 1)) continue;
                                er[i][b] = fma(f.x, c[i], er[i][b]);
                                ei[i][b] = fma(f.y, c[i], ei[i][b]);
                            }
                        }
                    }
                    ab = s_ab[t + 1];
                    rec_step<T, LPT, true>(ab.x, ab.y, x, y1, y2, k, c, gl);
                    if (__any_sync(kFull, kmin_of<T, LPT>(k) == 0)) {
#pragma unroll
                        for (int b = 0; b < BC; ++b) {
                            const T2 f = s_f[(t + 1) * BC + b];
#pragma unroll
                            for (int i = 0; i < LPT; ++i) {
                                if (!((gl >> i) & 1)) continue;
                                orr[i][b] = fma(f.x, c[i], orr[i][b]);
                                oi[i][b] = fma(f.y, c[i], oi[i][b]);
                            }
                        }
                    }
                }
            }
        }
    }

    T2 *eo2 = reinterpret_cast<T2 *>(eo);
#pragma unroll
    for (int i = 0; i < LPT; ++i) {
        if (p[i] >= npairs) continue;
#pragma unroll
        for (int b = 0; b < BC; ++b) {
            if (b0 + b >= batch) continue;
            const size_t o = (((size_t)(b0 + b) * (pv.mmax + 1) + m) * npairs + p[i]) * 2;
            T2 e, d;
            e.x = er[i][b]; e.y = ei[i][b];
            d.x = orr[i][b]; d.y = oi[i][b];
            eo2[o] = e;
            eo2[o + 1] = d;
        }
    }
}

template <typename T, int LPT, int BC, int NT>
__global__ void __launch_bounds__(NT)
k_synth(PlanView<T> pv, const T *__restrict__ spec, T *__restrict__ eo, int batch, int npb, int op)
{
    using T2 = typename Vec2<T>::type;
    __shared__ T2 s_ab[kSynthNch];
    __shared__ T2 s_f[kSynthNch * BC];
    __shared__ int s_first;
    const int m = blockIdx.x / npb;
    const int pb = blockIdx.x - m * npb;
    synth_tile<T, LPT, BC, NT>(pv, spec, eo, batch, m, pb, blockIdx.y * BC, op, s_ab, s_f, &s_first);
}

// ---------------------------------------------------------------------------
// Scalar analysis.  grid.x = m (heaviest first), grid.y = field chunk; the CTA
// covers all latitude pairs (NT * LPT >= npairs).
// ---------------------------------------------------------------------------
constexpr int kAnalysNch = 128;  // degrees staged per chunk (scalar analysis)
static_assert(kAnalysNch % kSeedSeg == 0 && kSeedSeg % 16 == 0, "restart segments must align with the chunks");

// One (order m, field chunk b0) tile of the scalar analysis, run by the whole
// CTA (blockDim.x * LPT >= npairs, at most 8 warps); s_ab[kAnalysNch] and
// s_red[8 * 32] are the CTA's buffers.
template <typename T, int LPT, int BC>
__device__ __forceinline__ void analys_tile(const PlanView<T> &pv, const T *__restrict__ sd, T *__restrict__ spec,
                                            int batch, int m, int b0, int op, typename Vec2<T>::type *s_ab,
                                            T (*s_red)[32])
{
    using T2 = typename Vec2<T>::type;
    constexpr int K = 16 / BC;   // degrees per reduction: 2*K*BC = 32 values
    constexpr int NCH = kAnalysNch;  // multiple of K

    const int NT = blockDim.x;
    const int nw = NT >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lmax = pv.lmax, npairs = pv.npairs;
    const int L = lmax - m * pv.mres + 1;   // order index m is the order m mres
    const long col = col_of_mres(lmax, m, pv.mres);

    T x[LPT], y1[LPT], y2[LPT], c[LPT];
    int k[LPT], p[LPT];
    T2 sv[LPT][BC], dv[LPT][BC];
    const T2 *sd2 = reinterpret_cast<const T2 *>(sd);
#pragma unroll
    for (int i = 0; i < LPT; ++i) {
        p[i] = i * NT + threadIdx.x;
        const bool v = p[i] < npairs;
        const size_t o = (size_t)m * npairs + p[i];
        x[i] = v ? pv.x[p[i]] : T(0);
        y2[i] = v ? pv.pmm[o] : T(0);
        k[i] = v ? pv.pmmk[o] : 0;
        y1[i] = T(0);
#pragma unroll
        for (int b = 0; b < BC; ++b) {
            T2 z;
            z.x = T(0); z.y = T(0);
            sv[i][b] = z;
            dv[i][b] = z;
            if (v && b0 + b < batch) {
                const size_t q = (((size_t)(b0 + b) * (pv.mmax + 1) + m) * npairs + p[i]) * 2;
                sv[i][b] = sd2[q];
                dv[i][b] = sd2[q + 1];
            }
        }
    }
    // output scale: c_m for the adjoint of synthesis
    const T outsc = (op == OP_SYNTH_ADJ && m > 0) ? T(2) : T(1);
    T2 *spec2 = reinterpret_cast<T2 *>(spec);
    int gf[LPT];
    group_first_live<T, LPT>(pv, m, p, gf);

    for (int n0 = 0; n0 < L; n0 += NCH) {
        const int cnt = min(NCH, L - n0);
        __syncthreads();
        for (int t = threadIdx.x; t < NCH; t += NT) {
            T2 ab;
            ab.x = T(0); ab.y = T(0);
            if (t < cnt) ab = pv.ab[col + n0 + t];
            s_ab[t] = ab;
        }
        __syncthreads();
        for (int t0 = 0; t0 < cnt; t0 += K) {
            // static polar optimisation: groups of 32 pairs with no live pair
            // in this segment run neither the recurrence nor the sums; a warp
            // with none contributes zeros
            const unsigned gl = live_groups<LPT>(gf, (n0 + t0) / kSeedSeg);
            const bool wlive = gl != 0;
            if (wlive && (n0 + t0) % kSeedSeg == 0) reseed<T, LPT>(pv, m, (n0 + t0) / kSeedSeg, p, y1, y2, k);
            T acc[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) acc[q] = T(0);
            const bool scaled = __any_sync(kFull, kmax_of<T, LPT>(k) > 0);
            if (wlive) {
#pragma unroll
                for (int kx = 0; kx < K; ++kx) {
                    const T2 ab = s_ab[t0 + kx];
                    bool live = true;
                    if (scaled) {
                        rec_step<T, LPT, true>(ab.x, ab.y, x, y1, y2, k, c, gl);
                        live = __any_sync(kFull, kmin_of<T, LPT>(k) == 0);
                    } else {
                        rec_step<T, LPT, false>(ab.x, ab.y, x, y1, y2, k, c, gl);
                    }
                    if (live) {
#pragma unroll
                        for (int b = 0; b < BC; ++b) {
#pragma unroll
                            for (int i = 0; i < LPT; ++i) {
                                if (!((gl >> i) & 1)) continue;
                                const T2 v = (kx & 1) ? dv[i][b] : sv[i][b];
                                acc[(kx * BC + b) * 2] = fma(c[i], v.x, acc[(kx * BC + b) * 2]);
                                acc[(kx * BC + b) * 2 + 1] = fma(c[i], v.y, acc[(kx * BC + b) * 2 + 1]);
                            }
                        }
                    }
                }
                warp_transpose_reduce<T, 32>(acc, lane);
            }
            s_red[warp][lane] = acc[0];
            __syncthreads();
            if (threadIdx.x < 2 * K * BC) {
                T tot = T(0);
                for (int w = 0; w < nw; ++w) tot += s_red[w][threadIdx.x];
                const int q = threadIdx.x;
                const int kx = q / (2 * BC), b = (q >> 1) % BC, part = q & 1;
                const int nn = n0 + t0 + kx;  // n - m
                if (nn < L && b0 + b < batch) {
                    T val = tot * outsc;
                    if (m == 0 && part == 1) val = T(0);
                    T *dst = reinterpret_cast<T *>(&spec2[(size_t)(b0 + b) * pv.nlm + col + nn]);
                    dst[part] = val;
                }
            }
            __syncthreads();
        }
    }
}

template <typename T, int LPT, int BC>
__global__ void __launch_bounds__(256)
k_analys(PlanView<T> pv, const T *__restrict__ sd, T *__restrict__ spec, int batch, int op)
{
    using T2 = typename Vec2<T>::type;
    __shared__ T2 s_ab[kAnalysNch];
    __shared__ T s_red[8][32];
    analys_tile<T, LPT, BC>(pv, sd, spec, batch, blockIdx.x, blockIdx.y * BC, op, s_ab, s_red);
}

// ---------------------------------------------------------------------------
// Scalar analysis, one warp per segment (FP64; npairs <= 32 PPL).
// grid.x = m (heaviest first), grid.y = field group of BC.  The CTA stages
// the folds s, d of its BC fields for all pairs in shared memory; each of its
// kSegWarps warps then takes kSeedSeg-degree segments from a shared counter,
// restarts the recurrence from the stored state and sums over every pair on
// its own: PPL pairs per lane, then one warp butterfly per K = 16 / BC
// degrees.  There is no CTA-wide barrier inside the sums, the recurrence is
// shared by BC fields, and the cross-lane reduction costs 1/PPL of the sums;
// the order of every sum is fixed, so results are bitwise reproducible.
// Groups of 32 pairs with no live pair in a segment (static polar
// optimisation, Sec. 3.1) run neither the recurrence nor the sums.
// ---------------------------------------------------------------------------
constexpr int kSegWarps = 8;

template <typename T, int PPL, int BC>
__global__ void __launch_bounds__(kSegWarps * 32, 1)
k_analys_seg(PlanView<T> pv, const T *__restrict__ sd, T *__restrict__ spec, int batch, int op)
{
    using T2 = typename Vec2<T>::type;
    constexpr int K = 16 / BC;        // degrees per butterfly: 2 K BC = 32 values
    constexpr int R = 32 * PPL;       // staged row: the pairs, zero-padded
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *s_v = reinterpret_cast<T2 *>(smem_raw);   // [BC][parity][R]: s (n - m even), d (odd)
    __shared__ int s_next;
    __shared__ int s_gfirst[PPL];                 // first live segment of each group of 32 pairs

    const int m = blockIdx.x, b0 = blockIdx.y * BC;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int npairs = pv.npairs;
    const int L = pv.lmax - m * pv.mres + 1;   // order index m is the order m mres
    const long col = col_of_mres(pv.lmax, m, pv.mres);
    const int nseg = (L + kSeedSeg - 1) / kSeedSeg;

    const T2 *sd2 = reinterpret_cast<const T2 *>(sd);
    for (int idx = threadIdx.x; idx < BC * 2 * R; idx += blockDim.x) {
        const int b = idx / (2 * R), r = idx - b * 2 * R;
        T2 v;
        v.x = T(0); v.y = T(0);
        if (r < 2 * npairs && b0 + b < batch) v = sd2[((size_t)(b0 + b) * (pv.mmax + 1) + m) * npairs * 2 + r];
        s_v[(b * 2 + (r & 1)) * R + (r >> 1)] = v;
    }
    for (int g = warp; g < PPL; g += kSegWarps) {
        const int pp = g * 32 + lane;
        const int f = pp < npairs ? (int)pv.live[(size_t)m * npairs + pp] : 0xffff;
        const int gm = __reduce_min_sync(kFull, f);
        if (lane == 0) s_gfirst[g] = gm;
    }
    if (threadIdx.x == 0) s_next = kSegWarps;
    __syncthreads();

    const T outsc = (op == OP_SYNTH_ADJ && m > 0) ? T(2) : T(1);   // c_m for the adjoint of synthesis
    T2 *spec2 = reinterpret_cast<T2 *>(spec);
    int p[PPL];
    T x[PPL];
#pragma unroll
    for (int i = 0; i < PPL; ++i) {
        p[i] = lane + 32 * i;
        x[i] = p[i] < npairs ? pv.x[p[i]] : T(0);
    }
    // value `lane` of the butterfly: degree t0 + kx, field b, real/imaginary part
    const int okx = lane / (2 * BC), ob = (lane >> 1) % BC, opart = lane & 1;

    for (int seg = warp; seg < nseg;) {
        const int nn0 = seg * kSeedSeg, cnt = min(kSeedSeg, L - nn0);
        unsigned live = 0;
#pragma unroll
        for (int i = 0; i < PPL; ++i)
            if (s_gfirst[i] <= seg) live |= 1u << i;
        if (live == 0) {
            for (int q = lane; q < cnt * 2 * BC; q += 32) {
                const int kx = q / (2 * BC), b = (q >> 1) % BC;
                if (b0 + b < batch)
                    reinterpret_cast<T *>(&spec2[(size_t)(b0 + b) * pv.nlm + col + nn0 + kx])[q & 1] = T(0);
            }
        } else {
            T y1[PPL], y2[PPL];
            int k[PPL];
#pragma unroll
            for (int i = 0; i < PPL; ++i) {
                y1[i] = y2[i] = T(0);
                k[i] = 0;
            }
            reseed<T, PPL>(pv, m, seg, p, y1, y2, k);
            unsigned scaled = 0;
#pragma unroll
            for (int i = 0; i < PPL; ++i)
                if (__any_sync(kFull, k[i] > 0)) scaled |= 1u << i;
            for (int t0 = 0; t0 < cnt; t0 += K) {
                T acc[32];
#pragma unroll
                for (int q = 0; q < 32; ++q) acc[q] = T(0);
#pragma unroll
                for (int kx = 0; kx < K; ++kx) {
                    if (t0 + kx >= cnt) break;
                    const T2 ab = __ldg(&pv.ab[col + nn0 + t0 + kx]);
                    const T2 *vrow = s_v + ((t0 + kx) & 1) * R;   // nn0 is even
#pragma unroll
                    for (int i = 0; i < PPL; ++i) {
                        if (!((live >> i) & 1)) continue;
                        const T yn = fma(ab.x * x[i], y1[i], ab.y * y2[i]);
                        y2[i] = y1[i];
                        y1[i] = yn;
                        T c = yn;
                        if ((scaled >> i) & 1) {
                            if (k[i] > 0 && abs_ge_one(yn)) {
                                y1[i] *= down_scale<T>();
                                y2[i] *= down_scale<T>();
                                k[i] -= 1;
                            }
                            c = (k[i] == 0) ? y1[i] : T(0);
                        }
#pragma unroll
                        for (int b = 0; b < BC; ++b) {
                            const T2 v = vrow[b * 2 * R + p[i]];
                            acc[(kx * BC + b) * 2] = fma(c, v.x, acc[(kx * BC + b) * 2]);
                            acc[(kx * BC + b) * 2 + 1] = fma(c, v.y, acc[(kx * BC + b) * 2 + 1]);
                        }
                    }
                }
                warp_transpose_reduce<T, 32>(acc, lane);
                if (t0 + okx < cnt && b0 + ob < batch) {
                    T val = acc[0] * outsc;
                    if (m == 0 && opart == 1) val = T(0);
                    reinterpret_cast<T *>(&spec2[(size_t)(b0 + ob) * pv.nlm + col + nn0 + t0 + okx])[opart] = val;
                }
            }
        }
        int nx = 0;
        if (lane == 0) nx = atomicAdd(&s_next, 1);
        seg = __shfl_sync(kFull, nx, 0);
    }
}

// More pairs than a warp holds (npairs <= 32 PPL TEAM): a team of TEAM warps
// takes each segment, every warp summing its own 32 PPL pairs; per butterfly
// the warps' partial sums meet in shared memory (double-buffered by
// butterfly, one named barrier per team each time) and the team's first warp
// adds them in a fixed order and writes the coefficients.  Teams take the
// segments t, t + teams, ... of the order.
template <typename T, int PPL, int BC, int TEAM>
__global__ void __launch_bounds__(kSegWarps * 32, 1)
k_analys_seg_team(PlanView<T> pv, const T *__restrict__ sd, T *__restrict__ spec, int batch, int op)
{
    using T2 = typename Vec2<T>::type;
    constexpr int K = 16 / BC;           // degrees per butterfly: 2 K BC = 32 values
    constexpr int R = 32 * PPL * TEAM;   // staged row: the pairs, zero-padded
    constexpr int NTEAM = kSegWarps / TEAM, NG = PPL * TEAM;
    static_assert(kSegWarps % TEAM == 0, "whole teams");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *s_v = reinterpret_cast<T2 *>(smem_raw);   // [BC][parity][R]: s (n - m even), d (odd)
    __shared__ int s_gfirst[NG];                  // first live segment of each group of 32 pairs
    __shared__ T s_part[NTEAM][2][TEAM][32];      // the warps' partial sums

    const int m = blockIdx.x, b0 = blockIdx.y * BC;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int team = warp / TEAM, wt = warp - team * TEAM;
    const int npairs = pv.npairs;
    const int L = pv.lmax - m * pv.mres + 1;   // order index m is the order m mres
    const long col = col_of_mres(pv.lmax, m, pv.mres);
    const int nseg = (L + kSeedSeg - 1) / kSeedSeg;

    const T2 *sd2 = reinterpret_cast<const T2 *>(sd);
    for (int idx = threadIdx.x; idx < BC * 2 * R; idx += blockDim.x) {
        const int b = idx / (2 * R), r = idx - b * 2 * R;
        T2 v;
        v.x = T(0); v.y = T(0);
        if (r < 2 * npairs && b0 + b < batch) v = sd2[((size_t)(b0 + b) * (pv.mmax + 1) + m) * npairs * 2 + r];
        s_v[(b * 2 + (r & 1)) * R + (r >> 1)] = v;
    }
    for (int g = warp; g < NG; g += kSegWarps) {
        const int pp = g * 32 + lane;
        const int f = pp < npairs ? (int)pv.live[(size_t)m * npairs + pp] : 0xffff;
        const int gm = __reduce_min_sync(kFull, f);
        if (lane == 0) s_gfirst[g] = gm;
    }
    __syncthreads();

    const T outsc = (op == OP_SYNTH_ADJ && m > 0) ? T(2) : T(1);   // c_m for the adjoint of synthesis
    T2 *spec2 = reinterpret_cast<T2 *>(spec);
    const int pbase = wt * 32 * PPL;
    int p[PPL];
    T x[PPL];
#pragma unroll
    for (int i = 0; i < PPL; ++i) {
        p[i] = pbase + lane + 32 * i;
        x[i] = p[i] < npairs ? pv.x[p[i]] : T(0);
    }
    const int okx = lane / (2 * BC), ob = (lane >> 1) % BC, opart = lane & 1;
    unsigned kb = 0;   // butterflies done by this team (selects the partial buffer)

    for (int seg = team; seg < nseg; seg += NTEAM) {
        const int nn0 = seg * kSeedSeg, cnt = min(kSeedSeg, L - nn0);
        unsigned live = 0;      // this warp's groups
        bool team_live = false;
#pragma unroll
        for (int i = 0; i < PPL; ++i)
            if (s_gfirst[wt * PPL + i] <= seg) live |= 1u << i;
        for (int g = 0; g < NG; ++g) team_live |= s_gfirst[g] <= seg;
        if (!team_live) {
            if (wt == 0) {
                for (int q = lane; q < cnt * 2 * BC; q += 32) {
                    const int kx = q / (2 * BC), b = (q >> 1) % BC;
                    if (b0 + b < batch)
                        reinterpret_cast<T *>(&spec2[(size_t)(b0 + b) * pv.nlm + col + nn0 + kx])[q & 1] = T(0);
                }
            }
            continue;
        }
        T y1[PPL], y2[PPL];
        int k[PPL];
#pragma unroll
        for (int i = 0; i < PPL; ++i) {
            y1[i] = y2[i] = T(0);
            k[i] = 0;
        }
        if (live) reseed<T, PPL>(pv, m, seg, p, y1, y2, k);
        unsigned scaled = 0;
#pragma unroll
        for (int i = 0; i < PPL; ++i)
            if (__any_sync(kFull, k[i] > 0)) scaled |= 1u << i;
        for (int t0 = 0; t0 < cnt; t0 += K, ++kb) {
            T acc[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) acc[q] = T(0);
            if (live) {
#pragma unroll
                for (int kx = 0; kx < K; ++kx) {
                    if (t0 + kx >= cnt) break;
                    const T2 ab = __ldg(&pv.ab[col + nn0 + t0 + kx]);
                    const T2 *vrow = s_v + ((t0 + kx) & 1) * R;   // nn0 is even
#pragma unroll
                    for (int i = 0; i < PPL; ++i) {
                        if (!((live >> i) & 1)) continue;
                        const T yn = fma(ab.x * x[i], y1[i], ab.y * y2[i]);
                        y2[i] = y1[i];
                        y1[i] = yn;
                        T c = yn;
                        if ((scaled >> i) & 1) {
                            if (k[i] > 0 && abs_ge_one(yn)) {
                                y1[i] *= down_scale<T>();
                                y2[i] *= down_scale<T>();
                                k[i] -= 1;
                            }
                            c = (k[i] == 0) ? y1[i] : T(0);
                        }
#pragma unroll
                        for (int b = 0; b < BC; ++b) {
                            const T2 v = vrow[b * 2 * R + p[i]];
                            acc[(kx * BC + b) * 2] = fma(c, v.x, acc[(kx * BC + b) * 2]);
                            acc[(kx * BC + b) * 2 + 1] = fma(c, v.y, acc[(kx * BC + b) * 2 + 1]);
                        }
                    }
                }
                warp_transpose_reduce<T, 32>(acc, lane);
            }
            s_part[team][kb & 1][wt][lane] = acc[0];
            // the team's warps: named barrier 1 + team over 32 TEAM threads
            asm volatile("bar.sync %0, %1;" ::"r"(1 + team), "r"(32 * TEAM) : "memory");
            if (wt == 0 && t0 + okx < cnt && b0 + ob < batch) {
                T tot = s_part[team][kb & 1][0][lane];
#pragma unroll
                for (int w = 1; w < TEAM; ++w) tot += s_part[team][kb & 1][w][lane];
                T val = tot * outsc;
                if (m == 0 && opart == 1) val = T(0);
                reinterpret_cast<T *>(&spec2[(size_t)(b0 + ob) * pv.nlm + col + nn0 + t0 + okx])[opart] = val;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Vector synthesis.  With dP = sin(theta) dP/dtheta = n x P_n - dc_n P_{n-1}:
//   sin * V_theta,m = sum [S dP - i m T P],   sin * V_phi,m = sum [i m S P + T dP].
// dP has the opposite mirror parity of P.  Outputs E/O for theta and phi.
// ---------------------------------------------------------------------------
template <typename T, int LPT, int BC, int NT>
__global__ void __launch_bounds__(NT)
k_synth_vec(PlanView<T> pv, const T *__restrict__ Sg, const T *__restrict__ Tg, T *__restrict__ eot,
            T *__restrict__ eop, int batch, int npb, int op)
{
    using T2 = typename Vec2<T>::type;
    constexpr int NCH = 64;
    __shared__ T2 s_ab[NCH];
    __shared__ T s_dc[NCH];
    __shared__ T2 s_S[NCH * BC];
    __shared__ T2 s_T[NCH * BC];

    const int m = blockIdx.x / npb;
    const int pb = blockIdx.x - m * npb;
    const int b0 = blockIdx.y * BC;
    const int lmax = pv.lmax, npairs = pv.npairs;
    const int L = lmax - m * pv.mres + 1;   // order index m is the order m mres
    const long col = col_of_mres(lmax, m, pv.mres);

    T x[LPT], y1[LPT], y2[LPT], c[LPT];
    int k[LPT], p[LPT];
#pragma unroll
    for (int i = 0; i < LPT; ++i) {
        p[i] = pb * NT * LPT + i * NT + threadIdx.x;
        const bool v = p[i] < npairs;
        const size_t o = (size_t)m * npairs + p[i];
        x[i] = v ? pv.x[p[i]] : T(0);
        y2[i] = v ? pv.pmm[o] : T(0);
        k[i] = v ? pv.pmmk[o] : 0;
        y1[i] = T(0);
    }
    // accumulators [pair][field][8 complex]: A_e A_o B_e B_o C_e C_o D_e D_o
    //   A: S dP, B: T P, C: S P, D: T dP; e/o = even/odd function of x
    T acc[LPT][BC][16];
#pragma unroll
    for (int i = 0; i < LPT; ++i)
#pragma unroll
        for (int b = 0; b < BC; ++b)
#pragma unroll
            for (int q = 0; q < 16; ++q) acc[i][b][q] = T(0);

    const T2 *S2 = reinterpret_cast<const T2 *>(Sg);
    const T2 *T2p = reinterpret_cast<const T2 *>(Tg);
    const T cadj = (op == OP_ANALYS_ADJ && m > 0) ? T(0.5) : T(1);

    for (int n0 = 0; n0 < L; n0 += NCH) {
        const int cnt = min(NCH, L - n0);
        __syncthreads();
        for (int t = threadIdx.x; t < NCH; t += NT) {
            T2 ab;
            ab.x = T(0); ab.y = T(0);
            T dcv = T(0);
            if (t < cnt) { ab = pv.ab[col + n0 + t]; dcv = pv.dc[col + n0 + t]; }
            s_ab[t] = ab;
            s_dc[t] = dcv;
            const int n = m * pv.mres + n0 + t;
            // adjoint of analysis: b / (c_m n(n+1)), nothing at n = 0
            T sc = T(1);
            if (op == OP_ANALYS_ADJ) sc = (n == 0) ? T(0) : cadj / (T(n) * T(n + 1));
#pragma unroll
            for (int b = 0; b < BC; ++b) {
                T2 fs, ft;
                fs.x = fs.y = ft.x = ft.y = T(0);
                if (t < cnt && b0 + b < batch) {
                    fs = S2[(size_t)(b0 + b) * pv.nlm + col + n0 + t];
                    ft = T2p[(size_t)(b0 + b) * pv.nlm + col + n0 + t];
                    fs.x *= sc; fs.y = (m == 0) ? T(0) : fs.y * sc;
                    ft.x *= sc; ft.y = (m == 0) ? T(0) : ft.y * sc;
                }
                s_S[t * BC + b] = fs;
                s_T[t * BC + b] = ft;
            }
        }
        __syncthreads();
        bool scaled = false;
        for (int t = 0; t < cnt; t += 2) {
            if (t % kSeedSeg == 0) {
                if constexpr (sizeof(T) == sizeof(float)) reseed<T, LPT>(pv, m, (n0 + t) / kSeedSeg, p, y1, y2, k);
                scaled = __any_sync(kFull, kmax_of<T, LPT>(k) > 0);
            }
#pragma unroll
            for (int par = 0; par < 2; ++par) {
                const int tt = t + par;
                const T2 ab = s_ab[tt];
                const T dcn = s_dc[tt];
                const T nf = T(m * pv.mres + n0 + tt);
                bool live = true;
                if (scaled) {
                    rec_step<T, LPT, true>(ab.x, ab.y, x, y1, y2, k, c);
                    live = __any_sync(kFull, kmin_of<T, LPT>(k) == 0);
                } else {
                    rec_step<T, LPT, false>(ab.x, ab.y, x, y1, y2, k, c);
                }
                if (!live) continue;
                T cd[LPT];
#pragma unroll
                for (int i = 0; i < LPT; ++i) {
                    // dP = n x P_n - dc_n P_{n-1}; zero whenever P itself is dropped
                    const T dpv = fma(nf * x[i], y1[i], -dcn * y2[i]);
                    cd[i] = (scaled && k[i] > 0) ? T(0) : dpv;
                }
#pragma unroll
                for (int b = 0; b < BC; ++b) {
                    const T2 fs = s_S[tt * BC + b];
                    const T2 ft = s_T[tt * BC + b];
#pragma unroll
                    for (int i = 0; i < LPT; ++i) {
                        // n-m even (par 0): P even, dP odd.  n-m odd: P odd, dP even.
                        const int iA = par == 0 ? 2 : 0;   // A_o : A_e
                        const int iB = par == 0 ? 4 : 6;   // B_e : B_o
                        const int iC = par == 0 ? 8 : 10;  // C_e : C_o
                        const int iD = par == 0 ? 14 : 12; // D_o : D_e
                        acc[i][b][iA] = fma(fs.x, cd[i], acc[i][b][iA]);
                        acc[i][b][iA + 1] = fma(fs.y, cd[i], acc[i][b][iA + 1]);
                        acc[i][b][iB] = fma(ft.x, c[i], acc[i][b][iB]);
                        acc[i][b][iB + 1] = fma(ft.y, c[i], acc[i][b][iB + 1]);
                        acc[i][b][iC] = fma(fs.x, c[i], acc[i][b][iC]);
                        acc[i][b][iC + 1] = fma(fs.y, c[i], acc[i][b][iC + 1]);
                        acc[i][b][iD] = fma(ft.x, cd[i], acc[i][b][iD]);
                        acc[i][b][iD + 1] = fma(ft.y, cd[i], acc[i][b][iD + 1]);
                    }
                }
            }
        }
    }

    T2 *eot2 = reinterpret_cast<T2 *>(eot);
    T2 *eop2 = reinterpret_cast<T2 *>(eop);
    const T fm = T(m * pv.mres);
#pragma unroll
    for (int i = 0; i < LPT; ++i) {
        if (p[i] >= npairs) continue;
        const T is = T(1) / pv.st[p[i]];
#pragma unroll
        for (int b = 0; b < BC; ++b) {
            if (b0 + b >= batch) continue;
            const T *a = acc[i][b];
            const size_t o = (((size_t)(b0 + b) * (pv.mmax + 1) + m) * npairs + p[i]) * 2;
            T2 v;
            // theta: (A - i m B) / sin ; E uses A_e,B_e ; O uses A_o,B_o
            v.x = (a[0] + fm * a[5]) * is; v.y = (a[1] - fm * a[4]) * is; eot2[o] = v;
            v.x = (a[2] + fm * a[7]) * is; v.y = (a[3] - fm * a[6]) * is; eot2[o + 1] = v;
            // phi: (i m C + D) / sin ; E uses C_e,D_e ; O uses C_o,D_o
            v.x = (a[12] - fm * a[9]) * is; v.y = (a[13] + fm * a[8]) * is; eop2[o] = v;
            v.x = (a[14] - fm * a[11]) * is; v.y = (a[15] + fm * a[10]) * is; eop2[o + 1] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Vector analysis.  With folds s/d of (w/sin) V_theta and V_phi:
//   S_n = sum [dP * fold(V_theta) - i m P * fold(V_phi)] / (n(n+1))
//   T_n = sum [i m P * fold(V_theta) + dP * fold(V_phi)] / (n(n+1))
// where the fold is s for an even function and d for an odd one.
// ---------------------------------------------------------------------------
template <typename T, int LPT, int BC>
__global__ void __launch_bounds__(256)
k_analys_vec(PlanView<T> pv, const T *__restrict__ sdt, const T *__restrict__ sdp, T *__restrict__ So,
             T *__restrict__ To, int batch, int op)
{
    using T2 = typename Vec2<T>::type;
    constexpr int K = 4 / BC;    // degrees per reduction: 8*K*BC = 32 values
    constexpr int NCH = 64;      // multiple of K
    static_assert(K % 2 == 0, "K must be even so that kx carries the parity of n - m");
    __shared__ T2 s_ab[NCH];
    __shared__ T s_dc[NCH];
    __shared__ T s_red[8][32];

    const int NT = blockDim.x;
    const int nw = NT >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = blockIdx.x;
    const int b0 = blockIdx.y * BC;
    const int lmax = pv.lmax, npairs = pv.npairs;
    const int L = lmax - m * pv.mres + 1;   // order index m is the order m mres
    const long col = col_of_mres(lmax, m, pv.mres);

    T x[LPT], y1[LPT], y2[LPT], c[LPT];
    int k[LPT], p[LPT];
    T2 st_[LPT][BC], dt_[LPT][BC], sp_[LPT][BC], dp_[LPT][BC];
    const T2 *sdt2 = reinterpret_cast<const T2 *>(sdt);
    const T2 *sdp2 = reinterpret_cast<const T2 *>(sdp);
#pragma unroll
    for (int i = 0; i < LPT; ++i) {
        p[i] = i * NT + threadIdx.x;
        const bool v = p[i] < npairs;
        const size_t o = (size_t)m * npairs + p[i];
        x[i] = v ? pv.x[p[i]] : T(0);
        y2[i] = v ? pv.pmm[o] : T(0);
        k[i] = v ? pv.pmmk[o] : 0;
        y1[i] = T(0);
#pragma unroll
        for (int b = 0; b < BC; ++b) {
            T2 z;
            z.x = T(0); z.y = T(0);
            st_[i][b] = dt_[i][b] = sp_[i][b] = dp_[i][b] = z;
            if (v && b0 + b < batch) {
                const size_t q = (((size_t)(b0 + b) * (pv.mmax + 1) + m) * npairs + p[i]) * 2;
                st_[i][b] = sdt2[q];
                dt_[i][b] = sdt2[q + 1];
                sp_[i][b] = sdp2[q];
                dp_[i][b] = sdp2[q + 1];
            }
        }
    }
    const T fm = T(m * pv.mres);
    T2 *S2 = reinterpret_cast<T2 *>(So);
    T2 *T2o = reinterpret_cast<T2 *>(To);

    for (int n0 = 0; n0 < L; n0 += NCH) {
        const int cnt = min(NCH, L - n0);
        __syncthreads();
        for (int t = threadIdx.x; t < NCH; t += NT) {
            T2 ab;
            ab.x = T(0); ab.y = T(0);
            T dcv = T(0);
            if (t < cnt) { ab = pv.ab[col + n0 + t]; dcv = pv.dc[col + n0 + t]; }
            s_ab[t] = ab;
            s_dc[t] = dcv;
        }
        __syncthreads();
        for (int t0 = 0; t0 < cnt; t0 += K) {
            if (sizeof(T) == sizeof(float) && (n0 + t0) % kSeedSeg == 0)
                reseed<T, LPT>(pv, m, (n0 + t0) / kSeedSeg, p, y1, y2, k);
            // per (kx, b): SA(2) SB(2) TA(2) TB(2)
            T acc[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) acc[q] = T(0);
            const bool scaled = __any_sync(kFull, kmax_of<T, LPT>(k) > 0);
#pragma unroll
            for (int kx = 0; kx < K; ++kx) {
                const T2 ab = s_ab[t0 + kx];
                const T dcn = s_dc[t0 + kx];
                const T nf = T(m * pv.mres + n0 + t0 + kx);
                bool live = true;
                if (scaled) {
                    rec_step<T, LPT, true>(ab.x, ab.y, x, y1, y2, k, c);
                    live = __any_sync(kFull, kmin_of<T, LPT>(k) == 0);
                } else {
                    rec_step<T, LPT, false>(ab.x, ab.y, x, y1, y2, k, c);
                }
                if (!live) continue;
#pragma unroll
                for (int i = 0; i < LPT; ++i) {
                    const T dpv = fma(nf * x[i], y1[i], -dcn * y2[i]);
                    const T cd = (scaled && k[i] > 0) ? T(0) : dpv;
#pragma unroll
                    for (int b = 0; b < BC; ++b) {
                        // n-m even (kx even): P even -> s folds; dP odd -> d folds
                        const T2 vt_dP = (kx & 1) ? st_[i][b] : dt_[i][b];
                        const T2 vp_P = (kx & 1) ? dp_[i][b] : sp_[i][b];
                        const T2 vt_P = (kx & 1) ? dt_[i][b] : st_[i][b];
                        const T2 vp_dP = (kx & 1) ? sp_[i][b] : dp_[i][b];
                        T *a = &acc[(kx * BC + b) * 8];
                        a[0] = fma(cd, vt_dP.x, a[0]);
                        a[1] = fma(cd, vt_dP.y, a[1]);
                        a[2] = fma(c[i], vp_P.x, a[2]);
                        a[3] = fma(c[i], vp_P.y, a[3]);
                        a[4] = fma(c[i], vt_P.x, a[4]);
                        a[5] = fma(c[i], vt_P.y, a[5]);
                        a[6] = fma(cd, vp_dP.x, a[6]);
                        a[7] = fma(cd, vp_dP.y, a[7]);
                    }
                }
            }
            warp_transpose_reduce<T, 32>(acc, lane);
            s_red[warp][lane] = acc[0];
            __syncthreads();
            if (threadIdx.x < K * BC) {
                T tot[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) tot[q] = T(0);
                for (int w = 0; w < nw; ++w)
#pragma unroll
                    for (int q = 0; q < 8; ++q) tot[q] += s_red[w][threadIdx.x * 8 + q];
                const int kx = threadIdx.x / BC, b = threadIdx.x % BC;
                const int nn = n0 + t0 + kx;
                const int n = m * pv.mres + nn;
                if (nn < L && b0 + b < batch) {
                    T sc;
                    if (op == OP_SYNTH_ADJ) sc = (m > 0) ? T(2) : T(1);
                    else sc = (n == 0) ? T(0) : T(1) / (T(n) * T(n + 1));
                    T2 sv, tv;
                    // S = SA - i m SB ; T = i m TA + TB
                    sv.x = sc * (tot[0] + fm * tot[3]);
                    sv.y = sc * (tot[1] - fm * tot[2]);
                    tv.x = sc * (tot[6] - fm * tot[5]);
                    tv.y = sc * (tot[7] + fm * tot[4]);
                    if (m == 0) { sv.y = T(0); tv.y = T(0); }
                    S2[(size_t)(b0 + b) * pv.nlm + col + nn] = sv;
                    T2o[(size_t)(b0 + b) * pv.nlm + col + nn] = tv;
                }
            }
            __syncthreads();
        }
    }
}

// Field chunk per CTA for a batch.
inline int pick_bc(int batch) { return batch >= 4 ? 4 : (batch >= 2 ? 2 : 1); }

template <typename T, int LPT, int BC>
cudaError_t synth_go(const PlanView<T> &pv, const T *spec, T *eo, int batch, Op op, cudaStream_t s)
{
    constexpr int NT = 128;
    const int npb = (pv.npairs + NT * LPT - 1) / (NT * LPT);
    dim3 grid((unsigned)((pv.mmax + 1) * npb), (unsigned)((batch + BC - 1) / BC));
    k_synth<T, LPT, BC, NT><<<grid, NT, 0, s>>>(pv, spec, eo, batch, npb, (int)op);
    return cudaGetLastError();
}

// Analysis CTAs hold every latitude pair of one order: nw warps of LPT pairs per thread.
inline int analys_warps(int npairs, int lpt) { int nw = (npairs + 32 * lpt - 1) / (32 * lpt); return nw < 1 ? 1 : nw; }

template <typename T, int LPT, int BC>
cudaError_t analys_go(const PlanView<T> &pv, const T *sd, T *spec, int batch, Op op, cudaStream_t s)
{
    const int nw = analys_warps(pv.npairs, LPT);
    if (nw > 8) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)(pv.mmax + 1), (unsigned)((batch + BC - 1) / BC));
    k_analys<T, LPT, BC><<<grid, nw * 32, 0, s>>>(pv, sd, spec, batch, (int)op);
    return cudaGetLastError();
}

// Pairs per lane of the segment analysis kernel (0: too many pairs for one warp).
inline int seg_ppl(int npairs) { return npairs <= 128 ? 4 : (npairs <= 256 ? 8 : (npairs <= 512 ? 16 : 0)); }

// FP64 analysis with 512 < npairs <= 2048: teams of 2 or 4 warps of 16 pairs per lane.
template <int TEAM, int BC>
cudaError_t analys_team_go(const PlanView<double> &pv, const double *sd, double *spec, int batch, Op op,
                           cudaStream_t s)
{
    const size_t smem = sizeof(double2) * BC * 2 * 32 * 16 * TEAM;
    cudaError_t e = cudaFuncSetAttribute(k_analys_seg_team<double, 16, BC, TEAM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(pv.mmax + 1), (unsigned)((batch + BC - 1) / BC));
    k_analys_seg_team<double, 16, BC, TEAM><<<grid, kSegWarps * 32, smem, s>>>(pv, sd, spec, batch, (int)op);
    return cudaGetLastError();
}

template <typename T, int PPL, int BC>
cudaError_t analys_seg_go(const PlanView<T> &pv, const T *sd, T *spec, int batch, Op op, cudaStream_t s)
{
    using T2 = typename Vec2<T>::type;
    const size_t smem = sizeof(T2) * BC * 2 * 32 * PPL;
    cudaError_t e = cudaFuncSetAttribute(k_analys_seg<T, PPL, BC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(pv.mmax + 1), (unsigned)((batch + BC - 1) / BC));
    k_analys_seg<T, PPL, BC><<<grid, kSegWarps * 32, smem, s>>>(pv, sd, spec, batch, (int)op);
    return cudaGetLastError();
}

template <typename T, int LPT, int BC>
cudaError_t synth_vec_go(const PlanView<T> &pv, const T *S, const T *Tc, T *eot, T *eop, int batch, Op op,
                         cudaStream_t s)
{
    constexpr int NT = 128;
    const int npb = (pv.npairs + NT * LPT - 1) / (NT * LPT);
    dim3 grid((unsigned)((pv.mmax + 1) * npb), (unsigned)((batch + BC - 1) / BC));
    k_synth_vec<T, LPT, BC, NT><<<grid, NT, 0, s>>>(pv, S, Tc, eot, eop, batch, npb, (int)op);
    return cudaGetLastError();
}

template <typename T, int LPT, int BC>
cudaError_t analys_vec_go(const PlanView<T> &pv, const T *sdt, const T *sdp, T *S, T *Tc, int batch, Op op,
                          cudaStream_t s)
{
    const int nw = analys_warps(pv.npairs, LPT);
    if (nw > 8) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)(pv.mmax + 1), (unsigned)((batch + BC - 1) / BC));
    k_analys_vec<T, LPT, BC><<<grid, nw * 32, 0, s>>>(pv, sdt, sdp, S, Tc, batch, (int)op);
    return cudaGetLastError();
}

// Pairs per thread for analysis: the cross-lane reduction costs ~1/LPT of the
// sums, so use 4 pairs per thread once there are enough pairs, 8 beyond 1024
// (at most 8 warps per CTA).
inline int analys_lpt(int npairs) { return npairs <= 64 ? 2 : (npairs <= 1024 ? 4 : 8); }

}  // namespace

template <typename T>
cudaError_t launch_legendre_synth_cfg(const PlanView<T> &pv, const T *spec, T *eo, int batch, Op op, int lpt, int bc,
                                      cudaStream_t s)
{
    if (!seeds_ok(pv, true)) return cudaErrorInvalidValue;
    // default shape: 2 pairs per thread, up to 4 fields per CTA (FP64: 1 pair
    // per thread, 8 fields, sharing each recurrence step among more sums)
    if (lpt <= 0) lpt = (sizeof(T) == sizeof(double) && batch >= 8) ? 1 : 2;
    if (bc <= 0) bc = (sizeof(T) == sizeof(double) && batch >= 8) ? 8 : pick_bc(batch);
#define SHT_SYN(L, B) if (lpt == L && bc == B) return synth_go<T, L, B>(pv, spec, eo, batch, op, s);
    SHT_SYN(1, 1) SHT_SYN(1, 2) SHT_SYN(1, 4)
    SHT_SYN(2, 1) SHT_SYN(2, 2) SHT_SYN(2, 4)
    SHT_SYN(4, 1) SHT_SYN(4, 2) SHT_SYN(4, 4)
#undef SHT_SYN
    if constexpr (sizeof(T) == sizeof(double)) {
        if (lpt == 1 && bc == 8) return synth_go<T, 1, 8>(pv, spec, eo, batch, op, s);
        if (lpt == 2 && bc == 8) return synth_go<T, 2, 8>(pv, spec, eo, batch, op, s);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_legendre_synth(const PlanView<T> &pv, const T *spec, T *eo, int batch, Op op, cudaStream_t s)
{
    return launch_legendre_synth_cfg<T>(pv, spec, eo, batch, op, 0, 0, s);
}

template <typename T>
cudaError_t launch_legendre_analys_cfg(const PlanView<T> &pv, const T *sd, T *spec, int batch, Op op, int lpt, int bc,
                                       cudaStream_t s)
{
    if (!seeds_ok(pv, true)) return cudaErrorInvalidValue;
    // default shape: FP64 up to 512 pairs, the segment kernel with up to 8
    // fields per CTA; otherwise LPT from the pair count (<= 8 warps), 2 fields
    // per CTA when batched
    if (lpt <= 0)
        lpt = (sizeof(T) == sizeof(double) && pv.npairs <= 2048) ? kAnalysSeg : analys_lpt(pv.npairs);
    if (lpt == kAnalysSeg) {
        if (sizeof(T) != sizeof(double)) return cudaErrorInvalidValue;
        const int ppl = seg_ppl(pv.npairs);
        if constexpr (sizeof(T) == sizeof(double)) {
            if (ppl == 0) {
                // teams: 2 warps and up to 4 fields per CTA, or 4 warps and 2 fields
                // (128 KB of staged folds either way)
                if (pv.npairs <= 1024) {
                    if (bc <= 0) bc = batch >= 4 ? 4 : (batch >= 2 ? 2 : 1);
                    if (bc == 4) return analys_team_go<2, 4>(pv, sd, spec, batch, op, s);
                    if (bc == 2) return analys_team_go<2, 2>(pv, sd, spec, batch, op, s);
                    if (bc == 1) return analys_team_go<2, 1>(pv, sd, spec, batch, op, s);
                } else if (pv.npairs <= 2048) {
                    if (bc <= 0) bc = batch >= 2 ? 2 : 1;
                    if (bc == 2) return analys_team_go<4, 2>(pv, sd, spec, batch, op, s);
                    if (bc == 1) return analys_team_go<4, 1>(pv, sd, spec, batch, op, s);
                }
                return cudaErrorInvalidValue;
            }
        }
        if (bc <= 0) bc = batch >= 8 ? 8 : (batch >= 4 ? 4 : (batch >= 2 ? 2 : 1));
        if constexpr (sizeof(T) == sizeof(double)) {
#define SHT_SEG(P, B) if (ppl == P && bc == B) return analys_seg_go<T, P, B>(pv, sd, spec, batch, op, s);
            SHT_SEG(4, 1) SHT_SEG(4, 2) SHT_SEG(4, 4) SHT_SEG(4, 8)
            SHT_SEG(8, 1) SHT_SEG(8, 2) SHT_SEG(8, 4) SHT_SEG(8, 8)
            SHT_SEG(16, 1) SHT_SEG(16, 2) SHT_SEG(16, 4) SHT_SEG(16, 8)
#undef SHT_SEG
        }
        return cudaErrorInvalidValue;
    }
    if (bc <= 0) bc = batch >= 2 ? 2 : 1;
    if (analys_warps(pv.npairs, lpt) > 8) return cudaErrorInvalidValue;
#define SHT_ANA(L, B) if (lpt == L && bc == B) return analys_go<T, L, B>(pv, sd, spec, batch, op, s);
    SHT_ANA(2, 1) SHT_ANA(2, 2) SHT_ANA(4, 1) SHT_ANA(4, 2) SHT_ANA(8, 1) SHT_ANA(8, 2)
#undef SHT_ANA
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_legendre_analys(const PlanView<T> &pv, const T *sd, T *spec, int batch, Op op, cudaStream_t s)
{
    return launch_legendre_analys_cfg<T>(pv, sd, spec, batch, op, 0, 0, s);
}

template <typename T>
cudaError_t launch_legendre_synth_vec(const PlanView<T> &pv, const T *S, const T *Tc, T *eot, T *eop, int batch,
                                      Op op, cudaStream_t s)
{
    if (!seeds_ok(pv, false)) return cudaErrorInvalidValue;
    if (batch >= 2) return synth_vec_go<T, 1, 2>(pv, S, Tc, eot, eop, batch, op, s);
    return synth_vec_go<T, 1, 1>(pv, S, Tc, eot, eop, batch, op, s);
}

template <typename T>
cudaError_t launch_legendre_analys_vec(const PlanView<T> &pv, const T *sdt, const T *sdp, T *S, T *Tc, int batch,
                                       Op op, cudaStream_t s)
{
    if (!seeds_ok(pv, false)) return cudaErrorInvalidValue;
    switch (analys_lpt(pv.npairs)) {
    case 2: return analys_vec_go<T, 2, 1>(pv, sdt, sdp, S, Tc, batch, op, s);
    case 4: return analys_vec_go<T, 4, 1>(pv, sdt, sdp, S, Tc, batch, op, s);
    default: return analys_vec_go<T, 8, 1>(pv, sdt, sdp, S, Tc, batch, op, s);
    }
}

// ---------------------------------------------------------------------------
// Persistent kernels for uneven batches (FP32, one field per tile).
// ---------------------------------------------------------------------------
namespace {

__global__ void __launch_bounds__(128) k_batch_synth(const BatchField *__restrict__ fields,
                                                     const int4 *__restrict__ tiles, int ntiles, int *counter)
{
    __shared__ float2 s_ab[kSynthNch];
    __shared__ float2 s_f[kSynthNch];
    __shared__ int s_tile, s_first;
    for (;;) {
        __syncthreads();  // the previous tile is done with the shared buffers
        if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1);
        __syncthreads();
        const int t = s_tile;
        if (t >= ntiles) break;
        const int4 tl = tiles[t];
        const BatchField f = fields[tl.x];
        synth_tile<float, 2, 1, 128>(f.pv, f.in, f.inter, 1, tl.y, tl.z, 0, OP_SYNTH, s_ab, s_f, &s_first);
    }
}

__global__ void __launch_bounds__(256) k_batch_analys(const BatchField *__restrict__ fields,
                                                      const int4 *__restrict__ tiles, int ntiles, int *counter)
{
    __shared__ float2 s_ab[kAnalysNch];
    __shared__ float s_red[8][32];
    __shared__ int s_tile;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1);
        __syncthreads();
        const int t = s_tile;
        if (t >= ntiles) break;
        const int4 tl = tiles[t];
        const BatchField f = fields[tl.x];
        analys_tile<float, 2, 1>(f.pv, f.inter, f.out, 1, tl.y, 0, OP_ANALYS, s_ab, s_red);
    }
}

}  // namespace

cudaError_t launch_batch_legendre(bool synth, const BatchField *fields, const int4 *tiles, int ntiles, int *counter,
                                  int ctas, cudaStream_t s)
{
    if (synth) k_batch_synth<<<ctas, 128, 0, s>>>(fields, tiles, ntiles, counter);
    else k_batch_analys<<<ctas, 256, 0, s>>>(fields, tiles, ntiles, counter);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Restart states of the recurrence and the first-live table of the static
// polar optimisation.  One thread per (order index m, pair): the FP64
// recurrence of Sec. 3.2 from P_m^m, carried as y 2^(-240 k) (Sec. 3.5).  At
// the start of every kSeedSeg-degree segment the state (y1, y2) =
// (P_{n0-1}, P_{n0-2}) is stored, either as it is with k (FP64 plans) or
// rewritten in the FP32 form y' 2^(-64 k'): k' = 0 when the larger of the two
// is at least 2^-63, else the k' that brings it into [2^-65, 1) -- the form in
// which the FP32 kernels carry it.  live[m][pair] is the first segment that
// holds a degree with |P_n^m| >= thr (all segments live when thr <= 0; the
// segment count when none is).
// ---------------------------------------------------------------------------
namespace {

__device__ float4 fp32_state(double y1, double y2, int k)
{
    const double mx = fmax(fabs(y1), fabs(y2));
    if (mx == 0.0) return make_float4(0.f, 0.f, __int_as_float(0), 0.f);
    int ex = 0;
    frexp(mx, &ex);
    const long E = (long)ex - (long)Scale<double>::S * k;   // the larger value < 2^E
    constexpr int S32 = Scale<float>::S;
    long k32 = 0;
    if (E < 1 - S32) k32 = (-E) / S32;
    const int sh = (int)(-(long)Scale<double>::S * k + (long)S32 * k32);
    return make_float4((float)scalbn(y1, sh), (float)scalbn(y2, sh), __int_as_float((int)k32), 0.f);
}

__global__ void __launch_bounds__(128)
k_build_restarts(PlanView<double> pv, const unsigned long long *__restrict__ segoff, float4 *__restrict__ seeds32,
                 double2 *__restrict__ seeds64, int *__restrict__ seeds64k, unsigned short *__restrict__ live,
                 double thr)
{
    const int m = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int npairs = pv.npairs;
    if (p >= npairs) return;
    const int L = pv.lmax - m * pv.mres + 1;
    const int nseg = (L + kSeedSeg - 1) / kSeedSeg;
    const long col = col_of_mres(pv.lmax, m, pv.mres);
    const double x = pv.x[p];
    double y1 = 0.0, y2 = pv.pmm[(size_t)m * npairs + p];
    int k = pv.pmmk[(size_t)m * npairs + p];
    int first = thr > 0.0 ? nseg : 0;
    for (int s = 0; s < nseg; ++s) {
        const size_t o = (segoff[m] + s) * npairs + p;
        if (seeds32) seeds32[o] = fp32_state(y1, y2, k);
        if (seeds64) {
            seeds64[o] = make_double2(y1, y2);
            seeds64k[o] = k;
        }
        for (int i = 0; i < kSeedSeg; ++i) {
            const int nn = kSeedSeg * s + i;
            if (nn >= L) break;
            const double2 ab = pv.ab[col + nn];
            const double yn = fma(ab.x * x, y1, ab.y * y2);
            y2 = y1;
            y1 = yn;
            if (k > 0 && fabs(yn) >= 1.0) {
                y1 *= down_scale<double>();
                y2 *= down_scale<double>();
                k -= 1;
            }
            if (k == 0 && fabs(y1) >= thr && s < first) first = s;
        }
    }
    live[(size_t)m * npairs + p] = (unsigned short)first;
}

}  // namespace

cudaError_t launch_build_restarts(const PlanView<double> &pv, const unsigned long long *segoff, float4 *seeds32,
                                  double2 *seeds64, int *seeds64k, unsigned short *live, double thr, cudaStream_t st)
{
    dim3 grid((unsigned)((pv.npairs + 127) / 128), (unsigned)(pv.mmax + 1));
    k_build_restarts<<<grid, 128, 0, st>>>(pv, segoff, seeds32, seeds64, seeds64k, live, thr);
    return cudaGetLastError();
}

template cudaError_t launch_legendre_synth_cfg<double>(const PlanView<double> &, const double *, double *, int, Op,
                                                       int, int, cudaStream_t);
template cudaError_t launch_legendre_synth_cfg<float>(const PlanView<float> &, const float *, float *, int, Op, int,
                                                      int, cudaStream_t);
template cudaError_t launch_legendre_analys_cfg<double>(const PlanView<double> &, const double *, double *, int, Op,
                                                        int, int, cudaStream_t);
template cudaError_t launch_legendre_analys_cfg<float>(const PlanView<float> &, const float *, float *, int, Op, int,
                                                       int, cudaStream_t);
template cudaError_t launch_legendre_synth<double>(const PlanView<double> &, const double *, double *, int, Op,
                                                   cudaStream_t);
template cudaError_t launch_legendre_synth<float>(const PlanView<float> &, const float *, float *, int, Op,
                                                  cudaStream_t);
template cudaError_t launch_legendre_analys<double>(const PlanView<double> &, const double *, double *, int, Op,
                                                    cudaStream_t);
template cudaError_t launch_legendre_analys<float>(const PlanView<float> &, const float *, float *, int, Op,
                                                   cudaStream_t);
template cudaError_t launch_legendre_synth_vec<double>(const PlanView<double> &, const double *, const double *,
                                                       double *, double *, int, Op, cudaStream_t);
template cudaError_t launch_legendre_synth_vec<float>(const PlanView<float> &, const float *, const float *, float *,
                                                      float *, int, Op, cudaStream_t);
template cudaError_t launch_legendre_analys_vec<double>(const PlanView<double> &, const double *, const double *,
                                                        double *, double *, int, Op, cudaStream_t);
template cudaError_t launch_legendre_analys_vec<float>(const PlanView<float> &, const float *, const float *, float *,
                                                       float *, int, Op, cudaStream_t);

}  // namespace sht
