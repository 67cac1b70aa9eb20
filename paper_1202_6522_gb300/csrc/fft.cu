// fft.cu -- the longitude stage of the SHT: batched real FFTs of length nphi
// (a power of two) over latitude rows, done in shared memory (Sec. 3.1: the
// longitude sum is a Fourier transform; real data use the Hermitian half).
//
// A CTA owns G latitude pairs of one field, i.e. the rows j and nlat-1-j of
// each pair, so the north/south mirror fold of Sec. 3.1 happens here:
//   synthesis: X_north = E + O, X_south = E - O from the Legendre stage, then
//              f_k = sum_m c_m Re(X_m e^{2 pi i m k / nphi})   (c2r);
//   analysis:  X_m = (2 pi / nphi) sum_k f_k e^{-2 pi i m k / nphi} (r2c), then
//              s = w (X_north + X_south), d = w (X_north - X_south).
// A real transform of length N = 2H is one complex transform of length H on
// z_n = f_{2n} + i f_{2n+1} plus a pre/post twiddle.  The complex transform is
// a sequence of Stockham (self-sorting) passes: each thread holds 16 values
// in registers, runs a radix-16 (or 2/4/8 for the remainder) DFT on them and
// writes them back permuted, so no bit reversal is needed.  The first r2c
// pass reads the grid straight from global memory and the last c2r pass
// writes it straight back; rows in shared memory are padded (one slot every
// 16) to spread the strided accesses over the banks.
#include <cuda_runtime.h>

#include "sht_internal.h"

namespace sht {
namespace {

constexpr double kTwoPiD = 6.283185307179586476925286766559;

template <typename T2> __device__ __forceinline__ T2 mk(decltype(T2::x) a, decltype(T2::x) b) { T2 r; r.x = a; r.y = b; return r; }
template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { return mk<T2>(a.x + b.x, a.y + b.y); }
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { return mk<T2>(a.x - b.x, a.y - b.y); }
template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b)
{
    return mk<T2>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T2> __device__ __forceinline__ T2 conj_(T2 a) { a.y = -a.y; return a; }
template <typename T2> __device__ __forceinline__ T2 mul_i(T2 a) { return mk<T2>(-a.y, a.x); }

__device__ __forceinline__ int padi(int i) { return i + (i >> 4); }

// Double-float numbers (used by the FFTs of the FP64-accurate tensor-core
// mode, further down): the unevaluated sum hi + lo of two FP32 numbers, after
// Dekker's double-length arithmetic (1971); normalised (|lo| <= ulp(hi) / 2)
// on the way in and out, possibly not in between (see operator+).
struct __align__(8) dfl {
    float hi, lo;
    dfl() = default;
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ explicit constexpr dfl(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};
struct __align__(16) dfl2 { dfl x, y; };

// s + e = a + b exactly for any a, b (Knuth)
__device__ __forceinline__ dfl two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return dfl(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
// The operations leave the pair unnormalised: the error-free sum or product
// of the high parts and the low-order terms added in FP32, without the final
// renormalisation, so |lo| can grow to a few units in the last place of hi
// (or exceed hi after a cancellation).  Each result still equals the exact
// one up to FP32 rounding of the low-order terms, an error of a few 2^-48
// times the magnitude of the operands -- the per-operation bound the
// normwise error analysis of an FFT rests on -- and the operations take the
// low part of their inputs at full weight, so they accept such pairs.
__device__ __forceinline__ dfl operator+(dfl x, dfl y)
{
    // Knuth's error-free sum of the high parts, then the low parts
    const dfl s = two_sum(x.hi, y.hi);
    return dfl(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dfl operator-(dfl x) { return dfl(-x.hi, -x.lo); }
__device__ __forceinline__ dfl operator-(dfl x, dfl y) { return x + (-y); }
__device__ __forceinline__ dfl operator*(dfl x, dfl y)
{
    // exact error of hi * hi by an FMA; the lo * lo term is below the result's precision
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return dfl(p, e);
}
// Complex product in double-float with each component formed as one sum:
// re = xr wr - xi wi from the two exact high products (FMA errors), one
// error-free sum of them and the cross terms accumulated into the low part.
__device__ __forceinline__ dfl dot2(dfl a, dfl b, dfl c, dfl d)   // a b + c d
{
    const float p1 = __fmul_rn(a.hi, b.hi), p2 = __fmul_rn(c.hi, d.hi);
    const float e1 = __fmaf_rn(a.hi, b.hi, -p1), e2 = __fmaf_rn(c.hi, d.hi, -p2);
    const dfl s = two_sum(p1, p2);
    float t = __fadd_rn(s.lo, __fadd_rn(e1, e2));
    t = __fmaf_rn(a.hi, b.lo, t);
    t = __fmaf_rn(a.lo, b.hi, t);
    t = __fmaf_rn(c.hi, d.lo, t);
    t = __fmaf_rn(c.lo, d.hi, t);
    return dfl(s.hi, t);
}
__device__ __forceinline__ dfl2 cmul(dfl2 a, dfl2 b)
{
    dfl2 r;
    r.x = dot2(a.x, b.x, -a.y, b.y);
    r.y = dot2(a.x, b.y, a.y, b.x);
    return r;
}
// x s for a power of two s (exact unless the low part leaves FP32's range)
__device__ __forceinline__ dfl scale2(dfl x, float s) { return dfl(x.hi * s, x.lo * s); }


// cos(pi j / 32), j = 0..16
__host__ __device__ constexpr double cospi32(int j)
{
    return j == 0 ? 1.0 : j == 1 ? 0.99518472667219688624 : j == 2 ? 0.98078528040323044913
         : j == 3 ? 0.95694033573220886494 : j == 4 ? 0.92387953251128675613 : j == 5 ? 0.88192126434835502971
         : j == 6 ? 0.83146961230254523708 : j == 7 ? 0.77301045336273696081 : j == 8 ? 0.70710678118654752440
         : j == 9 ? 0.63439328416364549822 : j == 10 ? 0.55557023301960222474 : j == 11 ? 0.47139673682599764856
         : j == 12 ? 0.38268343236508977173 : j == 13 ? 0.29028467725446236764 : j == 14 ? 0.19509032201612826785
         : j == 15 ? 0.09801714032956060199 : 0.0;
}
// cos and sin of 2 pi k / 64 for any integer k (cos(a) = cos(-a), cos(pi - a) = -cos(a))
__host__ __device__ constexpr double cos64_half(int k) { return k > 16 ? -cospi32(32 - k) : cospi32(k); }
__host__ __device__ constexpr double cos64(int k) { return cos64_half((k & 63) > 32 ? 64 - (k & 63) : (k & 63)); }
__host__ __device__ constexpr double sin64(int k) { return cos64(k - 16); }

// z e^{SIGN 2 pi i q / 64} for q < 32 (a constant once the DFT loops are
// unrolled).  In double-float the multiplications by +-i and by
// (+-1 + i) sqrt(1/2) are done as such (a general product costs four
// double-float products and two sums); other types keep the general form.
template <typename T2, int SIGN>
struct Tw64 {
    using T = decltype(T2::x);
    __device__ __forceinline__ static T2 mul(int q, T2 z)
    {
        // z (SIGN i): a swap and a sign (a general product by (0, +-1) keeps
        // its multiplications by zero, which IEEE arithmetic cannot drop)
        if (q == 16) return SIGN > 0 ? mk<T2>(-z.y, z.x) : mk<T2>(z.y, -z.x);
        return cmul(mk<T2>(T(cos64(q)), T(SIGN * sin64(q))), z);
    }
};
template <int SIGN>
struct Tw64<dfl2, SIGN> {
    __device__ __forceinline__ static dfl2 mul(int q, dfl2 z)
    {
        const dfl szr = SIGN > 0 ? z.x : -z.x, szi = SIGN > 0 ? z.y : -z.y;   // SIGN z
        if (q == 16) return mk<dfl2>(-szi, szr);
        const dfl c(0.70710678118654752440);
        if (q == 8) return mk<dfl2>(c * (z.x - szi), c * (szr + z.y));
        if (q == 24) return mk<dfl2>(c * (-z.x - szi), c * (szr - z.y));
        return cmul(mk<dfl2>(dfl(cos64(q)), dfl(SIGN * sin64(q))), z);
    }
};

// In-register DFT of size RD <= 64 (natural order in and out), split into
// even and odd halves recursively.  SIGN = +1: e^{+2 pi i ...} (inverse),
// -1: forward.
template <typename T2, int RD, int SIGN>
struct RegDft {
    using T = decltype(T2::x);
    __device__ __forceinline__ static void run(T2 (&v)[RD])
    {
        T2 e[RD / 2], o[RD / 2];
#pragma unroll
        for (int k = 0; k < RD / 2; ++k) { e[k] = v[2 * k]; o[k] = v[2 * k + 1]; }
        RegDft<T2, RD / 2, SIGN>::run(e);
        RegDft<T2, RD / 2, SIGN>::run(o);
#pragma unroll
        for (int k = 0; k < RD / 2; ++k) {
            const T2 t = (k == 0) ? o[k] : Tw64<T2, SIGN>::mul(k * (64 / RD), o[k]);
            v[k] = cadd(e[k], t);
            v[k + RD / 2] = csub(e[k], t);
        }
    }
};
template <typename T2, int SIGN>
struct RegDft<T2, 1, SIGN> {
    __device__ __forceinline__ static void run(T2 (&)[1]) {}
};
// Length 3 from the definition y_k = sum_r a_r w^(r k), w = e^(SIGN 2 pi i / 3):
// y_1,2 = a_0 - (a_1 + a_2) / 2 +- i SIGN (sqrt(3) / 2) (a_1 - a_2).
template <typename T2, int SIGN>
struct RegDft<T2, 3, SIGN> {
    using T = decltype(T2::x);
    __device__ __forceinline__ static void run(T2 (&a)[3])
    {
        const T s3 = T(SIGN * 0.86602540378443864676);
        const T2 t = cadd(a[1], a[2]), d = csub(a[1], a[2]);
        const T2 c = mk<T2>(a[0].x - T(0.5) * t.x, a[0].y - T(0.5) * t.y);
        const T2 id = mk<T2>(-s3 * d.y, s3 * d.x);   // i SIGN sqrt(3)/2 (a_1 - a_2)
        a[0] = cadd(a[0], t);
        a[1] = cadd(c, id);
        a[2] = csub(c, id);
    }
};
// Length 5 from the definition, with b_1 = a_1 + a_4, b_2 = a_2 + a_3,
// d_1 = a_1 - a_4, d_2 = a_2 - a_3, c_k = cos(2 pi k / 5), s_k = SIGN sin(2 pi k / 5):
// y_1,4 = a_0 + c_1 b_1 + c_2 b_2 +- i (s_1 d_1 + s_2 d_2),
// y_2,3 = a_0 + c_2 b_1 + c_1 b_2 +- i (s_2 d_1 - s_1 d_2).
template <typename T2, int SIGN>
struct RegDft<T2, 5, SIGN> {
    using T = decltype(T2::x);
    __device__ __forceinline__ static void run(T2 (&a)[5])
    {
        const T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);
        const T s1 = T(SIGN * 0.95105651629515357212), s2 = T(SIGN * 0.58778525229247312917);
        const T2 b1 = cadd(a[1], a[4]), b2 = cadd(a[2], a[3]);
        const T2 d1 = csub(a[1], a[4]), d2 = csub(a[2], a[3]);
        const T2 r1 = mk<T2>(a[0].x + c1 * b1.x + c2 * b2.x, a[0].y + c1 * b1.y + c2 * b2.y);
        const T2 r2 = mk<T2>(a[0].x + c2 * b1.x + c1 * b2.x, a[0].y + c2 * b1.y + c1 * b2.y);
        const T2 q1 = mk<T2>(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y);
        const T2 q2 = mk<T2>(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y);
        a[0] = cadd(a[0], cadd(b1, b2));
        a[1] = cadd(r1, mul_i(q1));
        a[4] = csub(r1, mul_i(q1));
        a[2] = cadd(r2, mul_i(q2));
        a[3] = csub(r2, mul_i(q2));
    }
};

// Registers per thread of a Stockham pass: ceil(16 / RD) items of RD values
// with TPR = ceil(H / 16) threads per row: 16 for power-of-two radices, 20
// once radix 3 or 5 passes occur (MIXED; compiled separately so that the
// power-of-two kernels keep their smaller register footprint).
template <bool MIXED> struct PassRegs { static constexpr int n = MIXED ? 20 : 16; };
__host__ __device__ inline int row_tpr(int H) { return (H + 15) / 16; }

// One Stockham pass of radix RD over a row of length H held in `row` (padded
// indices) or, for the first/last pass, in global memory.  Each thread owns
// up to ceil(16 / RD) items j = t + it * TPR; item j reads x[j + r H/RD],
// applies the twiddle W^(r (j mod Ns) H/(Ns RD)), runs the RD-point DFT and
// writes y[(j / Ns) Ns RD + j mod Ns + r Ns].
// log2 of a power of two
__device__ __forceinline__ int lg2(int v) { return __popc(v - 1); }

// P2: every length involved is a power of two, so the index arithmetic is
// masks and shifts (a division by a run-time value is a long instruction
// sequence on the integer pipe, which the FFT kernels are short of).
template <typename T2, int RD, int SIGN, int NR, bool P2>
__device__ __forceinline__ void stockham_load(const T2 *src, bool global_src, int t, int TPR, int H, int Ns,
                                              const T2 *__restrict__ wtab, T2 (&v)[NR])
{
    constexpr int IT = (16 + RD - 1) / RD;
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int j = t + it * TPR;
        if (j >= H / RD) break;
        T2 a[RD];
#pragma unroll
        for (int r = 0; r < RD; ++r) {
            const int idx = j + r * (H / RD);
            a[r] = global_src ? src[idx] : src[padi(idx)];
        }
        if (Ns > 1) {
            const int q0 = P2 ? (j & (Ns - 1)) << (lg2(H) - lg2(Ns) - lg2(RD)) : (j % Ns) * (H / (Ns * RD));
#pragma unroll
            for (int r = 1; r < RD; ++r) {
                T2 w = wtab[P2 ? (r * q0) & (H - 1) : (r * q0) % H];
                if (SIGN < 0) w = conj_(w);
                a[r] = cmul(a[r], w);
            }
        }
        RegDft<T2, RD, SIGN>::run(a);
#pragma unroll
        for (int r = 0; r < RD; ++r) v[it * RD + r] = a[r];
    }
}

template <typename T2, int RD, bool P2>
__device__ __forceinline__ int stockham_out(int j, int r, int Ns)
{
    if (P2) return ((j & ~(Ns - 1)) * RD) + (j & (Ns - 1)) + r * Ns;
    return (j / Ns) * Ns * RD + (j % Ns) + r * Ns;
}

template <typename T2, int RD, int NR, bool P2>
__device__ __forceinline__ void stockham_store_smem(T2 *row, int t, int TPR, int H, int Ns, const T2 (&v)[NR])
{
    constexpr int IT = (16 + RD - 1) / RD;
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int j = t + it * TPR;
        if (j >= H / RD) break;
#pragma unroll
        for (int r = 0; r < RD; ++r) row[padi(stockham_out<T2, RD, P2>(j, r, Ns))] = v[it * RD + r];
    }
}

// Runs a pass of the given radix (run-time selected).
template <typename T2, int SIGN, bool MIXED>
__device__ __forceinline__ void pass_load(int rd, const T2 *src, bool g, int t, int TPR, int H, int Ns,
                                          const T2 *wtab, T2 (&v)[PassRegs<MIXED>::n])
{
    constexpr int NR = PassRegs<MIXED>::n;
    constexpr bool P2 = !MIXED;
    if (MIXED && rd == 3) { stockham_load<T2, 3, SIGN, NR, P2>(src, g, t, TPR, H, Ns, wtab, v); return; }
    if (MIXED && rd == 5) { stockham_load<T2, 5, SIGN, NR, P2>(src, g, t, TPR, H, Ns, wtab, v); return; }
    switch (rd) {
    case 2: stockham_load<T2, 2, SIGN, NR, P2>(src, g, t, TPR, H, Ns, wtab, v); break;
    case 4: stockham_load<T2, 4, SIGN, NR, P2>(src, g, t, TPR, H, Ns, wtab, v); break;
    case 8: stockham_load<T2, 8, SIGN, NR, P2>(src, g, t, TPR, H, Ns, wtab, v); break;
    default: stockham_load<T2, 16, SIGN, NR, P2>(src, g, t, TPR, H, Ns, wtab, v); break;
    }
}

template <typename T2, bool MIXED>
__device__ __forceinline__ void pass_store(int rd, T2 *row, int t, int TPR, int H, int Ns,
                                           const T2 (&v)[PassRegs<MIXED>::n])
{
    constexpr int NR = PassRegs<MIXED>::n;
    constexpr bool P2 = !MIXED;
    if (MIXED && rd == 3) { stockham_store_smem<T2, 3, NR, P2>(row, t, TPR, H, Ns, v); return; }
    if (MIXED && rd == 5) { stockham_store_smem<T2, 5, NR, P2>(row, t, TPR, H, Ns, v); return; }
    switch (rd) {
    case 2: stockham_store_smem<T2, 2, NR, P2>(row, t, TPR, H, Ns, v); break;
    case 4: stockham_store_smem<T2, 4, NR, P2>(row, t, TPR, H, Ns, v); break;
    case 8: stockham_store_smem<T2, 8, NR, P2>(row, t, TPR, H, Ns, v); break;
    default: stockham_store_smem<T2, 16, NR, P2>(row, t, TPR, H, Ns, v); break;
    }
}

// Twiddle table W_H^q = e^{2 pi i q / H}, q < H, from the plan's e^{2 pi i k / nphi}.
template <typename T2>
__device__ __forceinline__ void fill_wtab(T2 *wtab, const T2 *__restrict__ tw, int H)
{
    for (int q = threadIdx.x; q < H; q += blockDim.x) {
        T2 w;
        if (2 * q < H) {
            w = tw[2 * q];
        } else {
            w = tw[2 * q - H];
            w.x = -w.x;
            w.y = -w.y;
        }
        wtab[q] = w;
    }
}

// Writes the last Stockham pass's outputs y[j + r H/RD] of a thread's items.
template <int RD, int NR, typename T2, typename F>
__device__ __forceinline__ void last_pass_out(const T2 (&v)[NR], int t, int TPR, int H, const F &put)
{
    constexpr int IT = (16 + RD - 1) / RD;
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int jj = t + it * TPR;
        if (jj >= H / RD) break;
#pragma unroll
        for (int rr = 0; rr < RD; ++rr) put(jj + rr * (H / RD), v[it * RD + rr]);
    }
}
template <bool MIXED, typename T2, typename F>
__device__ __forceinline__ void last_pass_out(int rd, const T2 (&v)[PassRegs<MIXED>::n], int t, int TPR, int H,
                                              const F &put)
{
    constexpr int NR = PassRegs<MIXED>::n;
    if (MIXED && rd == 3) { last_pass_out<3, NR>(v, t, TPR, H, put); return; }
    if (MIXED && rd == 5) { last_pass_out<5, NR>(v, t, TPR, H, put); return; }
    switch (rd) {
    case 2: last_pass_out<2, NR>(v, t, TPR, H, put); break;
    case 4: last_pass_out<4, NR>(v, t, TPR, H, put); break;
    case 8: last_pass_out<8, NR>(v, t, TPR, H, put); break;
    default: last_pass_out<16, NR>(v, t, TPR, H, put); break;
    }
}

// ---------------------------------------------------------------------------
// Synthesis: EO [batch][mmax+1][npairs][2] -> grid [batch][nlat][nphi]
// blockDim = R * TPR with TPR = max(1, H/16) threads per row, R = 2G rows.
// ---------------------------------------------------------------------------
// One tile (field b, pairs p0 .. p0+G-1) of the synthesis FFT, run by the
// whole CTA (blockDim.x >= 2 G max(1, H/16)); smem_raw holds the twiddle table
// and the 2G padded rows.
template <typename T, bool MIXED>
__device__ __forceinline__ void fft_synth_tile(const PlanView<T> &pv, const T *__restrict__ eo, T *__restrict__ grid,
                                               int b, int p0, int G, int op, unsigned char *smem_raw)
{
    using T2 = typename Vec2<T>::type;
    const int H = pv.nphi / 2, R = 2 * G;
    const int TPR = row_tpr(H);
    const int ld = padi(H) + 1;
    T2 *wtab = reinterpret_cast<T2 *>(smem_raw);
    T2 *buf = wtab + H;
    const int mmax = pv.mmax, npairs = pv.npairs, nlat = pv.nlat;
    const T2 *eo2 = reinterpret_cast<const T2 *>(eo);

    fill_wtab(wtab, pv.tw, H);
    // 1. spectra of the 2G rows, natural order, zero padded above mmax
    for (int q = threadIdx.x; q < G * H; q += blockDim.x) {
        const int m = q / G, i = q - m * G;
        const int p = p0 + i;
        T2 XN = mk<T2>(T(0), T(0)), XS = XN;
        if (m <= mmax && p < npairs) {
            const size_t o = (((size_t)b * (mmax + 1) + m) * npairs + p) * 2;
            const T2 E = eo2[o], O = eo2[o + 1];
            XN = cadd(E, O);
            XS = csub(E, O);
            if (m == 0) { XN.y = T(0); XS.y = T(0); }
        }
        buf[(2 * i) * ld + padi(m)] = XN;
        buf[(2 * i + 1) * ld + padi(m)] = XS;
    }
    __syncthreads();
    // 2. pre-twiddle: Z_k = (X_k + conj X_{H-k}) + i W^k (X_k - conj X_{H-k}), X_H = 0
    for (int q = threadIdx.x; q < R * (H / 2 + 1); q += blockDim.x) {
        const int r = q / (H / 2 + 1), k = q - r * (H / 2 + 1);
        T2 *row = buf + r * ld;
        if (k == 0) {
            const T2 X0 = row[0];
            row[0] = cadd(X0, mul_i(X0));
            continue;
        }
        const int k2 = H - k;
        const T2 Xa = row[padi(k)], Xb = row[padi(k2)];
        row[padi(k)] = cadd(cadd(Xa, conj_(Xb)), mul_i(cmul(pv.tw[k], csub(Xa, conj_(Xb)))));
        if (k2 != k) row[padi(k2)] = cadd(cadd(Xb, conj_(Xa)), mul_i(cmul(pv.tw[k2], csub(Xb, conj_(Xa)))));
    }
    __syncthreads();
    // 3. inverse complex FFT of length H by Stockham passes; the last one writes the grid
    const int r = threadIdx.x / TPR, t = threadIdx.x - r * TPR;
    const int p = p0 + (r >> 1);
    const int j = (r & 1) ? nlat - 1 - p : p;
    const bool live_row = r < R && p < npairs && !((r & 1) && j == p);
    T scale = T(1);
    if (op == OP_ANALYS_ADJ && p < npairs) scale = T(kTwoPiD) / T(pv.nphi) * pv.wq[p];
    T2 *row = buf + (r < R ? r : 0) * ld;
    T2 *out = reinterpret_cast<T2 *>(grid) + ((size_t)b * nlat + (live_row ? j : 0)) * H;
    if (H == 1) {
        if (threadIdx.x < R && live_row) {
            T2 z = row[0];
            z.x *= scale; z.y *= scale;
            out[0] = z;
        }
        return;
    }
    int Ns = 1;
    T2 v[PassRegs<MIXED>::n];
    for (int ps = 0;; ++ps) {
        const int rd = fft_plan_radix(pv.fftplan, ps);
        if (r < R) pass_load<T2, 1, MIXED>(rd, row, false, t, TPR, H, Ns, wtab, v);
        const bool last = Ns * rd == H;
        __syncthreads();
        if (last) {
            // last pass: y[j + r' H/RD] for item j -- contiguous over threads
            if (live_row)
                last_pass_out<MIXED>(rd, v, t, TPR, H, [&](int idx, T2 z) {
                    z.x *= scale; z.y *= scale;
                    out[idx] = z;
                });
            break;
        }
        if (r < R) pass_store<T2, MIXED>(rd, row, t, TPR, H, Ns, v);
        __syncthreads();
        Ns *= rd;
    }
}

template <typename T, bool MIXED>
__global__ void __launch_bounds__(512)
k_fft_synth(PlanView<T> pv, const T *__restrict__ eo, T *__restrict__ grid, int G, int op)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fft_synth_tile<T, MIXED>(pv, eo, grid, blockIdx.y, blockIdx.x * G, G, op, smem_raw);
}

// ---------------------------------------------------------------------------
// Analysis: grid [batch][nlat][nphi] -> SD [batch][mmax+1][npairs][2]
// ---------------------------------------------------------------------------
// One tile (field b, pairs p0 .. p0+G-1) of the analysis FFT (see fft_synth_tile).
template <typename T, bool MIXED>
__device__ __forceinline__ void fft_analys_tile(const PlanView<T> &pv, const T *__restrict__ grid, T *__restrict__ sd,
                                                int b, int p0, int G, int op, int vector, unsigned char *smem_raw)
{
    using T2 = typename Vec2<T>::type;
    const int H = pv.nphi / 2, R = 2 * G;
    const int TPR = row_tpr(H);
    const int ld = padi(H) + 1;
    T2 *wtab = reinterpret_cast<T2 *>(smem_raw);
    T2 *buf = wtab + H;
    const int mmax = pv.mmax, npairs = pv.npairs, nlat = pv.nlat;

    fill_wtab(wtab, pv.tw, H);
    __syncthreads();
    const int r = threadIdx.x / TPR, t = threadIdx.x - r * TPR;
    const int p = p0 + (r >> 1);
    const int j = (r & 1) ? nlat - 1 - p : p;
    const bool live_row = r < R && p < npairs && !((r & 1) && j == p);
    T2 *row = buf + (r < R ? r : 0) * ld;
    const T2 *in = reinterpret_cast<const T2 *>(grid) + ((size_t)b * nlat + (live_row ? j : 0)) * H;

    if (H == 1) {
        if (threadIdx.x < R) row[0] = live_row ? in[0] : mk<T2>(T(0), T(0));
    } else {
        // forward complex FFT of length H; the first pass reads the grid row
        int Ns = 1;
        T2 v[PassRegs<MIXED>::n];
        const int npass = fft_plan_npass(pv.fftplan);
        for (int ps = 0; ps < npass; ++ps) {
            const int rd = fft_plan_radix(pv.fftplan, ps);
            if (r < R) {
                if (ps == 0) {
                    if (live_row) {
                        pass_load<T2, -1, MIXED>(rd, in, true, t, TPR, H, Ns, wtab, v);
                    } else {
#pragma unroll
                        for (int q = 0; q < PassRegs<MIXED>::n; ++q) v[q] = mk<T2>(T(0), T(0));
                    }
                } else {
                    pass_load<T2, -1, MIXED>(rd, row, false, t, TPR, H, Ns, wtab, v);
                }
            }
            __syncthreads();
            if (r < R) pass_store<T2, MIXED>(rd, row, t, TPR, H, Ns, v);
            __syncthreads();
            Ns *= rd;
        }
    }
    __syncthreads();
    // post-twiddle, scale, fold north/south, weight
    T2 *sd2 = reinterpret_cast<T2 *>(sd);
    const T fscale = (op == OP_ANALYS) ? T(kTwoPiD) / T(pv.nphi) : T(1);
    for (int q = threadIdx.x; q < G * (mmax + 1); q += blockDim.x) {
        const int m = q / G, i = q - m * G;
        const int pp = p0 + i;
        if (pp >= npairs) continue;
        T2 X[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const T2 *rw = buf + (2 * i + h) * ld;
            const T2 Zk = rw[padi(m)];
            const T2 Zc = conj_(rw[padi(MIXED ? (H - m) % H : (H - m) & (H - 1))]);
            T2 E = cadd(Zk, Zc), O = csub(Zk, Zc);
            E.x *= T(0.5); E.y *= T(0.5);
            const T2 Od = mk<T2>(O.y * T(0.5), -O.x * T(0.5));  // O / (2i)
            X[h] = cadd(E, cmul(conj_(pv.tw[m]), Od));
        }
        T wf = fscale;
        if (op == OP_ANALYS) wf *= pv.wq[pp];
        if (vector) wf /= pv.st[pp];
        const bool equator = (nlat & 1) && pp == npairs - 1;
        T2 s, d;
        if (equator) {
            s = mk<T2>(wf * X[0].x, wf * X[0].y);
            d = s;
        } else {
            s = mk<T2>(wf * (X[0].x + X[1].x), wf * (X[0].y + X[1].y));
            d = mk<T2>(wf * (X[0].x - X[1].x), wf * (X[0].y - X[1].y));
        }
        const size_t o = (((size_t)b * (mmax + 1) + m) * npairs + pp) * 2;
        sd2[o] = s;
        sd2[o + 1] = d;
    }
}

template <typename T, bool MIXED>
__global__ void __launch_bounds__(512)
k_fft_analys(PlanView<T> pv, const T *__restrict__ grid, T *__restrict__ sd, int G, int op, int vector)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fft_analys_tile<T, MIXED>(pv, grid, sd, blockIdx.y, blockIdx.x * G, G, op, vector, smem_raw);
}

// ---------------------------------------------------------------------------
// Double-float FFTs for the FP64 data of the FP64-accurate tensor-core mode.
// A value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2 (Dekker's double-length arithmetic, 1971): 48
// significand bits from FP32 instructions only, which this GPU issues some
// seventy times faster than FP64 ones.  The sum is the short form (error-free
// sum of the high parts, the low parts added once, renormalised); its error is
// a small multiple of 2^-48 (|x| + |y|), which is the form of per-operation
// bound the normwise error analysis of an FFT rests on, so a transform keeps an
// error of order 2^-48 log2(H) of the row norm.  FP32's exponent range is kept
// out of the way by scaling each latitude pair by the power of two that brings
// its largest value into [1, 2) (found from the FP64 exponent bits, exact) and
// scaling back on the way out.  Conversions between FP64 and double-float work
// on the bits with integer operations, so no FP64 instruction runs per element.
// ---------------------------------------------------------------------------
// Biased FP64 exponent field of the larger part of v (0 for zeros and subnormals).
__device__ __forceinline__ int dexp2(double2 v)
{
    const int a = (int)((unsigned long long)__double_as_longlong(v.x) >> 52) & 0x7ff;
    const int b = (int)((unsigned long long)__double_as_longlong(v.y) >> 52) & 0x7ff;
    return a > b ? a : b;
}

// v 2^-u as a double-float, from the bits of v: hi takes the leading 24
// significand bits (truncated), lo the remaining 29 (rounded to 24 by the
// integer-to-float conversion), so 0 <= |lo| < ulp(hi), same sign: an
// unnormalised pair, which the operations above accept.  Scaled values below
// 2^-126 are flushed to zero (the scale puts the pair's largest value in
// [1, 2), so fe <= 0), as are FP64 subnormals.  Selects, not branches.
__device__ __forceinline__ dfl d2df(double v, int u)
{
    const unsigned hw = (unsigned)__double2hiint(v), lw = (unsigned)__double2loint(v);
    const int E = (int)((hw >> 20) & 0x7ffu), fe = E - 1023 - u;
    const unsigned sgn = hw & 0x80000000u;
    const unsigned top = __funnelshift_r(lw, hw, 29) & 0x7fffffu;           // significand bits 51..29
    const float hi = __uint_as_float(sgn | ((unsigned)(fe + 127) << 23) | top);
    // the low 29 bits weigh 2^(fe - 52) each; a scale below FP32's normal range gives 0
    float lo = __fmul_rn(__uint2float_rn(lw & 0x1fffffffu), __uint_as_float((unsigned)max(fe + 75, 0) << 23));
    lo = __uint_as_float(__float_as_uint(lo) | sgn);
    const bool zero = E == 0 || fe < -126;
    return dfl(zero ? 0.f : hi, zero ? 0.f : lo);
}
__device__ __forceinline__ dfl2 d2df2(double2 v, int u)
{
    dfl2 r;
    r.x = d2df(v.x, u);
    r.y = d2df(v.y, u);
    return r;
}

// f 2^u as an FP64 number, exactly: the float's sign and significand bits
// placed in a double whose exponent field is the float's raised by u
// (1023 - 127 = 896 re-biases it).  FP32 subnormals and zeros give 0, as do
// results below 2^-1022; results beyond the FP64 range give infinity.
__device__ __forceinline__ double f2d_pow2(float f, int u)
{
    const unsigned b = __float_as_uint(f), s = b & 0x80000000u;
    const int e = (int)((b >> 23) & 0xffu), E = e + 896 + u;
    unsigned hw = s | ((unsigned)E << 20) | ((b >> 3) & 0xfffffu), lw = b << 29;
    const bool zero = e == 0 || E <= 0, inf = E >= 2047;
    hw = zero ? s : (inf ? (s | 0x7ff00000u) : hw);
    lw = zero || inf ? 0u : lw;
    return __hiloint2double((int)hw, (int)lw);
}

// (z.hi + z.lo) 2^u as an FP64 number: both parts are exact in FP64, so one
// FP64 addition rounds their exact sum (to nearest, ties to even); the pair
// need not be normalised.  (A bit-level sum of the two significands in a
// 64-bit integer took about 60 integer instructions per value, a third of
// the synthesis FFT's instructions; this takes about 20 and one FP64 add.)
__device__ __forceinline__ double df2d(dfl z, int u) { return f2d_pow2(z.hi, u) + f2d_pow2(z.lo, u); }

__device__ __forceinline__ dfl2 ld_twdf(const float4 *__restrict__ tw, int k)
{
    const float4 t = tw[k];
    dfl2 r;
    r.x = dfl(t.x, t.y);
    r.y = dfl(t.z, t.w);
    return r;
}

// W_H^q = e^{2 pi i q / H}, q < H, from the plan's double-float e^{2 pi i k / nphi}.
__device__ __forceinline__ void fill_wtab_df(dfl2 *wtab, const float4 *__restrict__ twdf, int H)
{
    for (int q = threadIdx.x; q < H; q += blockDim.x) {
        dfl2 w;
        if (2 * q < H) {
            w = ld_twdf(twdf, 2 * q);
        } else {
            w = ld_twdf(twdf, 2 * q - H);
            w.x = -w.x;
            w.y = -w.y;
        }
        wtab[q] = w;
    }
}

// Shared memory of a double-float tile beyond the FP64 tile's (same row
// layout: a double-float complex is 16 bytes): per pair its exponent and a
// double-float scale factor.
__host__ __device__ constexpr size_t df_extra_smem(int G) { return (size_t)4 * (G + (G & 1)) + (size_t)8 * G; }

// Synthesis tile in double-float (see fft_synth_tile for the steps).  The
// Legendre output arrives as FP64 E, O; they are staged unconverted in the
// rows while the pair's largest exponent is found, then converted in the
// pre-twiddle.
template <bool MIXED, int LOGH = 0>
__device__ __forceinline__ void fft_synth_tile_df(const PlanView<double> &pv, const double *__restrict__ eo,
                                                  double *__restrict__ grid, int b, int p0, int G, int op,
                                                  unsigned char *smem_raw)
{
    const int H = LOGH ? (1 << LOGH) : pv.nphi / 2, R = 2 * G;
    const int TPR = row_tpr(H);
    const int ld = padi(H) + 1;
    dfl2 *wtab = reinterpret_cast<dfl2 *>(smem_raw);
    dfl2 *buf = wtab + H;
    int *s_e = reinterpret_cast<int *>(buf + R * ld);
    dfl *s_w = reinterpret_cast<dfl *>(s_e + G + (G & 1));
    const int mmax = pv.mmax, npairs = pv.npairs, nlat = pv.nlat;
    const double2 *eo2 = reinterpret_cast<const double2 *>(eo);
    double2 *raw = reinterpret_cast<double2 *>(buf);

    fill_wtab_df(wtab, pv.twdf, H);
    for (int i = threadIdx.x; i < G; i += blockDim.x) {
        s_e[i] = 0;
        const int p = p0 + i;
        const double sc = (op == OP_ANALYS_ADJ && p < npairs) ? kTwoPiD / pv.nphi * pv.wq[p] : 1.0;
        s_w[i] = dfl(sc);
    }
    __syncthreads();
    // 1. E (row 2i) and O (row 2i+1) of the G pairs in natural order, zero
    //    above mmax, and the largest exponent per pair (G is a power of two
    //    unless the plan has fewer pairs: shifts, not divisions, split q)
    const bool gp2 = (G & (G - 1)) == 0;
    const int lgG = __popc(G - 1);
    {
        // the loads of U items are issued before their stores (latency, not bandwidth, is the limit here)
        constexpr int U = 8;
        int cur = -1, emax = 0;
        for (int q0 = threadIdx.x; q0 < G * H; q0 += U * blockDim.x) {
            double2 E[U], O[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = q0 + u * blockDim.x;
                E[u] = make_double2(0.0, 0.0);
                O[u] = E[u];
                if (q < G * H) {
                    const int m = gp2 ? q >> lgG : q / G, i = q - m * G;
                    const int p = p0 + i;
                    if (m <= mmax && p < npairs) {
                        const size_t o = (((size_t)b * (mmax + 1) + m) * npairs + p) * 2;
                        E[u] = eo2[o];
                        O[u] = eo2[o + 1];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = q0 + u * blockDim.x;
                if (q >= G * H) break;
                const int m = gp2 ? q >> lgG : q / G, i = q - m * G;
                if (m == 0) { E[u].y = 0.0; O[u].y = 0.0; }
                raw[(2 * i) * ld + padi(m)] = E[u];
                raw[(2 * i + 1) * ld + padi(m)] = O[u];
                if (i != cur) {
                    if (cur >= 0) atomicMax(&s_e[cur], emax);
                    cur = i;
                    emax = 0;
                }
                emax = max(emax, max(dexp2(E[u]), dexp2(O[u])));
            }
        }
        if (cur >= 0) atomicMax(&s_e[cur], emax);
    }
    __syncthreads();
    // 2. X_N = E + O, X_S = E - O and the pre-twiddle, in double-float; a thread
    //    owns positions k and H - k of both rows of its pair (converted in place)
    for (int q = threadIdx.x; q < G * (H / 2 + 1); q += blockDim.x) {
        const int i = q / (H / 2 + 1), k = q - i * (H / 2 + 1);
        const int u = s_e[i] - 1023;
        const int k2 = k == 0 ? 0 : H - k;
        const double2 *rE = raw + (2 * i) * ld, *rO = raw + (2 * i + 1) * ld;
        const dfl2 Ea = d2df2(rE[padi(k)], u), Oa = d2df2(rO[padi(k)], u);
        const dfl2 Eb = d2df2(rE[padi(k2)], u), Ob = d2df2(rO[padi(k2)], u);
        dfl2 *dN = buf + (2 * i) * ld, *dS = buf + (2 * i + 1) * ld;
        const dfl2 XNa = cadd(Ea, Oa), XSa = csub(Ea, Oa);
        if (k == 0) {
            dN[0] = cadd(XNa, mul_i(XNa));
            dS[0] = cadd(XSa, mul_i(XSa));
            continue;
        }
        const dfl2 XNb = cadd(Eb, Ob), XSb = csub(Eb, Ob);
        // with A = X_k + conj X_{H-k} and P = W^k (X_k - conj X_{H-k}), W = e^{2 pi i / (2H)}:
        // Z_k = A + i P and, since W^{H-k} = -conj W^k, Z_{H-k} = conj A + i conj P
        const dfl2 wa = ld_twdf(pv.twdf, k);
        const dfl2 AN = cadd(XNa, conj_(XNb)), PN = cmul(wa, csub(XNa, conj_(XNb)));
        const dfl2 AS = cadd(XSa, conj_(XSb)), PS = cmul(wa, csub(XSa, conj_(XSb)));
        dN[padi(k)] = cadd(AN, mul_i(PN));
        dS[padi(k)] = cadd(AS, mul_i(PS));
        if (k2 != k) {
            dN[padi(k2)] = cadd(conj_(AN), mul_i(conj_(PN)));
            dS[padi(k2)] = cadd(conj_(AS), mul_i(conj_(PS)));
        }
    }
    __syncthreads();
    // 3. inverse complex FFT of length H; the last pass converts back to FP64 and writes the grid
    const int r = threadIdx.x / TPR, t = threadIdx.x - r * TPR;
    const int p = p0 + (r >> 1);
    const int j = (r & 1) ? nlat - 1 - p : p;
    const bool live_row = r < R && p < npairs && !((r & 1) && j == p);
    dfl2 *row = buf + (r < R ? r : 0) * ld;
    double2 *out = reinterpret_cast<double2 *>(grid) + ((size_t)b * nlat + (live_row ? j : 0)) * H;
    const int u = r < R ? s_e[r >> 1] - 1023 : 0;
    const bool scaled = op == OP_ANALYS_ADJ;
    const dfl sc = r < R ? s_w[r >> 1] : dfl(1.f, 0.f);
    const auto put = [&](int idx, dfl2 z) {
        if (scaled) { z.x = z.x * sc; z.y = z.y * sc; }
        out[idx] = make_double2(df2d(z.x, u), df2d(z.y, u));
    };
    if constexpr (LOGH == 10) {
        // inverse complex FFT of length 1024: radix 4, 16, 16, the last from registers to the grid
        constexpr int NR = PassRegs<false>::n;
        dfl2 v[NR];
        if (r < R) stockham_load<dfl2, 4, 1, NR, true>(row, false, t, TPR, H, 1, wtab, v);
        __syncthreads();
        if (r < R) stockham_store_smem<dfl2, 4, NR, true>(row, t, TPR, H, 1, v);
        __syncthreads();
        // the two radix-16 passes run one copy of their code (a smaller
        // instruction footprint for the two CTAs of an SM)
        int Ns = 4;
#pragma unroll 1
        for (;;) {
            if (r < R) stockham_load<dfl2, 16, 1, NR, true>(row, false, t, TPR, H, Ns, wtab, v);
            if (Ns == 64) break;
            __syncthreads();
            if (r < R) stockham_store_smem<dfl2, 16, NR, true>(row, t, TPR, H, Ns, v);
            __syncthreads();
            Ns = 64;
        }
        if (live_row) last_pass_out<16, NR>(v, t, TPR, H, put);
        return;
    }
    if (H == 1) {
        if (threadIdx.x < R && live_row) put(0, row[0]);
        return;
    }
    int Ns = 1;
    dfl2 v[PassRegs<MIXED>::n];
    for (int ps = 0;; ++ps) {
        const int rd = fft_plan_radix(pv.fftplan, ps);
        if (r < R) pass_load<dfl2, 1, MIXED>(rd, row, false, t, TPR, H, Ns, wtab, v);
        const bool last = Ns * rd == H;
        __syncthreads();
        if (last) {
            if (live_row) last_pass_out<MIXED>(rd, v, t, TPR, H, put);
            break;
        }
        if (r < R) pass_store<dfl2, MIXED>(rd, row, t, TPR, H, Ns, v);
        __syncthreads();
        Ns *= rd;
    }
}

// Analysis tile in double-float (see fft_analys_tile).  Each thread reads its
// share of its row into registers, the pair's largest exponent is found, and
// the values go to shared memory converted; the fold converts back to FP64.
// fmax (may be null): per field, the running maximum of frexp exponents of
// the folds written (the field scale of the FP64-accurate contraction).
// LOGH > 0: the row length is 2^LOGH, known at compile time, and the passes are
// spelled out (radix 4, 16, 16 for LOGH = 10, the plan's order), so the index
// arithmetic folds and no code of other radices sits in the kernel (the
// synthesis tile has the same form).
template <bool MIXED, int LOGH = 0>
__device__ __forceinline__ void fft_analys_tile_df(const PlanView<double> &pv, const double *__restrict__ grid,
                                                   double *__restrict__ sd, int b, int p0, int G, int op,
                                                   int vector, int *__restrict__ fmax, unsigned char *smem_raw)
{
    const int H = LOGH ? (1 << LOGH) : pv.nphi / 2, R = 2 * G;
    const int TPR = row_tpr(H);
    const int ld = padi(H) + 1;
    dfl2 *wtab = reinterpret_cast<dfl2 *>(smem_raw);
    dfl2 *buf = wtab + H;
    int *s_e = reinterpret_cast<int *>(buf + R * ld);
    dfl *s_w = reinterpret_cast<dfl *>(s_e + G + (G & 1));
    const int mmax = pv.mmax, npairs = pv.npairs, nlat = pv.nlat;

    fill_wtab_df(wtab, pv.twdf, H);
    for (int i = threadIdx.x; i < G; i += blockDim.x) {
        s_e[i] = 0;
        const int pp = p0 + i;
        double wf = (op == OP_ANALYS) ? kTwoPiD / pv.nphi : 1.0;
        if (pp < npairs) {
            if (op == OP_ANALYS) wf *= pv.wq[pp];
            if (vector) wf /= pv.st[pp];
        }
        s_w[i] = dfl(wf);
    }
    __syncthreads();
    const int r = threadIdx.x / TPR, t = threadIdx.x - r * TPR;
    const int p = p0 + (r >> 1);
    const int j = (r & 1) ? nlat - 1 - p : p;
    const bool live_row = r < R && p < npairs && !((r & 1) && j == p);
    dfl2 *row = buf + (r < R ? r : 0) * ld;
    const double2 *in = reinterpret_cast<const double2 *>(grid) + ((size_t)b * nlat + (live_row ? j : 0)) * H;
    // H <= 16 TPR: at most 16 values per thread
    double2 x[16];
    {
        int e = 0;
#pragma unroll
        for (int it = 0; it < 16; ++it) {
            const int k = t + it * TPR;
            x[it] = (live_row && k < H) ? in[k] : make_double2(0.0, 0.0);
            e = max(e, dexp2(x[it]));
        }
        if (live_row) atomicMax(&s_e[r >> 1], e);
    }
    __syncthreads();
    if (r < R) {
        const int u = s_e[r >> 1] - 1023;
#pragma unroll
        for (int it = 0; it < 16; ++it) {
            const int k = t + it * TPR;
            if (k < H) row[padi(k)] = d2df2(x[it], u);
        }
    }
    __syncthreads();
    if constexpr (LOGH == 10) {
        // forward complex FFT of length 1024: radix 4, 16, 16
        constexpr int NR = PassRegs<false>::n;
        dfl2 v[NR];
        if (r < R) stockham_load<dfl2, 4, -1, NR, true>(row, false, t, TPR, H, 1, wtab, v);
        __syncthreads();
        if (r < R) stockham_store_smem<dfl2, 4, NR, true>(row, t, TPR, H, 1, v);
        __syncthreads();
#pragma unroll 1
        for (int Ns = 4; Ns <= 64; Ns *= 16) {   // one copy of the radix-16 code
            if (r < R) stockham_load<dfl2, 16, -1, NR, true>(row, false, t, TPR, H, Ns, wtab, v);
            __syncthreads();
            if (r < R) stockham_store_smem<dfl2, 16, NR, true>(row, t, TPR, H, Ns, v);
            __syncthreads();
        }
    } else if (H > 1) {
        // forward complex FFT of length H
        int Ns = 1;
        dfl2 v[PassRegs<MIXED>::n];
        const int npass = fft_plan_npass(pv.fftplan);
        for (int ps = 0; ps < npass; ++ps) {
            const int rd = fft_plan_radix(pv.fftplan, ps);
            if (r < R) pass_load<dfl2, -1, MIXED>(rd, row, false, t, TPR, H, Ns, wtab, v);
            __syncthreads();
            if (r < R) pass_store<dfl2, MIXED>(rd, row, t, TPR, H, Ns, v);
            __syncthreads();
            Ns *= rd;
        }
    }
    // post-twiddle, fold north/south, weight, back to FP64.  Positions m and
    // H - m share their terms: with E = (Z_m + conj Z_{H-m}) / 2,
    // Od = (Z_m - conj Z_{H-m}) / (2i) and P = W^{-m} Od (W = e^{2 pi i / (2H)}),
    // X_m = E + P and X_{H-m} = conj(E - P), one product for both.
    double2 *sd2 = reinterpret_cast<double2 *>(sd);
    unsigned ebits = 0;   // largest biased exponent field written by this thread
    const auto emit = [&](int m, int i, int pp, const dfl2 (&X)[2]) {
        const dfl wf = s_w[i];
        const bool equator = (nlat & 1) && pp == npairs - 1;
        dfl2 s, d;
        if (equator) {
            s = mk<dfl2>(wf * X[0].x, wf * X[0].y);
            d = s;
        } else {
            s = mk<dfl2>(wf * (X[0].x + X[1].x), wf * (X[0].y + X[1].y));
            d = mk<dfl2>(wf * (X[0].x - X[1].x), wf * (X[0].y - X[1].y));
        }
        const int u = s_e[i] - 1023;
        const size_t o = (((size_t)b * (mmax + 1) + m) * npairs + pp) * 2;
        const double2 so = make_double2(df2d(s.x, u), df2d(s.y, u)), dd = make_double2(df2d(d.x, u), df2d(d.y, u));
        sd2[o] = so;
        sd2[o + 1] = dd;
        ebits = max(ebits, (unsigned)max(dexp2(so), dexp2(dd)));
    };
    const int mhalf = min(H / 2, mmax);
    const bool gp2 = (G & (G - 1)) == 0;
    const int lgG = __popc(G - 1);
    for (int q = threadIdx.x; q < G * (mhalf + 1); q += blockDim.x) {
        const int m = gp2 ? q >> lgG : q / G, i = q - m * G;
        const int pp = p0 + i;
        if (pp >= npairs) continue;
        const int m2 = H - m;   // its partner, when it is another position and an order of the plan
        const bool two = m2 != m && m2 < H && m2 <= mmax;
        const dfl2 wm = conj_(ld_twdf(pv.twdf, m));
        dfl2 X[2], X2[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const dfl2 *rw = buf + (2 * i + h) * ld;
            const dfl2 Zk = rw[padi(m)];
            const dfl2 Zc = conj_(rw[padi(MIXED ? (H - m) % H : (H - m) & (H - 1))]);
            dfl2 E = cadd(Zk, Zc), O = csub(Zk, Zc);
            E.x = scale2(E.x, 0.5f);
            E.y = scale2(E.y, 0.5f);
            const dfl2 Od = mk<dfl2>(scale2(O.y, 0.5f), scale2(O.x, -0.5f));  // O / (2i)
            const dfl2 P = cmul(wm, Od);
            X[h] = cadd(E, P);
            X2[h] = conj_(csub(E, P));
        }
        emit(m, i, pp, X);
        if (two) emit(m2, i, pp, X2);
    }
    if (fmax) {
        // outputs are normal or zero (df2d flushes below 2^-1022): frexp's
        // exponent of a normal double is its biased exponent field - 1022
        ebits = __reduce_max_sync(0xffffffffu, ebits);
        if ((threadIdx.x & 31) == 0 && ebits != 0) atomicMax(&fmax[b], (int)ebits - 1022);
    }
}

template <bool MIXED, int LOGH = 0>
__global__ void __launch_bounds__(512)
k_fft_synth_df(PlanView<double> pv, const double *__restrict__ eo, double *__restrict__ grid, int G, int op)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fft_synth_tile_df<MIXED, LOGH>(pv, eo, grid, blockIdx.y, blockIdx.x * G, G, op, smem_raw);
}

template <bool MIXED, int LOGH = 0>
__global__ void __launch_bounds__(512)
k_fft_analys_df(PlanView<double> pv, const double *__restrict__ grid, double *__restrict__ sd, int G, int op,
                int vector, int *__restrict__ fmax)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fft_analys_tile_df<MIXED, LOGH>(pv, grid, sd, blockIdx.y, blockIdx.x * G, G, op, vector, fmax, smem_raw);
}

// ---------------------------------------------------------------------------
// FP32 row FFTs for H <= 1024: one warp per grid row, no block barrier inside
// a transform.  Four-step split H = N1 N2 (N1 = 2^ceil(logH / 2)): lane
// n2 < N2 holds z[n2 + N2 n1] (n1 < N1) and runs a DFT of length N1 in
// registers; the results are multiplied by W_H^(n2 k1) (plan table rtw) and
// transposed through the warp's own shared-memory row; lane k1 < N1 then runs
// a DFT of length N2 over n2 and holds Z[k1 + N1 k2] (k2 < N2).  A CTA owns
// kRowPairs latitude pairs (2 kRowPairs warps), so the mirror unfold (synthesis)
// and fold (analysis) of Sec. 3.1 run on the CTA's rows in shared memory.
// ---------------------------------------------------------------------------
constexpr int kRowPairs = 4;
constexpr int kRowLogMax = 10;

template <int LOGH>
struct RowShape {
    static constexpr int H = 1 << LOGH;
    static constexpr int N1 = 1 << ((LOGH + 1) / 2);
    static constexpr int N2 = H / N1;
    static constexpr int LDT = N1 + 1;                      // stride of the transposed layout
    static constexpr int LDN = H + (H >> 4) + 1;            // natural layout (padi indices)
    static constexpr int LD = LDN > N2 * LDT ? LDN : N2 * LDT;
};

// Pairs per row-FFT tile (one CTA of 8 warps).  H = 512 = 32 x 16: one warp
// per latitude pair (8 pairs), each half-warp one of the pair's rows in the
// first DFT (lane 16 h + n2 holds z[n2 + 16 n1] of row h) and every lane both
// rows' columns in the second (lane k1 holds Z[k1 + 32 k2], k2 < 16, of both):
// no lane idles, where one warp per row leaves half the lanes idle in the
// first DFT.  Other lengths: one warp per row (4 pairs).
template <int LOGH> struct RowPairs { static constexpr int n = LOGH == 9 ? 8 : kRowPairs; };
__host__ __device__ inline int row_pairs(int logH) { return logH == 9 ? 8 : kRowPairs; }
__host__ __device__ constexpr size_t row_fft_smem(int ld, int rp) { return (size_t)2 * rp * ld * sizeof(float2); }

// Runtime row length of RowShape<logH>.
__host__ __device__ inline int row_ld(int logH)
{
    const int H = 1 << logH, N1 = 1 << ((logH + 1) / 2), N2 = H / N1;
    const int ldn = H + (H >> 4) + 1;
    return ldn > N2 * (N1 + 1) ? ldn : N2 * (N1 + 1);
}

// One synthesis tile (field b, pairs p0 .. p0 + RowPairs - 1), run by a CTA of
// 64 kRowPairs threads; smem_raw holds row_fft_smem(LD, RowPairs) bytes.
template <int LOGH>
__device__ __forceinline__ void fft_synth_rows_tile(const PlanView<float> &pv, const float *__restrict__ eo,
                                                    float *__restrict__ grid, int b, int p0, int op,
                                                    unsigned char *smem_raw)
{
    using S = RowShape<LOGH>;
    constexpr int H = S::H, N1 = S::N1, N2 = S::N2, LD = S::LD, LDT = S::LDT;
    constexpr int RP = RowPairs<LOGH>::n;
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    const int mmax = pv.mmax, npairs = pv.npairs, nlat = pv.nlat;
    // 1. spectra of the CTA's rows: X_north = E + O, X_south = E - O, zero above
    //    mmax; the loads of a batch of U items are issued before their stores
    constexpr int NT = 64 * kRowPairs, NQ = RP * H, U = 16;
    const float4 *eo4 = reinterpret_cast<const float4 *>(eo);
#pragma unroll 1
    for (int q0 = threadIdx.x; q0 < NQ; q0 += U * NT) {
        float4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = q0 + u * NT;
            const int m = q / RP, p = p0 + (q - m * RP);
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (q < NQ && m <= mmax && p < npairs) v[u] = eo4[((size_t)b * (mmax + 1) + m) * npairs + p];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = q0 + u * NT;
            if (q >= NQ) break;
            const int m = q / RP, i = q - m * RP;
            const float2 XN = make_float2(v[u].x + v[u].z, m == 0 ? 0.f : v[u].y + v[u].w);
            const float2 XS = make_float2(v[u].x - v[u].z, m == 0 ? 0.f : v[u].y - v[u].w);
            buf[(2 * i) * LD + padi(m)] = XN;
            buf[(2 * i + 1) * LD + padi(m)] = XS;
        }
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if constexpr (RP != kRowPairs) {
        // a warp per pair (see RowPairs): half-warp h, row h of pair p, in the first DFT
        static_assert(N1 == 32 && N2 == 16, "a half-warp per row in the first DFT");
        const int p = p0 + warp;
        if (p >= npairs) return;   // no barrier follows in this tile
        const int h = lane >> 4, n2 = lane & 15;
        const bool equator = (nlat & 1) && p == npairs - 1;   // one row only
        float2 *row = buf + (2 * warp + h) * LD;
        float2 v[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {
            const int k = n2 + N2 * n1;
            const float2 Xa = row[padi(k)];
            if (k == 0) {
                v[n1] = cadd(Xa, mul_i(Xa));
            } else {
                const float2 Xb = row[padi(H - k)];
                v[n1] = cadd(cadd(Xa, conj_(Xb)), mul_i(cmul(pv.tw[k], csub(Xa, conj_(Xb)))));
            }
        }
        RegDft<float2, N1, 1>::run(v);
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) row[n2 * LDT + k1] = k1 == 0 ? v[k1] : cmul(v[k1], pv.rtw[k1 * N2 + n2]);
        __syncwarp();
        const float2 *r0 = buf + (2 * warp) * LD, *r1 = r0 + LD;
        float2 u0[N2], u1[N2];
#pragma unroll
        for (int m2 = 0; m2 < N2; ++m2) {
            u0[m2] = r0[m2 * LDT + lane];
            u1[m2] = r1[m2 * LDT + lane];
        }
        RegDft<float2, N2, 1>::run(u0);
        RegDft<float2, N2, 1>::run(u1);
        float scale = 1.f;
        if (op == OP_ANALYS_ADJ) scale = float(kTwoPiD) / float(pv.nphi) * pv.wq[p];
        float2 *outN = reinterpret_cast<float2 *>(grid) + ((size_t)b * nlat + p) * H;
        float2 *outS = reinterpret_cast<float2 *>(grid) + ((size_t)b * nlat + (nlat - 1 - p)) * H;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) outN[lane + N1 * k2] = make_float2(u0[k2].x * scale, u0[k2].y * scale);
        if (!equator) {
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) outS[lane + N1 * k2] = make_float2(u1[k2].x * scale, u1[k2].y * scale);
        }
        return;
    }
    const int p = p0 + (warp >> 1);
    const int j = (warp & 1) ? nlat - 1 - p : p;
    if (p >= npairs || ((warp & 1) && j == p)) return;   // no barrier follows in this tile
    float2 *row = buf + warp * LD;
    // 2. Hermitian pre-twiddle Z_k = (X_k + conj X_{H-k}) + i W^k (X_k - conj X_{H-k}), X_H = 0,
    //    gathered in the phase-1 order k = n2 + N2 n1
    float2 v[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
        v[n1] = make_float2(0.f, 0.f);
        const int k = lane + N2 * n1;
        if (lane < N2) {
            const float2 Xa = row[padi(k)];
            if (k == 0) {
                v[n1] = cadd(Xa, mul_i(Xa));
            } else {
                const float2 Xb = row[padi(H - k)];
                v[n1] = cadd(cadd(Xa, conj_(Xb)), mul_i(cmul(pv.tw[k], csub(Xa, conj_(Xb)))));
            }
        }
    }
    // 3. inverse DFT of length H
    RegDft<float2, N1, 1>::run(v);
    __syncwarp();
    if (lane < N2) {
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
            const float2 y = k1 == 0 ? v[k1] : cmul(v[k1], pv.rtw[k1 * N2 + lane]);
            row[lane * LDT + k1] = y;
        }
    }
    __syncwarp();
    float2 u[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) u[n2] = lane < N1 ? row[n2 * LDT + lane] : make_float2(0.f, 0.f);
    RegDft<float2, N2, 1>::run(u);
    // 4. z_k = f_{2k} + i f_{2k+1}, k = k1 + N1 k2
    float scale = 1.f;
    if (op == OP_ANALYS_ADJ) scale = float(kTwoPiD) / float(pv.nphi) * pv.wq[p];
    if (lane < N1) {
        float2 *out = reinterpret_cast<float2 *>(grid) + ((size_t)b * nlat + j) * H;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) out[lane + N1 * k2] = make_float2(u[k2].x * scale, u[k2].y * scale);
    }
}

// One analysis tile (see fft_synth_rows_tile).
template <int LOGH>
__device__ __forceinline__ void fft_analys_rows_tile(const PlanView<float> &pv, const float *__restrict__ grid,
                                                     float *__restrict__ sd, int b, int p0, int op, int vector,
                                                     unsigned char *smem_raw)
{
    using S = RowShape<LOGH>;
    constexpr int H = S::H, N1 = S::N1, N2 = S::N2, LD = S::LD, LDT = S::LDT;
    constexpr int RP = RowPairs<LOGH>::n;
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    const int mmax = pv.mmax, npairs = pv.npairs, nlat = pv.nlat;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if constexpr (RP != kRowPairs) {
        // a warp per pair (see RowPairs); the south row of an equator pair is
        // the north one again, transformed and never folded in
        static_assert(N1 == 32 && N2 == 16, "a half-warp per row in the first DFT");
        const int p = p0 + warp;
        if (p < npairs) {
            const int h = lane >> 4, n2 = lane & 15;
            float2 *row = buf + (2 * warp + h) * LD;
            const float2 *in = reinterpret_cast<const float2 *>(grid) + ((size_t)b * nlat + (h ? nlat - 1 - p : p)) * H;
            float2 v[N1];
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) v[n1] = in[n2 + N2 * n1];
            RegDft<float2, N1, -1>::run(v);
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1)
                row[n2 * LDT + k1] = k1 == 0 ? v[k1] : cmul(v[k1], conj_(pv.rtw[k1 * N2 + n2]));
            __syncwarp();
            float2 *r0 = buf + (2 * warp) * LD, *r1 = r0 + LD;
            float2 u0[N2], u1[N2];
#pragma unroll
            for (int m2 = 0; m2 < N2; ++m2) {
                u0[m2] = r0[m2 * LDT + lane];
                u1[m2] = r1[m2 * LDT + lane];
            }
            RegDft<float2, N2, -1>::run(u0);
            RegDft<float2, N2, -1>::run(u1);
            __syncwarp();
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) {
                r0[padi(lane + N1 * k2)] = u0[k2];
                r1[padi(lane + N1 * k2)] = u1[k2];
            }
        }
    } else {
    const int p = p0 + (warp >> 1);
    const int j = (warp & 1) ? nlat - 1 - p : p;
    const bool live = p < npairs && !((warp & 1) && j == p);
    float2 *row = buf + warp * LD;
    if (live) {
        // 1. forward DFT of length H of z_n = f_{2n} + i f_{2n+1}
        const float2 *in = reinterpret_cast<const float2 *>(grid) + ((size_t)b * nlat + j) * H;
        float2 v[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) v[n1] = lane < N2 ? in[lane + N2 * n1] : make_float2(0.f, 0.f);
        RegDft<float2, N1, -1>::run(v);
        if (lane < N2) {
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) {
                const float2 y = k1 == 0 ? v[k1] : cmul(v[k1], conj_(pv.rtw[k1 * N2 + lane]));
                row[lane * LDT + k1] = y;
            }
        }
        __syncwarp();
        float2 u[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) u[n2] = lane < N1 ? row[n2 * LDT + lane] : make_float2(0.f, 0.f);
        RegDft<float2, N2, -1>::run(u);
        __syncwarp();
        if (lane < N1) {
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) row[padi(lane + N1 * k2)] = u[k2];
        }
    }
    }
    __syncthreads();
    // 2. post-twiddle, scale, fold north/south, weight
    float4 *sd4 = reinterpret_cast<float4 *>(sd);
    const float fscale = (op == OP_ANALYS) ? float(kTwoPiD) / float(pv.nphi) : 1.f;
    for (int q = threadIdx.x; q < RP * (mmax + 1); q += blockDim.x) {
        const int m = q / RP, i = q - m * RP;
        const int pp = p0 + i;
        if (pp >= npairs) continue;
        const bool equator = (nlat & 1) && pp == npairs - 1;
        float2 X[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            X[h] = make_float2(0.f, 0.f);
            if (h == 1 && equator) continue;
            const float2 *rw = buf + (2 * i + h) * LD;
            const float2 Zk = rw[padi(m)];
            const float2 Zc = conj_(rw[padi((H - m) & (H - 1))]);
            float2 E = cadd(Zk, Zc), O = csub(Zk, Zc);
            E.x *= 0.5f; E.y *= 0.5f;
            const float2 Od = make_float2(O.y * 0.5f, -O.x * 0.5f);  // O / (2i)
            X[h] = cadd(E, cmul(conj_(pv.tw[m]), Od));
        }
        float wf = fscale;
        if (op == OP_ANALYS) wf *= pv.wq[pp];
        if (vector) wf /= pv.st[pp];
        float4 o;
        if (equator) {
            o = make_float4(wf * X[0].x, wf * X[0].y, wf * X[0].x, wf * X[0].y);
        } else {
            o = make_float4(wf * (X[0].x + X[1].x), wf * (X[0].y + X[1].y), wf * (X[0].x - X[1].x),
                            wf * (X[0].y - X[1].y));
        }
        sd4[((size_t)b * (mmax + 1) + m) * npairs + pp] = o;
    }
}

template <int LOGH>
__global__ void __launch_bounds__(64 * kRowPairs, 2)
k_fft_synth_rows(PlanView<float> pv, const float *__restrict__ eo, float *__restrict__ grid, int op)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fft_synth_rows_tile<LOGH>(pv, eo, grid, blockIdx.y, blockIdx.x * RowPairs<LOGH>::n, op, smem_raw);
}

template <int LOGH>
__global__ void __launch_bounds__(64 * kRowPairs, 2)
k_fft_analys_rows(PlanView<float> pv, const float *__restrict__ grid, float *__restrict__ sd, int op, int vector)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fft_analys_rows_tile<LOGH>(pv, grid, sd, blockIdx.y, blockIdx.x * RowPairs<LOGH>::n, op, vector, smem_raw);
}

template <int LOGH>
cudaError_t launch_rows(bool synth, const PlanView<float> &pv, const float *in, float *out, int batch, Op op,
                        bool vector, cudaStream_t s)
{
    constexpr int RP = RowPairs<LOGH>::n;
    const size_t smem = row_fft_smem(RowShape<LOGH>::LD, RP);
    dim3 g((unsigned)((pv.npairs + RP - 1) / RP), (unsigned)batch);
    cudaError_t e;
    if (synth) {
        if (smem > 48 * 1024) {
            e = cudaFuncSetAttribute(k_fft_synth_rows<LOGH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k_fft_synth_rows<LOGH><<<g, 64 * kRowPairs, smem, s>>>(pv, in, out, (int)op);
    } else {
        if (smem > 48 * 1024) {
            e = cudaFuncSetAttribute(k_fft_analys_rows<LOGH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k_fft_analys_rows<LOGH><<<g, 64 * kRowPairs, smem, s>>>(pv, in, out, (int)op, vector ? 1 : 0);
    }
    return cudaGetLastError();
}

cudaError_t launch_rows_dispatch(int logH, bool synth, const PlanView<float> &pv, const float *in, float *out,
                                 int batch, Op op, bool vector, cudaStream_t s)
{
    switch (logH) {
    case 0: return launch_rows<0>(synth, pv, in, out, batch, op, vector, s);
    case 1: return launch_rows<1>(synth, pv, in, out, batch, op, vector, s);
    case 2: return launch_rows<2>(synth, pv, in, out, batch, op, vector, s);
    case 3: return launch_rows<3>(synth, pv, in, out, batch, op, vector, s);
    case 4: return launch_rows<4>(synth, pv, in, out, batch, op, vector, s);
    case 5: return launch_rows<5>(synth, pv, in, out, batch, op, vector, s);
    case 6: return launch_rows<6>(synth, pv, in, out, batch, op, vector, s);
    case 7: return launch_rows<7>(synth, pv, in, out, batch, op, vector, s);
    case 8: return launch_rows<8>(synth, pv, in, out, batch, op, vector, s);
    case 9: return launch_rows<9>(synth, pv, in, out, batch, op, vector, s);
    case 10: return launch_rows<10>(synth, pv, in, out, batch, op, vector, s);
    default: return cudaErrorInvalidValue;
    }
}

inline int ilog2(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }
inline bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Threads per row and pairs per CTA: TPR = ceil(H/16) threads per row and
// enough rows for 256 threads, capped so the CTA's buffer stays <= 96 KB.
// (512-thread CTAs read the intermediate in longer runs but fit one CTA per
// SM and measured slower: the kernel is latency-bound, not DRAM-bound.)
template <typename T>
void fft_shape(int H, int npairs, int &G, int &threads, size_t &smem)
{
    using T2 = typename Vec2<T>::type;
    const int TPR = row_tpr(H);
    int rows = 256 / TPR;
    if (rows < 2) rows = 2;
    const size_t row_bytes = (size_t)((H + (H >> 4)) + 1) * sizeof(T2);
    while (rows > 2 && (size_t)rows * row_bytes > 96 * 1024) rows /= 2;
    G = rows / 2;
    if (G > npairs) G = npairs < 1 ? 1 : npairs;
    threads = 2 * G * TPR;
    if (threads < 32) threads = 32;
    threads = (threads + 31) & ~31;
    smem = (size_t)H * sizeof(T2) + (size_t)2 * G * row_bytes;
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

template <typename T>
cudaError_t launch_fft_synth(const PlanView<T> &pv, const T *eo, T *grid, int batch, Op op, cudaStream_t s)
{
    const int H = pv.nphi / 2, logH = ilog2(H);
    if constexpr (sizeof(T) == 4) {
        if (pow2(H) && logH <= kRowLogMax) return launch_rows_dispatch(logH, true, pv, eo, grid, batch, op, false, s);
    }
    int G, threads;
    size_t smem;
    fft_shape<T>(H, pv.npairs, G, threads, smem);
    const bool mixed = !pow2(H);
    cudaError_t e = mixed ? set_smem(k_fft_synth<T, true>, smem) : set_smem(k_fft_synth<T, false>, smem);
    if (e != cudaSuccess) return e;
    dim3 gridd((unsigned)((pv.npairs + G - 1) / G), (unsigned)batch);
    if (mixed)
        k_fft_synth<T, true><<<gridd, threads, smem, s>>>(pv, eo, grid, G, (int)op);
    else
        k_fft_synth<T, false><<<gridd, threads, smem, s>>>(pv, eo, grid, G, (int)op);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fft_analys(const PlanView<T> &pv, const T *grid, T *sd, int batch, Op op, bool vector,
                              cudaStream_t s)
{
    const int H = pv.nphi / 2, logH = ilog2(H);
    if constexpr (sizeof(T) == 4) {
        if (pow2(H) && logH <= kRowLogMax)
            return launch_rows_dispatch(logH, false, pv, grid, sd, batch, op, vector, s);
    }
    int G, threads;
    size_t smem;
    fft_shape<T>(H, pv.npairs, G, threads, smem);
    const bool mixed = !pow2(H);
    cudaError_t e = mixed ? set_smem(k_fft_analys<T, true>, smem) : set_smem(k_fft_analys<T, false>, smem);
    if (e != cudaSuccess) return e;
    dim3 gridd((unsigned)((pv.npairs + G - 1) / G), (unsigned)batch);
    if (mixed)
        k_fft_analys<T, true><<<gridd, threads, smem, s>>>(pv, grid, sd, G, (int)op, vector ? 1 : 0);
    else
        k_fft_analys<T, false><<<gridd, threads, smem, s>>>(pv, grid, sd, G, (int)op, vector ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_fft_synth_df(const PlanView<double> &pv, const double *eo, double *grid, int batch, Op op,
                                cudaStream_t s)
{
    if (!pv.twdf) return cudaErrorInvalidValue;
    int G, threads;
    size_t smem;
    fft_shape<double>(pv.nphi / 2, pv.npairs, G, threads, smem);
    smem += df_extra_smem(G);
    const bool mixed = !pow2(pv.nphi / 2), h1024 = pv.nphi == 2048;
    cudaError_t e = mixed ? set_smem(k_fft_synth_df<true>, smem)
                          : (h1024 ? set_smem(k_fft_synth_df<false, 10>, smem) : set_smem(k_fft_synth_df<false>, smem));
    if (e != cudaSuccess) return e;
    dim3 gridd((unsigned)((pv.npairs + G - 1) / G), (unsigned)batch);
    if (mixed)
        k_fft_synth_df<true><<<gridd, threads, smem, s>>>(pv, eo, grid, G, (int)op);
    else if (h1024)
        k_fft_synth_df<false, 10><<<gridd, threads, smem, s>>>(pv, eo, grid, G, (int)op);
    else
        k_fft_synth_df<false><<<gridd, threads, smem, s>>>(pv, eo, grid, G, (int)op);
    return cudaGetLastError();
}

cudaError_t launch_fft_analys_df(const PlanView<double> &pv, const double *grid, double *sd, int batch, Op op,
                                 bool vector, cudaStream_t s, int *fmax)
{
    if (!pv.twdf) return cudaErrorInvalidValue;
    int G, threads;
    size_t smem;
    fft_shape<double>(pv.nphi / 2, pv.npairs, G, threads, smem);
    smem += df_extra_smem(G);
    const bool mixed = !pow2(pv.nphi / 2), h1024 = pv.nphi == 2048;
    cudaError_t e = mixed ? set_smem(k_fft_analys_df<true>, smem)
                          : (h1024 ? set_smem(k_fft_analys_df<false, 10>, smem) : set_smem(k_fft_analys_df<false>, smem));
    if (e != cudaSuccess) return e;
    dim3 gridd((unsigned)((pv.npairs + G - 1) / G), (unsigned)batch);
    if (mixed)
        k_fft_analys_df<true><<<gridd, threads, smem, s>>>(pv, grid, sd, G, (int)op, vector ? 1 : 0, fmax);
    else if (h1024)
        k_fft_analys_df<false, 10><<<gridd, threads, smem, s>>>(pv, grid, sd, G, (int)op, vector ? 1 : 0, fmax);
    else
        k_fft_analys_df<false><<<gridd, threads, smem, s>>>(pv, grid, sd, G, (int)op, vector ? 1 : 0, fmax);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Persistent FFT kernels for uneven batches (FP32, 256 threads, one field per tile).
// ---------------------------------------------------------------------------
namespace {

__global__ void __launch_bounds__(256, 2) k_batch_fft(int synth, const BatchField *__restrict__ fields,
                                                   const int4 *__restrict__ tiles, int ntiles, int *counter)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_tile;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1);
        __syncthreads();
        const int t = s_tile;
        if (t >= ntiles) break;
        const int4 tl = tiles[t];
        const BatchField f = fields[tl.x];
        if (f.logH <= kRowLogMax) {
            // the same tile functions as the per-field FP32 launches
            switch (f.logH) {
#define SHT_ROW_CASE(L)                                                                                \
    case L:                                                                                            \
        if (synth) fft_synth_rows_tile<L>(f.pv, f.inter, f.out, 0, tl.y, OP_SYNTH, smem_raw);          \
        else fft_analys_rows_tile<L>(f.pv, f.in, f.inter, 0, tl.y, OP_ANALYS, 0, smem_raw);            \
        break;
                SHT_ROW_CASE(0) SHT_ROW_CASE(1) SHT_ROW_CASE(2) SHT_ROW_CASE(3) SHT_ROW_CASE(4) SHT_ROW_CASE(5)
                SHT_ROW_CASE(6) SHT_ROW_CASE(7) SHT_ROW_CASE(8) SHT_ROW_CASE(9) SHT_ROW_CASE(10)
#undef SHT_ROW_CASE
            default: break;
            }
        } else if (synth) {
            fft_synth_tile<float, true>(f.pv, f.inter, f.out, 0, tl.y, f.G, OP_SYNTH, smem_raw);
        } else {
            fft_analys_tile<float, true>(f.pv, f.in, f.inter, 0, tl.y, f.G, OP_ANALYS, 0, smem_raw);
        }
    }
}

}  // namespace

// Pairs per FFT tile for a 256-thread CTA: kRowPairs for the row FFTs
// (logH <= 10), else 2G rows of max(1, H/16) threads.
int batch_fft_group(int H, int npairs)
{
    if (pow2(H) && ilog2(H) <= kRowLogMax) return row_pairs(ilog2(H));
    const int TPR = row_tpr(H);
    int G = 256 / (2 * TPR);
    if (G < 1) G = 1;
    if (G > npairs) G = npairs < 1 ? 1 : npairs;
    return G;
}

size_t batch_fft_smem(int H, int G)
{
    if (pow2(H) && ilog2(H) <= kRowLogMax) return row_fft_smem(row_ld(ilog2(H)), row_pairs(ilog2(H)));
    const size_t row_bytes = (size_t)((H + (H >> 4)) + 1) * sizeof(float2);
    return (size_t)H * sizeof(float2) + (size_t)2 * G * row_bytes;
}

cudaError_t batch_fft_prepare(size_t smem) { return set_smem(k_batch_fft, smem); }

cudaError_t launch_batch_fft(bool synth, const BatchField *fields, const int4 *tiles, int ntiles, int *counter,
                             int ctas, size_t smem, cudaStream_t s)
{
    k_batch_fft<<<ctas, 256, smem, s>>>(synth ? 1 : 0, fields, tiles, ntiles, counter);
    return cudaGetLastError();
}

template cudaError_t launch_fft_synth<double>(const PlanView<double> &, const double *, double *, int, Op,
                                              cudaStream_t);
template cudaError_t launch_fft_synth<float>(const PlanView<float> &, const float *, float *, int, Op, cudaStream_t);
template cudaError_t launch_fft_analys<double>(const PlanView<double> &, const double *, double *, int, Op, bool,
                                               cudaStream_t);
template cudaError_t launch_fft_analys<float>(const PlanView<float> &, const float *, float *, int, Op, bool,
                                              cudaStream_t);

}  // namespace sht
