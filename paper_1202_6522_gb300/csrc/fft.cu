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
            const int q = k * (64 / RD);
            const T2 w = mk<T2>(T(cos64(q)), T(SIGN * sin64(q)));
            const T2 t = (k == 0) ? o[k] : cmul(w, o[k]);
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
template <typename T2, int RD, int SIGN, int NR>
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
            const int q0 = (j % Ns) * (H / (Ns * RD));
#pragma unroll
            for (int r = 1; r < RD; ++r) {
                T2 w = wtab[(r * q0) % H];
                if (SIGN < 0) w = conj_(w);
                a[r] = cmul(a[r], w);
            }
        }
        RegDft<T2, RD, SIGN>::run(a);
#pragma unroll
        for (int r = 0; r < RD; ++r) v[it * RD + r] = a[r];
    }
}

template <typename T2, int RD>
__device__ __forceinline__ int stockham_out(int j, int r, int Ns)
{
    return (j / Ns) * Ns * RD + (j % Ns) + r * Ns;
}

template <typename T2, int RD, int NR>
__device__ __forceinline__ void stockham_store_smem(T2 *row, int t, int TPR, int H, int Ns, const T2 (&v)[NR])
{
    constexpr int IT = (16 + RD - 1) / RD;
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int j = t + it * TPR;
        if (j >= H / RD) break;
#pragma unroll
        for (int r = 0; r < RD; ++r) row[padi(stockham_out<T2, RD>(j, r, Ns))] = v[it * RD + r];
    }
}

// Runs a pass of the given radix (run-time selected).
template <typename T2, int SIGN, bool MIXED>
__device__ __forceinline__ void pass_load(int rd, const T2 *src, bool g, int t, int TPR, int H, int Ns,
                                          const T2 *wtab, T2 (&v)[PassRegs<MIXED>::n])
{
    constexpr int NR = PassRegs<MIXED>::n;
    if (MIXED && rd == 3) { stockham_load<T2, 3, SIGN, NR>(src, g, t, TPR, H, Ns, wtab, v); return; }
    if (MIXED && rd == 5) { stockham_load<T2, 5, SIGN, NR>(src, g, t, TPR, H, Ns, wtab, v); return; }
    switch (rd) {
    case 2: stockham_load<T2, 2, SIGN, NR>(src, g, t, TPR, H, Ns, wtab, v); break;
    case 4: stockham_load<T2, 4, SIGN, NR>(src, g, t, TPR, H, Ns, wtab, v); break;
    case 8: stockham_load<T2, 8, SIGN, NR>(src, g, t, TPR, H, Ns, wtab, v); break;
    default: stockham_load<T2, 16, SIGN, NR>(src, g, t, TPR, H, Ns, wtab, v); break;
    }
}

template <typename T2, bool MIXED>
__device__ __forceinline__ void pass_store(int rd, T2 *row, int t, int TPR, int H, int Ns,
                                           const T2 (&v)[PassRegs<MIXED>::n])
{
    constexpr int NR = PassRegs<MIXED>::n;
    if (MIXED && rd == 3) { stockham_store_smem<T2, 3, NR>(row, t, TPR, H, Ns, v); return; }
    if (MIXED && rd == 5) { stockham_store_smem<T2, 5, NR>(row, t, TPR, H, Ns, v); return; }
    switch (rd) {
    case 2: stockham_store_smem<T2, 2, NR>(row, t, TPR, H, Ns, v); break;
    case 4: stockham_store_smem<T2, 4, NR>(row, t, TPR, H, Ns, v); break;
    case 8: stockham_store_smem<T2, 8, NR>(row, t, TPR, H, Ns, v); break;
    default: stockham_store_smem<T2, 16, NR>(row, t, TPR, H, Ns, v); break;
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
            if (live_row) {
                const int IT = (16 + rd - 1) / rd;
                for (int it = 0; it < IT; ++it) {
                    const int jj = t + it * TPR;
                    if (jj >= H / rd) break;
                    for (int rr = 0; rr < rd; ++rr) {
                        T2 z = v[it * rd + rr];
                        z.x *= scale; z.y *= scale;
                        out[jj + rr * (H / rd)] = z;
                    }
                }
            }
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
            const T2 Zc = conj_(rw[padi((H - m) % H)]);
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

__host__ __device__ constexpr size_t row_fft_smem(int ld) { return (size_t)2 * kRowPairs * ld * sizeof(float2); }

// Runtime row length of RowShape<logH>.
__host__ __device__ inline int row_ld(int logH)
{
    const int H = 1 << logH, N1 = 1 << ((logH + 1) / 2), N2 = H / N1;
    const int ldn = H + (H >> 4) + 1;
    return ldn > N2 * (N1 + 1) ? ldn : N2 * (N1 + 1);
}

// One synthesis tile (field b, pairs p0 .. p0 + kRowPairs - 1), run by a CTA of
// 64 kRowPairs threads; smem_raw holds row_fft_smem(LD) bytes.
template <int LOGH>
__device__ __forceinline__ void fft_synth_rows_tile(const PlanView<float> &pv, const float *__restrict__ eo,
                                                    float *__restrict__ grid, int b, int p0, int op,
                                                    unsigned char *smem_raw)
{
    using S = RowShape<LOGH>;
    constexpr int H = S::H, N1 = S::N1, N2 = S::N2, LD = S::LD, LDT = S::LDT;
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    const int mmax = pv.mmax, npairs = pv.npairs, nlat = pv.nlat;
    // 1. spectra of the CTA's rows: X_north = E + O, X_south = E - O, zero above
    //    mmax; the loads of a batch of U items are issued before their stores
    constexpr int NT = 64 * kRowPairs, NQ = kRowPairs * H, U = 16;
    const float4 *eo4 = reinterpret_cast<const float4 *>(eo);
#pragma unroll 1
    for (int q0 = threadIdx.x; q0 < NQ; q0 += U * NT) {
        float4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = q0 + u * NT;
            const int m = q / kRowPairs, p = p0 + (q - m * kRowPairs);
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (q < NQ && m <= mmax && p < npairs) v[u] = eo4[((size_t)b * (mmax + 1) + m) * npairs + p];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = q0 + u * NT;
            if (q >= NQ) break;
            const int m = q / kRowPairs, i = q - m * kRowPairs;
            const float2 XN = make_float2(v[u].x + v[u].z, m == 0 ? 0.f : v[u].y + v[u].w);
            const float2 XS = make_float2(v[u].x - v[u].z, m == 0 ? 0.f : v[u].y - v[u].w);
            buf[(2 * i) * LD + padi(m)] = XN;
            buf[(2 * i + 1) * LD + padi(m)] = XS;
        }
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
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
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    const int mmax = pv.mmax, npairs = pv.npairs, nlat = pv.nlat;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
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
    __syncthreads();
    // 2. post-twiddle, scale, fold north/south, weight
    float4 *sd4 = reinterpret_cast<float4 *>(sd);
    const float fscale = (op == OP_ANALYS) ? float(kTwoPiD) / float(pv.nphi) : 1.f;
    for (int q = threadIdx.x; q < kRowPairs * (mmax + 1); q += blockDim.x) {
        const int m = q / kRowPairs, i = q - m * kRowPairs;
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
    fft_synth_rows_tile<LOGH>(pv, eo, grid, blockIdx.y, blockIdx.x * kRowPairs, op, smem_raw);
}

template <int LOGH>
__global__ void __launch_bounds__(64 * kRowPairs, 2)
k_fft_analys_rows(PlanView<float> pv, const float *__restrict__ grid, float *__restrict__ sd, int op, int vector)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fft_analys_rows_tile<LOGH>(pv, grid, sd, blockIdx.y, blockIdx.x * kRowPairs, op, vector, smem_raw);
}

template <int LOGH>
cudaError_t launch_rows(bool synth, const PlanView<float> &pv, const float *in, float *out, int batch, Op op,
                        bool vector, cudaStream_t s)
{
    const size_t smem = row_fft_smem(RowShape<LOGH>::LD);
    dim3 g((unsigned)((pv.npairs + kRowPairs - 1) / kRowPairs), (unsigned)batch);
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
    if (pow2(H) && ilog2(H) <= kRowLogMax) return kRowPairs;
    const int TPR = row_tpr(H);
    int G = 256 / (2 * TPR);
    if (G < 1) G = 1;
    if (G > npairs) G = npairs < 1 ? 1 : npairs;
    return G;
}

size_t batch_fft_smem(int H, int G)
{
    if (pow2(H) && ilog2(H) <= kRowLogMax) return row_fft_smem(row_ld(ilog2(H)));
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
