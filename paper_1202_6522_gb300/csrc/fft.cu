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
// an in-place radix-2 decimation-in-frequency pass sequence, which leaves the
// spectrum in bit-reversed order; the reads/writes around it undo that.
#include <cuda_runtime.h>

#include "sht_internal.h"

namespace sht {
namespace {

constexpr double kTwoPiD = 6.283185307179586476925286766559;

template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { T2 r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { T2 r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b)
{
    T2 r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename T2> __device__ __forceinline__ T2 conj_(T2 a) { a.y = -a.y; return a; }
template <typename T2> __device__ __forceinline__ T2 mul_i(T2 a) { T2 r; r.x = -a.y; r.y = a.x; return r; }

__device__ __forceinline__ int bitrev(int n, int logH) { return logH == 0 ? 0 : (int)(__brev((unsigned)n) >> (32 - logH)); }

// In-place radix-2 DIF over R rows of length H (row stride ld) in shared memory.
// INV: twiddles e^{+2 pi i ...} (inverse), else e^{-2 pi i ...}.
template <typename T, bool INV>
__device__ __forceinline__ void dif_fft(typename Vec2<T>::type *buf, int R, int H, int logH, int ld,
                                        const typename Vec2<T>::type *__restrict__ tw)
{
    using T2 = typename Vec2<T>::type;
    const int half_total = H >> 1;
    for (int lh = logH - 1; lh >= 0; --lh) {
        const int h = 1 << lh;
        const int tws = logH - lh;  // twiddle index stride: pos * (H / h)
        for (int t = threadIdx.x; t < R * half_total; t += blockDim.x) {
            const int r = t >> (logH - 1);
            const int u = t & (half_total - 1);
            const int pos = u & (h - 1);
            const int i0 = ((u >> lh) << (lh + 1)) + pos;
            T2 *row = buf + r * ld;
            const T2 a = row[i0], b = row[i0 + h];
            row[i0] = cadd(a, b);
            T2 w = tw[pos << tws];
            if (!INV) w = conj_(w);
            row[i0 + h] = cmul(csub(a, b), w);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Synthesis: EO [batch][mmax+1][npairs][2] -> grid [batch][nlat][nphi]
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_fft_synth(PlanView<T> pv, const T *__restrict__ eo, T *__restrict__ grid, int G, int logH, int op)
{
    using T2 = typename Vec2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *buf = reinterpret_cast<T2 *>(smem_raw);
    const int H = 1 << logH, ld = H + 1, R = 2 * G;
    const int b = blockIdx.y;
    const int p0 = blockIdx.x * G;
    const int mmax = pv.mmax, npairs = pv.npairs, nlat = pv.nlat;
    const T2 *eo2 = reinterpret_cast<const T2 *>(eo);

    // 1. spectra of the 2G rows, natural order, zero padded above mmax
    for (int q = threadIdx.x; q < R * H; q += blockDim.x) {
        const int m = q / R, r = q - m * R;
        const int p = p0 + (r >> 1);
        T2 X;
        X.x = T(0); X.y = T(0);
        if (m <= mmax && p < npairs) {
            const size_t o = (((size_t)b * (mmax + 1) + m) * npairs + p) * 2;
            const T2 E = eo2[o], O = eo2[o + 1];
            X = (r & 1) ? csub(E, O) : cadd(E, O);
            if (m == 0) X.y = T(0);
        }
        buf[r * ld + m] = X;
    }
    __syncthreads();
    // 2. pre-twiddle: Z_k = (X_k + conj X_{H-k}) + i W^k (X_k - conj X_{H-k}), X_H = 0
    for (int q = threadIdx.x; q < R * (H / 2 + 1); q += blockDim.x) {
        const int r = q / (H / 2 + 1), k = q - r * (H / 2 + 1);
        if (k > H - k && k != 0) continue;
        T2 *row = buf + r * ld;
        if (k == 0) {
            const T2 X0 = row[0];
            row[0] = cadd(X0, mul_i(X0));
            continue;
        }
        const int k2 = H - k;
        const T2 Xa = row[k], Xb = row[k2];
        const T2 Za = cadd(cadd(Xa, conj_(Xb)), mul_i(cmul(pv.tw[k], csub(Xa, conj_(Xb)))));
        row[k] = Za;
        if (k2 != k) {
            const T2 Zb = cadd(cadd(Xb, conj_(Xa)), mul_i(cmul(pv.tw[k2], csub(Xb, conj_(Xa)))));
            row[k2] = Zb;
        }
    }
    __syncthreads();
    // 3. inverse complex FFT of length H (output bit-reversed)
    dif_fft<T, true>(buf, R, H, logH, ld, pv.tw);
    // 4. f_{2n} = Re z_n, f_{2n+1} = Im z_n, scaled for the adjoint of analysis
    T2 *grid2 = reinterpret_cast<T2 *>(grid);
    for (int q = threadIdx.x; q < R * H; q += blockDim.x) {
        const int r = q >> logH, n = q & (H - 1);
        const int p = p0 + (r >> 1);
        if (p >= npairs) continue;
        const int j = (r & 1) ? nlat - 1 - p : p;
        if ((r & 1) && j == p) continue;  // equator row is written once
        T2 z = buf[r * ld + bitrev(n, logH)];
        if (op == OP_ANALYS_ADJ) {
            const T sc = T(kTwoPiD) / T(pv.nphi) * pv.wq[p];
            z.x *= sc;
            z.y *= sc;
        }
        grid2[((size_t)b * nlat + j) * H + n] = z;
    }
}

// ---------------------------------------------------------------------------
// Analysis: grid [batch][nlat][nphi] -> SD [batch][mmax+1][npairs][2]
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_fft_analys(PlanView<T> pv, const T *__restrict__ grid, T *__restrict__ sd, int G, int logH, int op, int vector)
{
    using T2 = typename Vec2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *buf = reinterpret_cast<T2 *>(smem_raw);
    const int H = 1 << logH, ld = H + 1, R = 2 * G;
    const int b = blockIdx.y;
    const int p0 = blockIdx.x * G;
    const int mmax = pv.mmax, npairs = pv.npairs, nlat = pv.nlat;
    const T2 *grid2 = reinterpret_cast<const T2 *>(grid);

    // 1. rows as complex z_n = f_{2n} + i f_{2n+1}
    for (int q = threadIdx.x; q < R * H; q += blockDim.x) {
        const int r = q >> logH, n = q & (H - 1);
        const int p = p0 + (r >> 1);
        const int j = (r & 1) ? nlat - 1 - p : p;
        T2 z;
        z.x = T(0); z.y = T(0);
        if (p < npairs && !((r & 1) && j == p)) z = grid2[((size_t)b * nlat + j) * H + n];
        buf[r * ld + n] = z;
    }
    __syncthreads();
    // 2. forward complex FFT of length H (output bit-reversed)
    dif_fft<T, false>(buf, R, H, logH, ld, pv.tw);
    // 3. post-twiddle, scale, fold north/south, weight
    T2 *sd2 = reinterpret_cast<T2 *>(sd);
    const T fscale = (op == OP_ANALYS) ? T(kTwoPiD) / T(pv.nphi) : T(1);
    for (int q = threadIdx.x; q < G * (mmax + 1); q += blockDim.x) {
        const int m = q / G, i = q - m * G;
        const int p = p0 + i;
        if (p >= npairs) continue;
        T2 X[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const T2 *row = buf + (2 * i + h) * ld;
            const T2 Zk = row[bitrev(m, logH)];
            const T2 Zc = conj_(row[bitrev((H - m) & (H - 1), logH)]);
            T2 E = cadd(Zk, Zc), O = csub(Zk, Zc);
            E.x *= T(0.5); E.y *= T(0.5);
            // O / (2i) = -i O / 2
            T2 Od;
            Od.x = O.y * T(0.5);
            Od.y = -O.x * T(0.5);
            X[h] = cadd(E, cmul(conj_(pv.tw[m]), Od));
        }
        T wf = fscale;
        if (op == OP_ANALYS) wf *= pv.wq[p];
        if (vector) wf /= pv.st[p];
        const bool equator = (nlat & 1) && p == npairs - 1;
        T2 s, d;
        if (equator) {
            s.x = wf * X[0].x; s.y = wf * X[0].y;
            d = s;
        } else {
            s.x = wf * (X[0].x + X[1].x); s.y = wf * (X[0].y + X[1].y);
            d.x = wf * (X[0].x - X[1].x); d.y = wf * (X[0].y - X[1].y);
        }
        const size_t o = (((size_t)b * (mmax + 1) + m) * npairs + p) * 2;
        sd2[o] = s;
        sd2[o + 1] = d;
    }
}

template <typename T>
int pick_group(int H)
{
    // rows of (H+1) complex values; keep the CTA's buffer within 64 KB
    const size_t row = (size_t)(H + 1) * sizeof(typename Vec2<T>::type);
    int g = (int)((64 * 1024) / (2 * row));
    if (g > 8) g = 8;
    if (g < 1) g = 1;
    return g;
}

inline int ilog2(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

template <typename T, typename K>
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
    const int G = pick_group<T>(H);
    const size_t smem = (size_t)2 * G * (H + 1) * sizeof(typename Vec2<T>::type);
    cudaError_t e = set_smem<T>(k_fft_synth<T>, smem);
    if (e != cudaSuccess) return e;
    dim3 gridd((unsigned)((pv.npairs + G - 1) / G), (unsigned)batch);
    k_fft_synth<T><<<gridd, 256, smem, s>>>(pv, eo, grid, G, logH, (int)op);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fft_analys(const PlanView<T> &pv, const T *grid, T *sd, int batch, Op op, bool vector,
                              cudaStream_t s)
{
    const int H = pv.nphi / 2, logH = ilog2(H);
    const int G = pick_group<T>(H);
    const size_t smem = (size_t)2 * G * (H + 1) * sizeof(typename Vec2<T>::type);
    cudaError_t e = set_smem<T>(k_fft_analys<T>, smem);
    if (e != cudaSuccess) return e;
    dim3 gridd((unsigned)((pv.npairs + G - 1) / G), (unsigned)batch);
    k_fft_analys<T><<<gridd, 256, smem, s>>>(pv, grid, sd, G, logH, (int)op, vector ? 1 : 0);
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
