// tc.cu -- the per-order Legendre contraction on the 5th-generation tensor
// cores (tcgen05), for batches of fields.
//
// For each order m and parity of n - m the Legendre stage is a small GEMM
// (mirror symmetry, Sec. 3.1):
//   synthesis  E/O[pair, col] = sum_k P[pair, k] * A[k, col]       (Eq. synth_direct)
//   analysis   f[k, col]      = sum_pair P[pair, k] * S[pair, col] (Eq. gauss)
// with k the index of n among degrees of that parity, col = (field, re/im),
// and S the weighted north/south folds (s for even, d for odd n - m).  The
// vector transforms run the same GEMMs with dP = sin(theta) dP/dtheta as a
// second matrix (k_tc_vec).
//
// The matrices P_n^m(x_j) (and dP) are built once per plan by the FP64
// recurrence of Sec. 3.2 with the rescaling of Sec. 3.5 (the precomputed
// variant of Sec. 3.1), split into bf16 hi + lo parts and stored in HBM
// already in the tensor core's shared-memory operand layout (K-major, no
// swizzle: 8-row x 16-byte core matrices), so each chunk is one bulk copy.
// A prep kernel converts the FP32 data into the same blocked hi/lo layout,
// and each product is hi*hi + hi*lo + lo*hi accumulated in FP32 in tensor
// memory.
//
// CTA: one (order m, 128-row tile).  A producer warp streams panel and data
// chunks with cp.async.bulk into a ring of stages, one thread issues the MMAs,
// four warps convert the analysis operand and run the epilogue (tcgen05.ld of
// the accumulators).  Every wait is bounded; on a timeout the kernel records
// an error code and returns.
// Leading panel chunks whose values are all below 2^-40 (high order, near
// the poles) are skipped: the static polar optimisation of Sec. 3.1.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include <algorithm>
#include <climits>
#include <vector>

#include "sht_internal.h"
#include "tc_common.cuh"
#include "tc_layout.cuh"
#include "tc_ptx.cuh"

namespace sht {
namespace {

constexpr int kRows = 128;            // MMA M
constexpr int kBlk = kRows * kKc * 2; // bytes of one bf16 [128 x kKc] panel block
constexpr int kChunkPanel = 4 * kBlk; // [parity][hi/lo] blocks per chunk = 16 KB
// A panel chunk interleaves its four blocks (parity x hi/lo) per 8-row group:
// group g of block kb at g * kPSbo + kb * kSbo, so that the rows from any group
// on are one contiguous byte range of the chunk.  kPSbo is the MMA's 8-row
// group stride for a panel block.
constexpr uint32_t kPSbo = 4 * kSbo;
__host__ __device__ __forceinline__ uint32_t pan_off(int kb, int row, int k)
{
    return (uint32_t)((row >> 3) * kPSbo + kb * kSbo + (k >> 3) * kLbo + (row & 7) * 16 + (k & 7) * 2);
}
using tcc::kWaitNs;
using tcc::raise_err;
using tcc::wait_or_abort;

__device__ __forceinline__ void split_bf16_d(double v, __nv_bfloat16 &hi, __nv_bfloat16 &lo)
{
    hi = __float2bfloat16_rn((float)v);
    lo = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hi)));
}

// ---------------------------------------------------------------------------
// Panel builder: one thread per (m, pair), FP64 recurrence with rescaling.
// deriv = 0: P_n^m; deriv = 1: dP = sin(theta) dP_n^m/dtheta = n x P_n - dc_n P_{n-1}
// (both factors carry the same scale, so the identity holds in scaled form).
// The panels must be zeroed beforehand; only non-zero entries are written.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128)
k_build_panels(PlanView<double> pv, const unsigned long long *__restrict__ off_s,
               const unsigned long long *__restrict__ off_a, unsigned char *__restrict__ ps,
               unsigned char *__restrict__ pa, int deriv)
{
    const int m = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int npairs = pv.npairs, lmax = pv.lmax;
    if (p >= npairs) return;
    const int mo = m * pv.mres;                      // the order of order index m
    const int L = lmax - mo + 1;
    const int Le = (L + 1) / 2;
    const int nch = (Le + kKc - 1) / kKc;            // synthesis chunks per tile
    const int kch = (npairs + kKc - 1) / kKc;        // analysis chunks (over pairs)
    const long col = col_of_mres(lmax, m, pv.mres);
    const double x = pv.x[p];
    double y2 = pv.pmm[(size_t)m * npairs + p], y1 = 0.0;
    int k = pv.pmmk[(size_t)m * npairs + p];
    const int t = p / kRows, row = p % kRows;
    unsigned char *sbase = ps + off_s[m] + ((size_t)t * nch) * kChunkPanel;
    const int kc = p / kKc, pc = p % kKc;
    unsigned char *abase = pa + off_a[m];
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
        if (k != 0) continue;
        const double P = deriv ? fma((double)(mo + nn) * x, y1, -pv.dc[col + nn] * y2) : y1;
        if (P == 0.0) continue;
        __nv_bfloat16 hi, lo;
        split_bf16_d(P, hi, lo);
        const int par = nn & 1, kk = nn >> 1;
        // synthesis panel: block (t, chunk kk/kKc, parity, hi|lo), element (row, kk%kKc)
        {
            unsigned char *b = sbase + (size_t)(kk / kKc) * kChunkPanel;
            *reinterpret_cast<__nv_bfloat16 *>(b + pan_off(par * 2, row, kk % kKc)) = hi;
            *reinterpret_cast<__nv_bfloat16 *>(b + pan_off(par * 2 + 1, row, kk % kKc)) = lo;
        }
        // analysis panel: block (M tile kk/128, pair chunk kc, parity, hi|lo), element (kk%128, pc)
        {
            const int mt = kk / kRows, r = kk % kRows;
            unsigned char *b = abase + ((size_t)mt * kch + kc) * kChunkPanel;
            *reinterpret_cast<__nv_bfloat16 *>(b + pan_off(par * 2, r, pc)) = hi;
            *reinterpret_cast<__nv_bfloat16 *>(b + pan_off(par * 2 + 1, r, pc)) = lo;
        }
    }
}

// ---------------------------------------------------------------------------
// Data operand: one chunk is [class][hi|lo] blocks of `rows` x kKc (rows a
// multiple of 32).  Synthesis chunk (m, c) holds degrees n - m in
// [2 kKc c, 2 kKc (c + 1)), class = parity of n - m; analysis chunk (m, kc)
// holds pairs [kKc kc, kKc (kc + 1)), class = fold (0: s, 1: d).
// Scalar rows: 2b + (re|im).  Vector rows: first quantity (S or theta)
// 2b + (re|im), second (T or phi) NH + 2b + (re|im), NH = rows / 2.
// Synthesis chunks are numbered from dchunk[m] per order; analysis chunks
// are m * kch + kc.
// ---------------------------------------------------------------------------
constexpr int kPrepThreads = 128;

// Packs 8 bf16 values into one 16-byte core-matrix row.
__device__ __forceinline__ uint4 pack8(const __nv_bfloat16 (&v)[8])
{
    uint4 r;
    r.x = (uint32_t)__bfloat16_as_ushort(v[0]) | ((uint32_t)__bfloat16_as_ushort(v[1]) << 16);
    r.y = (uint32_t)__bfloat16_as_ushort(v[2]) | ((uint32_t)__bfloat16_as_ushort(v[3]) << 16);
    r.z = (uint32_t)__bfloat16_as_ushort(v[4]) | ((uint32_t)__bfloat16_as_ushort(v[5]) << 16);
    r.w = (uint32_t)__bfloat16_as_ushort(v[6]) | ((uint32_t)__bfloat16_as_ushort(v[7]) << 16);
    return r;
}

// Writes the hi and lo rows of 8 consecutive K values of one operand row.
__device__ __forceinline__ void put_row8(unsigned char *bh, unsigned char *bl, int row, int h, const float (&v)[8])
{
    __nv_bfloat16 hv[8], lv[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) split_bf16(v[i], hv[i], lv[i]);
    const uint32_t o = blk_off(row, 8 * h);
    *reinterpret_cast<uint4 *>(bh + o) = pack8(hv);
    *reinterpret_cast<uint4 *>(bl + o) = pack8(lv);
}

// One thread per 8 consecutive K positions of one field (and quantity): it
// reads them (synthesis: 8 spectral coefficients of one parity; analysis: the
// s/d folds of 8 latitude pairs) and writes whole 16-byte core-matrix rows
// (re and im rows, hi and lo blocks).  The pad rows of the operand (fields
// beyond the batch) are left as they are: they only feed output columns that
// are never read.  grid = (ceil(max chunks * items / kPrepThreads), mmax + 1).
__global__ void __launch_bounds__(kPrepThreads)
k_tc_prep(int synth, int vec, int lmax, int mmax, int mres, int npairs, int nlm, int batch, int rows, int op,
          const float *__restrict__ in0, const float *__restrict__ in1, const unsigned long long *__restrict__ dchunk,
          unsigned char *__restrict__ data)
{
    const int m = blockIdx.y;   // order index: the order is m mres
    const int L = lmax - m * mres + 1, Le = (L + 1) / 2;
    const int nch = synth ? (Le + kKc - 1) / kKc : (npairs + kKc - 1) / kKc;
    const int nq = vec ? 2 : 1;
    // items per chunk: synthesis (quantity, field, parity, K half); analysis (quantity, field, K half)
    const int items = (synth ? 4 : 2) * batch * nq;
    const int gid = blockIdx.x * kPrepThreads + threadIdx.x;
    const int c = gid / items;
    if (c >= nch) return;
    int it = gid - c * items;
    const int h = it & 1;
    it >>= 1;
    const size_t db = data_chunk_bytes(rows);
    unsigned char *dat = data + (synth ? (dchunk[m] + c) : ((size_t)m * nch + c)) * db;
    const size_t blk = (size_t)rows * kKc * 2;
    const int NH = rows / 2;
    if (synth) {
        const int cls = it & 1;
        it >>= 1;
        const int b = it % batch, q = it / batch;
        const long col = col_of_mres(lmax, m, mres);
        const float2 *A = reinterpret_cast<const float2 *>(q ? in1 : in0) + (size_t)b * nlm + col;
        // adjoint of analysis: b / c_m (scalar) or b / (c_m n (n + 1)) (vector)
        const float cadj = (op == OP_ANALYS_ADJ && m > 0) ? 0.5f : 1.0f;
        float re[8], im[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int nn = 2 * (kKc * c + 8 * h + i) + cls;   // n - m
            float2 v = make_float2(0.f, 0.f);
            if (nn < L) v = A[nn];
            float sc = cadj;
            if (vec && op == OP_ANALYS_ADJ) {
                const int n = m * mres + nn;
                sc = (n == 0) ? 0.f : cadj / ((float)n * (float)(n + 1));
            }
            re[i] = v.x * sc;
            im[i] = m == 0 ? 0.f : v.y * sc;
        }
        unsigned char *bh = dat + (size_t)(cls * 2) * blk;
        const int r0 = q * NH + 2 * b;
        put_row8(bh, bh + blk, r0, h, re);
        put_row8(bh, bh + blk, r0 + 1, h, im);
    } else {
        const int b = it % batch, q = it / batch;
        const float4 *A = reinterpret_cast<const float4 *>(q ? in1 : in0) + ((size_t)b * (mmax + 1) + m) * npairs;
        float4 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int p = kKc * c + 8 * h + i;
            v[i] = p < npairs ? A[p] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const int r0 = q * NH + 2 * b;
        float t[8];
        // class 0: s folds (x: re, y: im); class 1: d folds (z: re, w: im)
#pragma unroll
        for (int i = 0; i < 8; ++i) t[i] = v[i].x;
        put_row8(dat, dat + blk, r0, h, t);
#pragma unroll
        for (int i = 0; i < 8; ++i) t[i] = v[i].y;
        put_row8(dat, dat + blk, r0 + 1, h, t);
#pragma unroll
        for (int i = 0; i < 8; ++i) t[i] = v[i].z;
        put_row8(dat + 2 * blk, dat + 3 * blk, r0, h, t);
#pragma unroll
        for (int i = 0; i < 8; ++i) t[i] = v[i].w;
        put_row8(dat + 2 * blk, dat + 3 * blk, r0 + 1, h, t);
    }
}

// ---------------------------------------------------------------------------
// Shared memory of the contraction kernels: a ring of S stages, each
// { NP panel chunks | data chunk }, then 2 S + 1 mbarriers and the TMEM slot.
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t stage_bytes_of(int npanels, int rows)
{
    return (size_t)npanels * kChunkPanel + data_chunk_bytes(rows);
}

__host__ __device__ inline size_t smem_bytes_of(int npanels, int rows, int stages)
{
    return 1024 + (size_t)stages * stage_bytes_of(npanels, rows) + 8 * (2 * stages + 2);
}

struct TcArgs {
    int lmax, mmax, npairs, nlm, batch, rows, ntiles, stages, op;
    int mres;                              // order stride: order index m is the order m mres
    int halves;                            // vector: field halves of kVecHalf per launch (CTA pairs)
    unsigned long long data_half;          // vector: bytes of one half's data operand
    const float *in;                       // raw FP32 s/d folds (warp-specialised analysis)
    int fused;                             // synthesis: spectra converted in the kernel (tensor map)
    const unsigned char *panel, *dpanel;   // dpanel: vector transforms only
    const unsigned long long *off;         // per-order panel byte offsets
    const int *c0;                         // per (m, tile): first chunk above the polar threshold
    const unsigned short *gf;              // per (m, tile, 8-row group): first chunk above it (or null)
    const unsigned char *data;             // data operand, blocked bf16 hi/lo
    const unsigned long long *dchunk;      // synthesis: first data chunk of each order
    float *out0, *out1;                    // outputs (vector: second quantity in out1)
    const float *st;                       // sin(theta) per pair (vector synthesis)
    const int *sched;                      // vector: work lists of the persistent CTAs (schedule_lpt)
    int *err;
};

// Common prologue: barriers, TMEM allocation.  Returns the TMEM base.
__device__ __forceinline__ uint32_t setup_ctas(int S, uint64_t *bar_load, uint64_t *bar_mma, uint64_t *bar_done,
                                               uint32_t *tslot, uint32_t ncols, int *s_ok)
{
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            tc::mbar_init(&bar_load[q], 1);
            tc::mbar_init(&bar_mma[q], 1);
        }
        tc::mbar_init(bar_done, 1);
        tc::mbar_fence_init();
        *s_ok = 1;
    }
    if ((tid >> 5) == 0) tc::tmem_alloc(tslot, ncols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    return *tslot;
}

// ---------------------------------------------------------------------------
// Warp-specialised panel contraction (the one the scalar transforms use).
// Warps 0-3 convert (analysis: the raw FP32 s/d folds of the chunk, brought in
// by bulk copy, into the blocked bf16 hi/lo operand) and run the epilogue;
// warp 4 lane 0 issues the MMAs; warp 5 streams the panel chunks and the data
// (synthesis: the prepped blocked chunk; analysis: the raw folds of all fields
// by one TMA tensor copy, fold_map).
// Stage: [panel chunk | blocked data | raw folds (analysis)].
// ---------------------------------------------------------------------------
constexpr int kWsThreads = 192;
constexpr int kWsCtasPerSm = 3;   // resident CTAs per SM: 3 x 3 stages beat 2 x 4
// Raw operand box per chunk: analysis kKc pairs (float4) per field; synthesis
// 2 kKc spectral coefficients (float2) per field plus one more, so that the
// box can start on a 16-byte boundary when the order's offset is odd.
constexpr int kSynthBoxFloats = 4 * kKc + 4;
__host__ __device__ inline size_t ws_raw_bytes(int batch, bool synth)
{
    return (size_t)batch * (synth ? kSynthBoxFloats * sizeof(float) : kKc * sizeof(float4));
}
// Stages are rounded up to 128 bytes: the TMA tensor copy into a stage's raw
// box needs a 128-byte aligned shared-memory destination.
__host__ __device__ inline size_t ws_stage_bytes(int rows, int batch, bool synth)
{
    return (kChunkPanel + data_chunk_bytes(rows) + ws_raw_bytes(batch, synth) + 127) & ~(size_t)127;
}
__host__ __device__ inline size_t ws_smem_bytes(int rows, int batch, int stages, bool synth)
{
    return 128 + (size_t)stages * ws_stage_bytes(rows, batch, synth) + 8 * (3 * stages + 2);
}

template <bool SYNTH>
__global__ void __launch_bounds__(kWsThreads, kWsCtasPerSm) k_tc_ws(TcArgs a, const __grid_constant__ CUtensorMap fold_map)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    const int S = a.stages, NC = a.rows;
    const size_t dbytes = data_chunk_bytes(NC);
    const size_t stage = ws_stage_bytes(NC, a.batch, SYNTH);
    const size_t blk = (size_t)NC * kKc * 2;
    uint64_t *bar_load = reinterpret_cast<uint64_t *>(smem + (size_t)S * stage);
    uint64_t *bar_conv = bar_load + S;
    uint64_t *bar_mma = bar_conv + S;
    uint64_t *bar_done = bar_mma + S;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_done + 1);
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int m = blockIdx.x / a.ntiles;
    const int tile = blockIdx.x - m * a.ntiles;
    const int lmax = a.lmax, npairs = a.npairs;
    const int L = lmax - m * a.mres + 1;   // m is the order index
    const int Le = (L + 1) / 2;
    const long col = col_of_mres(lmax, m, a.mres);
    if (!SYNTH && tile * kRows >= Le) return;
    const int nchunks = SYNTH ? (Le + kKc - 1) / kKc : (npairs + kKc - 1) / kKc;
    const unsigned char *panel = a.panel + a.off[m] + (size_t)tile * nchunks * kChunkPanel;
    const int cstart = a.c0 ? a.c0[m * a.ntiles + tile] : 0;
    const int nlive = nchunks - cstart;
    // wide: per parity, A_hi x [B_hi ; B_lo] as one MMA of N = 2 NC (columns
    // [hi.hi + lo.hi | hi.lo], summed by the epilogue) plus A_lo x B_hi, 4
    // MMAs per chunk; else 3 MMAs of N = NC per parity into NC columns
    const bool wide = 4 * NC <= 256;
    const int pcols = wide ? 2 * NC : NC;   // accumulator columns per parity
    const uint32_t ncols = 2 * pcols <= 64 ? 64 : (2 * pcols <= 128 ? 128 : (2 * pcols <= 256 ? 256 : 512));

    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            tc::mbar_init(&bar_load[q], 1);
            tc::mbar_init(&bar_conv[q], 4);
            tc::mbar_init(&bar_mma[q], 1);
        }
        tc::mbar_init(bar_done, 1);
        tc::mbar_fence_init();
        s_abort = 0;
    }
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    // Polar optimisation per 8-row group: a chunk's panel is copied from its
    // first group above the threshold, g0(c) = min{g : gf[g] <= c}, which never
    // grows with c.  Stage q first holds chunk cstart + q; its groups below that
    // chunk's g0 are zeroed once, and the later chunks of the stage write only
    // groups at or above their own (smaller or equal) g0, so the groups below it
    // stay zero and add nothing to the MMAs.
    const unsigned short *gf = a.gf ? a.gf + ((size_t)m * a.ntiles + tile) * (kRows / 8) : nullptr;
    if (gf) {
        for (int q = 0; q < min(S, nlive); ++q) {
            int g0 = 0;
            while (g0 < kRows / 8 && gf[g0] > cstart + q) ++g0;
            if (g0 == kRows / 8) g0 = 0;
            for (int w = tid; w < g0 * (int)(kPSbo / 16); w += kWsThreads)
                *reinterpret_cast<uint4 *>(smem + (size_t)q * stage + (size_t)w * 16) = make_uint4(0u, 0u, 0u, 0u);
        }
        tc::fence_proxy_async_smem();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp < 4) {
        // ---------------- converters ----------------
        if (SYNTH && a.fused) {
            // raw spectra of the chunk's 2 kKc degrees for every field -> blocked
            // hi/lo rows 2b (re), 2b + 1 (im), class = parity of n - m
            const int odd = (int)(col & 1);
            const float cadj = (a.op == OP_ANALYS_ADJ && m > 0) ? 0.5f : 1.0f;
            for (int u = 0; u < nlive; ++u) {
                const int q = u % S;
                const int c = cstart + u;
                if (!wait_or_abort(&bar_load[q], (uint32_t)((u / S) & 1), &s_abort)) break;
                unsigned char *st = smem + (size_t)q * stage;
                unsigned char *dat = st + kChunkPanel;
                const float *raw = reinterpret_cast<const float *>(dat + dbytes);
                // item = (field, parity class, pair of K positions 2 kp, 2 kp + 1):
                // two coefficients of the same parity, packed into 32-bit words
                for (int i = tid; i < a.batch * kKc; i += 128) {
                    const int b = i / kKc, r = i - b * kKc;
                    const int cls = r / (kKc / 2), kp = r - cls * (kKc / 2);
                    float re[2], im[2];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int j = 2 * (2 * kp + e) + cls;   // degree offset within the chunk
                        const int nn = 2 * kKc * c + j;
                        re[e] = im[e] = 0.f;
                        if (nn < L) {
                            const float *v = raw + (size_t)b * kSynthBoxFloats + 2 * (j + odd);
                            re[e] = v[0] * cadj;
                            im[e] = m == 0 ? 0.f : v[1] * cadj;
                        }
                    }
                    uint32_t rh, rl, ih, il;
                    split2(re[0], re[1], rh, rl);
                    split2(im[0], im[1], ih, il);
                    unsigned char *bh = dat + (size_t)(cls * 2) * blk;
                    *reinterpret_cast<uint32_t *>(bh + blk_off(2 * b, 2 * kp)) = rh;
                    *reinterpret_cast<uint32_t *>(bh + blk + blk_off(2 * b, 2 * kp)) = rl;
                    *reinterpret_cast<uint32_t *>(bh + blk_off(2 * b + 1, 2 * kp)) = ih;
                    *reinterpret_cast<uint32_t *>(bh + blk + blk_off(2 * b + 1, 2 * kp)) = il;
                }
                tc::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&bar_conv[q]);
            }
        }
        if (!SYNTH) {
            for (int u = 0; u < nlive; ++u) {
                const int q = u % S;
                const int c = cstart + u;
                if (!wait_or_abort(&bar_load[q], (uint32_t)((u / S) & 1), &s_abort)) break;
                unsigned char *st = smem + (size_t)q * stage;
                unsigned char *dat = st + kChunkPanel;
                const float4 *raw = reinterpret_cast<const float4 *>(dat + dbytes);
                const int np = min(kKc, npairs - kKc * c);
                // item = (field, pair of K positions 2 jp, 2 jp + 1): two pairs' folds
                // packed into 32-bit words per (fold, re|im, hi|lo)
                for (int i = tid; i < a.batch * (kKc / 2); i += 128) {
                    const int b = i / (kKc / 2), jp = i - b * (kKc / 2);
                    const int j0 = 2 * jp;
                    const float4 v0 = j0 < np ? raw[b * kKc + j0] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 v1 = j0 + 1 < np ? raw[b * kKc + j0 + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float a0[4] = {v0.x, v0.y, v0.z, v0.w};   // s.re s.im d.re d.im
                    const float a1[4] = {v1.x, v1.y, v1.z, v1.w};
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        uint32_t h, l;
                        split2(a0[t], a1[t], h, l);
                        const uint32_t o = blk_off(2 * b + (t & 1), j0);
                        unsigned char *bh = dat + (size_t)((t >> 1) * 2) * blk;
                        *reinterpret_cast<uint32_t *>(bh + o) = h;
                        *reinterpret_cast<uint32_t *>(bh + blk + o) = l;
                    }
                }
                tc::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&bar_conv[q]);
            }
        }
    } else if (warp == 4) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            const uint32_t idesc = tc::idesc_bf16_f32(kRows, NC);
            const uint32_t idesc2 = tc::idesc_bf16_f32(kRows, 2 * NC);
            uint64_t da0[2][2], db0[2][2];
#pragma unroll
            for (int par = 0; par < 2; ++par)
#pragma unroll
                for (int hl = 0; hl < 2; ++hl) {
                    da0[par][hl] = tc::smem_desc(smem + (size_t)(par * 2 + hl) * kSbo, kLbo, kPSbo);
                    db0[par][hl] = tc::smem_desc(smem + kChunkPanel + (size_t)(par * 2 + hl) * blk, kLbo, kSbo);
                }
            const uint64_t sstep = stage >> 4;
            bool ok = true;
            for (int u = 0; u < nlive; ++u) {
                const int q = u % S;
                if (!wait_or_abort(&bar_load[q], (uint32_t)((u / S) & 1), &s_abort)) { ok = false; break; }
                if ((!SYNTH || a.fused) && !wait_or_abort(&bar_conv[q], (uint32_t)((u / S) & 1), &s_abort)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const uint64_t so = sstep * (uint64_t)q;
                if (wide) {
                    // the blocked data holds B_lo right after B_hi: rows NC .. 2 NC - 1
#pragma unroll
                    for (int par = 0; par < 2; ++par) {
                        const uint32_t d = tmem + (uint32_t)(par * pcols);
                        tc::mma_bf16(d, da0[par][0] + so, db0[par][0] + so, idesc2, u != 0);
                        tc::mma_bf16(d, da0[par][1] + so, db0[par][0] + so, idesc, true);
                    }
                } else {
#pragma unroll
                    for (int par = 0; par < 2; ++par) {
                        const uint32_t d = tmem + (uint32_t)(par * pcols);
                        tc::mma_bf16(d, da0[par][0] + so, db0[par][0] + so, idesc, u != 0);
                        tc::mma_bf16(d, da0[par][0] + so, db0[par][1] + so, idesc, true);
                        tc::mma_bf16(d, da0[par][1] + so, db0[par][0] + so, idesc, true);
                    }
                }
                tc::mma_commit(&bar_mma[q]);
            }
            if (!ok) raise_err(a.err, SHT_ETIMEOUT);
            tc::mma_commit(bar_done);
        }
    } else {
        // ---------------- producer ----------------
        const unsigned char *data = a.data + (SYNTH ? a.dchunk[m] * dbytes : 0);
        const int rows_valid = SYNTH ? kRows : min(kRows, Le - kRows * tile);
        const uint32_t pgb = (uint32_t)((rows_valid + 7) / 8) * kPSbo;  // panel bytes up to the last used 8-row group
        // lane g < 16: first live chunk of 8-row group g
        const int gfl = (gf && lane < kRows / 8) ? (int)gf[lane] : 0;
        int issued = 0;
        bool ok = true;
        for (int u = 0; u < nlive; ++u) {
            const int q = u % S;
            const int c = cstart + u;
            if (lane == 0 && u >= S)
                ok = wait_or_abort(&bar_mma[q], (uint32_t)((u / S - 1) & 1), &s_abort);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) break;
            unsigned char *st = smem + (size_t)q * stage;
            const unsigned live = __ballot_sync(0xffffffffu, lane < kRows / 8 && gfl <= c);
            const uint32_t lo = min(live ? (uint32_t)(__ffs(live) - 1) * kPSbo : 0u, pgb);
            if (lane == 0) {
                // copied: the 8-row groups from g0(c) up to the last one holding
                // rows (analysis: the last degree tile of an order holds fewer
                // than 128 rows; the MMA rows above them read stale data and are
                // never written out)
                const uint32_t tx = (pgb - lo) + (uint32_t)(SYNTH && !a.fused ? dbytes : ws_raw_bytes(a.batch, SYNTH));
                tc::mbar_arrive_expect_tx(&bar_load[q], tx);
                if (pgb > lo) tc::bulk_g2s_stream(st + lo, panel + (size_t)c * kChunkPanel + lo, pgb - lo, &bar_load[q]);
                if (SYNTH && a.fused) {
                    // spectra of every field, degrees [2 kKc c, 2 kKc c + 2 kKc) of order
                    // m, from the 16-byte boundary at or below (one coefficient earlier
                    // when the order's offset is odd); degrees past the field arrive as zeros
                    const int x = 2 * (int)(col - (col & 1)) + 4 * kKc * c;
                    tc::tma_load_2d(st + kChunkPanel + dbytes, &fold_map, x, 0, &bar_load[q]);
                } else if (SYNTH) {
                    tc::bulk_g2s(st + kChunkPanel, data + (size_t)c * dbytes, (uint32_t)dbytes, &bar_load[q]);
                } else {
                    // raw folds of every field, pairs [kKc c, kKc c + kKc) of order m:
                    // one tensor copy of the box {4 kKc floats, 1 order, batch fields};
                    // pairs past npairs arrive as zeros
                    tc::tma_load_3d(st + kChunkPanel + dbytes, &fold_map, 4 * kKc * c, m, 0, &bar_load[q]);
                }
            }
            __syncwarp();
            issued = u + 1;
        }
        if (!ok && lane == 0) {
            raise_err(a.err, SHT_ETIMEOUT);
            for (int v = max(0, issued - S); v < issued; ++v)
                (void)tc::mbar_wait_bounded(&bar_load[v % S], (uint32_t)((v / S) & 1), 100000000ull);
        }
    }
    bool ok = true;
    if (warp < 4) {
        ok = wait_or_abort(bar_done, 0, &s_abort);
        if (!ok) {
            (void)tc::mbar_wait_bounded(bar_done, 0, 100000000ull);
            raise_err(a.err, SHT_ETIMEOUT);
        }
    }
    ok = __syncthreads_and(ok && !*(volatile int *)&s_abort);
    if (ok && warp < 4) {
        tc::tc_fence_after();
        const int row = tile * kRows + warp * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        for (int cb = 0; cb < NC; cb += 16) {
            float de[16], dd[16];
            if (nlive > 0) {
                tc::tmem_ld16(lane_base + (uint32_t)cb, de);
                tc::tmem_ld16(lane_base + (uint32_t)(pcols + cb), dd);
                if (wide) {
                    float t[16];
                    tc::tmem_ld16(lane_base + (uint32_t)(NC + cb), t);
#pragma unroll
                    for (int i = 0; i < 16; ++i) de[i] += t[i];
                    tc::tmem_ld16(lane_base + (uint32_t)(pcols + NC + cb), t);
#pragma unroll
                    for (int i = 0; i < 16; ++i) dd[i] += t[i];
                }
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) de[i] = dd[i] = 0.f;
            }
            for (int q = 0; q < 16; q += 2) {
                const int b = (cb + q) >> 1;
                if (b >= a.batch) break;
                if (SYNTH) {
                    if (row < npairs) {
                        float4 *eo = reinterpret_cast<float4 *>(a.out0);
                        eo[((size_t)b * (a.mmax + 1) + m) * npairs + row] = make_float4(de[q], de[q + 1], dd[q], dd[q + 1]);
                    }
                } else {
                    const int ne = 2 * row, no = 2 * row + 1;
                    const float sc = (a.op == OP_SYNTH_ADJ && m > 0) ? 2.f : 1.f;
                    float2 *spec = reinterpret_cast<float2 *>(a.out0);
                    if (ne < L) spec[(size_t)b * a.nlm + col + ne] = make_float2(sc * de[q], m == 0 ? 0.f : sc * de[q + 1]);
                    if (no < L) spec[(size_t)b * a.nlm + col + no] = make_float2(sc * dd[q], m == 0 ? 0.f : sc * dd[q + 1]);
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------
// Vector (spheroidal/toroidal) contraction.  dP = sin(theta) dP/dtheta has the
// mirror parity opposite to P.  Per order m and output class cls (0: E rows /
// even n - m, 1: O rows / odd n - m), with oth = 1 - cls:
//   synthesis  acc1 = P_cls [S|T]_cls,  acc2 = dP_oth [S|T]_oth
//     sin V_theta = acc2[S] - i m acc1[T],  sin V_phi = i m acc1[S] + acc2[T];
//   analysis   acc1 = P_cls^T [th|ph]_cls,  acc2 = dP_cls^T [th|ph]_oth
//     (data class 0: s folds, 1: d folds; the folds already carry 1/sin)
//     S_n = scale (acc2[th] - i m acc1[ph]),  T_n = scale (i m acc1[th] + acc2[ph]).
// Accumulators: [cls][acc][N columns], N = 2 NH (first | second quantity).
// ---------------------------------------------------------------------------
// Fields per CTA of the vector contraction (4 accumulators x 2 cols_of(32)
// columns fill the 512 TMEM columns).  A launch of up to 64 fields runs its
// field groups as adjacent CTAs of each (m, tile), so the later ones read the
// panel chunks the first brought into L2.
constexpr int kVecHalf = 32;

// Persistent: one CTA per SM walks its list of work items (order, tile,
// field half), the entries sched[gridDim.x + 1 + k] for k in
// [sched[blockIdx.x], sched[blockIdx.x + 1]) (schedule_lpt), with 192
// threads: warps 0-3 run the epilogue, warp 4 lane 0 issues the MMAs, warp 5
// lane 0 streams the P, dP and data chunks.  The ring of stages runs on across
// items, so the next item's chunks load while the epilogue drains the
// accumulators; the next item's MMAs start once the epilogue has read them.
template <bool SYNTH>
__global__ void __launch_bounds__(192, 1) k_tc_vec(TcArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int S = a.stages, NV = a.rows, NH = a.rows / 2;
    const size_t stage_bytes = stage_bytes_of(2, NV);
    const size_t blk = (size_t)NV * kKc * 2;
    uint64_t *bar_load = reinterpret_cast<uint64_t *>(smem + (size_t)S * stage_bytes);
    uint64_t *bar_mma = bar_load + S;
    uint64_t *bar_full = bar_mma + S;
    uint64_t *bar_free = bar_full + 1;
    uint64_t *bar_done = bar_free + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_done + 1);
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int k0 = a.sched[blockIdx.x], k1 = a.sched[blockIdx.x + 1];
    const int *items = a.sched + gridDim.x + 1;
    const uint32_t ncols = 4 * NV <= 256 ? 256 : 512;
    const int lmax = a.lmax, npairs = a.npairs;

    // item w: field half w % halves, then (order index, tile)
    struct Item {
        int m, tile, half, L, Le, nchunks, cstart, nlive;
        bool valid;
    };
    const auto item_of = [&](int w) {
        Item it;
        it.half = w % a.halves;
        const int mt = w / a.halves;
        it.m = mt / a.ntiles;
        it.tile = mt - it.m * a.ntiles;
        it.L = lmax - it.m * a.mres + 1;
        it.Le = (it.L + 1) / 2;
        it.valid = SYNTH || it.tile * kRows < it.Le;
        it.nchunks = SYNTH ? (it.Le + kKc - 1) / kKc : (npairs + kKc - 1) / kKc;
        it.cstart = it.valid && a.c0 ? a.c0[it.m * a.ntiles + it.tile] : 0;
        it.nlive = it.valid ? it.nchunks - it.cstart : 0;
        return it;
    };

    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            tc::mbar_init(&bar_load[q], 1);
            tc::mbar_init(&bar_mma[q], 1);
        }
        tc::mbar_init(bar_full, 1);
        tc::mbar_init(bar_free, 4);   // one arrival per epilogue warp
        tc::mbar_init(bar_done, 1);
        tc::mbar_fence_init();
        s_abort = 0;
    }
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 5) {
        if (lane == 0) {
            // ---------------- producer: P, dP and data chunks ----------------
            const uint32_t dbytes = (uint32_t)data_chunk_bytes(NV);
            bool ok = true;
            unsigned u = 0;
            for (int kk = k0; ok && kk < k1; ++kk) {
                const Item it = item_of(items[kk]);
                if (!it.valid) continue;
                const size_t poff = a.off[it.m] + (size_t)it.tile * it.nchunks * kChunkPanel;
                const unsigned char *p0 = a.panel + poff, *p1 = a.dpanel + poff;
                const unsigned char *data =
                    a.data + (size_t)it.half * a.data_half +
                    (SYNTH ? a.dchunk[it.m] : (unsigned long long)it.m * it.nchunks) * data_chunk_bytes(NV);
                // panel bytes up to the last 8-row group holding a pair (synthesis) or
                // a degree (analysis); the MMA rows above read stale data and are never
                // written out
                const int rows_valid = min(kRows, (SYNTH ? npairs : it.Le) - kRows * it.tile);
                const uint32_t pgb = (uint32_t)((rows_valid + 7) / 8) * kPSbo;
                for (int c = it.cstart; c < it.nchunks; ++c, ++u) {
                    const unsigned q = u % S;
                    if (u >= (unsigned)S && !wait_or_abort(&bar_mma[q], (u / S - 1) & 1, &s_abort)) {
                        ok = false;
                        break;
                    }
                    unsigned char *st = smem + (size_t)q * stage_bytes;
                    tc::mbar_arrive_expect_tx(&bar_load[q], 2u * pgb + dbytes);
                    if (it.half == a.halves - 1) {
                        // the tile's last use of these panel chunks: evict them first
                        tc::bulk_g2s_stream(st, p0 + (size_t)c * kChunkPanel, pgb, &bar_load[q]);
                        tc::bulk_g2s_stream(st + kChunkPanel, p1 + (size_t)c * kChunkPanel, pgb, &bar_load[q]);
                    } else {
                        // the next field half of the tile reads them again, from L2
                        tc::bulk_g2s(st, p0 + (size_t)c * kChunkPanel, pgb, &bar_load[q]);
                        tc::bulk_g2s(st + kChunkPanel, p1 + (size_t)c * kChunkPanel, pgb, &bar_load[q]);
                    }
                    tc::bulk_g2s(st + 2 * kChunkPanel, data + (size_t)c * dbytes, dbytes, &bar_load[q]);
                }
            }
            if (!ok) {
                raise_err(a.err, SHT_ETIMEOUT);
                for (unsigned v = u > (unsigned)S ? u - S : 0; v < u; ++v)
                    (void)tc::mbar_wait_bounded(&bar_load[v % S], (v / S) & 1, 100000000ull);
            }
        }
    } else if (warp == 4) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            const uint32_t idesc = tc::idesc_bf16_f32(kRows, NV);
            bool ok = true;
            unsigned u = 0, j = 0;
            for (int kk = k0; ok && kk < k1; ++kk) {
                const Item it = item_of(items[kk]);
                if (!it.valid) continue;
                if (j >= 1 && !wait_or_abort(bar_free, (j - 1) & 1, &s_abort)) { ok = false; break; }
                tc::tc_fence_after();
                for (int c = 0; c < it.nlive; ++c, ++u) {
                    const unsigned q = u % S;
                    if (!wait_or_abort(&bar_load[q], (u / S) & 1, &s_abort)) { ok = false; break; }
                    tc::tc_fence_after();
                    unsigned char *st = smem + (size_t)q * stage_bytes;
                    unsigned char *dat = st + 2 * kChunkPanel;
                    const bool first = c == 0;   // the item's first chunk overwrites the accumulators
#pragma unroll
                    for (int cls = 0; cls < 2; ++cls) {
                        const int dp = SYNTH ? 1 - cls : cls;   // parity of n - m of the dP block
                        const unsigned char *aph = st + (size_t)(cls * 2) * kSbo, *apl = aph + kSbo;
                        const unsigned char *adh = st + kChunkPanel + (size_t)(dp * 2) * kSbo, *adl = adh + kSbo;
                        const unsigned char *b1h = dat + (size_t)(cls * 2) * blk, *b1l = b1h + blk;
                        const unsigned char *b2h = dat + (size_t)((1 - cls) * 2) * blk, *b2l = b2h + blk;
                        const uint32_t d1 = tmem + (uint32_t)((cls * 2 + 0) * NV);
                        const uint32_t d2 = tmem + (uint32_t)((cls * 2 + 1) * NV);
                        const uint64_t Aph = tc::smem_desc(aph, kLbo, kPSbo), Apl = tc::smem_desc(apl, kLbo, kPSbo);
                        const uint64_t Adh = tc::smem_desc(adh, kLbo, kPSbo), Adl = tc::smem_desc(adl, kLbo, kPSbo);
                        const uint64_t B1h = tc::smem_desc(b1h, kLbo, kSbo), B1l = tc::smem_desc(b1l, kLbo, kSbo);
                        const uint64_t B2h = tc::smem_desc(b2h, kLbo, kSbo), B2l = tc::smem_desc(b2l, kLbo, kSbo);
                        tc::mma_bf16(d1, Aph, B1h, idesc, !first);
                        tc::mma_bf16(d1, Aph, B1l, idesc, true);
                        tc::mma_bf16(d1, Apl, B1h, idesc, true);
                        tc::mma_bf16(d2, Adh, B2h, idesc, !first);
                        tc::mma_bf16(d2, Adh, B2l, idesc, true);
                        tc::mma_bf16(d2, Adl, B2h, idesc, true);
                    }
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
    } else {
        // ---------------- epilogue (warps 0-3: TMEM lanes 32 warp ..) ----------------
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        unsigned j = 0;
        for (int kk = k0; kk < k1; ++kk) {
            const Item it = item_of(items[kk]);
            if (!it.valid) continue;
            if (!wait_or_abort(bar_full, j & 1, &s_abort)) {
                raise_err(a.err, SHT_ETIMEOUT);
                break;
            }
            tc::tc_fence_after();
            ++j;
            const int m = it.m, L = it.L;
            const long col = col_of_mres(lmax, m, a.mres);
            const int fb0 = it.half * kVecHalf, nbh = min(kVecHalf, a.batch - fb0);
            const int row = it.tile * kRows + warp * 32 + lane;
            const float fm = (float)(m * a.mres);
            float isn = 1.f;
            if (SYNTH && row < npairs) isn = 1.f / a.st[row];
            for (int cls = 0; cls < 2; ++cls) {
                for (int cb = 0; cb < NH; cb += 32) {
                    float v[2][2][32];  // [acc][first|second quantity][col]
#pragma unroll
                    for (int ac = 0; ac < 2; ++ac)
#pragma unroll
                        for (int hf = 0; hf < 2; ++hf) {
                            if (it.nlive > 0) {
                                tc::tmem_ld32(lane_base + (uint32_t)((cls * 2 + ac) * NV + hf * NH + cb), v[ac][hf]);
                            } else {
#pragma unroll
                                for (int i = 0; i < 32; ++i) v[ac][hf][i] = 0.f;
                            }
                        }
                    if (cls == 1 && cb + 32 >= NH) {
                        // the accumulators are read: the next item's MMAs may overwrite them
                        tc::tc_fence_before();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(bar_free);
                    }
                    for (int q = 0; q < 32; q += 2) {
                        const int bl = (cb + q) >> 1;   // field within the half
                        if (bl >= nbh) break;
                        const int b = fb0 + bl;
                        if (SYNTH) {
                            if (row >= npairs) continue;
                            const float psr = v[0][0][q], psi = v[0][0][q + 1];   // sum P S
                            const float ptr = v[0][1][q], pti = v[0][1][q + 1];   // sum P T
                            const float dsr = v[1][0][q], dsi = v[1][0][q + 1];   // sum dP S
                            const float dtr = v[1][1][q], dti = v[1][1][q + 1];   // sum dP T
                            const size_t oi = (((size_t)b * (a.mmax + 1) + m) * npairs + row) * 2 + cls;
                            reinterpret_cast<float2 *>(a.out0)[oi] =
                                make_float2((dsr + fm * pti) * isn, (dsi - fm * ptr) * isn);
                            reinterpret_cast<float2 *>(a.out1)[oi] =
                                make_float2((dtr - fm * psi) * isn, (dti + fm * psr) * isn);
                        } else {
                            const int nn = 2 * row + cls;
                            if (nn >= L) continue;
                            const int n = m * a.mres + nn;
                            float sc;
                            if (a.op == OP_SYNTH_ADJ) sc = (m > 0) ? 2.f : 1.f;
                            else sc = (n == 0) ? 0.f : 1.f / ((float)n * (float)(n + 1));
                            const float pthr = v[0][0][q], pthi = v[0][0][q + 1];   // P^T theta folds
                            const float pphr = v[0][1][q], pphi = v[0][1][q + 1];   // P^T phi folds
                            const float dthr = v[1][0][q], dthi = v[1][0][q + 1];   // dP^T theta folds
                            const float dphr = v[1][1][q], dphi = v[1][1][q + 1];   // dP^T phi folds
                            float2 sv = make_float2(sc * (dthr + fm * pphi), sc * (dthi - fm * pphr));
                            float2 tv = make_float2(sc * (dphr - fm * pthi), sc * (dphi + fm * pthr));
                            if (m == 0) {
                                sv.y = 0.f;
                                tv.y = 0.f;
                            }
                            reinterpret_cast<float2 *>(a.out0)[(size_t)b * a.nlm + col + nn] = sv;
                            reinterpret_cast<float2 *>(a.out1)[(size_t)b * a.nlm + col + nn] = tv;
                        }
                    }
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------
// On-the-fly P_n^m for the contraction (mode SHT_TC_OTF): instead of streaming
// precomputed panels from HBM, four warps run the recurrence of Sec. 3.2 in
// FP32 and write the bf16 hi/lo operand straight into shared memory -- the
// on-the-fly variant of Sec. 3.1 feeding the tensor cores.  The FP32
// recurrence restarts every kSeg degrees from a seed computed once per plan
// by the FP64 recurrence with the rescaling of Sec. 3.5, so its rounding
// errors grow over at most kSeg steps instead of N.
//
// Seed (m, segment s, pair p), s covering n - m in [kSeg s, kSeg s + kSeg):
// the recurrence state entering the segment, (P_{n0-1}, P_{n0-2}) at
// n0 = m + kSeg s ((0, P_m^m) for s = 0), as FP32 (y1, y2) times a power of
// two 2^E held as the FP32 value `scale` (0 when 2^E is below the FP32
// range), E the exponent of the largest |P_n^m| of the segment, and the
// pair's FP32 cos(theta): float4 (y1, y2, scale, x).
// ---------------------------------------------------------------------------
constexpr int kSeg = 2 * kKc;                // degrees per segment = one synthesis chunk
constexpr int kSegPerTile = 2 * kRows / kSeg; // segments per analysis tile (128 rows per parity)
constexpr int kOtfGrowthLog2 = 120;           // largest growth within a segment (FP32 range of the seed)

// One thread per (m, pair).  Also records, for the polar optimisation, the
// first live synthesis chunk of each (m, pair tile) and the first live pair
// chunk of each (m, degree tile) (atomicMin into tables initialised to the
// chunk counts), and sets *flag when a seed would fall below the FP32 range
// (a segment growing by more than 2^120).
__global__ void __launch_bounds__(128)
k_build_seeds(PlanView<double> pv, const unsigned long long *__restrict__ segoff, float4 *__restrict__ seeds,
              float thr, int *__restrict__ c0s, int *__restrict__ c0a, int ntiles_s, int ntiles_a,
              int *__restrict__ flag)
{
    const int m = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int npairs = pv.npairs, lmax = pv.lmax;
    if (p >= npairs) return;
    const int L = lmax - m * pv.mres + 1;   // m is the order index
    const int nseg = (L + kSeg - 1) / kSeg;
    const long col = col_of_mres(lmax, m, pv.mres);
    const double x = pv.x[p];
    double y2 = pv.pmm[(size_t)m * npairs + p], y1 = 0.0;
    int k = pv.pmmk[(size_t)m * npairs + p];
    int first_s = nseg;
    bool tile_live = false;
    bool underflow = false;
    for (int s = 0; s < nseg; ++s) {
        // state entering the segment
        const double s1 = y1, s2 = y2;
        const int sk = k;
        // run the segment: largest exponent of its values, liveness
        int emax = INT_MIN;
        bool live = false;
        for (int i = 0; i < kSeg; ++i) {
            const int nn = kSeg * s + i;
            if (nn >= L) break;
            const double2 ab = pv.ab[col + nn];
            const double yn = fma(ab.x * x, y1, ab.y * y2);
            y2 = y1;
            y1 = yn;
            if (k > 0 && fabs(yn) >= 1.0) {
                y1 *= 0x1p-240;
                y2 *= 0x1p-240;
                k -= 1;
            }
            if (y1 != 0.0) emax = max(emax, ilogb(y1) - Scale<double>::S * k);
            if ((k == 0 && fabs(y1) >= (double)thr) || thr == 0.f) live = true;
        }
        // seed normalised so that the largest value of the segment is in [1, 2):
        // the FP32 chain then stays below 2 and the seed, at most ~2^116 smaller
        // at lmax = 1023, stays a normal FP32 number
        float4 sd = make_float4(0.f, 0.f, 0.f, 0.f);
        if (emax != INT_MIN) {
            const int sh = -Scale<double>::S * sk - emax;   // true value * 2^-emax = y * 2^sh
            const double t1 = scalbn(s1, sh), t2 = scalbn(s2, sh);
            sd.x = (float)t1;
            sd.y = (float)t2;
            sd.z = emax >= -149 ? scalbnf(1.0f, emax) : 0.0f;
            const double tmax = fmax(fabs(t1), fabs(t2));
            if (tmax > 0.0 && ilogb(tmax) < -kOtfGrowthLog2) underflow = true;
        }
        sd.w = (float)x;
        seeds[(segoff[m] + s) * npairs + p] = sd;
        if (live && first_s == nseg) first_s = s;
        tile_live |= live;
        // end of a degree tile of the analysis: record this pair's chunk if live
        if ((s + 1) % kSegPerTile == 0 || s + 1 == nseg) {
            if (tile_live) atomicMin(&c0a[m * ntiles_a + s / kSegPerTile], p / kKc);
            tile_live = false;
        }
    }
    atomicMin(&c0s[m * ntiles_s + p / kRows], first_s);
    if (underflow) atomicOr(flag, 1);
}

// c0 tables before k_build_seeds: the chunk counts (nothing live).
__global__ void k_init_c0(int lmax, int mmax, int mres, int npairs, int ntiles_s, int ntiles_a, int *c0s, int *c0a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = i / (ntiles_s + ntiles_a);
    if (m > mmax) return;
    const int t = i - m * (ntiles_s + ntiles_a);
    const int Le = (lmax - m * mres + 2) / 2;
    if (t < ntiles_s) c0s[m * ntiles_s + t] = (Le + kKc - 1) / kKc;
    else c0a[m * ntiles_a + (t - ntiles_s)] = (npairs + kKc - 1) / kKc;
}

struct OtfArgs {
    int lmax, mmax, npairs, nlm, batch, rows, ntiles, stages, op, nab;
    int mres;                           // order stride: order index m is the order m mres
    const float4 *seeds;
    const unsigned long long *segoff;   // first segment (= synthesis data chunk) of each order
    const int *c0;                      // per (m, tile): first live chunk
    const float2 *ab;                   // FP32 recurrence coefficients (a, b) per packed index
    const float *x;                     // FP32 cos(theta) per pair
    const unsigned char *data;          // data operand, blocked bf16 hi/lo
    float *out;
    int *err;
};

// Shared memory of the on-the-fly kernels: SA operand stages of kChunkPanel
// bytes, SD data stages (data chunk + one seed per generator thread), the
// (a, b) table, 2 SA + 2 SD + 1 mbarriers and the TMEM slot.
constexpr size_t kOtfSeedBytes = kRows * sizeof(float4);
__host__ __device__ inline size_t otf_dstage_bytes(int rows) { return data_chunk_bytes(rows) + kOtfSeedBytes; }
// Synthesis keeps its operand stages in tensor memory (A from TMEM), analysis
// in shared memory.
__host__ __device__ inline size_t otf_smem_bytes(int rows, int sa, int sd, int nab, bool synth)
{
    return 1024 + (synth ? 0 : (size_t)sa * kChunkPanel) + (size_t)sd * otf_dstage_bytes(rows) +
           (size_t)nab * sizeof(float2) + 8 * (2 * sa + 2 * sd + 2);
}

// TMEM columns: accumulators [0, 4 rows) (per parity: hi (x) [data hi | data
// lo] in 2 rows columns), then (synthesis) SA operand stages of 4 blocks x
// kKc / 2 columns (M = 128 rows in the lanes, two bf16 per column).
__host__ __device__ inline uint32_t otf_tmem_cols(int rows, int sa, bool synth)
{
    const int need = 4 * rows + (synth ? sa * 4 * (kKc / 2) : 0);
    return need <= 64 ? 64 : need <= 128 ? 128 : need <= 256 ? 256 : 512;
}

// Threads of the on-the-fly kernel: two groups of 4 generator warps (group g
// generates the chunks u with u % 2 == g) and one producer / MMA warp.
constexpr int kOtfGroups = 2;
constexpr int kOtfThreads = 32 * (4 * kOtfGroups + 2);   // + MMA warp + producer warp

// kSeg steps of the FP32 recurrence from a seed (y1, y2, scale, x); P = y *
// scale split into bf16 hi/lo and packed per parity: w[par][j] holds the
// values of parity par at K positions 2j and 2j + 1 (j < kKc / 2).
__device__ __forceinline__ void otf_segment(const float2 *__restrict__ ab, float4 sd, uint32_t (&hw)[2][kKc / 2],
                                            uint32_t (&lw)[2][kKc / 2])
{
    float y1 = sd.x, y2 = sd.y;
    const float sc = sd.z, x = sd.w;
#pragma unroll
    for (int j = 0; j < kKc / 2; ++j) {
        float P[4];   // degrees 4j .. 4j + 3: (par 0, k 2j), (par 1, k 2j), (par 0, k 2j+1), (par 1, k 2j+1)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 c = ab[4 * j + i];
            const float yn = fmaf(c.x * x, y1, c.y * y2);
            y2 = y1;
            y1 = yn;
            P[i] = yn * sc;
        }
        split2(P[0], P[2], hw[0][j], lw[0][j]);
        split2(P[1], P[3], hw[1][j], lw[1][j]);
    }
}

// Writes one generator thread's packed words into an operand stage.
template <bool SYNTH>
__device__ __forceinline__ void otf_store(unsigned char *st, int tid, const uint32_t (&hw)[2][kKc / 2],
                                          const uint32_t (&lw)[2][kKc / 2])
{
#pragma unroll
    for (int par = 0; par < 2; ++par) {
        unsigned char *bh = st + (size_t)(par * 2) * kBlk, *bl = bh + kBlk;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t off;
            if (SYNTH) {
                off = blk_off(tid, 8 * h);   // row = pair, K = degrees of this parity
            } else {
                // MN-major: 8 degrees contiguous per pair; core matrices 128 B
                // apart along the degrees, 2 KB apart along the pairs
                const int kr = 2 * (tid / kKc) + h;
                const int j = tid % kKc;
                off = (uint32_t)(kr * 128 + (j >> 3) * 2048 + (j & 7) * 16);
            }
            *reinterpret_cast<uint4 *>(bh + off) =
                make_uint4(hw[par][4 * h], hw[par][4 * h + 1], hw[par][4 * h + 2], hw[par][4 * h + 3]);
            *reinterpret_cast<uint4 *>(bl + off) =
                make_uint4(lw[par][4 * h], lw[par][4 * h + 1], lw[par][4 * h + 2], lw[par][4 * h + 3]);
        }
    }
}

// The contraction with on-the-fly P.  Warps 0-7 generate the operand (two
// groups of four, alternate chunks; group 0 also runs the epilogue); warp 8
// lane 0 issues the MMAs; warp 9 lane 0 streams the data chunks and their
// seeds, up to SD chunks ahead of the MMAs.  Synthesis writes its operand
// into tensor memory (tcgen05.st; the MMA reads A from TMEM), analysis into
// shared memory.  Synthesis: CTA
// (m, 128-pair tile), chunk = 32 degrees, generator thread = pair row, operand
// K-major.  Analysis: CTA (m, 128-row degree tile per parity), chunk = 16
// pairs, generator thread = (degree segment of the tile, pair), operand
// MN-major (degrees contiguous).
// Barriers: bar_load[SD] (data + seeds arrived), bar_dfree[SD] (MMAs that read
// the data stage done), bar_gen[SA] (operand written, 4 warp arrivals),
// bar_mma[SA] (MMAs that read the operand stage done), bar_done.
template <bool SYNTH>
__global__ void __launch_bounds__(kOtfThreads, 2) k_tc_otf(OtfArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int SA = a.stages & 0xff, SD = a.stages >> 8, NC = a.rows;
    const size_t dbytes = data_chunk_bytes(NC);
    const size_t dstage = otf_dstage_bytes(NC);
    const size_t blk = (size_t)NC * kKc * 2;
    unsigned char *opnd = smem;                                  // analysis: SA x kChunkPanel
    unsigned char *dst = opnd + (SYNTH ? 0 : (size_t)SA * kChunkPanel);   // SD x (data | seeds)
    float2 *ab_s = reinterpret_cast<float2 *>(dst + (size_t)SD * dstage);
    uint64_t *bar_load = reinterpret_cast<uint64_t *>(ab_s + a.nab);
    uint64_t *bar_dfree = bar_load + SD;
    uint64_t *bar_gen = bar_dfree + SD;
    uint64_t *bar_mma = bar_gen + SA;
    uint64_t *bar_done = bar_mma + SA;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_done + 1);
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int m = blockIdx.x / a.ntiles;
    const int tile = blockIdx.x - m * a.ntiles;
    const int lmax = a.lmax, npairs = a.npairs;
    const int L = lmax - m * a.mres + 1;   // m is the order index
    const int Le = (L + 1) / 2;
    const long col = col_of_mres(lmax, m, a.mres);
    if (!SYNTH && tile * kRows >= Le) return;
    const int nseg = (L + kSeg - 1) / kSeg;
    const int kch = (npairs + kKc - 1) / kKc;
    const int nchunks = SYNTH ? nseg : kch;
    const int cstart = a.c0[m * a.ntiles + tile];
    const int nlive = nchunks - cstart;
    const uint32_t ncols = otf_tmem_cols(NC, SA, SYNTH);
    // degrees held in the (a, b) table: the whole order (synthesis) or the tile (analysis)
    const int nn_base = SYNTH ? 0 : 2 * kRows * tile;

    const unsigned char *data = a.data + (SYNTH ? a.segoff[m] : (unsigned long long)m * kch) * dbytes;
    // data chunk + seeds of chunk un into data stage un % SD (producer thread only)
    auto issue = [&](int un) {
        const int sn = un % SD;
        const int c = cstart + un;
        unsigned char *ds = dst + (size_t)sn * dstage;
        float4 *sd = reinterpret_cast<float4 *>(ds + dbytes);
        // seed runs: synthesis one run of the tile's pairs; analysis one run
        // of the chunk's pairs per segment of the tile
        int np, ns;
        if (SYNTH) {
            np = min(kRows, npairs - tile * kRows);
            ns = 1;
        } else {
            np = min(kKc, npairs - kKc * c);
            ns = min(kSegPerTile, nseg - kSegPerTile * tile);
        }
        const uint32_t sbytes = (uint32_t)(np * ns) * (uint32_t)sizeof(float4);
        tc::mbar_arrive_expect_tx(&bar_load[sn], (uint32_t)dbytes + sbytes);
        tc::bulk_g2s(ds, data + (size_t)c * dbytes, (uint32_t)dbytes, &bar_load[sn]);
        if (SYNTH) {
            tc::bulk_g2s(sd, a.seeds + (a.segoff[m] + c) * npairs + tile * kRows, sbytes, &bar_load[sn]);
        } else {
            for (int sg = 0; sg < ns; ++sg)
                tc::bulk_g2s(sd + sg * kKc, a.seeds + (a.segoff[m] + kSegPerTile * tile + sg) * npairs + kKc * c,
                             (uint32_t)np * (uint32_t)sizeof(float4), &bar_load[sn]);
        }
    };
    // the producer fills all SD data stages ahead; a stage is refilled once the
    // MMAs of the chunk that last used it are done
    const int DD = SD;
    if (tid == 32 * (4 * kOtfGroups + 1)) {   // the producer thread
        for (int q = 0; q < SD; ++q) {
            tc::mbar_init(&bar_load[q], 1);
            tc::mbar_init(&bar_dfree[q], 1);
        }
        for (int q = 0; q < SA; ++q) {
            tc::mbar_init(&bar_gen[q], 4);
            tc::mbar_init(&bar_mma[q], 1);
        }
        tc::mbar_init(bar_done, 1);
        tc::mbar_fence_init();
        s_abort = 0;
        for (int u = 0; u < DD && u < nlive; ++u) issue(u);   // overlaps the table load below
    }
    {
        // (a, b) of the degrees this CTA needs: loads first, then stores
        constexpr int kAbIter = 4;   // nab <= kAbIter * kOtfThreads
        float2 v[kAbIter];
#pragma unroll
        for (int k = 0; k < kAbIter; ++k) {
            const int i = tid + k * kOtfThreads, nn = nn_base + i;
            v[k] = (i < a.nab && nn < L) ? a.ab[col + nn] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < kAbIter; ++k) {
            const int i = tid + k * kOtfThreads;
            if (i < a.nab) ab_s[i] = v[k];
        }
    }
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp < 4 * kOtfGroups) {
        // ---------------- operand generators ----------------
        // group g generates chunks u = g, g + 2, ...; thread r = row within the
        // group; seed slot: synthesis = pair row, analysis = segment * kKc + pair
        const int g = warp / 4, r = tid - 128 * g;
        for (int u = g; u < nlive; u += kOtfGroups) {
            const int qa = u % SA, qd = u % SD;
            const int c = cstart + u;
            if (u >= SA && !wait_or_abort(&bar_mma[qa], (uint32_t)((u / SA - 1) & 1), &s_abort)) break;
            if (!wait_or_abort(&bar_load[qd], (uint32_t)((u / SD) & 1), &s_abort)) break;
            int pp, ss;
            if (SYNTH) {
                pp = tile * kRows + r;
                ss = c;
            } else {
                pp = kKc * c + r % kKc;
                ss = kSegPerTile * tile + r / kKc;
            }
            float4 sd = reinterpret_cast<const float4 *>(dst + (size_t)qd * dstage + dbytes)[r];
            if (pp >= npairs || ss >= nseg) sd = make_float4(0.f, 0.f, 0.f, 0.f);
            uint32_t hw[2][kKc / 2], lw[2][kKc / 2];
            otf_segment(ab_s + (SYNTH ? kSeg * c : kSeg * (r / kKc)), sd, hw, lw);
            if (SYNTH) {
                // row r of the operand = TMEM lane r: block (par, hi|lo) of stage qa
                tc::tc_fence_after();   // after the wait on the MMAs that read this stage
                const uint32_t ta = tmem + ((uint32_t)(32 * (warp % 4)) << 16) + (uint32_t)(4 * NC + 32 * qa);
                tc::tmem_st8(ta, hw[0]);
                tc::tmem_st8(ta + 8, lw[0]);
                tc::tmem_st8(ta + 16, hw[1]);
                tc::tmem_st8(ta + 24, lw[1]);
                tc::tmem_wait_st();
                tc::tc_fence_before();
            } else {
                otf_store<SYNTH>(opnd + (size_t)qa * kChunkPanel, r, hw, lw);
                tc::fence_proxy_async_smem();
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&bar_gen[qa]);
        }
    } else if (warp == 4 * kOtfGroups && lane == 0) {
        // ---------------- MMA issuer ----------------
        // descriptors of stage 0; a stage adds its byte offset / 16 to the
        // start-address field (stage offsets stay far below the 256 KB field)
        // per parity two MMAs: P_hi x [data_hi ; data_lo] (N = 2 NC: the hi and lo
        // blocks are adjacent, one 2 NC-row operand) and P_lo x data_hi (N = NC),
        // both into the parity's accumulator; the epilogue adds its two halves
        const uint32_t idesc2 = tc::idesc_bf16_f32(kRows, 2 * NC, !SYNTH);
        const uint32_t idesc1 = tc::idesc_bf16_f32(kRows, NC, !SYNTH);
        uint64_t da0[2][2], db0[2][2];
#pragma unroll
        for (int par = 0; par < 2; ++par)
#pragma unroll
            for (int hl = 0; hl < 2; ++hl) {
                const unsigned char *ap = opnd + (size_t)(par * 2 + hl) * kBlk;
                da0[par][hl] = SYNTH ? tc::smem_desc(ap, kLbo, kSbo) : tc::smem_desc(ap, 2048, 128);
                db0[par][hl] = tc::smem_desc(dst + (size_t)(par * 2 + hl) * blk, kLbo, kSbo);
            }
        const uint64_t astep = kChunkPanel >> 4, dstep = dstage >> 4;
        bool ok = true;
        for (int u = 0; u < nlive; ++u) {
            const int qa = u % SA, qd = u % SD;
            if (!wait_or_abort(&bar_load[qd], (uint32_t)((u / SD) & 1), &s_abort)) { ok = false; break; }
            if (!wait_or_abort(&bar_gen[qa], (uint32_t)((u / SA) & 1), &s_abort)) { ok = false; break; }
            tc::tc_fence_after();
            const uint64_t ao = astep * (uint64_t)qa, bo = dstep * (uint64_t)qd;
#pragma unroll
            for (int par = 0; par < 2; ++par) {
                const uint32_t d = tmem + (uint32_t)(par * 2 * NC);
                if (SYNTH) {
                    const uint32_t ah = tmem + (uint32_t)(4 * NC + 32 * qa + 16 * par), al = ah + 8;
                    tc::mma_bf16_ts(d, ah, db0[par][0] + bo, idesc2, u != 0);
                    tc::mma_bf16_ts(d, al, db0[par][0] + bo, idesc1, true);
                } else {
                    tc::mma_bf16(d, da0[par][0] + ao, db0[par][0] + bo, idesc2, u != 0);
                    tc::mma_bf16(d, da0[par][1] + ao, db0[par][0] + bo, idesc1, true);
                }
            }
            tc::mma_commit(&bar_mma[qa]);
            tc::mma_commit(&bar_dfree[qd]);
        }
        if (!ok) raise_err(a.err, SHT_ETIMEOUT);
        tc::mma_commit(bar_done);
    } else if (warp == 4 * kOtfGroups + 1 && lane == 0) {
        // ---------------- data producer ----------------
        // refills data stage un % SD once the MMAs of chunk un - SD are done
        int issued_upto = min(DD, nlive);   // chunks 0 .. issued_upto - 1 already issued
        bool ok = true;
        for (int un = issued_upto; un < nlive; ++un) {
            if (un >= SD) {
                const int up = un - SD;
                if (!wait_or_abort(&bar_dfree[up % SD], (uint32_t)((up / SD) & 1), &s_abort)) { ok = false; break; }
            }
            issue(un);
            issued_upto = un + 1;
        }
        if (!ok) {
            raise_err(a.err, SHT_ETIMEOUT);
            // wait (bounded) for this CTA's own copies in flight: the last
            // chunk issued to each data stage
            for (int v = max(0, issued_upto - SD); v < issued_upto; ++v)
                (void)tc::mbar_wait_bounded(&bar_load[v % SD], (uint32_t)((v / SD) & 1), 100000000ull);
        }
    }
    bool ok = true;
    if (warp < 4 * kOtfGroups) {
        ok = wait_or_abort(bar_done, 0, &s_abort);
        if (!ok) {
            (void)tc::mbar_wait_bounded(bar_done, 0, 100000000ull);   // MMAs in flight
            raise_err(a.err, SHT_ETIMEOUT);
        }
    }
    ok = __syncthreads_and(ok && !*(volatile int *)&s_abort);
    if (ok && warp < 4) {   // epilogue: generator group 0 (warp w reads TMEM lanes 32 w ..)
        tc::tc_fence_after();
        const int row = tile * kRows + warp * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        for (int cb = 0; cb < NC; cb += 32) {
            float de[32], dd[32];
            if (nlive > 0) {
                float t[32];
                // parity accumulators: columns [par 2 NC, par 2 NC + 2 NC); sum of the two halves
                tc::tmem_ld32(lane_base + (uint32_t)cb, de);
                tc::tmem_ld32(lane_base + (uint32_t)(NC + cb), t);
#pragma unroll
                for (int i = 0; i < 32; ++i) de[i] += t[i];
                tc::tmem_ld32(lane_base + (uint32_t)(2 * NC + cb), dd);
                tc::tmem_ld32(lane_base + (uint32_t)(3 * NC + cb), t);
#pragma unroll
                for (int i = 0; i < 32; ++i) dd[i] += t[i];
            } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) de[i] = dd[i] = 0.f;
            }
            for (int q = 0; q < 32; q += 2) {
                const int b = (cb + q) >> 1;
                if (b >= a.batch) break;
                if (SYNTH) {
                    if (row < npairs) {
                        float4 *eo = reinterpret_cast<float4 *>(a.out);
                        eo[((size_t)b * (a.mmax + 1) + m) * npairs + row] = make_float4(de[q], de[q + 1], dd[q], dd[q + 1]);
                    }
                } else {
                    const int ne = 2 * row, no = 2 * row + 1;
                    const float sc = (a.op == OP_SYNTH_ADJ && m > 0) ? 2.f : 1.f;
                    float2 *spec = reinterpret_cast<float2 *>(a.out);
                    if (ne < L) spec[(size_t)b * a.nlm + col + ne] = make_float2(sc * de[q], m == 0 ? 0.f : sc * de[q + 1]);
                    if (no < L) spec[(size_t)b * a.nlm + col + no] = make_float2(sc * dd[q], m == 0 ? 0.f : sc * dd[q + 1]);
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------
// Static polar optimisation (Sec. 3.1): for each (m, tile), the first chunk
// whose panel blocks hold a value >= thr.  One CTA per (m, tile).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128)
k_panel_first_live(int synth, int lmax, int mres, int npairs, int ntiles, const unsigned long long *__restrict__ off,
                   const unsigned char *__restrict__ panel, float thr, int *__restrict__ c0,
                   unsigned short *__restrict__ gfirst)
{
    const int m = blockIdx.y, tile = blockIdx.x;   // m: order index
    const int L = lmax - m * mres + 1, Le = (L + 1) / 2;
    const int nchunks = synth ? (Le + kKc - 1) / kKc : (npairs + kKc - 1) / kKc;
    const bool valid = synth || tile * kRows < Le;
    constexpr int NG = kRows / 8;
    __shared__ int s_live[NG], s_first[NG], s_open;
    if (threadIdx.x < NG) s_first[threadIdx.x] = nchunks;
    __syncthreads();
    if (valid) {
        // rows of the tile that hold a latitude pair (synthesis) or a degree (analysis)
        const int rows_valid = synth ? min(kRows, npairs - kRows * tile) : min(kRows, Le - kRows * tile);
        const int ng = (rows_valid + 7) / 8;
        const unsigned char *base = panel + off[m] + (size_t)tile * nchunks * kChunkPanel;
        for (int c = 0; c < nchunks; ++c) {
            if (threadIdx.x < NG) s_live[threadIdx.x] = 0;
            if (threadIdx.x == 0) s_open = 0;
            __syncthreads();
            // hi blocks of both parities (the lo parts are ~2^-8 smaller): the
            // 8 kKc values of 8-row group g of block kb start at g kPSbo + kb kSbo
            const unsigned char *cp = base + (size_t)c * kChunkPanel;
            for (int par = 0; par < 2; ++par) {
                for (int i = threadIdx.x; i < kBlk / 2; i += blockDim.x) {
                    const int g = i / (8 * kKc), e = i - g * (8 * kKc);
                    const __nv_bfloat16 v =
                        *reinterpret_cast<const __nv_bfloat16 *>(cp + (size_t)g * kPSbo + (size_t)(par * 2) * kSbo + 2 * e);
                    if (fabsf(__bfloat162float(v)) >= thr) s_live[g] = 1;
                }
            }
            __syncthreads();
            if (threadIdx.x < ng) {
                if (s_live[threadIdx.x] && s_first[threadIdx.x] == nchunks) s_first[threadIdx.x] = c;
                if (s_first[threadIdx.x] == nchunks) s_open = 1;
            }
            __syncthreads();
            const int open = s_open;
            __syncthreads();
            if (!open) break;   // every group of the tile has its first live chunk
        }
    }
    if (threadIdx.x == 0) {
        int first = nchunks;
        for (int g = 0; g < NG; ++g) first = min(first, s_first[g]);
        c0[m * ntiles + tile] = first;
    }
    if (gfirst && threadIdx.x < NG) gfirst[((size_t)m * ntiles + tile) * NG + threadIdx.x] = (unsigned short)s_first[threadIdx.x];
}

__global__ void k_min_int(const int *__restrict__ a, const int *__restrict__ b, int *__restrict__ out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = min(a[i], b[i]);
}

// Self-test of the timeout path: one thread waits on an mbarrier that nothing
// will ever arrive on, with a bound of `max_ns`, exactly like the waits of the
// tensor-core kernels, then records the timeout in the error word and returns.
__global__ void k_selftest_timeout(int *err, unsigned long long max_ns)
{
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    tc::mbar_init(&bar, 1);
    tc::mbar_fence_init();
    if (!tc::mbar_wait_bounded(&bar, 0, max_ns)) raise_err(err, SHT_ETIMEOUT);
}

int cols_of(int batch) { return tc_rows(batch, false); }

// Launch of the vector contraction (two panels per stage, one CTA per SM:
// its accumulators take the SM's tensor memory): up to 4 stages within 200 KB,
// a.halves field groups per (m, tile).
cudaError_t launch_prep(bool synth, bool vec, int lmax, int mmax, int mres, int npairs, int nlm, int batch, int rows,
                        Op op, const float *in0, const float *in1, const unsigned long long *dchunk,
                        unsigned char *data, cudaStream_t st)
{
    const int Le0 = (lmax + 2) / 2;
    const int maxch = synth ? (Le0 + kKc - 1) / kKc : (npairs + kKc - 1) / kKc;
    const long items = (long)(synth ? 4 : 2) * batch * (vec ? 2 : 1);
    dim3 g((unsigned)((maxch * items + kPrepThreads - 1) / kPrepThreads), (unsigned)(mmax + 1));
    k_tc_prep<<<g, kPrepThreads, 0, st>>>(synth ? 1 : 0, vec ? 1 : 0, lmax, mmax, mres, npairs, nlm, batch, rows,
                                          (int)op, in0, in1, dchunk, data);
    return cudaGetLastError();
}

// Tensor map over the s/d folds [batch][mmax+1][npairs] float4 seen as FP32
// [batch][mmax+1][4 npairs], box {4 kKc, 1, batch}: one chunk of kKc pairs of
// one order for every field.  cuTensorMapEncodeTiled is reached through the
// runtime's driver entry point (no link against the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return nullptr;
        encode = reinterpret_cast<EncodeTiledFn>(fn);
    }
    return encode;
}

cudaError_t make_fold_map(CUtensorMap *map, const float *sd, int npairs, int norders, int batch)
{
    EncodeTiledFn encode = encode_tiled();
    if (!encode) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {(cuuint64_t)4 * npairs, (cuuint64_t)norders, (cuuint64_t)batch};
    const cuuint64_t strides[2] = {(cuuint64_t)npairs * sizeof(float4), (cuuint64_t)norders * npairs * sizeof(float4)};
    const cuuint32_t box[3] = {(cuuint32_t)(4 * kKc), 1u, (cuuint32_t)batch};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(sd), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tensor map over the spectra [batch][nlm] complex seen as FP32 [batch][2 nlm]
// (nlm even), box {kSynthBoxFloats, batch}.
cudaError_t make_spec_map(CUtensorMap *map, const float *spec, int nlm, int batch)
{
    EncodeTiledFn encode = encode_tiled();
    if (!encode) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)2 * nlm, (cuuint64_t)batch};
    const cuuint64_t strides[1] = {(cuuint64_t)nlm * 2 * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kSynthBoxFloats, (cuuint32_t)batch};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(spec), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
int tc_max_batch() { return 64; }
// the on-the-fly kernel keeps 4 x 2 batch accumulator columns (+ the synthesis
// operand) in tensor memory: at most 32 fields per launch
int tc_otf_max_batch() { return 32; }
int tc_vec_max_batch() { return 64; }   // in launches of 64 / kVecHalf adjacent CTAs per (m, tile)

void tc_panel_layout(int lmax, int mmax, int mres, int npairs, std::vector<unsigned long long> &off_s,
                     std::vector<unsigned long long> &off_a, size_t &bytes_s, size_t &bytes_a,
                     std::vector<unsigned long long> &dchunk, size_t &nchunk_s)
{
    off_s.assign(mmax + 1, 0);
    off_a.assign(mmax + 1, 0);
    dchunk.assign(mmax + 1, 0);
    const int T = (npairs + kRows - 1) / kRows;
    const int kch = (npairs + kKc - 1) / kKc;
    unsigned long long s = 0, q = 0, ch = 0;
    for (int m = 0; m <= mmax; ++m) {   // order index m, order m mres
        const int L = lmax - m * mres + 1, Le = (L + 1) / 2;
        const int nch = (Le + kKc - 1) / kKc;
        const int Mt = (Le + kRows - 1) / kRows;
        off_s[m] = s;
        off_a[m] = q;
        dchunk[m] = ch;
        s += (unsigned long long)T * nch * kChunkPanel;
        q += (unsigned long long)Mt * kch * kChunkPanel;
        ch += (unsigned long long)nch;
    }
    bytes_s = s;
    bytes_a = q;
    nchunk_s = (size_t)ch;
}

size_t tc_data_bytes(int mmax, int npairs, size_t nchunk_s, int batch, bool vec)
{
    // vector: one operand per half of kVecHalf fields, each of 2 cols_of(half) rows
    const int halves = (batch + kVecHalf - 1) / kVecHalf;
    const int rows = vec ? halves * 2 * cols_of(halves > 1 ? kVecHalf : batch) : cols_of(batch);
    const size_t kch = (size_t)(npairs + kKc - 1) / kKc;
    const size_t an = (size_t)(mmax + 1) * kch;
    return (nchunk_s > an ? nchunk_s : an) * data_chunk_bytes(rows);
}

cudaError_t launch_build_panels(const PlanView<double> &pv, const unsigned long long *off_s,
                                const unsigned long long *off_a, unsigned char *ps, unsigned char *pa, bool deriv,
                                cudaStream_t st)
{
    dim3 grid((unsigned)((pv.npairs + 127) / 128), (unsigned)(pv.mmax + 1));
    k_build_panels<<<grid, 128, 0, st>>>(pv, off_s, off_a, ps, pa, deriv ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_min_int(const int *a, const int *b, int *out, int n, cudaStream_t st)
{
    k_min_int<<<(n + 255) / 256, 256, 0, st>>>(a, b, out, n);
    return cudaGetLastError();
}

cudaError_t launch_selftest_timeout(int *err, unsigned long long max_ns, cudaStream_t st)
{
    k_selftest_timeout<<<1, 32, 0, st>>>(err, max_ns);
    return cudaGetLastError();
}

void tc_tile_counts(int lmax, int npairs, int &ntiles_s, int &ntiles_a)
{
    ntiles_s = (npairs + kRows - 1) / kRows;
    ntiles_a = (((lmax + 2) / 2) + kRows - 1) / kRows;
}

cudaError_t tc_polar_stats(int lmax, int mmax, int mres, int npairs, const int *d_c0_s, const int *d_c0_a, double &frac_s,
                           double &frac_a, const unsigned short *d_gf_s, const unsigned short *d_gf_a)
{
    int T_s, T_a;
    tc_tile_counts(lmax, npairs, T_s, T_a);
    constexpr int NG = kRows / 8;
    const int kch = (npairs + kKc - 1) / kKc;
    double sk_s = 0, tot_s = 0, sk_a = 0, tot_a = 0;
    if (d_gf_s && d_gf_a) {
        // panel bytes skipped: 8-row groups of a chunk before the group's first live chunk
        std::vector<unsigned short> gs((size_t)(mmax + 1) * T_s * NG), ga((size_t)(mmax + 1) * T_a * NG);
        cudaError_t e = cudaMemcpy(gs.data(), d_gf_s, sizeof(unsigned short) * gs.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(ga.data(), d_gf_a, sizeof(unsigned short) * ga.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return e;
        for (int m = 0; m <= mmax; ++m) {
            const int Le = (lmax - m * mres + 2) / 2, nch = (Le + kKc - 1) / kKc;
            for (int t = 0; t < T_s; ++t) {
                const int ng = (std::min(kRows, npairs - kRows * t) + 7) / 8;
                for (int g = 0; g < ng; ++g) {
                    sk_s += std::min<int>(gs[((size_t)m * T_s + t) * NG + g], nch);
                    tot_s += nch;
                }
            }
            for (int t = 0; t < T_a; ++t) {
                if (t * kRows >= Le) continue;
                const int ng = (std::min(kRows, Le - kRows * t) + 7) / 8;
                for (int g = 0; g < ng; ++g) {
                    sk_a += std::min<int>(ga[((size_t)m * T_a + t) * NG + g], kch);
                    tot_a += kch;
                }
            }
        }
    } else {
        // whole chunks skipped
        std::vector<int> c0s((size_t)(mmax + 1) * T_s), c0a((size_t)(mmax + 1) * T_a);
        cudaError_t e = cudaMemcpy(c0s.data(), d_c0_s, sizeof(int) * c0s.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(c0a.data(), d_c0_a, sizeof(int) * c0a.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return e;
        for (int m = 0; m <= mmax; ++m) {
            const int Le = (lmax - m * mres + 2) / 2, nch = (Le + kKc - 1) / kKc;
            for (int t = 0; t < T_s; ++t) { sk_s += c0s[(size_t)m * T_s + t]; tot_s += nch; }
            for (int t = 0; t < T_a; ++t)
                if (t * kRows < Le) { sk_a += c0a[(size_t)m * T_a + t]; tot_a += kch; }
        }
    }
    frac_s = tot_s > 0 ? sk_s / tot_s : 0.0;
    frac_a = tot_a > 0 ? sk_a / tot_a : 0.0;
    return cudaSuccess;
}

cudaError_t launch_panel_first_live(bool synth, int lmax, int mmax, int mres, int npairs, const unsigned long long *off,
                                    const unsigned char *panel, float thr, int *c0, int &ntiles, cudaStream_t st,
                                    unsigned short *gfirst)
{
    int ts, ta;
    tc_tile_counts(lmax, npairs, ts, ta);
    ntiles = synth ? ts : ta;
    dim3 g((unsigned)ntiles, (unsigned)(mmax + 1));
    k_panel_first_live<<<g, 128, 0, st>>>(synth ? 1 : 0, lmax, mres, npairs, ntiles, off, panel, thr, c0, gfirst);
    return cudaGetLastError();
}

cudaError_t launch_tc_legendre(bool synth, int lmax, int mmax, int mres, int npairs, int nlm, const unsigned char *panel,
                               const unsigned long long *off, const int *c0, const unsigned short *gfirst,
                               const unsigned long long *dchunk,
                               unsigned char *data, const float *in, float *out, int batch, Op op, int *err,
                               bool prepped, cudaStream_t st)
{
    if (batch < 1 || batch > tc_max_batch()) return cudaErrorInvalidValue;
    const int rows = cols_of(batch);
    // synthesis: prep the spectra into the blocked layout; analysis: the
    // contraction converts the raw folds itself
    // the spectra's tensor map needs a 16-byte row pitch: nlm even
    const bool fuse_synth = synth && (nlm % 2 == 0);
    if (synth && !fuse_synth && !prepped) {
        cudaError_t e =
            launch_prep(synth, false, lmax, mmax, mres, npairs, nlm, batch, rows, op, in, nullptr, dchunk, data, st);
        if (e != cudaSuccess) return e;
    }
    TcArgs a{};
    a.lmax = lmax;
    a.mmax = mmax;
    a.mres = mres;
    a.npairs = npairs;
    a.nlm = nlm;
    a.batch = batch;
    a.rows = rows;
    a.op = (int)op;
    a.panel = panel;
    a.off = off;
    a.c0 = c0;
    a.gf = c0 ? gfirst : nullptr;
    a.data = data;
    a.dchunk = dchunk;
    a.out0 = out;
    a.err = err;
    a.in = in;
    CUtensorMap fold_map;
    memset(&fold_map, 0, sizeof(fold_map));
    a.fused = fuse_synth ? 1 : 0;
    if (!synth) {
        cudaError_t em = make_fold_map(&fold_map, in, npairs, mmax + 1, batch);
        if (em != cudaSuccess) return em;
    } else if (fuse_synth) {
        cudaError_t em = make_spec_map(&fold_map, in, nlm, batch);
        if (em != cudaSuccess) return em;
    }
    // kWsCtasPerSm CTAs of up to 3 stages per SM (228 KB, 1 KB reserved per
    // CTA, a little static shared memory); wider batches fall back to fewer CTAs
    const size_t cap = (size_t)228 * 1024 / kWsCtasPerSm - 1024 - 256;
    int stages = 3;
    while (stages > 2 && ws_smem_bytes(rows, batch, stages, synth) > cap) --stages;
    if (ws_smem_bytes(rows, batch, stages, synth) > cap) {
        stages = 4;
        while (stages > 2 && ws_smem_bytes(rows, batch, stages, synth) > 110 * 1024) --stages;
    }
    a.stages = stages;
    const size_t smem = ws_smem_bytes(rows, batch, stages, synth);
    int ts, ta;
    tc_tile_counts(lmax, npairs, ts, ta);
    a.ntiles = synth ? ts : ta;
    const unsigned blocks = (unsigned)((mmax + 1) * a.ntiles);
    cudaError_t e2;
    if (synth) {
        e2 = cudaFuncSetAttribute(k_tc_ws<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e2 != cudaSuccess) return e2;
        k_tc_ws<true><<<blocks, kWsThreads, smem, st>>>(a, fold_map);
    } else {
        e2 = cudaFuncSetAttribute(k_tc_ws<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e2 != cudaSuccess) return e2;
        k_tc_ws<false><<<blocks, kWsThreads, smem, st>>>(a, fold_map);
    }
    return cudaGetLastError();
}

cudaError_t launch_tc_vec(bool synth, int lmax, int mmax, int mres, int npairs, int nlm, const unsigned char *panel,
                          const unsigned char *dpanel, const unsigned long long *off, const int *c0,
                          const int *const sched[2], int nctas,
                          const unsigned long long *dchunk, unsigned char *data, const float *in0, const float *in1,
                          float *out0, float *out1, const float *st_pairs, int batch, Op op, int *err, bool prepped,
                          cudaStream_t st)
{
    if (batch < 1 || batch > tc_vec_max_batch()) return cudaErrorInvalidValue;
    const int halves = (batch + kVecHalf - 1) / kVecHalf;
    const int rows = 2 * cols_of(halves > 1 ? kVecHalf : batch);   // 4 accumulators x rows columns <= 512
    // one half's data operand: the larger of the two chunk numberings
    size_t nch_s = 0;
    for (int m = 0; m <= mmax; ++m) nch_s += (size_t)(((lmax - m * mres + 2) / 2 + kKc - 1) / kKc);
    const size_t nch_a = (size_t)(mmax + 1) * ((npairs + kKc - 1) / kKc);
    const size_t data_half = (nch_s > nch_a ? nch_s : nch_a) * data_chunk_bytes(rows);
    if (!prepped) {
        for (int h = 0; h < halves; ++h) {
            const int hb = std::min(kVecHalf, batch - h * kVecHalf);
            const size_t fo = (size_t)h * kVecHalf * (synth ? (size_t)nlm * 2 : (size_t)(mmax + 1) * npairs * 4);
            cudaError_t e = launch_prep(synth, true, lmax, mmax, mres, npairs, nlm, hb, rows, op, in0 + fo, in1 + fo,
                                        dchunk, data + (size_t)h * data_half, st);
            if (e != cudaSuccess) return e;
        }
    }
    TcArgs a{};
    a.halves = halves;
    a.data_half = data_half;
    a.lmax = lmax;
    a.mmax = mmax;
    a.mres = mres;
    a.npairs = npairs;
    a.nlm = nlm;
    a.batch = batch;
    a.rows = rows;
    a.op = (int)op;
    a.panel = panel;
    a.dpanel = dpanel;
    a.off = off;
    a.c0 = c0;
    a.data = data;
    a.dchunk = dchunk;
    a.out0 = out0;
    a.out1 = out1;
    a.st = st_pairs;
    a.err = err;
    a.sched = sched[halves - 1];
    if (!a.sched || nctas < 1) return cudaErrorInvalidValue;
    int stages = 4;
    while (stages > 2 && smem_bytes_of(2, rows, stages) + 16 > 200 * 1024) --stages;
    a.stages = stages;
    const size_t smem = smem_bytes_of(2, rows, stages) + 16;   // + the accumulator barriers
    int ts, ta;
    tc_tile_counts(lmax, npairs, ts, ta);
    a.ntiles = synth ? ts : ta;
    cudaError_t e;
    if (synth) {
        e = cudaFuncSetAttribute(k_tc_vec<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_tc_vec<true><<<(unsigned)nctas, 192, smem, st>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_tc_vec<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_tc_vec<false><<<(unsigned)nctas, 192, smem, st>>>(a);
    }
    return cudaGetLastError();
}

// Work items of the vector contraction, (order index, tile) x field half,
// costed as their live chunks plus two for the epilogue (-1: no rows),
// grouped by order index.
void tc_vec_costs(int lmax, int mmax, int mres, int npairs, bool synth, int halves, const std::vector<int> &c0,
                  std::vector<int> &cost, std::vector<int> &group)
{
    int ts, ta;
    tc_tile_counts(lmax, npairs, ts, ta);
    const int ntiles = synth ? ts : ta;
    cost.assign((size_t)(mmax + 1) * ntiles * halves, -1);
    group.assign(cost.size(), 0);
    for (size_t w = 0; w < group.size(); ++w) group[w] = (int)(w / ((size_t)ntiles * halves));
    for (int m = 0; m <= mmax; ++m)
        for (int t = 0; t < ntiles; ++t) {
            const int L = lmax - m * mres + 1, Le = (L + 1) / 2;
            if (!synth && t * kRows >= Le) continue;
            const int nchunks = synth ? (Le + kKc - 1) / kKc : (npairs + kKc - 1) / kKc;
            for (int h = 0; h < halves; ++h) cost[((size_t)m * ntiles + t) * halves + h] = nchunks - c0[(size_t)m * ntiles + t] + 2;
        }
}

// ---------------------------------------------------------------------------
// On-the-fly mode (host side)
// ---------------------------------------------------------------------------
size_t otf_segment_offsets(int lmax, int mmax, int mres, std::vector<unsigned long long> &segoff)
{
    segoff.assign(mmax + 1, 0);
    unsigned long long s = 0;
    for (int m = 0; m <= mmax; ++m) {
        segoff[m] = s;
        s += (unsigned long long)((lmax - m * mres + 1 + kSeg - 1) / kSeg);
    }
    return (size_t)s;
}

cudaError_t launch_build_seeds(const PlanView<double> &pv, const unsigned long long *segoff, float4 *seeds,
                               float thr, int *c0s, int *c0a, int *flag, cudaStream_t st)
{
    int ts, ta;
    tc_tile_counts(pv.lmax, pv.npairs, ts, ta);
    const int n = (pv.mmax + 1) * (ts + ta);
    k_init_c0<<<(n + 255) / 256, 256, 0, st>>>(pv.lmax, pv.mmax, pv.mres, pv.npairs, ts, ta, c0s, c0a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 g((unsigned)((pv.npairs + 127) / 128), (unsigned)(pv.mmax + 1));
    k_build_seeds<<<g, 128, 0, st>>>(pv, segoff, seeds, thr, c0s, c0a, ts, ta, flag);
    return cudaGetLastError();
}

cudaError_t launch_tc_otf(bool synth, int lmax, int mmax, int mres, int npairs, int nlm, const float4 *seeds,
                          const unsigned long long *segoff, const int *c0, const float2 *ab32, const float *x32,
                          unsigned char *data, const float *in, float *out, int batch, Op op, int *err,
                          cudaStream_t st)
{
    if (batch < 1 || batch > tc_otf_max_batch()) return cudaErrorInvalidValue;
    const int rows = cols_of(batch);
    // synthesis data chunks are numbered like the segments (one chunk = one segment)
    cudaError_t e = launch_prep(synth, false, lmax, mmax, mres, npairs, nlm, batch, rows, op, in, nullptr, segoff, data, st);
    if (e != cudaSuccess) return e;
    OtfArgs a{};
    a.lmax = lmax;
    a.mmax = mmax;
    a.mres = mres;
    a.npairs = npairs;
    a.nlm = nlm;
    a.batch = batch;
    a.rows = rows;
    a.op = (int)op;
    a.nab = synth ? kSeg * ((lmax + 1 + kSeg - 1) / kSeg) : 2 * kRows;
    a.seeds = seeds;
    a.segoff = segoff;
    a.c0 = c0;
    a.ab = ab32;
    a.x = x32;
    a.data = data;
    a.out = out;
    a.err = err;
    // operand stages SA (4: generators fill two per round) and data stages SD
    // (up to 8), within 110 KB so that two CTAs share an SM
    int sa = 4, sd = 8;
    while (sd > 3 && otf_smem_bytes(rows, sa, sd, a.nab, synth) > 110 * 1024) --sd;
    while (sa > 2 && otf_smem_bytes(rows, sa, sd, a.nab, synth) > 110 * 1024) --sa;
    a.stages = sa | (sd << 8);
    const size_t smem = otf_smem_bytes(rows, sa, sd, a.nab, synth);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    int ts, ta;
    tc_tile_counts(lmax, npairs, ts, ta);
    a.ntiles = synth ? ts : ta;
    const unsigned blocks = (unsigned)((mmax + 1) * a.ntiles);
    if (synth) {
        e = cudaFuncSetAttribute(k_tc_otf<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_tc_otf<true><<<blocks, kOtfThreads, smem, st>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_tc_otf<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_tc_otf<false><<<blocks, kOtfThreads, smem, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace sht
