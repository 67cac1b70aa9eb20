// tc.cu -- the per-order Legendre contraction on the 5th-generation tensor
// cores (tcgen05), for batches of fields.
//
// For each order m and parity of n - m the Legendre stage is a small GEMM
// (mirror symmetry, Sec. 3.1):
//   synthesis  E/O[pair, col] = sum_k P[pair, k] * A[k, col]       (Eq. synth_direct)
//   analysis   f[k, col]      = sum_pair P[pair, k] * S[pair, col] (Eq. gauss)
// with k the index of n among degrees of that parity, col = (field, re/im),
// and S the weighted north/south folds (s for even, d for odd n - m).
//
// The matrices P_n^m(x_j) are built once per plan by the FP64 recurrence of
// Sec. 3.2 with the rescaling of Sec. 3.5 (the precomputed variant of
// Sec. 3.1), split into bf16 hi + lo parts and stored in
// HBM already in the tensor core's shared-memory operand layout (K-major,
// no swizzle: 8-row x 16-byte core matrices), so each chunk is one bulk copy.
// The data operand is split the same way by the CTA's threads, and each
// product is hi*hi + hi*lo + lo*hi accumulated in FP32 in tensor memory.
//
// CTA: 128 threads, one (order m, 128-row tile).  Thread 0 issues the bulk
// copies and the MMAs; all threads stage the data operand and run the
// epilogue (tcgen05.ld of the accumulators).  Every wait is bounded; on a
// timeout the kernel records an error code and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "sht_internal.h"
#include "tc_ptx.cuh"

namespace sht {
namespace {

constexpr int kRows = 128;            // MMA M
constexpr int kKc = 32;               // K per chunk (per parity)
constexpr int kBlk = kRows * kKc * 2; // bytes of one bf16 [128 x 32] operand block
constexpr int kChunkPanel = 4 * kBlk; // [parity][hi/lo] blocks per chunk = 32 KB
constexpr uint32_t kSbo = (kKc / 8) * 128;  // 8-row group stride in a [rows x 32] block
constexpr uint32_t kLbo = 128;              // K-adjacent core matrices
constexpr uint64_t kWaitNs = 2000000000ull; // 2 s

// byte offset of element (row, k) in a K-major [rows x 32] bf16 block
__host__ __device__ __forceinline__ uint32_t blk_off(int row, int k)
{
    return (uint32_t)((row >> 3) * kSbo + (k >> 3) * kLbo + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16 &hi, __nv_bfloat16 &lo)
{
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

__device__ __forceinline__ void split_bf16_d(double v, __nv_bfloat16 &hi, __nv_bfloat16 &lo)
{
    hi = __float2bfloat16_rn((float)v);
    lo = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hi)));
}

__device__ __forceinline__ long col_of(int lmax, int m) { return (long)m * (2 * lmax + 3 - m) / 2; }

__device__ __forceinline__ void raise_err(int *err, int code)
{
    if (err) atomicCAS(err, 0, code);
}

// ---------------------------------------------------------------------------
// Panel builder: one thread per (m, pair), FP64 recurrence with rescaling.
// Both panel sets must be zeroed beforehand; only non-zero entries are written.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128)
k_build_panels(PlanView<double> pv, const unsigned long long *__restrict__ off_s,
               const unsigned long long *__restrict__ off_a, unsigned char *__restrict__ ps,
               unsigned char *__restrict__ pa)
{
    const int m = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int npairs = pv.npairs, lmax = pv.lmax;
    if (p >= npairs) return;
    const int L = lmax - m + 1;
    const int Le = (L + 1) / 2;
    const int nch = (Le + kKc - 1) / kKc;            // synthesis chunks per tile
    const int kch = (npairs + kKc - 1) / kKc;        // analysis chunks (over pairs)
    const long col = col_of(lmax, m);
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
        const double P = (k == 0) ? y1 : 0.0;
        if (P == 0.0) continue;
        __nv_bfloat16 hi, lo;
        split_bf16_d(P, hi, lo);
        const int par = nn & 1, kk = nn >> 1;
        // synthesis panel: block (t, chunk kk/32, parity, hi|lo), element (row, kk%32)
        {
            unsigned char *b = sbase + (size_t)(kk / kKc) * kChunkPanel + (size_t)(par * 2) * kBlk;
            const uint32_t o = blk_off(row, kk % kKc);
            *reinterpret_cast<__nv_bfloat16 *>(b + o) = hi;
            *reinterpret_cast<__nv_bfloat16 *>(b + kBlk + o) = lo;
        }
        // analysis panel: block (M tile kk/128, pair chunk kc, parity, hi|lo), element (kk%128, pc)
        {
            const int mt = kk / kRows, r = kk % kRows;
            unsigned char *b = abase + ((size_t)mt * kch + kc) * kChunkPanel + (size_t)(par * 2) * kBlk;
            const uint32_t o = blk_off(r, pc);
            *reinterpret_cast<__nv_bfloat16 *>(b + o) = hi;
            *reinterpret_cast<__nv_bfloat16 *>(b + kBlk + o) = lo;
        }
    }
}

struct TcArgs {
    int lmax, mmax, npairs, nlm, batch, nc, ntiles, stages, op;
    const unsigned char *panel;
    const unsigned long long *off;     // per-order panel byte offsets
    const unsigned char *data;         // data operand, blocked bf16 hi/lo
    const unsigned long long *dchunk;  // synthesis: first data chunk of each order
    float *out;                        // synthesis: E/O; analysis: spectra
    int *err;
};

// Bytes of one chunk of the data operand: [parity][hi|lo] blocks of nc rows x 32.
__host__ __device__ inline size_t tc_data_chunk(int nc) { return 4 * (size_t)nc * kKc * 2; }

// Shared memory: [stages] x { panel chunk (32 KB) | data chunk } then 2*stages+1
// mbarriers and the TMEM address slot.
__host__ __device__ inline size_t tc_stage_bytes(int nc) { return (size_t)kChunkPanel + tc_data_chunk(nc); }

__host__ __device__ inline size_t tc_smem_bytes(int nc, int stages)
{
    return 1024 + (size_t)stages * tc_stage_bytes(nc) + 8 * (2 * stages + 2);
}

// ---------------------------------------------------------------------------
// Data operand preparation: FP32 -> bf16 hi/lo, blocked like the panels.
// Synthesis: chunk (m, c) holds degrees n - m in [64c, 64c + 64), row 2b + part.
// Analysis:  chunk (m, kc) holds pairs [32kc, 32kc + 32), folds s (even) / d (odd).
// grid = (chunk, m) with chunk < max chunks; one CTA of 128 threads per chunk.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128)
k_tc_prep(int synth, int lmax, int mmax, int npairs, int nlm, int batch, int nc, int op, const float *__restrict__ in,
          const unsigned long long *__restrict__ dchunk, unsigned char *__restrict__ data)
{
    const int m = blockIdx.y, c = blockIdx.x;
    const int L = lmax - m + 1, Le = (L + 1) / 2;
    const int nch = synth ? (Le + kKc - 1) / kKc : (npairs + kKc - 1) / kKc;
    if (c >= nch) return;
    const size_t db = tc_data_chunk(nc);
    unsigned char *dat = data + (synth ? (dchunk[m] + c) : ((size_t)m * nch + c)) * db;
    const size_t blk = (size_t)nc * kKc * 2;
    // zero the chunk first: rows >= 2*batch are the MMA's pad columns
    for (int i = threadIdx.x; i < (int)(db / 16); i += blockDim.x)
        *reinterpret_cast<uint4 *>(dat + (size_t)i * 16) = make_uint4(0, 0, 0, 0);
    __syncthreads();
    if (synth) {
        const long col = col_of(lmax, m);
        const float cm_in = (op == OP_ANALYS_ADJ && m > 0) ? 0.5f : 1.0f;
        const float2 *spec = reinterpret_cast<const float2 *>(in);
        for (int i = threadIdx.x; i < batch * 2 * kKc; i += blockDim.x) {
            const int b = i / (2 * kKc), j = i - b * (2 * kKc);
            const int nn = 2 * kKc * c + j;
            float2 v = make_float2(0.f, 0.f);
            if (nn < L) v = spec[(size_t)b * nlm + col + nn];
            v.x *= cm_in;
            v.y = (m == 0) ? 0.f : v.y * cm_in;
            const int par = j & 1, kk = j >> 1;
            __nv_bfloat16 hr, lr, hi_, li;
            split_bf16(v.x, hr, lr);
            split_bf16(v.y, hi_, li);
            unsigned char *bh = dat + (size_t)(par * 2) * blk;
            unsigned char *bl = bh + blk;
            *reinterpret_cast<__nv_bfloat16 *>(bh + blk_off(2 * b, kk)) = hr;
            *reinterpret_cast<__nv_bfloat16 *>(bl + blk_off(2 * b, kk)) = lr;
            *reinterpret_cast<__nv_bfloat16 *>(bh + blk_off(2 * b + 1, kk)) = hi_;
            *reinterpret_cast<__nv_bfloat16 *>(bl + blk_off(2 * b + 1, kk)) = li;
        }
    } else {
        const float4 *sd = reinterpret_cast<const float4 *>(in);
        for (int i = threadIdx.x; i < batch * kKc; i += blockDim.x) {
            const int b = i / kKc, j = i - b * kKc;
            const int p = kKc * c + j;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (p < npairs) v = sd[((size_t)b * (mmax + 1) + m) * npairs + p];
            const float vals[4] = {v.x, v.y, v.z, v.w};  // s.re s.im d.re d.im
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int par = q >> 1, part = q & 1;
                __nv_bfloat16 h, l;
                split_bf16(vals[q], h, l);
                unsigned char *bh = dat + (size_t)(par * 2) * blk;
                unsigned char *bl = bh + blk;
                *reinterpret_cast<__nv_bfloat16 *>(bh + blk_off(2 * b + part, j)) = h;
                *reinterpret_cast<__nv_bfloat16 *>(bl + blk_off(2 * b + part, j)) = l;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The contraction.  Thread 0 is the producer and MMA issuer: for each chunk it
// waits until the stage is free (the MMAs that read it completed), issues the
// two bulk copies (panel chunk and data chunk) D = S - 1 chunks ahead, waits
// for the current chunk and issues its 12 MMAs.  The other threads only run
// the epilogue once every MMA has completed.
// ---------------------------------------------------------------------------
template <bool SYNTH>
__global__ void __launch_bounds__(128, 1) k_tc_legendre(TcArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int S = a.stages, NC = a.nc;
    const size_t stage_bytes = tc_stage_bytes(NC);
    const uint32_t dbytes = (uint32_t)tc_data_chunk(NC);
    uint64_t *bar_load = reinterpret_cast<uint64_t *>(smem + (size_t)S * stage_bytes);
    uint64_t *bar_mma = bar_load + S;
    uint64_t *bar_done = bar_mma + S;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_done + 1);
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int m = blockIdx.x / a.ntiles;
    const int tile = blockIdx.x - m * a.ntiles;
    const int lmax = a.lmax, npairs = a.npairs;
    const int L = lmax - m + 1;
    const int Le = (L + 1) / 2;
    const long col = col_of(lmax, m);
    // analysis tiles run over degrees of this order: tiles past them have no panel
    if (!SYNTH && tile * kRows >= Le) return;
    // chunks: synthesis over degrees (per parity), analysis over latitude pairs
    const int nchunks = SYNTH ? (Le + kKc - 1) / kKc : (npairs + kKc - 1) / kKc;
    const unsigned char *panel = a.panel + a.off[m] + (size_t)tile * nchunks * kChunkPanel;
    const unsigned char *data = a.data + (SYNTH ? a.dchunk[m] : (unsigned long long)m * nchunks) * dbytes;
    const uint32_t ncols = NC * 2 <= 64 ? 64 : (NC * 2 <= 128 ? 128 : 256);

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&bar_load[s], 1);
            tc::mbar_init(&bar_mma[s], 1);
        }
        tc::mbar_init(bar_done, 1);
        tc::mbar_fence_init();
        s_ok = 1;
    }
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;

    if (tid == 0) {
        bool ok = true;
        int issued[4] = {0, 0, 0, 0}, waited[4] = {0, 0, 0, 0};
        const uint32_t idesc = tc::idesc_bf16_f32(kRows, NC);
        const int D = S - 1;
        auto issue = [&](int cn) {
            const int sn = cn % S;
            unsigned char *st = smem + (size_t)sn * stage_bytes;
            tc::mbar_arrive_expect_tx(&bar_load[sn], (uint32_t)kChunkPanel + dbytes);
            tc::bulk_g2s(st, panel + (size_t)cn * kChunkPanel, kChunkPanel, &bar_load[sn]);
            tc::bulk_g2s(st + kChunkPanel, data + (size_t)cn * dbytes, dbytes, &bar_load[sn]);
            issued[sn] += 1;
        };
        for (int c = 0; c < D && c < nchunks; ++c) issue(c);
        for (int c = 0; c < nchunks; ++c) {
            const int s = c % S;
            // refill the stage of chunk c - 1 with chunk c + D once its MMAs are done
            const int cn = c + D;
            if (cn < nchunks) {
                if (cn >= S) {
                    const int cp = cn - S;  // == c - 1
                    if (!tc::mbar_wait_bounded(&bar_mma[cp % S], (uint32_t)((cp / S) & 1), kWaitNs)) {
                        ok = false;
                        break;
                    }
                }
                issue(cn);
            }
            if (!tc::mbar_wait_bounded(&bar_load[s], (uint32_t)((c / S) & 1), kWaitNs)) {
                ok = false;
                break;
            }
            waited[s] += 1;
            tc::tc_fence_after();
            unsigned char *st = smem + (size_t)s * stage_bytes;
            unsigned char *dat = st + kChunkPanel;
#pragma unroll
            for (int par = 0; par < 2; ++par) {
                const unsigned char *ah = st + (size_t)(par * 2) * kBlk;
                const unsigned char *al = ah + kBlk;
                const unsigned char *bh = dat + (size_t)(par * 2) * NC * kKc * 2;
                const unsigned char *bl = bh + (size_t)NC * kKc * 2;
                const uint32_t d = tmem + (uint32_t)(par * NC);
#pragma unroll
                for (int ks = 0; ks < kKc / 16; ++ks) {
                    const uint32_t ko = (uint32_t)ks * 2 * kLbo;  // 16 K = 2 core matrices
                    const uint64_t dah = tc::smem_desc(ah + ko, kLbo, kSbo);
                    const uint64_t dal = tc::smem_desc(al + ko, kLbo, kSbo);
                    const uint64_t dbh = tc::smem_desc(bh + ko, kLbo, kSbo);
                    const uint64_t dbl = tc::smem_desc(bl + ko, kLbo, kSbo);
                    tc::mma_bf16(d, dah, dbh, idesc, !(c == 0 && ks == 0));
                    tc::mma_bf16(d, dah, dbl, idesc, true);
                    tc::mma_bf16(d, dal, dbh, idesc, true);
                }
            }
            tc::mma_commit(&bar_mma[s]);
        }
        if (ok) {
            tc::mma_commit(bar_done);
        } else {
            raise_err(a.err, SHT_ETIMEOUT);
            s_ok = 0;
            // wait (bounded) for this CTA's own copies and MMAs before TMEM is freed
            for (int s = 0; s < S; ++s)
                if (issued[s] > waited[s])
                    (void)tc::mbar_wait_bounded(&bar_load[s], (uint32_t)((issued[s] - 1) & 1), 100000000ull);
            tc::mma_commit(bar_done);
        }
    }
    // everyone waits for the last MMAs (bounded), then reads the accumulators
    bool ok = tc::mbar_wait_bounded(bar_done, 0, 2 * kWaitNs);
    if (!ok) raise_err(a.err, SHT_ETIMEOUT);
    ok = __syncthreads_and(ok && s_ok);
    if (ok) {
        tc::tc_fence_after();
        const int row = tile * kRows + warp * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < NC; c0 += 32) {
            float de[32], dd[32];
            tc::tmem_ld32(lane_base + (uint32_t)c0, de);
            tc::tmem_ld32(lane_base + (uint32_t)(NC + c0), dd);
            for (int q = 0; q < 32; q += 2) {
                const int b = (c0 + q) >> 1;
                if (b >= a.batch) break;
                if (SYNTH) {
                    if (row < npairs) {
                        float4 *eo = reinterpret_cast<float4 *>(a.out);
                        eo[((size_t)b * (a.mmax + 1) + m) * npairs + row] = make_float4(de[q], de[q + 1], dd[q], dd[q + 1]);
                    }
                } else {
                    const int ne = 2 * row, no = 2 * row + 1;   // n - m of the two rows
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

// Self-test of the timeout path: one thread waits on an mbarrier that nothing
// will ever arrive on, with a bound of `max_ns`, exactly like the waits of the
// tensor-core kernel, then records the timeout in the error word and returns.
__global__ void k_selftest_timeout(int *err, unsigned long long max_ns)
{
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    tc::mbar_init(&bar, 1);
    tc::mbar_fence_init();
    if (!tc::mbar_wait_bounded(&bar, 0, max_ns)) raise_err(err, SHT_ETIMEOUT);
}

}  // namespace

cudaError_t launch_selftest_timeout(int *err, unsigned long long max_ns, cudaStream_t st)
{
    k_selftest_timeout<<<1, 32, 0, st>>>(err, max_ns);
    return cudaGetLastError();
}

// Sizes of the two panel sets and per-order byte offsets.
void tc_panel_layout(int lmax, int mmax, int npairs, std::vector<unsigned long long> &off_s,
                     std::vector<unsigned long long> &off_a, size_t &bytes_s, size_t &bytes_a,
                     std::vector<unsigned long long> &dchunk, size_t &nchunk_s)
{
    off_s.assign(mmax + 1, 0);
    off_a.assign(mmax + 1, 0);
    dchunk.assign(mmax + 1, 0);
    unsigned long long ch = 0;
    const int T = (npairs + kRows - 1) / kRows;
    const int kch = (npairs + kKc - 1) / kKc;
    unsigned long long s = 0, q = 0;
    for (int m = 0; m <= mmax; ++m) {
        const int L = lmax - m + 1, Le = (L + 1) / 2;
        const int nch = (Le + kKc - 1) / kKc;
        const int Mt = (Le + kRows - 1) / kRows;
        off_s[m] = s;
        off_a[m] = q;
        dchunk[m] = ch;
        ch += (unsigned long long)nch;
        s += (unsigned long long)T * nch * kChunkPanel;
        q += (unsigned long long)Mt * kch * kChunkPanel;
    }
    bytes_s = s;
    bytes_a = q;
    nchunk_s = (size_t)ch;
}

// Bytes of the data-operand buffer for a batch: synthesis and analysis layouts.
size_t tc_data_bytes(int lmax, int mmax, int npairs, size_t nchunk_s, int batch)
{
    const int nc = ((2 * batch + 31) / 32) * 32;
    const size_t kch = (size_t)(npairs + kKc - 1) / kKc;
    const size_t a = (size_t)(mmax + 1) * kch;
    return (nchunk_s > a ? nchunk_s : a) * tc_data_chunk(nc);
}

cudaError_t launch_build_panels(const PlanView<double> &pv, const unsigned long long *off_s,
                                const unsigned long long *off_a, unsigned char *ps, unsigned char *pa,
                                cudaStream_t st)
{
    dim3 grid((unsigned)((pv.npairs + 127) / 128), (unsigned)(pv.mmax + 1));
    k_build_panels<<<grid, 128, 0, st>>>(pv, off_s, off_a, ps, pa);
    return cudaGetLastError();
}

// Columns of the data operand: 2 per field, rounded up to 32 (N of the MMA).
static int tc_cols(int batch) { return ((2 * batch + 31) / 32) * 32; }

int tc_max_batch() { return 64; }

cudaError_t launch_tc_legendre(bool synth, int lmax, int mmax, int npairs, int nlm, const unsigned char *panel,
                               const unsigned long long *off, const unsigned long long *dchunk,
                               unsigned char *data, const float *in, float *out, int batch, Op op, int *err,
                               cudaStream_t st)
{
    // data operand in the blocked bf16 layout
    {
        const int Le0 = (lmax + 2) / 2;
        const int maxch = synth ? (Le0 + kKc - 1) / kKc : (npairs + kKc - 1) / kKc;
        dim3 g((unsigned)maxch, (unsigned)(mmax + 1));
        k_tc_prep<<<g, 128, 0, st>>>(synth ? 1 : 0, lmax, mmax, npairs, nlm, batch, ((2 * batch + 31) / 32) * 32,
                                    (int)op, in, dchunk, data);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    TcArgs a;
    a.lmax = lmax;
    a.mmax = mmax;
    a.npairs = npairs;
    a.nlm = nlm;
    a.batch = batch;
    a.nc = tc_cols(batch);
    a.op = (int)op;
    a.panel = panel;
    a.off = off;
    a.data = data;
    a.dchunk = dchunk;
    a.out = out;
    a.err = err;
    if (a.nc > 256) return cudaErrorInvalidValue;
    int stages = 4;
    while (stages > 2 && tc_smem_bytes(a.nc, stages) > 200 * 1024) --stages;
    a.stages = stages;
    const size_t smem = tc_smem_bytes(a.nc, stages);
    unsigned blocks;
    if (synth) {
        a.ntiles = (npairs + kRows - 1) / kRows;
        blocks = (unsigned)((mmax + 1) * a.ntiles);
    } else {
        // analysis tiles run over degrees; the largest order count (m = 0) sets the tile count
        const int Le0 = (lmax + 2) / 2;
        a.ntiles = (Le0 + kRows - 1) / kRows;
        blocks = (unsigned)((mmax + 1) * a.ntiles);
    }
    cudaError_t e;
    if (synth) {
        e = cudaFuncSetAttribute(k_tc_legendre<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_tc_legendre<true><<<blocks, 128, smem, st>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_tc_legendre<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_tc_legendre<false><<<blocks, 128, smem, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace sht
