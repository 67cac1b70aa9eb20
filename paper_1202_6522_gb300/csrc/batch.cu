// batch.cu -- uneven batches: many scalar fields of different truncations
// transformed by one graph launch.
//
// Each distinct (lmax, nlat, nphi) gets one plan; every field keeps its own
// intermediate buffer.  The host builds, once, a tile list per stage covering
// all fields -- synthesis Legendre tiles (field, m, pair block), analysis
// Legendre tiles (field, m), FFT tiles (field, pair group) -- sorted longest
// first (the load-balancing concern of Sec. 3.3, applied to CTAs instead of
// threads).  A transform is then: copy the per-field pointer table, reset the
// work counters, one persistent Legendre kernel and one persistent FFT kernel
// (in the order of Sec. 2.2 / 2.3).  That sequence is captured once into a
// CUDA graph and replayed on every call.  The persistent kernels take tiles
// with atomicAdd on a counter and never wait on each other.
//
// Tensor-core mode: the fields of one shape form a group whose spectra (a
// gather kernel copies them in, or the results out) and intermediates are
// contiguous, so each group's Legendre stage is one batched tcgen05
// contraction against that plan's P panels; the FFTs stay one persistent
// launch over all fields.  The captured graph then holds the pointer-table
// copy, the gather (or scatter), one contraction per group and the FFT.  The
// automatic mode times both and keeps the faster.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "sht_internal.h"

namespace {
// One copy of the gather (synthesis) or scatter (analysis) of the tensor-core mode.
struct BatchCopy {
    const float2 *src;
    float2 *dst;
    long long n;   // complex values
};
}  // namespace

struct sht_batch_plan {
    int nfields = 0;
    int device = 0;
    int mode = SHT_F32;                    // SHT_F32 (persistent CUDA-core kernels) or SHT_TC_BF16X3
    std::vector<std::vector<int>> group_fields;   // tensor cores: the fields of each plan, in order
    float *d_gspec = nullptr;              // ... contiguous spectra of each group
    std::vector<size_t> gspec_off;         // ... per group, floats
    std::vector<size_t> field_gspec;       // ... per field: its slot in d_gspec, floats
    std::vector<size_t> ginter_off;        // ... per group: its contiguous intermediate in d_inter, floats
    std::vector<size_t> inter_tc;          // ... per field: its intermediate in that layout
    BatchCopy *h_copies = nullptr, *d_copies = nullptr;
    float tuned_ms[2] = {0.f, 0.f};        // automatic mode: round trip per path (CUDA cores, tensor cores)
    std::vector<std::unique_ptr<sht::Plan>> plans;   // one per distinct shape
    std::vector<int> field_plan;
    std::vector<int> lmax, nlat, nphi;
    sht::BatchField *h_fields = nullptr;   // pinned staging of the pointer table
    sht::BatchField *d_fields = nullptr;
    int4 *d_tiles = nullptr;               // [synth legendre | synth fft | analys fft | analys legendre]
    int ntile[4] = {0, 0, 0, 0};
    size_t tile_off[4] = {0, 0, 0, 0};
    int *d_counters = nullptr;             // 4 counters
    float *d_inter = nullptr;
    std::vector<size_t> inter_off;
    size_t fft_smem = 0;
    int ctas_legendre_syn = 0, ctas_legendre_ana = 0, ctas_fft = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};   // synthesis, analysis
    cudaEvent_t done = nullptr;                      // last launch (guards h_fields reuse)
};

namespace {

int bfail(int code, const std::string &msg) { return sht::set_error(code, msg); }

void free_batch(sht_batch_plan *b)
{
    if (!b) return;
    for (auto &g : b->graph)
        if (g) cudaGraphExecDestroy(g);
    if (b->done) cudaEventDestroy(b->done);
    if (b->h_fields) cudaFreeHost(b->h_fields);
    if (b->h_copies) cudaFreeHost(b->h_copies);
    cudaFree(b->d_copies);
    cudaFree(b->d_gspec);
    cudaFree(b->d_fields);
    cudaFree(b->d_tiles);
    cudaFree(b->d_counters);
    cudaFree(b->d_inter);
    for (auto &p : b->plans)
        if (p) sht::plan_free(*p);
    delete b;
}

// Gather / scatter of the tensor-core mode: blockIdx.y = copy.
__global__ void __launch_bounds__(256) k_batch_copy(const BatchCopy *__restrict__ copies)
{
    const BatchCopy c = copies[blockIdx.y];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < c.n; i += (long long)gridDim.x * blockDim.x)
        c.dst[i] = c.src[i];
}

// Fill the pointer table (and the tensor-core mode's copy list) for one call.
void fill_fields(sht_batch_plan *b, bool synth, void *const *in, void *const *out)
{
    const bool tc = b->mode == SHT_TC_BF16X3;
    for (int f = 0; f < b->nfields; ++f) {
        sht::BatchField &bf = b->h_fields[f];
        const sht::Plan &p = *b->plans[b->field_plan[f]];
        bf.pv = p.view32();
        bf.in = static_cast<const float *>(in[f]);
        bf.out = static_cast<float *>(out[f]);
        bf.inter = b->d_inter + (tc ? b->inter_tc[f] : b->inter_off[f]);
        if (tc) {
            BatchCopy &c = b->h_copies[f];
            float2 *slot = reinterpret_cast<float2 *>(b->d_gspec + b->field_gspec[f]);
            c.n = p.nlm;
            c.src = synth ? static_cast<const float2 *>(in[f]) : slot;
            c.dst = synth ? slot : static_cast<float2 *>(out[f]);
        }
        // row FFT tiles for power-of-two lengths <= 2^10, else the mixed-radix kernel
        const int H = p.nphi / 2;
        int logH = 0;
        while ((1 << logH) < H) ++logH;
        bf.logH = (1 << logH) == H ? logH : 31;
        bf.G = sht::batch_fft_group(H, p.npairs);
    }
}

cudaError_t launch_copies(sht_batch_plan *b, cudaStream_t s)
{
    k_batch_copy<<<dim3(16, (unsigned)b->nfields), 256, 0, s>>>(b->d_copies);
    return cudaGetLastError();
}

// Tensor-core mode: one contraction per group of equal shape.
cudaError_t group_contractions(sht_batch_plan *b, bool synth, cudaStream_t s)
{
    for (size_t g = 0; g < b->group_fields.size(); ++g) {
        sht::Plan &p = *b->plans[g];
        float *spec = b->d_gspec + b->gspec_off[g], *inter = b->d_inter + b->ginter_off[g];
        const int nb = (int)b->group_fields[g].size();
        cudaError_t e = synth ? sht::tc_batch_legendre(p, true, spec, inter, nb, s)
                              : sht::tc_batch_legendre(p, false, inter, spec, nb, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Enqueue the steps of one direction on stream s.
cudaError_t enqueue(sht_batch_plan *b, bool synth, cudaStream_t s)
{
    cudaError_t e = cudaMemcpyAsync(b->d_fields, b->h_fields, sizeof(sht::BatchField) * b->nfields,
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b->d_counters, 0, 4 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (b->mode == SHT_TC_BF16X3) {
        e = cudaMemcpyAsync(b->d_copies, b->h_copies, sizeof(BatchCopy) * b->nfields, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
        if (synth) {
            if ((e = launch_copies(b, s)) != cudaSuccess) return e;
            if ((e = group_contractions(b, true, s)) != cudaSuccess) return e;
            return sht::launch_batch_fft(true, b->d_fields, b->d_tiles + b->tile_off[1], b->ntile[1],
                                         b->d_counters + 1, b->ctas_fft, b->fft_smem, s);
        }
        e = sht::launch_batch_fft(false, b->d_fields, b->d_tiles + b->tile_off[2], b->ntile[2], b->d_counters + 2,
                                  b->ctas_fft, b->fft_smem, s);
        if (e != cudaSuccess) return e;
        if ((e = group_contractions(b, false, s)) != cudaSuccess) return e;
        return launch_copies(b, s);
    }
    if (synth) {
        e = sht::launch_batch_legendre(true, b->d_fields, b->d_tiles + b->tile_off[0], b->ntile[0], b->d_counters + 0,
                                       b->ctas_legendre_syn, s);
        if (e != cudaSuccess) return e;
        return sht::launch_batch_fft(true, b->d_fields, b->d_tiles + b->tile_off[1], b->ntile[1], b->d_counters + 1,
                                     b->ctas_fft, b->fft_smem, s);
    }
    e = sht::launch_batch_fft(false, b->d_fields, b->d_tiles + b->tile_off[2], b->ntile[2], b->d_counters + 2,
                              b->ctas_fft, b->fft_smem, s);
    if (e != cudaSuccess) return e;
    return sht::launch_batch_legendre(false, b->d_fields, b->d_tiles + b->tile_off[3], b->ntile[3], b->d_counters + 3,
                                      b->ctas_legendre_ana, s);
}

int run(sht_batch_plan *b, bool synth, void *const *in, void *const *out, int use_graph, void *stream)
{
    if (!b) return bfail(SHT_EINVAL, "null batch handle");
    if (!in || !out) return bfail(SHT_EINVAL, "null pointer array");
    for (int f = 0; f < b->nfields; ++f)
        if (!in[f] || !out[f]) return bfail(SHT_EINVAL, "null data pointer for field " + std::to_string(f));
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device)
        return bfail(SHT_EINVAL, "current CUDA device differs from the batch plan's device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the previous launch copies h_fields when it runs: wait for it before overwriting
    cudaError_t e = cudaEventSynchronize(b->done);
    if (e != cudaSuccess) return bfail(SHT_ECUDA, std::string("waiting for the previous batch call: ") + cudaGetErrorString(e));
    fill_fields(b, synth, in, out);
    const int dir = synth ? 0 : 1;
    if (use_graph) {
        if (!b->graph[dir]) {
            cudaStream_t cs;
            e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
            if (e != cudaSuccess) return bfail(SHT_ECUDA, "cudaStreamCreate failed");
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e2 = enqueue(b, synth, cs);
                e = cudaStreamEndCapture(cs, &g);
                if (e == cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph[dir], g, 0);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
            if (e != cudaSuccess) {
                b->graph[dir] = nullptr;
                return bfail(SHT_ECUDA, std::string("capturing the batch graph: ") + cudaGetErrorString(e));
            }
        }
        e = cudaGraphLaunch(b->graph[dir], s);
    } else {
        e = enqueue(b, synth, s);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->done, s);
    if (e != cudaSuccess) return bfail(SHT_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    return SHT_OK;
}

// Automatic mode: time a synthesis + analysis of zero fields on each path
// (direct launches, after a warm-up) and keep the faster.
int choose_mode(sht_batch_plan *b)
{
    const int nf = b->nfields;
    std::vector<size_t> so(nf), go(nf);
    size_t bytes = 0;
    for (int f = 0; f < nf; ++f) {
        const sht::Plan &p = *b->plans[b->field_plan[f]];
        so[f] = bytes;
        bytes = (bytes + (size_t)p.nlm * 8 + 255) & ~(size_t)255;
        go[f] = bytes;
        bytes = (bytes + (size_t)p.nlat * p.nphi * 4 + 255) & ~(size_t)255;
    }
    unsigned char *buf = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&buf, bytes);
    if (e == cudaSuccess) e = cudaMemset(buf, 0, bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    std::vector<void *> spec(nf), grid(nf);
    for (int f = 0; f < nf && buf; ++f) {
        spec[f] = buf + so[f];
        grid[f] = buf + go[f];
    }
    int rc = SHT_OK;
    float best = 0.f;
    int best_mode = SHT_F32;
    const int modes[2] = {SHT_F32, SHT_TC_BF16X3};
    for (int k = 0; k < 2 && e == cudaSuccess && rc == SHT_OK; ++k) {
        b->mode = modes[k];
        for (int it = 0; it < 5 && rc == SHT_OK; ++it) {
            if (it == 2) e = cudaEventRecord(e0, s);
            rc = run(b, true, spec.data(), grid.data(), 0, s);
            if (rc == SHT_OK) rc = run(b, false, grid.data(), spec.data(), 0, s);
        }
        if (rc != SHT_OK) break;
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        b->tuned_ms[k] = ms / 3.f;
        if (e == cudaSuccess && (k == 0 || ms < best)) {
            best = ms;
            best_mode = modes[k];
        }
    }
    if (s) cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(buf);
    b->mode = best_mode;
    if (rc != SHT_OK) return rc;
    if (e != cudaSuccess) return bfail(SHT_ECUDA, std::string("timing the batch paths: ") + cudaGetErrorString(e));
    return SHT_OK;
}

}  // namespace

extern "C" {

int sht_batch_create(int nfields, const int *lmax, const int *nlat, const int *nphi, sht_batch *out)
{
    return sht_batch_create_mode(nfields, lmax, nlat, nphi, SHT_F32, out);
}

int sht_batch_create_mode(int nfields, const int *lmax, const int *nlat, const int *nphi, int mode, sht_batch *out)
{
    if (!out) return bfail(SHT_EINVAL, "out is NULL");
    *out = nullptr;
    if (nfields < 1 || !lmax || !nlat || !nphi) return bfail(SHT_EINVAL, "need nfields >= 1 and size arrays");
    if (mode != SHT_F32 && mode != SHT_TC_BF16X3 && mode != SHT_F32_AUTO)
        return bfail(SHT_EINVAL, "batch mode must be SHT_F32, SHT_TC_BF16X3 or SHT_F32_AUTO");
    for (int f = 0; f < nfields; ++f) {
        if (lmax[f] < 0 || nlat[f] < lmax[f] + 1 || nphi[f] < 2 * lmax[f] + 1)
            return bfail(SHT_EINVAL, "field " + std::to_string(f) + ": need nlat >= lmax+1 and nphi >= 2 lmax + 1");
        if (nphi[f] < 2 || nphi[f] > 4096 || nphi[f] % 2 != 0 || sht::fft_plan_of(nphi[f] / 2) == sht::kFftPlanBad)
            return bfail(SHT_EUNSUPPORTED, "field " + std::to_string(f) + ": nphi must be 2 x 2^a 3^b 5^c in [2, 4096]");
        if ((nlat[f] + 1) / 2 > sht::kBatchMaxPairs)
            return bfail(SHT_EUNSUPPORTED, "field " + std::to_string(f) + ": nlat > 1024 is not supported in a batch");
    }
    sht_batch_plan *b = new (std::nothrow) sht_batch_plan;
    if (!b) return bfail(SHT_ENOMEM, "host allocation failed");
    b->nfields = nfields;
    b->lmax.assign(lmax, lmax + nfields);
    b->nlat.assign(nlat, nlat + nfields);
    b->nphi.assign(nphi, nphi + nfields);
    cudaGetDevice(&b->device);
    std::map<std::tuple<int, int, int>, int> shape_plan;
    for (int f = 0; f < nfields; ++f) {
        auto key = std::make_tuple(lmax[f], nlat[f], nphi[f]);
        auto it = shape_plan.find(key);
        if (it == shape_plan.end()) {
            auto p = std::make_unique<sht::Plan>();
            p->lmax = lmax[f];
            p->mmax = lmax[f];
            p->nlat = nlat[f];
            p->nphi = nphi[f];
            std::string err;
            int rc = sht::plan_build(*p, err);
            if (!rc) rc = sht::plan_seeds32(*p, err);   // the CUDA-core kernels restart from these
            if (rc) {
                sht::plan_free(*p);
                free_batch(b);
                return bfail(rc, err);
            }
            it = shape_plan.emplace(key, (int)b->plans.size()).first;
            b->plans.push_back(std::move(p));
        }
        b->field_plan.push_back(it->second);
    }
    b->group_fields.assign(b->plans.size(), std::vector<int>());
    for (int f = 0; f < nfields; ++f) b->group_fields[b->field_plan[f]].push_back(f);
    // intermediates, tile lists (longest first)
    size_t inter = 0;
    std::vector<std::pair<double, int4>> syn, ffts, ana;
    size_t smem = 0;
    for (int f = 0; f < nfields; ++f) {
        const sht::Plan &p = *b->plans[b->field_plan[f]];
        b->inter_off.push_back(inter);
        inter += (size_t)(p.mmax + 1) * p.npairs * 4;  // floats
        inter = (inter + 63) & ~(size_t)63;
        const int npb = (p.npairs + sht::kBatchSynthPairs - 1) / sht::kBatchSynthPairs;
        for (int m = 0; m <= p.mmax; ++m) {
            for (int pb = 0; pb < npb; ++pb) {
                const int np = std::min(sht::kBatchSynthPairs, p.npairs - pb * sht::kBatchSynthPairs);
                syn.push_back({(double)(p.lmax - m + 1) * (np + 32), make_int4(f, m, pb, 0)});
            }
            ana.push_back({(double)(p.lmax - m + 1) * (p.npairs + 32), make_int4(f, m, 0, 0)});
        }
        int logH = 0;
        while ((1 << logH) < p.nphi / 2) ++logH;
        const int G = sht::batch_fft_group(p.nphi / 2, p.npairs);
        smem = std::max(smem, sht::batch_fft_smem(p.nphi / 2, G));
        for (int p0 = 0; p0 < p.npairs; p0 += G)
            ffts.push_back({(double)G * p.nphi * (logH + 2) + p.mmax, make_int4(f, p0, 0, 0)});
    }
    // tensor-core layout: each group's intermediates and spectra contiguous
    bool tc_ok = mode != SHT_F32;
    size_t inter_tc = 0, gspec = 0;
    b->inter_tc.assign(nfields, 0);
    b->field_gspec.assign(nfields, 0);
    for (size_t g = 0; g < b->plans.size() && tc_ok; ++g) {
        const sht::Plan &p = *b->plans[g];
        const size_t stride = (size_t)(p.mmax + 1) * p.npairs * 4;
        b->ginter_off.push_back(inter_tc);
        b->gspec_off.push_back(gspec);
        for (size_t i = 0; i < b->group_fields[g].size(); ++i) {
            b->inter_tc[b->group_fields[g][i]] = inter_tc + i * stride;
            b->field_gspec[b->group_fields[g][i]] = gspec + i * (size_t)p.nlm * 2;
        }
        inter_tc = (inter_tc + b->group_fields[g].size() * stride + 63) & ~(size_t)63;
        gspec = (gspec + b->group_fields[g].size() * (size_t)p.nlm * 2 + 63) & ~(size_t)63;
        const int rc = sht::tc_batch_prepare(*b->plans[g], (int)b->group_fields[g].size());
        if (rc) {
            if (mode == SHT_TC_BF16X3) {
                free_batch(b);
                return rc;   // message set by the preparation
            }
            tc_ok = false;   // automatic mode: keep the CUDA-core path
        }
    }
    if (tc_ok) inter = std::max(inter, inter_tc);
    auto by_cost = [](const std::pair<double, int4> &a, const std::pair<double, int4> &c) { return a.first > c.first; };
    std::stable_sort(syn.begin(), syn.end(), by_cost);
    std::stable_sort(ffts.begin(), ffts.end(), by_cost);
    std::stable_sort(ana.begin(), ana.end(), by_cost);
    std::vector<int4> tiles;
    auto append = [&](int k, const std::vector<std::pair<double, int4>> &v) {
        b->tile_off[k] = tiles.size();
        b->ntile[k] = (int)v.size();
        for (auto &x : v) tiles.push_back(x.second);
    };
    append(0, syn);
    append(1, ffts);
    append(2, ffts);
    append(3, ana);
    b->fft_smem = smem;
    if (sht::batch_fft_prepare(smem) != cudaSuccess) {
        free_batch(b);
        return bfail(SHT_ECUDA, "setting the FFT kernel's shared-memory size failed");
    }
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    b->ctas_legendre_syn = sms * 8;   // 128-thread CTAs
    b->ctas_legendre_ana = sms * 4;   // 256-thread CTAs
    b->ctas_fft = sms * std::max(1, (int)std::min<size_t>(8, (200 * 1024) / std::max<size_t>(smem, 1)));
    cudaError_t e = cudaMallocHost(&b->h_fields, sizeof(sht::BatchField) * nfields);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_fields, sizeof(sht::BatchField) * nfields);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tiles, sizeof(int4) * tiles.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counters, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_inter, sizeof(float) * std::max<size_t>(inter, 64));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && tc_ok) e = cudaMallocHost(&b->h_copies, sizeof(BatchCopy) * nfields);
    if (e == cudaSuccess && tc_ok) e = cudaMalloc(&b->d_copies, sizeof(BatchCopy) * nfields);
    if (e == cudaSuccess && tc_ok) e = cudaMalloc(&b->d_gspec, sizeof(float) * std::max<size_t>(gspec, 64));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        free_batch(b);
        return bfail(SHT_ENOMEM, std::string("allocating the batch plan: ") + cudaGetErrorString(e));
    }
    b->mode = mode == SHT_TC_BF16X3 ? SHT_TC_BF16X3 : SHT_F32;
    if (mode == SHT_F32_AUTO && tc_ok) {
        const int rc = choose_mode(b);
        if (rc) {
            sht_batch_destroy(b);
            return rc;
        }
    }
    *out = b;
    return SHT_OK;
}

int sht_batch_mode(sht_batch b, float *ms_f32, float *ms_tc)
{
    if (!b) return bfail(SHT_EINVAL, "null batch handle");
    if (ms_f32) *ms_f32 = b->tuned_ms[0];
    if (ms_tc) *ms_tc = b->tuned_ms[1];
    return b->mode;
}

void sht_batch_destroy(sht_batch b)
{
    if (!b) return;
    cudaEventSynchronize(b->done);
    free_batch(b);
}

int sht_batch_synth(sht_batch b, void *const *spec, void *const *grid, int use_graph, void *stream)
{
    return run(b, true, spec, grid, use_graph, stream);
}

int sht_batch_analys(sht_batch b, void *const *grid, void *const *spec, int use_graph, void *stream)
{
    return run(b, false, grid, spec, use_graph, stream);
}

}  // extern "C"
