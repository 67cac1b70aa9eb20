// capi.cu -- the extern "C" entry points declared in include/sht.h.
// Argument checking, scratch management and the launch sequence of each
// transform (Legendre stage + longitude FFT, in the order of Sec. 2.2/2.3).
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <new>
#include <string>

#include "sht_internal.h"

struct sht_plan {
    sht::Plan p;
};

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}


int check_handle(sht_handle h)
{
    if (!h) return fail(SHT_EINVAL, "null handle");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(SHT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev != h->p.device)
        return fail(SHT_EINVAL, "current CUDA device differs from the device the plan was created on");
    return SHT_OK;
}

int check_mode(int mode)
{
    if (mode != SHT_F64 && mode != SHT_F32 && mode != SHT_TC_BF16X3 && mode != SHT_F32_AUTO && mode != SHT_TC_OTF &&
        mode != SHT_TC_F64)
        return fail(SHT_EINVAL, "unknown mode");
    return SHT_OK;
}

// Frees whatever ensure_panels / ensure_vec_panels allocated.
void free_panels(sht::Plan &p)
{
    cudaFree(p.panel_s); cudaFree(p.panel_a); cudaFree(p.d_off_s); cudaFree(p.d_off_a); cudaFree(p.d_dchunk);
    cudaFree(p.d_c0_s); cudaFree(p.d_c0_a); cudaFree(p.d_gf_s); cudaFree(p.d_gf_a);
    p.panel_s = p.panel_a = nullptr;
    p.d_off_s = p.d_off_a = p.d_dchunk = nullptr;
    p.d_c0_s = p.d_c0_a = nullptr;
    p.d_gf_s = p.d_gf_a = nullptr;
}

// Static polar optimisation (Sec. 3.1): per (m, tile) and per 8-row group of
// the tile, the first panel chunk holding a value >= the plan's threshold;
// the fractions of panel bytes skipped.
cudaError_t first_live_scalar(sht::Plan &p)
{
    int ts = 0, ta = 0;
    cudaError_t e = sht::launch_panel_first_live(true, p.lmax, p.mmax, p.mres, p.npairs, p.d_off_s, p.panel_s, p.polar_thr,
                                                 p.d_c0_s, ts, 0, p.d_gf_s);
    if (e == cudaSuccess)
        e = sht::launch_panel_first_live(false, p.lmax, p.mmax, p.mres, p.npairs, p.d_off_a, p.panel_a, p.polar_thr,
                                         p.d_c0_a, ta, 0, p.d_gf_a);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = sht::tc_polar_stats(p.lmax, p.mmax, p.mres, p.npairs, p.d_c0_s, p.d_c0_a, p.polar_skip_s, p.polar_skip_a,
                                p.d_gf_s, p.d_gf_a);
    return e;
}

// Vector transforms: the first chunk live in P or in dP (tmp: scratch of
// (mmax+1) * max(tiles) ints; the scalar tables must be current).
cudaError_t first_live_vector(sht::Plan &p, int *tmp)
{
    int T_s = 0, T_a = 0, nt = 0;
    sht::tc_tile_counts(p.lmax, p.npairs, T_s, T_a);
    const int ns = (p.mmax + 1) * T_s, na = (p.mmax + 1) * T_a;
    cudaError_t e = sht::launch_panel_first_live(true, p.lmax, p.mmax, p.mres, p.npairs, p.d_off_s, p.dpanel_s, p.polar_thr,
                                                 tmp, nt, 0);
    if (e == cudaSuccess) e = sht::launch_min_int(p.d_c0_s, tmp, p.d_c0v_s, ns, 0);
    if (e == cudaSuccess)
        e = sht::launch_panel_first_live(false, p.lmax, p.mmax, p.mres, p.npairs, p.d_off_a, p.dpanel_a, p.polar_thr, tmp,
                                         nt, 0);
    if (e == cudaSuccess) e = sht::launch_min_int(p.d_c0_a, tmp, p.d_c0v_a, na, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e;
}

// Build the tensor-core panels once (allocates about (lmax+1)^3 bytes): the
// P_n^m panels in both operand layouts, per-order offsets, and the first
// chunk above the polar threshold of every (m, tile).
int ensure_panels(sht::Plan &p)
{
    if (p.panel_s) return SHT_OK;
    std::vector<unsigned long long> off_s, off_a, dchunk;
    size_t bs = 0, ba = 0, nch = 0;
    sht::tc_panel_layout(p.lmax, p.mmax, p.mres, p.npairs, off_s, off_a, bs, ba, dchunk, nch);
    const size_t ob = off_s.size() * sizeof(unsigned long long);
    int T_s = 0, T_a = 0;
    sht::tc_tile_counts(p.lmax, p.npairs, T_s, T_a);
    cudaError_t e = cudaMalloc(&p.panel_s, bs);
    if (e == cudaSuccess) e = cudaMalloc(&p.panel_a, ba);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_off_s, ob);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_off_a, ob);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_dchunk, ob);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_c0_s, sizeof(int) * (size_t)(p.mmax + 1) * T_s);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_c0_a, sizeof(int) * (size_t)(p.mmax + 1) * T_a);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_gf_s, sizeof(unsigned short) * 16 * (size_t)(p.mmax + 1) * T_s);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_gf_a, sizeof(unsigned short) * 16 * (size_t)(p.mmax + 1) * T_a);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_panels(p);
        return fail(SHT_ENOMEM, std::string("cudaMalloc(tensor-core panels): ") + cudaGetErrorString(e));
    }
    p.tc_nchunk_s = nch;
    e = cudaMemcpy(p.d_off_s, off_s.data(), ob, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p.d_off_a, off_a.data(), ob, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p.d_dchunk, dchunk.data(), ob, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p.panel_s, 0, bs);
    if (e == cudaSuccess) e = cudaMemset(p.panel_a, 0, ba);
    if (e == cudaSuccess)
        e = sht::launch_build_panels(p.view64(), p.d_off_s, p.d_off_a, p.panel_s, p.panel_a, false, 0);
    if (e == cudaSuccess) e = first_live_scalar(p);
    if (e != cudaSuccess) {
        free_panels(p);
        return fail(SHT_ECUDA, std::string("building tensor-core panels: ") + cudaGetErrorString(e));
    }
    return SHT_OK;
}

void free_vec_panels(sht::Plan &p)
{
    cudaFree(p.dpanel_s); cudaFree(p.dpanel_a); cudaFree(p.d_c0v_s); cudaFree(p.d_c0v_a);
    p.dpanel_s = p.dpanel_a = nullptr;
    p.d_c0v_s = p.d_c0v_a = nullptr;
    for (int h = 0; h < 2; ++h) {
        cudaFree(p.d_schedv_s[h]);
        cudaFree(p.d_schedv_a[h]);
        p.d_schedv_s[h] = p.d_schedv_a[h] = nullptr;
    }
    p.schedv_ctas = 0;
}

// Work lists of the persistent vector contraction (one CTA per SM) for one
// and two field halves, from the current first-live chunks; rebuilt when
// the polar threshold changes (the lists only balance the work).
cudaError_t vec_schedules(sht::Plan &p)
{
    int T_s = 0, T_a = 0, dev = 0, sms = 0;
    sht::tc_tile_counts(p.lmax, p.npairs, T_s, T_a);
    std::vector<int> c0s((size_t)(p.mmax + 1) * T_s), c0a((size_t)(p.mmax + 1) * T_a), cost, group, sc;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMemcpy(c0s.data(), p.d_c0v_s, sizeof(int) * c0s.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(c0a.data(), p.d_c0v_a, sizeof(int) * c0a.size(), cudaMemcpyDeviceToHost);
    for (int dir = 0; dir < 2 && e == cudaSuccess; ++dir)
        for (int h = 0; h < 2 && e == cudaSuccess; ++h) {
            sht::tc_vec_costs(p.lmax, p.mmax, p.mres, p.npairs, dir == 0, h + 1, dir == 0 ? c0s : c0a, cost, group);
            sht::schedule_lpt(cost, group, sms, sc);
            int *&d = dir == 0 ? p.d_schedv_s[h] : p.d_schedv_a[h];
            cudaFree(d);
            d = nullptr;
            e = cudaMalloc(&d, sizeof(int) * sc.size());
            if (e == cudaSuccess) e = cudaMemcpy(d, sc.data(), sizeof(int) * sc.size(), cudaMemcpyHostToDevice);
        }
    if (e == cudaSuccess) p.schedv_ctas = sms;
    return e;
}

// The sin(theta) dP/dtheta panels of the vector transforms (same layouts and
// offsets as the P panels) and the first chunk live in either matrix.
int ensure_vec_panels(sht::Plan &p)
{
    int rc = ensure_panels(p);
    if (rc) return rc;
    if (p.dpanel_s) return SHT_OK;
    std::vector<unsigned long long> off_s, off_a, dchunk;
    size_t bs = 0, ba = 0, nch = 0;
    sht::tc_panel_layout(p.lmax, p.mmax, p.mres, p.npairs, off_s, off_a, bs, ba, dchunk, nch);
    int T_s = 0, T_a = 0;
    sht::tc_tile_counts(p.lmax, p.npairs, T_s, T_a);
    const size_t ns = (size_t)(p.mmax + 1) * T_s, na = (size_t)(p.mmax + 1) * T_a;
    int *tmp = nullptr;
    cudaError_t e = cudaMalloc(&p.dpanel_s, bs);
    if (e == cudaSuccess) e = cudaMalloc(&p.dpanel_a, ba);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_c0v_s, sizeof(int) * ns);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_c0v_a, sizeof(int) * na);
    if (e == cudaSuccess) e = cudaMalloc(&tmp, sizeof(int) * (ns > na ? ns : na));
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(tmp);
        free_vec_panels(p);
        return fail(SHT_ENOMEM, std::string("cudaMalloc(vector tensor-core panels): ") + cudaGetErrorString(e));
    }
    e = cudaMemset(p.dpanel_s, 0, bs);
    if (e == cudaSuccess) e = cudaMemset(p.dpanel_a, 0, ba);
    if (e == cudaSuccess)
        e = sht::launch_build_panels(p.view64(), p.d_off_s, p.d_off_a, p.dpanel_s, p.dpanel_a, true, 0);
    if (e == cudaSuccess) e = first_live_vector(p, tmp);
    cudaFree(tmp);
    if (e == cudaSuccess) e = vec_schedules(p);
    if (e != cudaSuccess) {
        free_vec_panels(p);
        return fail(SHT_ECUDA, std::string("building vector tensor-core panels: ") + cudaGetErrorString(e));
    }
    return SHT_OK;
}

void free_otf(sht::Plan &p)
{
    cudaFree(p.otf_seeds); cudaFree(p.d_segoff); cudaFree(p.d_c0o_s); cudaFree(p.d_c0o_a);
    p.otf_seeds = nullptr;
    p.d_segoff = nullptr;
    p.d_c0o_s = p.d_c0o_a = nullptr;
}

// Seeds of the on-the-fly mode (float4 per pair and 32-degree segment, about
// 16 (lmax+1)^2 npairs / 64 bytes: 138 MB at lmax = 1023) and its polar-skip
// tables, built once by the FP64 recurrence.
cudaError_t otf_build(sht::Plan &p, int *flag_dev)
{
    cudaError_t e = cudaMemset(flag_dev, 0, sizeof(int));
    if (e == cudaSuccess)
        e = sht::launch_build_seeds(p.view64(), p.d_segoff, p.otf_seeds, p.polar_thr, p.d_c0o_s, p.d_c0o_a, flag_dev,
                                    0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = sht::tc_polar_stats(p.lmax, p.mmax, p.mres, p.npairs, p.d_c0o_s, p.d_c0o_a, p.otf_skip_s, p.otf_skip_a);
    return e;
}

int ensure_otf(sht::Plan &p)
{
    if (p.otf_state > 0) return SHT_OK;
    if (p.otf_state < 0)
        return fail(SHT_EUNSUPPORTED, "on-the-fly mode: the FP32 recurrence would leave the FP32 range for this plan");
    std::vector<unsigned long long> segoff;
    const size_t nseg = sht::otf_segment_offsets(p.lmax, p.mmax, p.mres, segoff);
    std::vector<unsigned long long> off_s, off_a, dchunk;
    size_t bs = 0, ba = 0, nch = 0;
    sht::tc_panel_layout(p.lmax, p.mmax, p.mres, p.npairs, off_s, off_a, bs, ba, dchunk, nch);
    int T_s = 0, T_a = 0;
    sht::tc_tile_counts(p.lmax, p.npairs, T_s, T_a);
    int *flag = nullptr;
    cudaError_t e = cudaMalloc(&p.otf_seeds, sizeof(float4) * nseg * (size_t)p.npairs);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_segoff, sizeof(unsigned long long) * segoff.size());
    if (e == cudaSuccess) e = cudaMalloc(&p.d_c0o_s, sizeof(int) * (size_t)(p.mmax + 1) * T_s);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_c0o_a, sizeof(int) * (size_t)(p.mmax + 1) * T_a);
    if (e == cudaSuccess) e = cudaMalloc(&flag, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(flag);
        free_otf(p);
        return fail(SHT_ENOMEM, std::string("cudaMalloc(on-the-fly seeds): ") + cudaGetErrorString(e));
    }
    p.tc_nchunk_s = nch;
    e = cudaMemcpy(p.d_segoff, segoff.data(), sizeof(unsigned long long) * segoff.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = otf_build(p, flag);
    int hflag = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(flag);
    if (e != cudaSuccess) {
        free_otf(p);
        return fail(SHT_ECUDA, std::string("building on-the-fly seeds: ") + cudaGetErrorString(e));
    }
    if (hflag) {
        free_otf(p);
        p.otf_state = -1;
        return fail(SHT_EUNSUPPORTED, "on-the-fly mode: the FP32 recurrence would leave the FP32 range for this plan");
    }
    p.otf_state = 1;
    return SHT_OK;
}

// FP32 CUDA-core path: the recurrence restart states (plan_seeds32), built on
// the first call that needs them.
int ensure_seeds32(sht::Plan &p)
{
    std::string err;
    const int rc = sht::plan_seeds32(p, err);
    return rc ? fail(rc, err) : SHT_OK;
}

// FP64 CUDA-core scalar path: the restart states and first-live table of the
// static polar optimisation (plan_seeds64), built on the first call that needs them.
int ensure_seeds64(sht::Plan &p)
{
    std::string err;
    const int rc = sht::plan_seeds64(p, err);
    return rc ? fail(rc, err) : SHT_OK;
}

size_t elem_size(int mode) { return (mode == SHT_F64 || mode == SHT_TC_F64) ? sizeof(double) : sizeof(float); }

// FP64-accurate tensor-core mode: digit-slice panels (about 6 (lmax+1)^3
// bytes), row exponents and first nonzero chunks, built once per plan.
int ensure_panels64(sht::Plan &p)
{
    if (p.p64_s) return SHT_OK;
    if (p.lmax > 1023 || p.npairs > 512)
        return fail(SHT_EUNSUPPORTED, "SHT_TC_F64 needs lmax <= 1023 and nlat <= 1024");
    std::vector<unsigned long long> off_s, off_a, dchunk;
    size_t bs = 0, ba = 0, nch = 0;
    sht::tc64_panel_layout(p.lmax, p.mmax, p.mres, p.npairs, off_s, off_a, bs, ba, dchunk, nch);
    const size_t ob = off_s.size() * sizeof(unsigned long long);
    int T_s = 0, T_a = 0;
    sht::tc_tile_counts(p.lmax, p.npairs, T_s, T_a);
    cudaError_t e = cudaMalloc(&p.p64_s, bs);
    if (e == cudaSuccess) e = cudaMalloc(&p.p64_a, ba);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_off64_s, ob);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_off64_a, ob);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_dchunk64, ob);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_e64_s, sizeof(int) * (size_t)(p.mmax + 1) * p.npairs);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_e64_a, sizeof(int) * (size_t)p.nlm);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_c064_s, sizeof(int) * (size_t)(p.mmax + 1) * T_s);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_c064_a, sizeof(int) * (size_t)(p.mmax + 1) * T_a);
    const size_t ngs = (size_t)(p.mmax + 1) * T_s * 32, nga = (size_t)(p.mmax + 1) * T_a * 32;   // 2 parities x 16 groups
    if (e == cudaSuccess) e = cudaMalloc(&p.d_gf64_s, sizeof(unsigned short) * ngs);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_gf64_a, sizeof(unsigned short) * nga);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_zero64, sht::tc64_zero_bytes());
    if (e == cudaSuccess) e = cudaMemset(p.d_zero64, 0, sht::tc64_zero_bytes());
    if (e == cudaSuccess) e = cudaMalloc(&p.d_fcol, sizeof(int) * (size_t)sht::tc64_max_batch());
    if (e == cudaSuccess) e = cudaMemcpy(p.d_off64_s, off_s.data(), ob, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p.d_off64_a, off_a.data(), ob, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p.d_dchunk64, dchunk.data(), ob, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p.p64_s, 0, bs);
    if (e == cudaSuccess) e = cudaMemset(p.p64_a, 0, ba);
    if (e == cudaSuccess)
        e = sht::tc64_build(p.view64(), p.d_off64_s, p.d_off64_a, p.p64_s, p.p64_a, p.d_e64_s, p.d_e64_a, p.d_c064_s,
                            p.d_c064_a, p.d_gf64_s, p.d_gf64_a, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaGetLastError();
        sht::plan_free_tc64(p);
        return fail(SHT_ENOMEM, std::string("building the digit-slice panels: ") + cudaGetErrorString(e));
    }
    p.nchunk64_s = nch;
    {
        // balanced work lists of the persistent contraction, two CTAs per SM
        int dev = 0, sms = 0;
        std::vector<int> c0s((size_t)(p.mmax + 1) * T_s), c0a((size_t)(p.mmax + 1) * T_a), ss, sa;
        std::vector<unsigned short> gfs(ngs), gfa(nga);
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaMemcpy(c0s.data(), p.d_c064_s, sizeof(int) * c0s.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(c0a.data(), p.d_c064_a, sizeof(int) * c0a.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(gfs.data(), p.d_gf64_s, sizeof(unsigned short) * ngs, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(gfa.data(), p.d_gf64_a, sizeof(unsigned short) * nga, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) {
            sms *= sht::tc64_ctas_per_sm();
            std::vector<int> cost, group;
            sht::tc64_costs(p.lmax, p.mmax, p.mres, p.npairs, true, c0s, gfs, cost, group);
            sht::schedule_lpt(cost, group, sms, ss);
            sht::tc64_costs(p.lmax, p.mmax, p.mres, p.npairs, false, c0a, gfa, cost, group);
            sht::schedule_lpt(cost, group, sms, sa);
            // fractions of the panel bytes the contraction does not read
            sht::tc64_skip_stats(p.lmax, p.mmax, p.mres, p.npairs, c0s, c0a, gfs, gfa, p.skip64_s, p.skip64_a);
            e = cudaMalloc(&p.d_sched64_s, sizeof(int) * ss.size());
        }
        if (e == cudaSuccess) e = cudaMalloc(&p.d_sched64_a, sizeof(int) * sa.size());
        if (e == cudaSuccess) e = cudaMemcpy(p.d_sched64_s, ss.data(), sizeof(int) * ss.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(p.d_sched64_a, sa.data(), sizeof(int) * sa.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaGetLastError();
            sht::plan_free_tc64(p);
            return fail(SHT_ENOMEM, std::string("scheduling the digit-slice contraction: ") + cudaGetErrorString(e));
        }
        p.sched64_ctas = sms;
    }
    return SHT_OK;
}

// Scratch of SHT_TC_F64: the FP64 intermediate of up to 16 fields, then the
// blocked digit data.
size_t tc64_data_offset(const sht::Plan &p, int batch)
{
    const int nb = batch > sht::tc64_max_batch() ? sht::tc64_max_batch() : batch;
    return ((size_t)nb * (p.mmax + 1) * p.npairs * 4 * sizeof(double) + 255) & ~(size_t)255;
}
size_t tc64_work_bytes(const sht::Plan &p, int batch)
{
    return tc64_data_offset(p, batch) + sht::tc64_data_bytes(p.mmax, p.npairs, p.nchunk64_s);
}

int run_tc64(sht::Plan &p, bool synth, const void *in_, void *out_, int batch, sht::Op op, cudaStream_t s);

// Tensor-core scalar transforms: the Legendre contraction on tcgen05, FFTs in FP32.
int run_synth_tc(sht::Plan &p, const void *spec, void *grid, int batch, sht::Op op, cudaStream_t s);
int run_analys_tc(sht::Plan &p, const void *grid, void *spec, int batch, sht::Op op, cudaStream_t s);
int run_otf(sht::Plan &p, bool synth, const void *in_, void *out_, int batch, sht::Op op, cudaStream_t s);
int run_synth_vec_tc(sht::Plan &p, const void *S, const void *T, void *vt, void *vp, int batch, sht::Op op,
                     cudaStream_t s);
int run_analys_vec_tc(sht::Plan &p, const void *vt, const void *vp, void *S, void *T, int batch, sht::Op op,
                      cudaStream_t s);

// Bytes of one [batch][mmax+1][npairs][2] complex intermediate.
size_t inter_bytes(const sht::Plan &p, int batch, int mode)
{
    if (mode == SHT_TC_BF16X3 && batch > sht::tc_max_batch()) batch = sht::tc_max_batch();
    return (size_t)batch * (p.mmax + 1) * p.npairs * 4 * elem_size(mode);
}

// Tensor-core mode scratch: the FP32 intermediate(s) of up to the tensor-core
// batch limit of fields, then the blocked bf16 data operand.  Size and offset
// depend only on min(batch, limit) and on whether the transform is a vector one.
int tc_chunk(bool vec) { return vec ? sht::tc_vec_max_batch() : sht::tc_max_batch(); }

size_t tc_data_offset(const sht::Plan &p, int batch, bool vec)
{
    const int nb = batch > tc_chunk(vec) ? tc_chunk(vec) : batch;
    const size_t inter = (size_t)nb * (p.mmax + 1) * p.npairs * 4 * sizeof(float);
    return ((vec ? 2 : 1) * inter + 255) & ~(size_t)255;
}

size_t tc_work_bytes(const sht::Plan &p, int batch, bool vec)
{
    const int nb = batch > tc_chunk(vec) ? tc_chunk(vec) : batch;
    return tc_data_offset(p, batch, vec) + sht::tc_data_bytes(p.mmax, p.npairs, p.tc_nchunk_s, nb, vec);
}

int ensure_work(sht::Plan &p, size_t bytes)
{
    if (bytes <= p.work_bytes) return SHT_OK;
    if (p.work) {
        cudaError_t e = cudaFree(p.work);  // cudaFree waits for work using the old buffer
        p.work = nullptr;
        p.work_bytes = 0;
        if (e != cudaSuccess) return fail(SHT_ECUDA, std::string("cudaFree(scratch): ") + cudaGetErrorString(e));
    }
    cudaError_t e = cudaMalloc(&p.work, bytes);
    if (e != cudaSuccess) {
        p.work = nullptr;
        cudaGetLastError();
        return fail(SHT_ENOMEM, std::string("cudaMalloc(scratch): ") + cudaGetErrorString(e));
    }
    p.work_bytes = bytes;
    return SHT_OK;
}

int launched(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) return fail(SHT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return SHT_OK;
}

// Launch through f(), bracketed by timing events when profiling is enabled.
template <typename F>
int timed(sht::Plan &p, int kind, cudaStream_t s, const char *what, F &&f)
{
    sht::KernelTimer &t = p.timer;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (t.enabled) {
        while (t.pool.size() < t.used + 2) {
            cudaEvent_t ev;
            if (cudaEventCreate(&ev) != cudaSuccess) return fail(SHT_ECUDA, "cudaEventCreate failed");
            t.pool.push_back(ev);
        }
        e0 = t.pool[t.used];
        e1 = t.pool[t.used + 1];
        cudaEventRecord(e0, s);
    }
    cudaError_t e = f();
    if (t.enabled) {
        cudaEventRecord(e1, s);
        t.used += 2;
        t.kinds.push_back(kind);
    }
    return launched(e, what);
}

int prologue(sht_handle h, int batch, int mode, int nptr, const void *const *ptrs)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if ((rc = check_mode(mode))) return rc;
    if (batch < 1) return fail(SHT_EINVAL, "batch must be >= 1");
    for (int i = 0; i < nptr; ++i)
        if (!ptrs[i]) return fail(SHT_EINVAL, "null data pointer");
    return SHT_OK;
}

// Tuned kernel shape for (mode, batch), or the defaults.
sht::TunedShape tuned_shape(const sht::Plan &p, int mode, int batch)
{
    const long long key = ((long long)mode << 32) | (unsigned)batch;
    for (const auto &kv : p.tuned)
        if (kv.first == key) return kv.second;
    return sht::TunedShape();
}

void set_tuned(sht::Plan &p, int mode, int batch, const sht::TunedShape &t)
{
    const long long key = ((long long)mode << 32) | (unsigned)batch;
    for (auto &kv : p.tuned)
        if (kv.first == key) { kv.second = t; return; }
    p.tuned.push_back({key, t});
}

template <typename T> constexpr int mode_of_type() { return sizeof(T) == 8 ? SHT_F64 : SHT_F32; }

// The two directions of the scalar transform, parameterised by precision.
template <typename T>
int run_synth(sht::Plan &p, const sht::PlanView<T> &pv, const void *spec, void *grid, int batch, sht::Op op,
              cudaStream_t s)
{
    T *eo = static_cast<T *>(p.work);
    const sht::TunedShape ts = tuned_shape(p, mode_of_type<T>(), batch);
    int rc = timed(p, SHT_K_LEGENDRE_SYNTH, s, "legendre synthesis launch", [&] {
        return sht::launch_legendre_synth_cfg<T>(pv, static_cast<const T *>(spec), eo, batch, op, ts.synth_lpt,
                                                 ts.synth_bc, s);
    });
    if (rc) return rc;
    return timed(p, SHT_K_FFT_SYNTH, s, "fft synthesis launch", [&] {
        return sht::launch_fft_synth<T>(pv, eo, static_cast<T *>(grid), batch, op, s);
    });
}

template <typename T>
int run_analys(sht::Plan &p, const sht::PlanView<T> &pv, const void *grid, void *spec, int batch, sht::Op op,
               cudaStream_t s)
{
    T *sd = static_cast<T *>(p.work);
    int rc = timed(p, SHT_K_FFT_ANALYS, s, "fft analysis launch", [&] {
        return sht::launch_fft_analys<T>(pv, static_cast<const T *>(grid), sd, batch, op, false, s);
    });
    if (rc) return rc;
    const sht::TunedShape ts = tuned_shape(p, mode_of_type<T>(), batch);
    return timed(p, SHT_K_LEGENDRE_ANALYS, s, "legendre analysis launch", [&] {
        return sht::launch_legendre_analys_cfg<T>(pv, sd, static_cast<T *>(spec), batch, op, ts.analys_lpt,
                                                  ts.analys_bc, s);
    });
}

template <typename T>
int run_synth_vec(sht::Plan &p, const sht::PlanView<T> &pv, const void *S, const void *Tc, void *vt, void *vp,
                  int batch, sht::Op op, cudaStream_t s)
{
    T *eot = static_cast<T *>(p.work);
    T *eop = eot + (size_t)batch * (p.mmax + 1) * p.npairs * 4;
    int rc = timed(p, SHT_K_LEGENDRE_SYNTH_VEC, s, "legendre vector synthesis launch", [&] {
        return sht::launch_legendre_synth_vec<T>(pv, static_cast<const T *>(S), static_cast<const T *>(Tc), eot, eop,
                                                 batch, op, s);
    });
    if (rc) return rc;
    rc = timed(p, SHT_K_FFT_SYNTH, s, "fft synthesis launch",
               [&] { return sht::launch_fft_synth<T>(pv, eot, static_cast<T *>(vt), batch, op, s); });
    if (rc) return rc;
    return timed(p, SHT_K_FFT_SYNTH, s, "fft synthesis launch",
                 [&] { return sht::launch_fft_synth<T>(pv, eop, static_cast<T *>(vp), batch, op, s); });
}

template <typename T>
int run_analys_vec(sht::Plan &p, const sht::PlanView<T> &pv, const void *vt, const void *vp, void *S, void *Tc,
                   int batch, sht::Op op, cudaStream_t s)
{
    T *sdt = static_cast<T *>(p.work);
    T *sdp = sdt + (size_t)batch * (p.mmax + 1) * p.npairs * 4;
    int rc = timed(p, SHT_K_FFT_ANALYS, s, "fft analysis launch", [&] {
        return sht::launch_fft_analys<T>(pv, static_cast<const T *>(vt), sdt, batch, op, true, s);
    });
    if (rc) return rc;
    rc = timed(p, SHT_K_FFT_ANALYS, s, "fft analysis launch", [&] {
        return sht::launch_fft_analys<T>(pv, static_cast<const T *>(vp), sdp, batch, op, true, s);
    });
    if (rc) return rc;
    return timed(p, SHT_K_LEGENDRE_ANALYS_VEC, s, "legendre vector analysis launch", [&] {
        return sht::launch_legendre_analys_vec<T>(pv, sdt, sdp, static_cast<T *>(S), static_cast<T *>(Tc), batch, op,
                                                  s);
    });
}

// SHT_F32_AUTO resolves to the path sht_tune found faster for this batch.
int resolve_mode(const sht::Plan &p, int mode, int batch, bool vector)
{
    if (vector) {
        if (mode == SHT_F32_AUTO) return SHT_F32;
        if (mode == SHT_TC_OTF) return SHT_TC_BF16X3;   // vector transforms use the panels
        if (mode == SHT_TC_F64) return SHT_F64;         // ... and the FP64 recurrence
        return mode;
    }
    if (mode != SHT_F32_AUTO) return mode;
    return tuned_shape(p, SHT_F32_AUTO, batch).auto_mode;
}

int scalar_s2g(sht_handle h, const void *spec, void *grid, int batch, int mode, void *stream, sht::Op op)
{
    const void *ptrs[2] = {spec, grid};
    int rc = prologue(h, batch, mode, 2, ptrs);
    if (rc) return rc;
    mode = resolve_mode(h->p, mode, batch, false);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (mode == SHT_TC_BF16X3) {
        if ((rc = ensure_panels(h->p))) return rc;
        if ((rc = ensure_work(h->p, tc_work_bytes(h->p, batch, false)))) return rc;
        return run_synth_tc(h->p, spec, grid, batch, op, s);
    }
    if (mode == SHT_TC_OTF) {
        if ((rc = ensure_otf(h->p))) return rc;
        if ((rc = ensure_work(h->p, tc_work_bytes(h->p, batch, false)))) return rc;
        return run_otf(h->p, true, spec, grid, batch, op, s);
    }
    if (mode == SHT_TC_F64) {
        if ((rc = ensure_panels64(h->p))) return rc;
        if ((rc = ensure_work(h->p, tc64_work_bytes(h->p, batch)))) return rc;
        return run_tc64(h->p, true, spec, grid, batch, op, s);
    }
    if (mode == SHT_F32 && (rc = ensure_seeds32(h->p))) return rc;
    if (mode == SHT_F64 && (rc = ensure_seeds64(h->p))) return rc;
    if ((rc = ensure_work(h->p, inter_bytes(h->p, batch, mode)))) return rc;
    if (mode == SHT_F64) return run_synth<double>(h->p, h->p.view64(), spec, grid, batch, op, s);
    return run_synth<float>(h->p, h->p.view32(), spec, grid, batch, op, s);
}

int scalar_g2s(sht_handle h, const void *grid, void *spec, int batch, int mode, void *stream, sht::Op op)
{
    const void *ptrs[2] = {grid, spec};
    int rc = prologue(h, batch, mode, 2, ptrs);
    if (rc) return rc;
    mode = resolve_mode(h->p, mode, batch, false);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (mode == SHT_TC_BF16X3) {
        if ((rc = ensure_panels(h->p))) return rc;
        if ((rc = ensure_work(h->p, tc_work_bytes(h->p, batch, false)))) return rc;
        return run_analys_tc(h->p, grid, spec, batch, op, s);
    }
    if (mode == SHT_TC_OTF) {
        if ((rc = ensure_otf(h->p))) return rc;
        if ((rc = ensure_work(h->p, tc_work_bytes(h->p, batch, false)))) return rc;
        return run_otf(h->p, false, grid, spec, batch, op, s);
    }
    if (mode == SHT_TC_F64) {
        if ((rc = ensure_panels64(h->p))) return rc;
        if ((rc = ensure_work(h->p, tc64_work_bytes(h->p, batch)))) return rc;
        return run_tc64(h->p, false, grid, spec, batch, op, s);
    }
    if (mode == SHT_F32 && (rc = ensure_seeds32(h->p))) return rc;
    if (mode == SHT_F64 && (rc = ensure_seeds64(h->p))) return rc;
    if ((rc = ensure_work(h->p, inter_bytes(h->p, batch, mode)))) return rc;
    if (mode == SHT_F64) return run_analys<double>(h->p, h->p.view64(), grid, spec, batch, op, s);
    return run_analys<float>(h->p, h->p.view32(), grid, spec, batch, op, s);
}

int vector_s2g(sht_handle h, const void *S, const void *T, void *vt, void *vp, int batch, int mode, void *stream,
               sht::Op op)
{
    const void *ptrs[4] = {S, T, vt, vp};
    int rc = prologue(h, batch, mode, 4, ptrs);
    if (rc) return rc;
    mode = resolve_mode(h->p, mode, batch, true);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (mode == SHT_TC_BF16X3) {
        if ((rc = ensure_vec_panels(h->p))) return rc;
        if ((rc = ensure_work(h->p, tc_work_bytes(h->p, batch, true)))) return rc;
        return run_synth_vec_tc(h->p, S, T, vt, vp, batch, op, s);
    }
    if (mode == SHT_F32 && (rc = ensure_seeds32(h->p))) return rc;
    if ((rc = ensure_work(h->p, 2 * inter_bytes(h->p, batch, mode)))) return rc;
    if (mode == SHT_F64) return run_synth_vec<double>(h->p, h->p.view64(), S, T, vt, vp, batch, op, s);
    return run_synth_vec<float>(h->p, h->p.view32(), S, T, vt, vp, batch, op, s);
}

int vector_g2s(sht_handle h, const void *vt, const void *vp, void *S, void *T, int batch, int mode, void *stream,
               sht::Op op)
{
    const void *ptrs[4] = {vt, vp, S, T};
    int rc = prologue(h, batch, mode, 4, ptrs);
    if (rc) return rc;
    mode = resolve_mode(h->p, mode, batch, true);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (mode == SHT_TC_BF16X3) {
        if ((rc = ensure_vec_panels(h->p))) return rc;
        if ((rc = ensure_work(h->p, tc_work_bytes(h->p, batch, true)))) return rc;
        return run_analys_vec_tc(h->p, vt, vp, S, T, batch, op, s);
    }
    if (mode == SHT_F32 && (rc = ensure_seeds32(h->p))) return rc;
    if ((rc = ensure_work(h->p, 2 * inter_bytes(h->p, batch, mode)))) return rc;
    if (mode == SHT_F64) return run_analys_vec<double>(h->p, h->p.view64(), vt, vp, S, T, batch, op, s);
    return run_analys_vec<float>(h->p, h->p.view32(), vt, vp, S, T, batch, op, s);
}

// Tensor-core transforms run in chunks of at most tc_chunk() fields: the
// contraction (prep + tcgen05 kernel) and the FP32 FFTs of each chunk.
int run_synth_tc(sht::Plan &p, const void *spec, void *grid, int batch, sht::Op op, cudaStream_t s)
{
    const int chunk = tc_chunk(false);
    float *eo = static_cast<float *>(p.work);
    unsigned char *data = static_cast<unsigned char *>(p.work) + tc_data_offset(p, batch, false);
    for (int b0 = 0; b0 < batch; b0 += chunk) {
        const int nb = batch - b0 < chunk ? batch - b0 : chunk;
        const float *in = static_cast<const float *>(spec) + (size_t)b0 * p.nlm * 2;
        float *out = static_cast<float *>(grid) + (size_t)b0 * p.nlat * p.nphi;
        int rc = timed(p, SHT_K_TC_SYNTH, s, "tensor-core synthesis launch", [&] {
            return sht::launch_tc_legendre(true, p.lmax, p.mmax, p.mres, p.npairs, p.nlm, p.panel_s, p.d_off_s, p.d_c0_s,
                                           p.d_gf_s, p.d_dchunk, data, in, eo, nb, op, p.d_err, false, s);
        });
        if (rc) return rc;
        rc = timed(p, SHT_K_FFT_SYNTH, s, "fft synthesis launch",
                   [&] { return sht::launch_fft_synth<float>(p.view32(), eo, out, nb, op, s); });
        if (rc) return rc;
    }
    return SHT_OK;
}

int run_analys_tc(sht::Plan &p, const void *grid, void *spec, int batch, sht::Op op, cudaStream_t s)
{
    const int chunk = tc_chunk(false);
    float *sd = static_cast<float *>(p.work);
    unsigned char *data = static_cast<unsigned char *>(p.work) + tc_data_offset(p, batch, false);
    for (int b0 = 0; b0 < batch; b0 += chunk) {
        const int nb = batch - b0 < chunk ? batch - b0 : chunk;
        const float *in = static_cast<const float *>(grid) + (size_t)b0 * p.nlat * p.nphi;
        float *out = static_cast<float *>(spec) + (size_t)b0 * p.nlm * 2;
        int rc = timed(p, SHT_K_FFT_ANALYS, s, "fft analysis launch",
                       [&] { return sht::launch_fft_analys<float>(p.view32(), in, sd, nb, op, false, s); });
        if (rc) return rc;
        rc = timed(p, SHT_K_TC_ANALYS, s, "tensor-core analysis launch", [&] {
            return sht::launch_tc_legendre(false, p.lmax, p.mmax, p.mres, p.npairs, p.nlm, p.panel_a, p.d_off_a, p.d_c0_a,
                                           p.d_gf_a, p.d_dchunk, data, sd, out, nb, op, p.d_err, false, s);
        });
        if (rc) return rc;
    }
    return SHT_OK;
}

// FP64-accurate tensor-core mode: synthesis = contraction then the
// double-float FFT; analysis = double-float FFT then contraction; groups of up
// to 16 fields.
int run_tc64(sht::Plan &p, bool synth, const void *in_, void *out_, int batch, sht::Op op, cudaStream_t s)
{
    const int chunk = sht::tc64_max_batch();
    double *inter = static_cast<double *>(p.work);
    unsigned char *data = static_cast<unsigned char *>(p.work) + tc64_data_offset(p, batch);
    const size_t spec_n = (size_t)p.nlm * 2, grid_n = (size_t)p.nlat * p.nphi;
    for (int b0 = 0; b0 < batch; b0 += chunk) {
        const int nb = batch - b0 < chunk ? batch - b0 : chunk;
        int rc;
        if (synth) {
            const double *in = static_cast<const double *>(in_) + (size_t)b0 * spec_n;
            double *out = static_cast<double *>(out_) + (size_t)b0 * grid_n;
            rc = timed(p, SHT_K_TC_SYNTH, s, "FP64 tensor-core synthesis launch", [&] {
                return sht::launch_tc64(true, p.lmax, p.mmax, p.mres, p.npairs, p.nlm, p.p64_s, p.d_off64_s, p.d_c064_s,
                                        p.d_gf64_s, p.d_zero64, p.d_sched64_s, p.sched64_ctas, p.d_e64_s, p.d_dchunk64, p.d_fcol, data, in, inter, nb, op, p.d_err, s);
            });
            if (rc) return rc;
            rc = timed(p, SHT_K_FFT_SYNTH, s, "fft synthesis launch",
                       [&] { return sht::launch_fft_synth_df(p.view64(), inter, out, nb, op, s); });
        } else {
            const double *in = static_cast<const double *>(in_) + (size_t)b0 * grid_n;
            double *out = static_cast<double *>(out_) + (size_t)b0 * spec_n;
            // the FFT also finds the folds' field exponents for the digit pass
            rc = timed(p, SHT_K_FFT_ANALYS, s, "fft analysis launch", [&] {
                cudaError_t e = sht::tc64_reset_fcol(p.d_fcol, nb, s);
                return e != cudaSuccess ? e : sht::launch_fft_analys_df(p.view64(), in, inter, nb, op, false, s, p.d_fcol);
            });
            if (rc) return rc;
            rc = timed(p, SHT_K_TC_ANALYS, s, "FP64 tensor-core analysis launch", [&] {
                return sht::launch_tc64(false, p.lmax, p.mmax, p.mres, p.npairs, p.nlm, p.p64_a, p.d_off64_a, p.d_c064_a,
                                        p.d_gf64_a, p.d_zero64, p.d_sched64_a, p.sched64_ctas, p.d_e64_a, p.d_dchunk64, p.d_fcol, data, inter, out, nb, op,
                                        p.d_err, s, true);
            });
        }
        if (rc) return rc;
    }
    return SHT_OK;
}

// On-the-fly mode: synthesis = contraction then FFT; analysis = FFT then contraction.
int run_otf(sht::Plan &p, bool synth, const void *in_, void *out_, int batch, sht::Op op, cudaStream_t s)
{
    const int chunk = sht::tc_otf_max_batch();
    float *inter = static_cast<float *>(p.work);
    unsigned char *data = static_cast<unsigned char *>(p.work) + tc_data_offset(p, batch, false);
    const sht::PlanView<float> pv = p.view32();
    for (int b0 = 0; b0 < batch; b0 += chunk) {
        const int nb = batch - b0 < chunk ? batch - b0 : chunk;
        const size_t so = (size_t)b0 * p.nlm * 2, go = (size_t)b0 * p.nlat * p.nphi;
        int rc;
        if (synth) {
            const float *in = static_cast<const float *>(in_) + so;
            float *out = static_cast<float *>(out_) + go;
            rc = timed(p, SHT_K_TC_SYNTH, s, "on-the-fly tensor-core synthesis launch", [&] {
                return sht::launch_tc_otf(true, p.lmax, p.mmax, p.mres, p.npairs, p.nlm, p.otf_seeds, p.d_segoff, p.d_c0o_s,
                                          pv.ab, pv.x, data, in, inter, nb, op, p.d_err, s);
            });
            if (rc) return rc;
            rc = timed(p, SHT_K_FFT_SYNTH, s, "fft synthesis launch",
                       [&] { return sht::launch_fft_synth<float>(pv, inter, out, nb, op, s); });
        } else {
            const float *in = static_cast<const float *>(in_) + go;
            float *out = static_cast<float *>(out_) + so;
            rc = timed(p, SHT_K_FFT_ANALYS, s, "fft analysis launch",
                       [&] { return sht::launch_fft_analys<float>(pv, in, inter, nb, op, false, s); });
            if (rc) return rc;
            rc = timed(p, SHT_K_TC_ANALYS, s, "on-the-fly tensor-core analysis launch", [&] {
                return sht::launch_tc_otf(false, p.lmax, p.mmax, p.mres, p.npairs, p.nlm, p.otf_seeds, p.d_segoff, p.d_c0o_a,
                                          pv.ab, pv.x, data, inter, out, nb, op, p.d_err, s);
            });
        }
        if (rc) return rc;
    }
    return SHT_OK;
}

int run_synth_vec_tc(sht::Plan &p, const void *S, const void *T, void *vt, void *vp, int batch, sht::Op op,
                     cudaStream_t s)
{
    const int chunk = tc_chunk(true);
    const size_t inter = (size_t)(batch < chunk ? batch : chunk) * (p.mmax + 1) * p.npairs * 4;
    float *eot = static_cast<float *>(p.work);
    float *eop = eot + inter;
    unsigned char *data = static_cast<unsigned char *>(p.work) + tc_data_offset(p, batch, true);
    for (int b0 = 0; b0 < batch; b0 += chunk) {
        const int nb = batch - b0 < chunk ? batch - b0 : chunk;
        const size_t so = (size_t)b0 * p.nlm * 2, go = (size_t)b0 * p.nlat * p.nphi;
        int rc = timed(p, SHT_K_TC_SYNTH_VEC, s, "tensor-core vector synthesis launch", [&] {
            return sht::launch_tc_vec(true, p.lmax, p.mmax, p.mres, p.npairs, p.nlm, p.panel_s, p.dpanel_s, p.d_off_s,
                                      p.d_c0v_s, p.d_schedv_s, p.schedv_ctas, p.d_dchunk, data, static_cast<const float *>(S) + so,
                                      static_cast<const float *>(T) + so, eot, eop, p.t32.st, nb, op, p.d_err, false,
                                      s);
        });
        if (rc) return rc;
        rc = timed(p, SHT_K_FFT_SYNTH, s, "fft synthesis launch", [&] {
            return sht::launch_fft_synth<float>(p.view32(), eot, static_cast<float *>(vt) + go, nb, op, s);
        });
        if (rc) return rc;
        rc = timed(p, SHT_K_FFT_SYNTH, s, "fft synthesis launch", [&] {
            return sht::launch_fft_synth<float>(p.view32(), eop, static_cast<float *>(vp) + go, nb, op, s);
        });
        if (rc) return rc;
    }
    return SHT_OK;
}

int run_analys_vec_tc(sht::Plan &p, const void *vt, const void *vp, void *S, void *T, int batch, sht::Op op,
                      cudaStream_t s)
{
    const int chunk = tc_chunk(true);
    const size_t inter = (size_t)(batch < chunk ? batch : chunk) * (p.mmax + 1) * p.npairs * 4;
    float *sdt = static_cast<float *>(p.work);
    float *sdp = sdt + inter;
    unsigned char *data = static_cast<unsigned char *>(p.work) + tc_data_offset(p, batch, true);
    for (int b0 = 0; b0 < batch; b0 += chunk) {
        const int nb = batch - b0 < chunk ? batch - b0 : chunk;
        const size_t so = (size_t)b0 * p.nlm * 2, go = (size_t)b0 * p.nlat * p.nphi;
        int rc = timed(p, SHT_K_FFT_ANALYS, s, "fft analysis launch", [&] {
            return sht::launch_fft_analys<float>(p.view32(), static_cast<const float *>(vt) + go, sdt, nb, op, true, s);
        });
        if (rc) return rc;
        rc = timed(p, SHT_K_FFT_ANALYS, s, "fft analysis launch", [&] {
            return sht::launch_fft_analys<float>(p.view32(), static_cast<const float *>(vp) + go, sdp, nb, op, true, s);
        });
        if (rc) return rc;
        rc = timed(p, SHT_K_TC_ANALYS_VEC, s, "tensor-core vector analysis launch", [&] {
            return sht::launch_tc_vec(false, p.lmax, p.mmax, p.mres, p.npairs, p.nlm, p.panel_a, p.dpanel_a, p.d_off_a,
                                      p.d_c0v_a, p.d_schedv_a, p.schedv_ctas, p.d_dchunk, data, sdt, sdp, static_cast<float *>(S) + so,
                                      static_cast<float *>(T) + so, p.t32.st, nb, op, p.d_err, false, s);
        });
        if (rc) return rc;
    }
    return SHT_OK;
}

}  // namespace

int sht::set_error(int code, const std::string &msg) { return fail(code, msg); }

// Uneven batches on the tensor cores (batch.cu): panels and the contraction's
// operand scratch for `batch` fields of this plan, built outside any capture.
int sht::tc_batch_prepare(sht::Plan &p, int batch)
{
    int rc = ensure_panels(p);
    if (rc) return rc;
    const int nb = batch > tc_chunk(false) ? tc_chunk(false) : batch;
    return ensure_work(p, sht::tc_data_bytes(p.mmax, p.npairs, p.tc_nchunk_s, nb, false));
}

// The contraction alone, in chunks: synthesis spectra [batch][nlm] -> E/O
// [batch][mmax+1][npairs][4]; analysis folds (same layout) -> spectra.
cudaError_t sht::tc_batch_legendre(sht::Plan &p, bool synth, const float *in, float *out, int batch, cudaStream_t s)
{
    const int chunk = tc_chunk(false);
    unsigned char *data = static_cast<unsigned char *>(p.work);
    const size_t spec_n = (size_t)p.nlm * 2, inter_n = (size_t)(p.mmax + 1) * p.npairs * 4;
    for (int b0 = 0; b0 < batch; b0 += chunk) {
        const int nb = batch - b0 < chunk ? batch - b0 : chunk;
        const float *i = in + (size_t)b0 * (synth ? spec_n : inter_n);
        float *o = out + (size_t)b0 * (synth ? inter_n : spec_n);
        cudaError_t e = synth ? sht::launch_tc_legendre(true, p.lmax, p.mmax, p.mres, p.npairs, p.nlm, p.panel_s, p.d_off_s,
                                                        p.d_c0_s, p.d_gf_s, p.d_dchunk, data, i, o, nb,
                                                        sht::OP_SYNTH, p.d_err, false, s)
                              : sht::launch_tc_legendre(false, p.lmax, p.mmax, p.mres, p.npairs, p.nlm, p.panel_a, p.d_off_a,
                                                        p.d_c0_a, p.d_gf_a, p.d_dchunk, data, i, o, nb,
                                                        sht::OP_ANALYS, p.d_err, false, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

namespace {
int static_scratch_refresh(int device);
}  // namespace

extern "C" {

const char *sht_last_error(void) { return g_err.c_str(); }

int sht_create(int lmax, int mmax, int nlat, int nphi, sht_handle *out)
{
    return sht_create_mres(lmax, mmax, 1, nlat, nphi, out);
}

int sht_create_mres(int lmax, int mmax, int mres, int nlat, int nphi, sht_handle *out)
{
    if (!out) return fail(SHT_EINVAL, "out is NULL");
    *out = nullptr;
    if (mres < 1) return fail(SHT_EINVAL, "need mres >= 1");
    if (lmax < 0 || mmax < 0 || (long)mmax * mres > lmax) return fail(SHT_EINVAL, "need 0 <= mmax mres <= lmax");
    if (nlat < lmax + 1) return fail(SHT_EINVAL, "need nlat >= lmax + 1 for an exact Gauss-Legendre quadrature");
    if (nphi < 2 * mmax + 1) return fail(SHT_EINVAL, "need nphi >= 2 mmax + 1");
    if (nlat > 4096 || lmax > 4095) return fail(SHT_EUNSUPPORTED, "nlat > 4096 is not supported");
    if (nphi < 2 || nphi > 8192 || nphi % 2 != 0 || sht::fft_plan_of(nphi / 2) == sht::kFftPlanBad)
        return fail(SHT_EUNSUPPORTED, "nphi must be 2 x 2^a 3^b 5^c in [2, 8192]");
    sht_plan *h = new (std::nothrow) sht_plan;
    if (!h) return fail(SHT_ENOMEM, "host allocation failed");
    h->p.lmax = lmax;
    h->p.mmax = mmax;
    h->p.mres = mres;
    h->p.nlat = nlat;
    h->p.nphi = nphi;
    std::string err;
    int rc = sht::plan_build(h->p, err);
    if (rc) {
        sht::plan_free(h->p);
        delete h;
        return fail(rc, err);
    }
    // device address of the fixed array of sht_synth_static, looked up here
    // with the plan's device current (see static_scratch_refresh)
    if ((rc = static_scratch_refresh(h->p.device))) {
        sht::plan_free(h->p);
        delete h;
        return rc;
    }
    *out = h;
    return SHT_OK;
}

void sht_destroy(sht_handle h)
{
    if (!h) return;
    sht::plan_free(h->p);
    delete h;
}

int sht_reserve(sht_handle h, int batch, int mode)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if ((rc = check_mode(mode))) return rc;
    if (batch < 1) return fail(SHT_EINVAL, "batch must be >= 1");
    if (mode == SHT_TC_BF16X3) {
        if ((rc = ensure_vec_panels(h->p))) return rc;
        const size_t a = tc_work_bytes(h->p, batch, false), b = tc_work_bytes(h->p, batch, true);
        return ensure_work(h->p, a > b ? a : b);
    }
    if (mode == SHT_TC_OTF) {
        if ((rc = ensure_otf(h->p))) return rc;
        return ensure_work(h->p, tc_work_bytes(h->p, batch, false));
    }
    if (mode == SHT_TC_F64) {
        if ((rc = ensure_panels64(h->p))) return rc;
        return ensure_work(h->p, tc64_work_bytes(h->p, batch));
    }
    if ((mode == SHT_F32 || mode == SHT_F32_AUTO) && (rc = ensure_seeds32(h->p))) return rc;
    if (mode == SHT_F64 && (rc = ensure_seeds64(h->p))) return rc;
    return ensure_work(h->p, 2 * inter_bytes(h->p, batch, mode));
}

int sht_synth(sht_handle h, const void *spec, void *grid, int batch, int mode, void *stream)
{
    return scalar_s2g(h, spec, grid, batch, mode, stream, sht::OP_SYNTH);
}

int sht_analys(sht_handle h, const void *grid, void *spec, int batch, int mode, void *stream)
{
    return scalar_g2s(h, grid, spec, batch, mode, stream, sht::OP_ANALYS);
}

int sht_synth_adj(sht_handle h, const void *grid, void *spec, int batch, int mode, void *stream)
{
    return scalar_g2s(h, grid, spec, batch, mode, stream, sht::OP_SYNTH_ADJ);
}

int sht_analys_adj(sht_handle h, const void *spec, void *grid, int batch, int mode, void *stream)
{
    return scalar_s2g(h, spec, grid, batch, mode, stream, sht::OP_ANALYS_ADJ);
}

int sht_synth_vec(sht_handle h, const void *S, const void *T, void *vt, void *vp, int batch, int mode, void *stream)
{
    return vector_s2g(h, S, T, vt, vp, batch, mode, stream, sht::OP_SYNTH);
}

int sht_analys_vec(sht_handle h, const void *vt, const void *vp, void *S, void *T, int batch, int mode, void *stream)
{
    return vector_g2s(h, vt, vp, S, T, batch, mode, stream, sht::OP_ANALYS);
}

int sht_synth_vec_adj(sht_handle h, const void *gt, const void *gp, void *S, void *T, int batch, int mode,
                      void *stream)
{
    return vector_g2s(h, gt, gp, S, T, batch, mode, stream, sht::OP_SYNTH_ADJ);
}

int sht_analys_vec_adj(sht_handle h, const void *S, const void *T, void *gt, void *gp, int batch, int mode,
                       void *stream)
{
    return vector_s2g(h, S, T, gt, gp, batch, mode, stream, sht::OP_ANALYS_ADJ);
}

int sht_nlm(sht_handle h)
{
    if (!h) return fail(SHT_EINVAL, "null handle");
    return h->p.nlm;
}

int sht_lm_index(sht_handle h, int n, int m)
{
    if (!h) return fail(SHT_EINVAL, "null handle");
    const int mres = h->p.mres;
    if (m < 0 || m % mres != 0 || m / mres > h->p.mmax || n < m || n > h->p.lmax) return -1;
    return (int)sht::col_of_mres(h->p.lmax, m / mres, mres) + (n - m);
}

int sht_gauss(sht_handle h, double *x, double *w)
{
    if (!h) return fail(SHT_EINVAL, "null handle");
    if (!x || !w) return fail(SHT_EINVAL, "null output pointer");
    for (int j = 0; j < h->p.nlat; ++j) {
        x[j] = h->p.x[j];
        w[j] = h->p.w[j];
    }
    return SHT_OK;
}

int sht_tc_polar_skip(sht_handle h, double *synth_frac, double *analys_frac)
{
    if (!h) return fail(SHT_EINVAL, "null handle");
    if (!synth_frac || !analys_frac) return fail(SHT_EINVAL, "null output pointer");
    // the panels' tables if built, else those of the on-the-fly mode, else the
    // FP64-accurate mode's digit groups it does not read (all-zero 8-row groups)
    const sht::Plan &p = h->p;
    *synth_frac = p.panel_s ? p.polar_skip_s : (p.otf_state > 0 ? p.otf_skip_s : (p.p64_s ? p.skip64_s : -1.0));
    *analys_frac = p.panel_s ? p.polar_skip_a : (p.otf_state > 0 ? p.otf_skip_a : (p.p64_s ? p.skip64_a : -1.0));
    return SHT_OK;
}

int sht_cc_polar_skip(sht_handle h, int mode, double *frac)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!frac) return fail(SHT_EINVAL, "sht_cc_polar_skip: null output");
    const sht::Plan &p = h->p;
    const unsigned short *live = mode == SHT_F64 ? p.live64 : (mode == SHT_F32 ? p.live32 : nullptr);
    if (mode != SHT_F64 && mode != SHT_F32) return fail(SHT_EINVAL, "sht_cc_polar_skip: mode SHT_F64 or SHT_F32");
    if (!live) {
        *frac = -1.0;
        return SHT_OK;
    }
    std::vector<unsigned short> t((size_t)(p.mmax + 1) * p.npairs);
    cudaError_t e = cudaMemcpy(t.data(), live, sizeof(unsigned short) * t.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(SHT_ECUDA, std::string("sht_cc_polar_skip: ") + cudaGetErrorString(e));
    double skipped = 0.0, total = 0.0;
    for (int m = 0; m <= p.mmax; ++m) {
        const int L = p.lmax - m * p.mres + 1;
        for (int q = 0; q < p.npairs; ++q) {
            const long dead = (long)t[(size_t)m * p.npairs + q] * sht::kSeedSeg;
            skipped += (double)(dead < L ? dead : L);
            total += L;
        }
    }
    *frac = total > 0 ? skipped / total : 0.0;
    return SHT_OK;
}

int sht_set_polar_threshold(sht_handle h, double threshold)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!(threshold >= 0.0) || threshold > 1.0) return fail(SHT_EINVAL, "polar threshold must be in [0, 1]");
    sht::Plan &p = h->p;
    p.polar_thr = (float)threshold;
    p.polar_thr_set = true;
    cudaError_t e = cudaDeviceSynchronize();   // no transform may be reading the tables
    if (e == cudaSuccess) {
        std::string err;
        if ((rc = sht::plan_relive(p, err))) return fail(rc, "sht_set_polar_threshold: " + err);
    }
    if (e == cudaSuccess && p.panel_s) e = first_live_scalar(p);
    if (e == cudaSuccess && p.dpanel_s) {
        int T_s = 0, T_a = 0;
        sht::tc_tile_counts(p.lmax, p.npairs, T_s, T_a);
        int *tmp = nullptr;
        e = cudaMalloc(&tmp, sizeof(int) * (size_t)(p.mmax + 1) * (T_s > T_a ? T_s : T_a));
        if (e == cudaSuccess) e = first_live_vector(p, tmp);
        cudaFree(tmp);
        if (e == cudaSuccess) e = vec_schedules(p);
    }
    if (e == cudaSuccess && p.otf_state > 0) {
        int *flag = nullptr;
        e = cudaMalloc(&flag, sizeof(int));
        if (e == cudaSuccess) e = otf_build(p, flag);
        cudaFree(flag);
    }
    if (e != cudaSuccess) return fail(SHT_ECUDA, std::string("sht_set_polar_threshold: ") + cudaGetErrorString(e));
    return SHT_OK;
}

int sht_selftest_timeout(sht_handle h, int timeout_us, void *stream)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (timeout_us < 1 || timeout_us > 2000000) return fail(SHT_EINVAL, "timeout_us must be in [1, 2e6]");
    return launched(sht::launch_selftest_timeout(h->p.d_err, (unsigned long long)timeout_us * 1000ull,
                                                 static_cast<cudaStream_t>(stream)),
                    "self-test launch");
}

int sht_profile(sht_handle h, int enable)
{
    if (!h) return fail(SHT_EINVAL, "null handle");
    h->p.timer.enabled = enable != 0;
    h->p.timer.used = 0;
    h->p.timer.kinds.clear();
    return SHT_OK;
}

int sht_profile_read(sht_handle h, double *ms, int *count, int cap)
{
    if (!h) return fail(SHT_EINVAL, "null handle");
    if (cap < 0 || (cap > 0 && (!ms || !count))) return fail(SHT_EINVAL, "bad output arrays");
    for (int k = 0; k < cap; ++k) { ms[k] = 0.0; count[k] = 0; }
    sht::KernelTimer &t = h->p.timer;
    int rc = SHT_OK;
    for (size_t i = 0; i < t.kinds.size(); ++i) {
        cudaEvent_t e0 = t.pool[2 * i], e1 = t.pool[2 * i + 1];
        float el = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&el, e0, e1) != cudaSuccess) {
            rc = fail(SHT_ECUDA, "reading timing events failed");
            break;
        }
        const int k = t.kinds[i];
        if (k < cap) { ms[k] += el; count[k] += 1; }
    }
    t.used = 0;
    t.kinds.clear();
    return rc;
}

const char *sht_kernel_name(int kind)
{
    static const char *names[SHT_NKERNELS] = {"legendre_synth", "legendre_analys", "legendre_synth_vec",
                                              "legendre_analys_vec", "fft_synth",       "fft_analys",
                                              "tc_synth",       "tc_analys",          "tc_synth_vec",
                                              "tc_analys_vec"};
    if (kind < 0 || kind >= SHT_NKERNELS) return "";
    return names[kind];
}

int sht_sync_status(sht_handle h, void *stream)
{
    int rc = check_handle(h);
    if (rc) return rc;
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SHT_ECUDA, std::string("CUDA error: ") + cudaGetErrorString(e));
    int code = 0;
    e = cudaMemcpy(&code, h->p.d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(SHT_ECUDA, std::string("reading the error word: ") + cudaGetErrorString(e));
    if (code != 0) {
        cudaMemset(h->p.d_err, 0, sizeof(int));
        return fail(SHT_ETIMEOUT, "a tensor-core kernel gave up waiting for its copies or MMAs");
    }
    return SHT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// sht_tune: time candidate shapes / paths and keep the fastest.
// ---------------------------------------------------------------------------
namespace {

template <typename F>
double time_ms(F &&launch, cudaStream_t s, int reps, bool &ok)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    ok = launch() == cudaSuccess;  // warm-up
    cudaEventRecord(e0, s);
    for (int i = 0; i < reps && ok; ++i) ok = launch() == cudaSuccess;
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (ok) ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ok ? ms / reps : 1e30;
}

}  // namespace

extern "C" int sht_tune(sht_handle h, int batch, int mode, double *report, void *stream)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if ((rc = check_mode(mode))) return rc;
    if (mode == SHT_TC_BF16X3) return fail(SHT_EINVAL, "tune SHT_F64, SHT_F32 or SHT_F32_AUTO");
    if (batch < 1) return fail(SHT_EINVAL, "batch must be >= 1");
    sht::Plan &p = h->p;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int shape_mode = mode == SHT_F64 ? SHT_F64 : SHT_F32;
    if (shape_mode == SHT_F32 && (rc = ensure_seeds32(p))) return rc;
    if (shape_mode == SHT_F64 && (rc = ensure_seeds64(p))) return rc;
    const size_t es = elem_size(shape_mode);
    void *spec = nullptr, *grid = nullptr;
    cudaError_t e = cudaMalloc(&spec, (size_t)batch * p.nlm * 2 * es);
    if (e == cudaSuccess) e = cudaMalloc(&grid, (size_t)batch * p.nlat * p.nphi * es);
    if (e == cudaSuccess) e = cudaMemsetAsync(spec, 0, (size_t)batch * p.nlm * 2 * es, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(grid, 0, (size_t)batch * p.nlat * p.nphi * es, s);
    if (e != cudaSuccess) {
        cudaFree(spec);
        cudaFree(grid);
        return fail(SHT_ENOMEM, "sht_tune: allocating test buffers failed");
    }
    if ((rc = ensure_work(p, inter_bytes(p, batch, shape_mode)))) { cudaFree(spec); cudaFree(grid); return rc; }
    sht::TunedShape best;
    double best_syn = 1e30, best_ana = 1e30;
    const int reps = 3;
    const int lpts_s[3] = {1, 2, 4}, bcs_s[4] = {1, 2, 4, 8};
    for (int li = 0; li < 3; ++li)
        for (int bi = 0; bi < 4; ++bi) {
            const int lpt = lpts_s[li], bc = bcs_s[bi];
            if (bc > batch && bc > 1) continue;
            if (bc == 8 && (shape_mode != SHT_F64 || lpt > 2)) continue;
            bool ok = false;
            double ms;
            if (shape_mode == SHT_F64)
                ms = time_ms([&] { return sht::launch_legendre_synth_cfg<double>(p.view64(), (const double *)spec, (double *)p.work, batch, sht::OP_SYNTH, lpt, bc, s); }, s, reps, ok);
            else
                ms = time_ms([&] { return sht::launch_legendre_synth_cfg<float>(p.view32(), (const float *)spec, (float *)p.work, batch, sht::OP_SYNTH, lpt, bc, s); }, s, reps, ok);
            if (ok && ms < best_syn) { best_syn = ms; best.synth_lpt = lpt; best.synth_bc = bc; }
        }
    const int lpts_a[4] = {2, 4, 8, sht::kAnalysSeg}, bcs_a[4] = {1, 2, 4, 8};
    for (int li = 0; li < 4; ++li)
        for (int bi = 0; bi < 4; ++bi) {
            const int lpt = lpts_a[li], bc = bcs_a[bi];
            if (bc > batch && bc > 1) continue;
            if (lpt == sht::kAnalysSeg
                    ? (shape_mode != SHT_F64 || p.npairs > 2048 || (p.npairs > 1024 && bc > 2) ||
                       (p.npairs > 512 && bc > 4))
                    : (bc > 2 || (p.npairs + 32 * lpt - 1) / (32 * lpt) > 8))
                continue;
            bool ok = false;
            double ms;
            if (shape_mode == SHT_F64)
                ms = time_ms([&] { return sht::launch_legendre_analys_cfg<double>(p.view64(), (const double *)p.work, (double *)spec, batch, sht::OP_ANALYS, lpt, bc, s); }, s, reps, ok);
            else
                ms = time_ms([&] { return sht::launch_legendre_analys_cfg<float>(p.view32(), (const float *)p.work, (float *)spec, batch, sht::OP_ANALYS, lpt, bc, s); }, s, reps, ok);
            if (ok && ms < best_ana) { best_ana = ms; best.analys_lpt = lpt; best.analys_bc = bc; }
        }
    cudaGetLastError();
    set_tuned(p, shape_mode, batch, best);
    if (report) { report[0] = best_syn; report[1] = best_ana; report[2] = -1.0; }
    if (mode == SHT_F32_AUTO) {
        // the paper's choice: on-the-fly recurrence (FP32 cores) vs precomputed P (tensor cores)
        bool ok1 = false, ok2 = false;
        const double ms_f32 = time_ms([&] {
            if (scalar_s2g(h, spec, grid, batch, SHT_F32, s, sht::OP_SYNTH)) return cudaErrorUnknown;
            return scalar_g2s(h, grid, spec, batch, SHT_F32, s, sht::OP_ANALYS) ? cudaErrorUnknown : cudaSuccess;
        }, s, reps, ok1);
        double ms_tc = 1e30, ms_otf = 1e30;
        bool ok3 = false;
        if (ensure_panels(p) == SHT_OK) {
            ms_tc = time_ms([&] {
                if (scalar_s2g(h, spec, grid, batch, SHT_TC_BF16X3, s, sht::OP_SYNTH)) return cudaErrorUnknown;
                return scalar_g2s(h, grid, spec, batch, SHT_TC_BF16X3, s, sht::OP_ANALYS) ? cudaErrorUnknown : cudaSuccess;
            }, s, reps, ok2);
        }
        if (ensure_otf(p) == SHT_OK) {
            ms_otf = time_ms([&] {
                if (scalar_s2g(h, spec, grid, batch, SHT_TC_OTF, s, sht::OP_SYNTH)) return cudaErrorUnknown;
                return scalar_g2s(h, grid, spec, batch, SHT_TC_OTF, s, sht::OP_ANALYS) ? cudaErrorUnknown : cudaSuccess;
            }, s, reps, ok3);
        }
        cudaGetLastError();
        sht::TunedShape a = best;
        a.auto_mode = SHT_F32;
        double best_ms = ok1 ? ms_f32 : 1e30;
        if (ok2 && ms_tc < best_ms) { best_ms = ms_tc; a.auto_mode = SHT_TC_BF16X3; }
        if (ok3 && ms_otf < best_ms) { best_ms = ms_otf; a.auto_mode = SHT_TC_OTF; }
        set_tuned(p, SHT_F32_AUTO, batch, a);
        if (report) {
            report[0] = ok1 ? ms_f32 : -1.0;
            report[1] = ok2 ? ms_tc : -1.0;
            report[2] = ok3 ? ms_otf : -1.0;
        }
    }
    cudaStreamSynchronize(s);
    cudaFree(spec);
    cudaFree(grid);
    return SHT_OK;
}

// ---------------------------------------------------------------------------
// sht_synth_static: the scalar synthesis with its intermediate in a fixed
// device array instead of the handle's scratch (see include/sht.h for who
// needs it).  The array below is the only storage it uses besides the plan
// tables and the caller's buffers.
// ---------------------------------------------------------------------------
namespace {

static __device__ __align__(256) unsigned char g_static_scratch[SHT_STATIC_SCRATCH_BYTES];

// Device address of g_static_scratch on each device.  In host code the
// symbol's name is only a stand-in for the device object, so kernels must be
// given the address cudaGetSymbolAddress returns with that device current.
// sht_create looks it up (static_scratch_refresh) for the device it builds the
// plan on -- the current device, which every later call on the handle must
// also have current (check_handle) -- and stores it under that ordinal; a plan
// created after a device reset thus stores the address of the reloaded
// module.  sht_synth_static only reads the stored address.
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_ptr[kMaxDevices] = {};

int static_scratch_refresh(int device)
{
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return fail(SHT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (cur != device) return fail(SHT_EINVAL, "static scratch: the plan's device is not current");
    if (device < 0 || device >= kMaxDevices) return fail(SHT_EUNSUPPORTED, "device ordinal too large");
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || !ptr)
        return fail(SHT_ECUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(g_static_mu);
    g_static_ptr[device] = ptr;
    return SHT_OK;
}

// The stored address for the current device (the handle's, see check_handle).
int static_scratch(void **out)
{
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return fail(SHT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (cur < 0 || cur >= kMaxDevices) return fail(SHT_EUNSUPPORTED, "device ordinal too large");
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[cur]) return fail(SHT_EINVAL, "sht_synth_static: no plan was created on this device");
    *out = g_static_ptr[cur];
    return SHT_OK;
}

}  // namespace

extern "C" int sht_synth_static(sht_handle h, const void *spec, void *grid, int batch, int mode, void *stream)
{
    const void *ptrs[2] = {spec, grid};
    int rc = prologue(h, batch, mode, 2, ptrs);
    if (rc) return rc;
    if (mode == SHT_TC_BF16X3 || mode == SHT_TC_OTF || mode == SHT_TC_F64)
        return fail(SHT_EUNSUPPORTED, "sht_synth_static: the tensor-core modes need tables allocated by the handle");
    if (mode == SHT_F32_AUTO) mode = SHT_F32;
    const size_t need = inter_bytes(h->p, batch, mode);
    if (need > (size_t)SHT_STATIC_SCRATCH_BYTES)
        return fail(SHT_EINVAL, "sht_synth_static: this call needs " + std::to_string(need) +
                                    " bytes of intermediate storage, more than the fixed " +
                                    std::to_string((size_t)SHT_STATIC_SCRATCH_BYTES) + "-byte array");
    if (mode == SHT_F32 && !h->p.seeds32)
        return fail(SHT_EUNSUPPORTED, "sht_synth_static: SHT_F32 needs the plan's FP32 recurrence restart states; "
                                      "build them first with sht_reserve(h, batch, SHT_F32) or any SHT_F32 call");
    if (mode == SHT_F64 && !h->p.seeds64)
        return fail(SHT_EUNSUPPORTED, "sht_synth_static: SHT_F64 needs the plan's FP64 restart states and polar "
                                      "table; build them first with sht_reserve(h, batch, SHT_F64) or any SHT_F64 "
                                      "call");
    void *scratch = nullptr;
    if ((rc = static_scratch(&scratch))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (mode == SHT_F64) {
        const sht::PlanView<double> pv = h->p.view64();
        double *eo = static_cast<double *>(scratch);
        rc = launched(sht::launch_legendre_synth<double>(pv, static_cast<const double *>(spec), eo, batch,
                                                         sht::OP_SYNTH, s),
                      "legendre synthesis launch");
        if (rc) return rc;
        return launched(sht::launch_fft_synth<double>(pv, eo, static_cast<double *>(grid), batch, sht::OP_SYNTH, s),
                        "fft synthesis launch");
    }
    const sht::PlanView<float> pv = h->p.view32();
    float *eo = static_cast<float *>(scratch);
    rc = launched(sht::launch_legendre_synth<float>(pv, static_cast<const float *>(spec), eo, batch, sht::OP_SYNTH, s),
                  "legendre synthesis launch");
    if (rc) return rc;
    return launched(sht::launch_fft_synth<float>(pv, eo, static_cast<float *>(grid), batch, sht::OP_SYNTH, s),
                    "fft synthesis launch");
}
