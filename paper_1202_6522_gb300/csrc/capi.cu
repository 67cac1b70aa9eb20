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

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

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
    if (mode != SHT_F64 && mode != SHT_F32) return fail(SHT_EINVAL, "unknown mode");
    return SHT_OK;
}

size_t elem_size(int mode) { return mode == SHT_F64 ? sizeof(double) : sizeof(float); }

// Bytes of one [batch][mmax+1][npairs][2] complex intermediate.
size_t inter_bytes(const sht::Plan &p, int batch, int mode)
{
    return (size_t)batch * (p.mmax + 1) * p.npairs * 4 * elem_size(mode);
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

// The two directions of the scalar transform, parameterised by precision.
template <typename T>
int run_synth(sht::Plan &p, const sht::PlanView<T> &pv, const void *spec, void *grid, int batch, sht::Op op,
              cudaStream_t s)
{
    T *eo = static_cast<T *>(p.work);
    int rc = timed(p, SHT_K_LEGENDRE_SYNTH, s, "legendre synthesis launch", [&] {
        return sht::launch_legendre_synth<T>(pv, static_cast<const T *>(spec), eo, batch, op, s);
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
    return timed(p, SHT_K_LEGENDRE_ANALYS, s, "legendre analysis launch", [&] {
        return sht::launch_legendre_analys<T>(pv, sd, static_cast<T *>(spec), batch, op, s);
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

int scalar_s2g(sht_handle h, const void *spec, void *grid, int batch, int mode, void *stream, sht::Op op)
{
    const void *ptrs[2] = {spec, grid};
    int rc = prologue(h, batch, mode, 2, ptrs);
    if (rc) return rc;
    if ((rc = ensure_work(h->p, inter_bytes(h->p, batch, mode)))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (mode == SHT_F64) return run_synth<double>(h->p, h->p.view64(), spec, grid, batch, op, s);
    return run_synth<float>(h->p, h->p.view32(), spec, grid, batch, op, s);
}

int scalar_g2s(sht_handle h, const void *grid, void *spec, int batch, int mode, void *stream, sht::Op op)
{
    const void *ptrs[2] = {grid, spec};
    int rc = prologue(h, batch, mode, 2, ptrs);
    if (rc) return rc;
    if ((rc = ensure_work(h->p, inter_bytes(h->p, batch, mode)))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (mode == SHT_F64) return run_analys<double>(h->p, h->p.view64(), grid, spec, batch, op, s);
    return run_analys<float>(h->p, h->p.view32(), grid, spec, batch, op, s);
}

int vector_s2g(sht_handle h, const void *S, const void *T, void *vt, void *vp, int batch, int mode, void *stream,
               sht::Op op)
{
    const void *ptrs[4] = {S, T, vt, vp};
    int rc = prologue(h, batch, mode, 4, ptrs);
    if (rc) return rc;
    if ((rc = ensure_work(h->p, 2 * inter_bytes(h->p, batch, mode)))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (mode == SHT_F64) return run_synth_vec<double>(h->p, h->p.view64(), S, T, vt, vp, batch, op, s);
    return run_synth_vec<float>(h->p, h->p.view32(), S, T, vt, vp, batch, op, s);
}

int vector_g2s(sht_handle h, const void *vt, const void *vp, void *S, void *T, int batch, int mode, void *stream,
               sht::Op op)
{
    const void *ptrs[4] = {vt, vp, S, T};
    int rc = prologue(h, batch, mode, 4, ptrs);
    if (rc) return rc;
    if ((rc = ensure_work(h->p, 2 * inter_bytes(h->p, batch, mode)))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (mode == SHT_F64) return run_analys_vec<double>(h->p, h->p.view64(), vt, vp, S, T, batch, op, s);
    return run_analys_vec<float>(h->p, h->p.view32(), vt, vp, S, T, batch, op, s);
}

}  // namespace

extern "C" {

const char *sht_last_error(void) { return g_err.c_str(); }

int sht_create(int lmax, int mmax, int nlat, int nphi, sht_handle *out)
{
    if (!out) return fail(SHT_EINVAL, "out is NULL");
    *out = nullptr;
    if (lmax < 0 || mmax < 0 || mmax > lmax) return fail(SHT_EINVAL, "need 0 <= mmax <= lmax");
    if (nlat < lmax + 1) return fail(SHT_EINVAL, "need nlat >= lmax + 1 for an exact Gauss-Legendre quadrature");
    if (nphi < 2 * mmax + 1) return fail(SHT_EINVAL, "need nphi >= 2 mmax + 1");
    if (nlat > 4096 || lmax > 4095) return fail(SHT_EUNSUPPORTED, "nlat > 4096 is not supported");
    if (!is_pow2(nphi) || nphi < 2 || nphi > 8192)
        return fail(SHT_EUNSUPPORTED, "nphi must be a power of two in [2, 8192]");
    sht_plan *h = new (std::nothrow) sht_plan;
    if (!h) return fail(SHT_ENOMEM, "host allocation failed");
    h->p.lmax = lmax;
    h->p.mmax = mmax;
    h->p.nlat = nlat;
    h->p.nphi = nphi;
    std::string err;
    int rc = sht::plan_build(h->p, err);
    if (rc) {
        sht::plan_free(h->p);
        delete h;
        return fail(rc, err);
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
    if (m < 0 || m > h->p.mmax || n < m || n > h->p.lmax) return -1;
    return m * (2 * h->p.lmax + 3 - m) / 2 + (n - m);
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
                                              "legendre_analys_vec", "fft_synth", "fft_analys"};
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
    return SHT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// sht_synth_static: the scalar synthesis with its intermediate in a fixed
// device array instead of the handle's scratch (see include/sht.h for who
// needs it).  The array below is the only storage it uses besides the plan
// tables and the caller's buffers.
// ---------------------------------------------------------------------------
namespace {

static __device__ __align__(256) unsigned char g_static_scratch[SHT_STATIC_SCRATCH_BYTES];

// Device address of g_static_scratch, looked up once per device.  In host code
// the symbol name is only a stand-in for the device object, so kernels must
// be given the address returned by cudaGetSymbolAddress.
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_ptr[kMaxDevices] = {};

int static_scratch(int device, void **out)
{
    if (device < 0 || device >= kMaxDevices) return fail(SHT_EUNSUPPORTED, "device ordinal too large");
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || !ptr)
            return fail(SHT_ECUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
        g_static_ptr[device] = ptr;
    }
    *out = g_static_ptr[device];
    return SHT_OK;
}

}  // namespace

extern "C" int sht_synth_static(sht_handle h, const void *spec, void *grid, int batch, int mode, void *stream)
{
    const void *ptrs[2] = {spec, grid};
    int rc = prologue(h, batch, mode, 2, ptrs);
    if (rc) return rc;
    const size_t need = inter_bytes(h->p, batch, mode);
    if (need > (size_t)SHT_STATIC_SCRATCH_BYTES)
        return fail(SHT_EINVAL, "sht_synth_static: this call needs " + std::to_string(need) +
                                    " bytes of intermediate storage, more than the fixed " +
                                    std::to_string((size_t)SHT_STATIC_SCRATCH_BYTES) + "-byte array");
    void *scratch = nullptr;
    if ((rc = static_scratch(h->p.device, &scratch))) return rc;
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
