// plan.cpp -- host construction of an SHT plan: Gauss nodes and weights
// (Sec. 2.3), recurrence coefficients a_n^m, b_n^m (Sec. 3.2), the starting
// values P_m^m(x_j) with their rescaling counters (Sec. 3.5), derivative
// coefficients for the vector transforms and the FFT twiddles.  Everything is
// computed in FP64 on the host once and copied to the device; FP32 copies are
// rounded from the FP64 values.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <vector>

#include "sht_internal.h"

namespace sht {

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

// P_n(x) and P_{n-1}(x) by the three-term recurrence of Sec. 2.1.
void legendre_pair(int n, double x, double &pn, double &pn1)
{
    double a = 1.0, b = x;  // P_0, P_1
    if (n == 0) { pn = 1.0; pn1 = 0.0; return; }
    for (int k = 2; k <= n; ++k) {
        double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
        a = b;
        b = c;
    }
    pn = b;
    pn1 = a;
}

// Nodes of the nlat-point Gauss-Legendre rule, largest first, and weights
// w = 2 / ((1 - x^2) P_n'(x)^2) with (1 - x^2) P_n' = n (P_{n-1} - x P_n).
// Keeping the -x P_n term (zero at the exact root) cancels the first-order
// effect of rounding the node to a double, which near the poles would
// otherwise be amplified by ~ 2(n+1)/(1 - x^2).  Newton on P_n started from
// Tricomi's asymptotic estimate.
void gauss_nodes(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double th = kPi * (4.0 * i + 3.0) / (4.0 * n + 2.0);
        double z = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * std::cos(th);
        double pn = 0.0, pn1 = 0.0;
        for (int it = 0; it < 60; ++it) {
            legendre_pair(n, z, pn, pn1);
            double dp = n * (pn1 - z * pn) / ((1.0 - z) * (1.0 + z));
            double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) <= 2e-16 * std::fabs(z) + 1e-300 && it > 2) break;
        }
        legendre_pair(n, z, pn, pn1);
        const double omx2 = (1.0 - z) * (1.0 + z);
        const double q = n * (pn1 - z * pn);   // (1 - x^2) P_n'(x)
        const double wt = 2.0 * omx2 / (q * q);
        if (n % 2 == 1 && i == n / 2) z = 0.0;  // the equatorial node
        x[i] = z;
        x[n - 1 - i] = -z;
        w[i] = wt;
        w[n - 1 - i] = wt;
    }
}

// Round the double table into a float copy.
std::vector<float> to_f32(const std::vector<double> &v)
{
    std::vector<float> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = (float)v[i];
    return o;
}

// Bump allocator over a single device allocation.
struct DevArena {
    char *base = nullptr;
    size_t off = 0, cap = 0;
    template <typename U>
    U *take(size_t count)
    {
        size_t bytes = (count * sizeof(U) + 255) & ~size_t(255);
        U *p = reinterpret_cast<U *>(base + off);
        off += bytes;
        return p;
    }
};

template <typename U>
size_t padded(size_t count) { return (count * sizeof(U) + 255) & ~size_t(255); }

}  // namespace

PlanView<double> Plan::view64() const
{
    PlanView<double> v{lmax, mmax, nlat, nphi, npairs, nlm,
                       t64.ab, t64.dc, t64.x, t64.st, t64.wq, t64.pmm, t64.pmmk, t64.tw, t64.rtw, fft_plan_of(nphi / 2), mres, twdf,
                       nullptr, d_seg32, seeds64, seeds64k, live64};
    return v;
}

PlanView<float> Plan::view32() const
{
    PlanView<float> v{lmax, mmax, nlat, nphi, npairs, nlm,
                      t32.ab, t32.dc, t32.x, t32.st, t32.wq, t32.pmm, t32.pmmk, t32.tw, t32.rtw, fft_plan_of(nphi / 2), mres, nullptr,
                      seeds32, d_seg32, nullptr, nullptr, live32};
    return v;
}

int plan_build(Plan &p, std::string &err)
{
    const int lmax = p.lmax, mmax = p.mmax, nlat = p.nlat, nphi = p.nphi, mres = p.mres;
    p.npairs = (nlat + 1) / 2;
    // orders m = k mres, k = 0 .. mmax, each with degrees m .. lmax
    p.nlm = (int)col_of_mres(lmax, mmax + 1, mres);
    const int npairs = p.npairs, nlm = p.nlm;
    gauss_nodes(nlat, p.x, p.w);

    // Recurrence coefficients of Sec. 3.2, packed like the spectral arrays.
    std::vector<double> ab((size_t)2 * nlm), dc(nlm);
    for (int kq = 0; kq <= mmax; ++kq) {
        const int m = kq * mres;
        const size_t col = (size_t)col_of_mres(lmax, kq, mres);
        for (int n = m; n <= lmax; ++n) {
            const size_t i = col + (n - m);
            const double dn = n, dm = m;
            double a, b;
            if (n == m) {            // P_m^m is loaded as the starting value
                a = 0.0; b = 1.0;
            } else if (n == m + 1) { // P_{m+1}^m = sqrt(2m+3) x P_m^m
                a = std::sqrt(2.0 * m + 3.0); b = 0.0;
            } else {
                a = std::sqrt((4.0 * dn * dn - 1.0) / (dn * dn - dm * dm));
                b = -std::sqrt((2.0 * dn + 1.0) / (2.0 * dn - 3.0) *
                               ((dn - 1.0) * (dn - 1.0) - dm * dm) / (dn * dn - dm * dm));
            }
            ab[2 * i] = a;
            ab[2 * i + 1] = b;
            dc[i] = (n == m) ? 0.0 : std::sqrt((2.0 * dn + 1.0) * (dn * dn - dm * dm) / (2.0 * dn - 1.0));
        }
    }

    // Per latitude pair: northern node, sin(theta), weight.
    std::vector<double> xp(npairs), sp(npairs), wp(npairs);
    for (int j = 0; j < npairs; ++j) {
        xp[j] = p.x[j];
        sp[j] = std::sqrt((1.0 - p.x[j]) * (1.0 + p.x[j]));
        wp[j] = p.w[j];
    }

    // Starting values P_m^m(x_j) = sqrt(1/4pi) prod_{k<=m} sqrt((2k+1)/(2k)) sin^m,
    // carried as mantissa * 2^e, then written as y * 2^(-S k) with y in [2^-S, 1)
    // when the value is below 2^-S (k > 0), else y = value, k = 0.
    std::vector<double> pmm64((size_t)(mmax + 1) * npairs), pmm32d((size_t)(mmax + 1) * npairs);
    std::vector<int> k64((size_t)(mmax + 1) * npairs), k32((size_t)(mmax + 1) * npairs);
    auto split = [](double mant, long e, int S, double &y, int &k) {
        if (mant == 0.0) { y = 0.0; k = 0; return; }
        if (e >= 1 - S) { y = std::ldexp(mant, (int)e); k = 0; return; }
        long kk = (-e) / S;  // equals ceil((1 - S - e) / S) when e < 1 - S
        y = std::ldexp(mant, (int)(e + S * kk));
        k = (int)kk;
    };
    for (int j = 0; j < npairs; ++j) {
        int ex = 0;
        double mant = std::frexp(std::sqrt(1.0 / (4.0 * kPi)), &ex);
        long e = ex;
        for (int m = 0; m <= mmax * mres; ++m) {
            if (m > 0) {
                mant *= std::sqrt((2.0 * m + 1.0) / (2.0 * m)) * sp[j];
                int ee = 0;
                mant = std::frexp(mant, &ee);
                e += ee;
            }
            if (m % mres) continue;   // only the orders of the plan are stored
            const size_t o = (size_t)(m / mres) * npairs + j;
            split(mant, e, Scale<double>::S, pmm64[o], k64[o]);
            split(mant, e, Scale<float>::S, pmm32d[o], k32[o]);
        }
    }

    // FFT twiddles e^{2 pi i k / nphi}, k < nphi/2.
    const int H = nphi / 2;
    std::vector<double> tw((size_t)2 * (H > 0 ? H : 1));
    for (int k = 0; k < H; ++k) {
        const double ang = 2.0 * kPi * k / nphi;
        tw[2 * k] = std::cos(ang);
        tw[2 * k + 1] = std::sin(ang);
    }

    // Twiddles of the four-step FFT of length H: rtw[k1 N2 + n2] = e^{2 pi i n2 k1 / H}.
    const size_t H1 = H > 0 ? H : 1;
    std::vector<double> rtw(2 * H1, 0.0);
    {
        int logH = 0;
        while ((1 << logH) < H) ++logH;
        const int N1 = fft_n1(logH), N2 = H / N1;
        for (int k1 = 0; k1 < N1 && H > 0; ++k1)
            for (int n2 = 0; n2 < N2; ++n2) {
                const double ang = 2.0 * kPi * (double)(n2 * k1) / H;
                rtw[2 * ((size_t)k1 * N2 + n2)] = std::cos(ang);
                rtw[2 * ((size_t)k1 * N2 + n2) + 1] = std::sin(ang);
            }
    }

    // One device allocation holding both precisions' tables.
    size_t bytes = padded<double2>(nlm) + padded<double>(nlm) + 3 * padded<double>(npairs) +
                   padded<double>((size_t)(mmax + 1) * npairs) + padded<int>((size_t)(mmax + 1) * npairs) +
                   2 * padded<double2>(H1);
    bytes += padded<float2>(nlm) + padded<float>(nlm) + 3 * padded<float>(npairs) +
             padded<float>((size_t)(mmax + 1) * npairs) + padded<int>((size_t)(mmax + 1) * npairs) +
             2 * padded<float2>(H1);
    bytes += padded<float4>(H1) + padded<int>(1);
    DevArena ar;
    cudaError_t ce = cudaGetDevice(&p.device);
    if (ce != cudaSuccess) { err = std::string("cudaGetDevice: ") + cudaGetErrorString(ce); return SHT_ECUDA; }
    ce = cudaMalloc(&ar.base, bytes);
    if (ce != cudaSuccess) { err = std::string("cudaMalloc(plan tables): ") + cudaGetErrorString(ce); return SHT_ENOMEM; }
    ar.cap = bytes;
    p.tables_base = ar.base;

    auto up = [&](void *dst, const void *src, size_t n) -> bool {
        return cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    bool ok = true;
    p.t64.ab = ar.take<double2>(nlm);
    ok &= up(p.t64.ab, ab.data(), sizeof(double) * 2 * nlm);
    p.t64.dc = ar.take<double>(nlm);
    ok &= up(p.t64.dc, dc.data(), sizeof(double) * nlm);
    p.t64.x = ar.take<double>(npairs);
    ok &= up(p.t64.x, xp.data(), sizeof(double) * npairs);
    p.t64.st = ar.take<double>(npairs);
    ok &= up(p.t64.st, sp.data(), sizeof(double) * npairs);
    p.t64.wq = ar.take<double>(npairs);
    ok &= up(p.t64.wq, wp.data(), sizeof(double) * npairs);
    p.t64.pmm = ar.take<double>((size_t)(mmax + 1) * npairs);
    ok &= up(p.t64.pmm, pmm64.data(), sizeof(double) * pmm64.size());
    p.t64.pmmk = ar.take<int>((size_t)(mmax + 1) * npairs);
    ok &= up(p.t64.pmmk, k64.data(), sizeof(int) * k64.size());
    p.t64.tw = ar.take<double2>(H1);
    ok &= up(p.t64.tw, tw.data(), sizeof(double) * 2 * H1);
    p.t64.rtw = ar.take<double2>(H1);
    ok &= up(p.t64.rtw, rtw.data(), sizeof(double) * 2 * H1);

    std::vector<float> ab32 = to_f32(ab), dc32 = to_f32(dc), x32 = to_f32(xp), s32 = to_f32(sp),
                       w32 = to_f32(wp), pmm32 = to_f32(pmm32d), tw32 = to_f32(tw),
                       rtw32 = to_f32(rtw);
    p.t32.ab = ar.take<float2>(nlm);
    ok &= up(p.t32.ab, ab32.data(), sizeof(float) * 2 * nlm);
    p.t32.dc = ar.take<float>(nlm);
    ok &= up(p.t32.dc, dc32.data(), sizeof(float) * nlm);
    p.t32.x = ar.take<float>(npairs);
    ok &= up(p.t32.x, x32.data(), sizeof(float) * npairs);
    p.t32.st = ar.take<float>(npairs);
    ok &= up(p.t32.st, s32.data(), sizeof(float) * npairs);
    p.t32.wq = ar.take<float>(npairs);
    ok &= up(p.t32.wq, w32.data(), sizeof(float) * npairs);
    p.t32.pmm = ar.take<float>((size_t)(mmax + 1) * npairs);
    ok &= up(p.t32.pmm, pmm32.data(), sizeof(float) * pmm32.size());
    p.t32.pmmk = ar.take<int>((size_t)(mmax + 1) * npairs);
    ok &= up(p.t32.pmmk, k32.data(), sizeof(int) * k32.size());
    p.t32.tw = ar.take<float2>(H1);
    ok &= up(p.t32.tw, tw32.data(), sizeof(float) * 2 * H1);
    p.t32.rtw = ar.take<float2>(H1);
    ok &= up(p.t32.rtw, rtw32.data(), sizeof(float) * 2 * H1);
    // the same twiddles as double-float pairs: hi = fl32(w), lo = fl32(w - hi)
    std::vector<float> twdf(4 * H1, 0.f);
    for (size_t k = 0; k < 2 * H1; ++k) {
        const float hi = (float)tw[k];
        twdf[2 * k] = hi;
        twdf[2 * k + 1] = (float)(tw[k] - (double)hi);
    }
    p.twdf = ar.take<float4>(H1);
    ok &= up(p.twdf, twdf.data(), sizeof(float) * 4 * H1);
    p.d_err = ar.take<int>(1);
    ok &= cudaMemset(p.d_err, 0, sizeof(int)) == cudaSuccess;
    if (!ok) {
        err = "cudaMemcpy of plan tables failed";
        cudaFree(ar.base);
        p.tables_base = nullptr;
        return SHT_ECUDA;
    }
    return 0;
}

size_t seed_segment_offsets(int lmax, int mmax, int mres, std::vector<unsigned long long> &segoff)
{
    segoff.assign(mmax + 1, 0);
    unsigned long long s = 0;
    for (int m = 0; m <= mmax; ++m) {
        segoff[m] = s;
        s += (unsigned long long)((lmax - m * mres + 1 + kSeedSeg - 1) / kSeedSeg);
    }
    return (size_t)s;
}

namespace {

// The segment offsets (shared by both precisions).
int plan_segments(Plan &p, std::string &err)
{
    if (p.d_seg32) return SHT_OK;
    std::vector<unsigned long long> segoff;
    seed_segment_offsets(p.lmax, p.mmax, p.mres, segoff);
    cudaError_t e = cudaMalloc(&p.d_seg32, sizeof(unsigned long long) * segoff.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(p.d_seg32, segoff.data(), sizeof(unsigned long long) * segoff.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p.d_seg32);
        p.d_seg32 = nullptr;
        err = std::string("segment table: ") + cudaGetErrorString(e);
        return SHT_ENOMEM;
    }
    return SHT_OK;
}

size_t plan_nseg(const Plan &p)
{
    std::vector<unsigned long long> segoff;
    return seed_segment_offsets(p.lmax, p.mmax, p.mres, segoff);
}

}  // namespace

int plan_seeds32(Plan &p, std::string &err)
{
    if (p.seeds32) return SHT_OK;
    int rc = plan_segments(p, err);
    if (rc) return rc;
    const size_t nseg = plan_nseg(p);
    cudaError_t e = cudaMalloc(&p.seeds32, sizeof(float4) * nseg * (size_t)p.npairs);
    if (e == cudaSuccess) e = cudaMalloc(&p.live32, sizeof(unsigned short) * (size_t)(p.mmax + 1) * p.npairs);
    if (e == cudaSuccess)
        e = launch_build_restarts(p.view64(), p.d_seg32, p.seeds32, nullptr, nullptr, p.live32, p.thr_cc32(), 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p.seeds32);
        cudaFree(p.live32);
        p.seeds32 = nullptr;
        p.live32 = nullptr;
        err = std::string("building FP32 recurrence seeds: ") + cudaGetErrorString(e);
        return SHT_ENOMEM;
    }
    return SHT_OK;
}

int plan_seeds64(Plan &p, std::string &err)
{
    if (p.seeds64) return SHT_OK;
    int rc = plan_segments(p, err);
    if (rc) return rc;
    const size_t nseg = plan_nseg(p);
    cudaError_t e = cudaMalloc(&p.seeds64, sizeof(double2) * nseg * (size_t)p.npairs);
    if (e == cudaSuccess) e = cudaMalloc(&p.seeds64k, sizeof(int) * nseg * (size_t)p.npairs);
    if (e == cudaSuccess) e = cudaMalloc(&p.live64, sizeof(unsigned short) * (size_t)(p.mmax + 1) * p.npairs);
    if (e == cudaSuccess)
        e = launch_build_restarts(p.view64(), p.d_seg32, nullptr, p.seeds64, p.seeds64k, p.live64, p.thr_cc64(), 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p.seeds64);
        cudaFree(p.seeds64k);
        cudaFree(p.live64);
        p.seeds64 = nullptr;
        p.seeds64k = nullptr;
        p.live64 = nullptr;
        err = std::string("building FP64 recurrence seeds: ") + cudaGetErrorString(e);
        return SHT_ENOMEM;
    }
    return SHT_OK;
}

int plan_relive(Plan &p, std::string &err)
{
    cudaError_t e = cudaSuccess;
    if (p.seeds32)
        e = launch_build_restarts(p.view64(), p.d_seg32, p.seeds32, nullptr, nullptr, p.live32, p.thr_cc32(), 0);
    if (e == cudaSuccess && p.seeds64)
        e = launch_build_restarts(p.view64(), p.d_seg32, nullptr, p.seeds64, p.seeds64k, p.live64, p.thr_cc64(), 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
        err = std::string("rebuilding the polar tables: ") + cudaGetErrorString(e);
        return SHT_ECUDA;
    }
    return SHT_OK;
}

void schedule_lpt(const std::vector<int> &cost, const std::vector<int> &group, int nctas, std::vector<int> &sched)
{
    // groups in order of first appearance, their items in ascending order
    std::vector<int> gid(cost.size(), -1);
    std::vector<std::vector<int>> members;
    std::vector<long long> gcost;
    std::vector<int> slot;   // group id -> index in members
    for (int w = 0; w < (int)cost.size(); ++w) {
        if (cost[w] < 0) continue;
        const int g = group[w];
        if (g >= (int)slot.size()) slot.resize(g + 1, -1);
        if (slot[g] < 0) {
            slot[g] = (int)members.size();
            members.emplace_back();
            gcost.push_back(0);
        }
        members[slot[g]].push_back(w);
        gcost[slot[g]] += cost[w];
    }
    std::vector<int> order(members.size());
    for (int i = 0; i < (int)order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return gcost[x] > gcost[y]; });
    std::vector<long long> load(nctas, 0);
    std::vector<std::vector<int>> lists(nctas);
    for (const int g : order) {
        int best = 0;
        for (int i = 1; i < nctas; ++i)
            if (load[i] < load[best]) best = i;
        load[best] += gcost[g];
        lists[best].insert(lists[best].end(), members[g].begin(), members[g].end());
    }
    sched.assign(nctas + 1, 0);
    for (int i = 0; i < nctas; ++i) sched[i + 1] = sched[i] + (int)lists[i].size();
    for (int i = 0; i < nctas; ++i) sched.insert(sched.end(), lists[i].begin(), lists[i].end());
}

void plan_free_tc64(Plan &p)
{
    cudaFree(p.p64_s); cudaFree(p.p64_a); cudaFree(p.d_off64_s); cudaFree(p.d_off64_a); cudaFree(p.d_dchunk64);
    cudaFree(p.d_e64_s); cudaFree(p.d_e64_a); cudaFree(p.d_c064_s); cudaFree(p.d_c064_a); cudaFree(p.d_fcol);
    cudaFree(p.d_sched64_s); cudaFree(p.d_sched64_a);
    cudaFree(p.d_gf64_s); cudaFree(p.d_gf64_a); cudaFree(p.d_zero64);
    p.d_gf64_s = p.d_gf64_a = nullptr;
    p.d_zero64 = nullptr;
    p.p64_s = p.p64_a = nullptr;
    p.d_off64_s = p.d_off64_a = p.d_dchunk64 = nullptr;
    p.d_e64_s = p.d_e64_a = p.d_c064_s = p.d_c064_a = p.d_fcol = nullptr;
    p.d_sched64_s = p.d_sched64_a = nullptr;
    p.sched64_ctas = 0;
}

void plan_free(Plan &p)
{
    cudaFree(p.seeds32);
    cudaFree(p.d_seg32);
    cudaFree(p.seeds64);
    cudaFree(p.seeds64k);
    cudaFree(p.live32);
    cudaFree(p.live64);
    p.seeds32 = nullptr;
    p.d_seg32 = nullptr;
    p.seeds64 = nullptr;
    p.seeds64k = nullptr;
    p.live32 = p.live64 = nullptr;
    for (cudaEvent_t e : p.timer.pool) cudaEventDestroy(e);
    p.timer.pool.clear();
    if (p.tables_base) cudaFree(p.tables_base);
    if (p.work) cudaFree(p.work);
    if (p.panel_s) cudaFree(p.panel_s);
    if (p.panel_a) cudaFree(p.panel_a);
    if (p.d_off_s) cudaFree(p.d_off_s);
    if (p.d_off_a) cudaFree(p.d_off_a);
    if (p.d_dchunk) cudaFree(p.d_dchunk);
    if (p.d_c0_s) cudaFree(p.d_c0_s);
    if (p.d_c0_a) cudaFree(p.d_c0_a);
    plan_free_tc64(p);
    if (p.d_gf_s) cudaFree(p.d_gf_s);
    if (p.d_gf_a) cudaFree(p.d_gf_a);
    p.d_gf_s = p.d_gf_a = nullptr;
    for (int h = 0; h < 2; ++h) {
        cudaFree(p.d_schedv_s[h]);
        cudaFree(p.d_schedv_a[h]);
        p.d_schedv_s[h] = p.d_schedv_a[h] = nullptr;
    }
    if (p.dpanel_s) cudaFree(p.dpanel_s);
    if (p.dpanel_a) cudaFree(p.dpanel_a);
    if (p.d_c0v_s) cudaFree(p.d_c0v_s);
    if (p.d_c0v_a) cudaFree(p.d_c0v_a);
    if (p.otf_seeds) cudaFree(p.otf_seeds);
    if (p.d_segoff) cudaFree(p.d_segoff);
    if (p.d_c0o_s) cudaFree(p.d_c0o_s);
    if (p.d_c0o_a) cudaFree(p.d_c0o_a);
    p.otf_seeds = nullptr;
    p.d_segoff = nullptr;
    p.d_c0o_s = p.d_c0o_a = nullptr;
    p.panel_s = p.panel_a = p.dpanel_s = p.dpanel_a = nullptr;
    p.d_off_s = p.d_off_a = p.d_dchunk = nullptr;
    p.d_c0_s = p.d_c0_a = p.d_c0v_s = p.d_c0v_a = nullptr;
    p.tables_base = nullptr;
    p.work = nullptr;
    p.work_bytes = 0;
}

}  // namespace sht
