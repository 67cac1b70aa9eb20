// sht_internal.h -- plan structure and kernel launchers shared by the
// translation units of libsht.  Not part of the public ABI (see include/sht.h).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "sht.h"

namespace sht {

// Exponent step of the underflow rescaling (Sec. 3.5): a value is carried as
// y * 2^(-S k) with an integer k >= 0.  While k > 0 the true value is below
// 2^-S: it is left out of the Legendre sums but still advanced by the
// recurrence.  Dropped terms are < 2^-240 (FP64) or 2^-64 (FP32).
template <typename T> struct Scale;
template <> struct Scale<double> { static constexpr int S = 240; };
template <> struct Scale<float> { static constexpr int S = 64; };

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

// Device tables of one precision.
template <typename T>
struct Tables {
    using T2 = typename Vec2<T>::type;
    T2 *ab = nullptr;    // [nlm] (a_n^m, b_n^m); (0, 1) at n = m, (sqrt(2m+3), 0) at n = m+1
    T *dc = nullptr;     // [nlm] sqrt((2n+1)(n^2-m^2)/(2n-1)); 0 at n = m
    T *x = nullptr;      // [npairs] cos(theta) of the northern node of each pair (>= 0)
    T *st = nullptr;     // [npairs] sin(theta)
    T *wq = nullptr;     // [npairs] Gauss weight of that node
    T *pmm = nullptr;    // [mmax+1][npairs] P_m^m(x_p) * 2^(S k) (mantissa)
    int *pmmk = nullptr; // [mmax+1][npairs] k (number of 2^S steps)
    T2 *tw = nullptr;    // [nphi/2] e^{2 pi i k / nphi}
};

// Kernel-side view of a plan in precision T.
template <typename T>
struct PlanView {
    using T2 = typename Vec2<T>::type;
    int lmax, mmax, nlat, nphi, npairs, nlm;
    const T2 *ab;
    const T *dc;
    const T *x;
    const T *st;
    const T *wq;
    const T *pmm;
    const int *pmmk;
    const T2 *tw;
};

// What a Legendre or FFT launch computes; selects the scale factors.
enum Op {
    OP_SYNTH = 0,       // forward synthesis
    OP_ANALYS = 1,      // forward analysis
    OP_SYNTH_ADJ = 2,   // adjoint of synthesis (an unweighted analysis times c_m)
    OP_ANALYS_ADJ = 3   // adjoint of analysis (a weighted synthesis of b / c_m)
};

// Event pairs recorded around kernel launches while profiling is enabled.
struct KernelTimer {
    bool enabled = false;
    std::vector<cudaEvent_t> pool;   // created on demand, reused
    std::vector<int> kinds;          // kind of each recorded pair
    size_t used = 0;                 // events in use (2 per launch)
};

struct Plan {
    int lmax, mmax, nlat, nphi, npairs, nlm;
    std::vector<double> x, w;        // host nodes (descending) and weights, all nlat
    Tables<double> t64;
    Tables<float> t32;
    void *tables_base = nullptr;     // single device allocation holding t64 and t32
    void *work = nullptr;            // scratch (grown on demand)
    size_t work_bytes = 0;
    int device = 0;
    KernelTimer timer;

    PlanView<double> view64() const;
    PlanView<float> view32() const;
};

// Host plan construction (plan.cpp).
int plan_build(Plan &p, std::string &err);
void plan_free(Plan &p);

// Launchers (legendre.cu, fft.cu).  `eo` / `sd` are intermediate buffers of
// [batch][mmax+1][npairs][2] complex values of precision T.
template <typename T>
cudaError_t launch_legendre_synth(const PlanView<T> &pv, const T *spec, T *eo, int batch, Op op,
                                  cudaStream_t s);
template <typename T>
cudaError_t launch_legendre_analys(const PlanView<T> &pv, const T *sd, T *spec, int batch, Op op,
                                   cudaStream_t s);
template <typename T>
cudaError_t launch_legendre_synth_vec(const PlanView<T> &pv, const T *S, const T *Tc, T *eot,
                                      T *eop, int batch, Op op, cudaStream_t s);
template <typename T>
cudaError_t launch_legendre_analys_vec(const PlanView<T> &pv, const T *sdt, const T *sdp, T *S,
                                       T *Tc, int batch, Op op, cudaStream_t s);
template <typename T>
cudaError_t launch_fft_synth(const PlanView<T> &pv, const T *eo, T *grid, int batch, Op op,
                             cudaStream_t s);
template <typename T>
cudaError_t launch_fft_analys(const PlanView<T> &pv, const T *grid, T *sd, int batch, Op op,
                              bool vector, cudaStream_t s);

}  // namespace sht
