// sfh_inst.cu -- kernel instantiation unit.  Compiled once per (mode, d,
// flux family, nodal or modal): -DSFH_INST_D=<2|3>, one of -DSFH_INST_FP64 /
// -DSFH_INST_FP32K / -DSFH_INST_MIXED / -DSFH_INST_VJP, -DSFH_INST_CH for the
// units of Chandrashekar's flux (entry points suffixed _ch; the others hold
// Burgers and Ranocha's flux), and -DSFH_INST_MODAL for the modal entry
// points (suffixed _modal).  Splitting the instances over several objects
// keeps the build parallel.
#include "sfh_internal.h"
#include "sfh_volume.cuh"
#include "sfh_vjp.cuh"
#include "sfh_volume_tma.cuh"
#include "sfh_volume_ws.cuh"
#include "sfh_volume_row.cuh"
#include "sfh_volume_row64.cuh"

#ifndef SFH_INST_D
#error "SFH_INST_D must be defined"
#endif

#include <type_traits>

#define SFH_CAT2(a, b) a##b
#define SFH_CAT(a, b) SFH_CAT2(a, b)
#if defined(SFH_INST_MODAL)
#define SFH_MSUF _modal
#else
#define SFH_MSUF
#endif
#if defined(SFH_INST_CH)
#define SFH_NAME(base) SFH_CAT(SFH_CAT(SFH_CAT(base, SFH_INST_D), _ch), SFH_MSUF)
#else
#define SFH_NAME(base) SFH_CAT(SFH_CAT(base, SFH_INST_D), SFH_MSUF)
#endif

namespace sfh {

// Calls fn(std::integral_constant<int, FLUX>) for the fluxes this unit
// instantiates.
template <class Fn>
static cudaError_t pick_flux(int flux, Fn fn) {
#if defined(SFH_INST_CH)
    if (flux == kFluxEulerCh) return fn(std::integral_constant<int, kFluxEulerCh>{});
#else
    if (flux == kFluxEuler) return fn(std::integral_constant<int, kFluxEuler>{});
    if (flux == kFluxBurgers) return fn(std::integral_constant<int, kFluxBurgers>{});
#endif
    return cudaErrorInvalidValue;
}

#if defined(SFH_INST_VJP)

#if defined(SFH_INST_MODAL)
cudaError_t SFH_NAME(vjp_d)(int n, int flux, const double *u, const double *Ja, const double *lam, double *g,
                           int64_t n_elem, const OpTab<double> &tab, const BasisTab<double> &bt, int *err,
                           cudaStream_t stream) {
    constexpr int D = SFH_INST_D;
#define SFH_CASE(N)                                                                                       \
    case N:                                                                                               \
        return pick_flux(flux, [&](auto F) {                                                              \
            return launch_vjp_modal<D, N, decltype(F)::value>(u, Ja, lam, g, n_elem, tab, bt, err, stream); \
        });
#else
cudaError_t SFH_NAME(vjp_d)(int n, int flux, const double *u, const double *Ja, const double *lam, double *g,
                           int64_t n_elem, const OpTab<double> &tab, int *err, cudaStream_t stream) {
    constexpr int D = SFH_INST_D;
#define SFH_CASE(N)                                                                                  \
    case N:                                                                                          \
        return pick_flux(flux, [&](auto F) {                                                         \
            return launch_vjp<D, N, decltype(F)::value>(u, Ja, lam, g, n_elem, tab, err, stream);  \
        });
#endif
    switch (n) {
        SFH_CASE(2) SFH_CASE(3) SFH_CASE(4) SFH_CASE(5) SFH_CASE(6) SFH_CASE(7) SFH_CASE(8) SFH_CASE(9)
        default: return cudaErrorInvalidValue;
    }
#undef SFH_CASE
}

#else

#if defined(SFH_INST_FP32K)
template <int D, int N, int FLUX>
cudaError_t launch_fp32k(const void *u, const double *Ja, void *r, int64_t n_elem, const OpTab<float> &tab, int *err,
                         cudaStream_t stream) {
    if constexpr (use_row_kernel<D, N, FLUX>())
        return launch_volume_fp32_row<N>(u, Ja, r, n_elem, tab, err, stream);
    else if constexpr (use_ws_kernel<D, N, FLUX>())
        return launch_volume_fp32_ws<D, N, FLUX>(u, Ja, r, n_elem, tab, err, stream);
    else
        return launch_volume_fp32_tma<D, N, FLUX>(u, Ja, r, n_elem, tab, err, stream);
}
#endif

#if defined(SFH_INST_MIXED) && !defined(SFH_INST_MODAL)
// Mixed mode: the warp-specialized kernel for 3D Euler at n = 3..8 (FP64
// metric pair sums and log-mean islands in its sweep), the thread-per-line
// kernel otherwise.
template <int D, int N, int FLUX>
cudaError_t launch_mixed(const void *u, const double *Ja, void *r, int64_t n_elem, const OpTab<float> &tab, int *err,
                         cudaStream_t stream) {
    if constexpr (use_ws_mixed<D, N, FLUX>())
        return launch_volume_fp32_ws<D, N, FLUX, true>(u, Ja, r, n_elem, tab, err, stream);
    else
        return launch_volume<D, N, FLUX, ModeMixed>(u, Ja, r, n_elem, tab, err, stream);
}
#endif

#if defined(SFH_INST_FP64)
// FP64 tile shape of the thread-per-line kernel: 3D n = 6, 7 take 256-line
// tiles with a 200 KB budget (one CTA of 7-8 warps per SM, 84-98 % of the
// lanes busy, against 77-84 % with the default two 4-warp CTAs; 5-6 % faster)
template <int D, int N, int FLUX>
constexpr bool fp64_big_tiles() { return D == 3 && (N == 6 || N == 7); }
template <int D, int N, int FLUX>
using Fp64Shape = Shape<D, N, FLUX, ModeFP64, fp64_big_tiles<D, N, FLUX>() ? 200 * 1024 : 96 * 1024,
                        fp64_big_tiles<D, N, FLUX>() ? 256 : 0>;

template <int D, int N, int FLUX>
cudaError_t launch_fp64(const void *u, const double *Ja, void *r, int64_t n_elem, const OpTab<double> &tab, int *err,
                        cudaStream_t stream) {
    // The thread-per-line kernel keeps the FP64 pipe busier on large meshes;
    // the row kernel wins where the former's element blocks would not fill
    // two CTAs per SM (e.g. 512 elements at n = 6: 0.25 against 0.31 ms).
    if constexpr (use_row64_kernel<D, N, FLUX>()) {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return cudaErrorInvalidDevice;
        using S = Fp64Shape<D, N, FLUX>;
        if ((n_elem + S::EPB - 1) / S::EPB < 2 * (int64_t)sms)
            return launch_volume_fp64_row<N>(u, Ja, r, n_elem, tab, err, stream);
    }
    return launch_volume<D, N, FLUX, ModeFP64, Fp64Shape<D, N, FLUX>>(u, Ja, r, n_elem, tab, err, stream);
}
#endif

#if defined(SFH_INST_FP64)
using Mode = ModeFP64;
#define SFH_FN SFH_NAME(volume_fp64_d)
#elif defined(SFH_INST_FP32K)
using Mode = ModeFP32K;
#define SFH_FN SFH_NAME(volume_fp32k_d)
#elif defined(SFH_INST_MIXED)
using Mode = ModeMixed;
#define SFH_FN SFH_NAME(volume_mixed_d)
#else
#error "no instantiation mode"
#endif

#if defined(SFH_INST_MODAL)
// Modal / uncollocated entry: u holds basis coefficients, r receives V^T r_v
// (the basis transforms fused into the kernels).  FP32-Kahan always takes the
// persistent line kernel.
cudaError_t SFH_FN(int n, int flux, const void *u, const double *Ja, void *r, int64_t n_elem,
                   const OpTab<typename Mode::T> &tab, const BasisTab<typename Mode::T> &bt, int *err,
                   cudaStream_t stream) {
    constexpr int D = SFH_INST_D;
#if defined(SFH_INST_FP32K)
#define SFH_MCALL(N, F) launch_volume_fp32_tma<D, N, F, true>(u, Ja, r, n_elem, tab, err, stream, &bt)
#elif defined(SFH_INST_FP64)
#define SFH_MCALL(N, F) launch_volume_modal<D, N, F, Mode, Fp64Shape<D, N, F>>(u, Ja, r, n_elem, tab, bt, err, stream)
#else
#define SFH_MCALL(N, F) launch_volume_modal<D, N, F, Mode>(u, Ja, r, n_elem, tab, bt, err, stream)
#endif
#define SFH_CASE(N)                                                                                    \
    case N:                                                                                            \
        return pick_flux(flux, [&](auto F) { return SFH_MCALL(N, decltype(F)::value); });
    switch (n) {
        SFH_CASE(2) SFH_CASE(3) SFH_CASE(4) SFH_CASE(5) SFH_CASE(6) SFH_CASE(7) SFH_CASE(8) SFH_CASE(9)
        default: return cudaErrorInvalidValue;
    }
#undef SFH_CASE
#undef SFH_MCALL
}
#else
cudaError_t SFH_FN(int n, int flux, const void *u, const double *Ja, void *r, int64_t n_elem,
                   const OpTab<typename Mode::T> &tab, int *err, cudaStream_t stream) {
    constexpr int D = SFH_INST_D;
#if defined(SFH_INST_FP32K)
    // FP32-Kahan: the persistent TMA-staged kernels (warp-specialized for 3D
    // Euler at n = 3..7, a thread per line and node for 3D Euler at n = 8, a
    // thread per line otherwise)
#define SFH_VCALL(N, F) launch_fp32k<D, N, F>(u, Ja, r, n_elem, tab, err, stream)
#elif defined(SFH_INST_FP64)
#define SFH_VCALL(N, F) launch_fp64<D, N, F>(u, Ja, r, n_elem, tab, err, stream)
#else
#define SFH_VCALL(N, F) launch_mixed<D, N, F>(u, Ja, r, n_elem, tab, err, stream)
#endif
#define SFH_CASE(N)                                                                                    \
    case N:                                                                                            \
        return pick_flux(flux, [&](auto F) { return SFH_VCALL(N, decltype(F)::value); });
    switch (n) {
        SFH_CASE(2) SFH_CASE(3) SFH_CASE(4) SFH_CASE(5) SFH_CASE(6) SFH_CASE(7) SFH_CASE(8) SFH_CASE(9)
        default: return cudaErrorInvalidValue;
    }
#undef SFH_CASE
#undef SFH_VCALL
}
#endif

#endif

}  // namespace sfh
