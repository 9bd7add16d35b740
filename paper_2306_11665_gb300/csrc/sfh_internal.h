// sfh_internal.h -- declarations shared by the host API and the kernel
// instantiation units of libsfhad (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sfh_device.cuh"

namespace sfh {

// One entry point per (precision mode, dimension, flux family) instantiation
// unit; each dispatches on n = p + 1 (2..9) and the flux.
#define SFH_DECL_VOLUME(name, T)                                                                   \
    cudaError_t name(int n, int flux, const void *u, const double *Ja, void *r, int64_t n_elem,     \
                     const OpTab<T> &tab, int *err, cudaStream_t stream);
SFH_DECL_VOLUME(volume_fp64_d2, double)
SFH_DECL_VOLUME(volume_fp64_d3, double)
SFH_DECL_VOLUME(volume_fp32k_d2, float)
SFH_DECL_VOLUME(volume_fp32k_d3, float)
SFH_DECL_VOLUME(volume_mixed_d2, float)
SFH_DECL_VOLUME(volume_mixed_d3, float)
// Chandrashekar's flux (flux == kFluxEulerCh only)
SFH_DECL_VOLUME(volume_fp64_d2_ch, double)
SFH_DECL_VOLUME(volume_fp64_d3_ch, double)
SFH_DECL_VOLUME(volume_fp32k_d2_ch, float)
SFH_DECL_VOLUME(volume_fp32k_d3_ch, float)
SFH_DECL_VOLUME(volume_mixed_d2_ch, float)
SFH_DECL_VOLUME(volume_mixed_d3_ch, float)
#undef SFH_DECL_VOLUME

// Modal entry points (basis coefficients in, V^T r_v out).
#define SFH_DECL_MODAL(name, T)                                                                    \
    cudaError_t name(int n, int flux, const void *u, const double *Ja, void *r, int64_t n_elem,     \
                     const OpTab<T> &tab, const BasisTab<T> &bt, int *err, cudaStream_t stream);
SFH_DECL_MODAL(volume_fp64_d2_modal, double)
SFH_DECL_MODAL(volume_fp64_d3_modal, double)
SFH_DECL_MODAL(volume_fp32k_d2_modal, float)
SFH_DECL_MODAL(volume_fp32k_d3_modal, float)
SFH_DECL_MODAL(volume_mixed_d2_modal, float)
SFH_DECL_MODAL(volume_mixed_d3_modal, float)
SFH_DECL_MODAL(volume_fp64_d2_ch_modal, double)
SFH_DECL_MODAL(volume_fp64_d3_ch_modal, double)
SFH_DECL_MODAL(volume_fp32k_d2_ch_modal, float)
SFH_DECL_MODAL(volume_fp32k_d3_ch_modal, float)
SFH_DECL_MODAL(volume_mixed_d2_ch_modal, float)
SFH_DECL_MODAL(volume_mixed_d3_ch_modal, float)
#undef SFH_DECL_MODAL

// Basis transforms of the modal residual as kernels of their own (3D, FP32
// state, n = 3..8, five variables): u_hat -> V u_hat, or (backward) r_v ->
// V^T r_v (sfh_modal.cu).
cudaError_t modal_xform_3d(int n, bool backward, const float *in, float *out, int64_t n_elem,
                           const BasisTab<float> &bt, int *err, cudaStream_t stream);

using ModalFn64 = cudaError_t (*)(int, int, const void *, const double *, void *, int64_t, const OpTab<double> &,
                                  const BasisTab<double> &, int *, cudaStream_t);
using ModalFn32 = cudaError_t (*)(int, int, const void *, const double *, void *, int64_t, const OpTab<float> &,
                                  const BasisTab<float> &, int *, cudaStream_t);
inline ModalFn64 modal_fp64_fn(int d, int flux) {
    if (flux == kFluxEulerCh) return d == 3 ? volume_fp64_d3_ch_modal : volume_fp64_d2_ch_modal;
    return d == 3 ? volume_fp64_d3_modal : volume_fp64_d2_modal;
}
inline ModalFn32 modal_fp32k_fn(int d, int flux) {
    if (flux == kFluxEulerCh) return d == 3 ? volume_fp32k_d3_ch_modal : volume_fp32k_d2_ch_modal;
    return d == 3 ? volume_fp32k_d3_modal : volume_fp32k_d2_modal;
}
inline ModalFn32 modal_mixed_fn(int d, int flux) {
    if (flux == kFluxEulerCh) return d == 3 ? volume_mixed_d3_ch_modal : volume_mixed_d2_ch_modal;
    return d == 3 ? volume_mixed_d3_modal : volume_mixed_d2_modal;
}

// The instantiation unit's entry point for a (d, flux).
using VolumeFn64 = cudaError_t (*)(int, int, const void *, const double *, void *, int64_t, const OpTab<double> &,
                                   int *, cudaStream_t);
using VolumeFn32 = cudaError_t (*)(int, int, const void *, const double *, void *, int64_t, const OpTab<float> &,
                                   int *, cudaStream_t);
inline VolumeFn64 volume_fp64_fn(int d, int flux) {
    if (flux == kFluxEulerCh) return d == 3 ? volume_fp64_d3_ch : volume_fp64_d2_ch;
    return d == 3 ? volume_fp64_d3 : volume_fp64_d2;
}
inline VolumeFn32 volume_fp32k_fn(int d, int flux) {
    if (flux == kFluxEulerCh) return d == 3 ? volume_fp32k_d3_ch : volume_fp32k_d2_ch;
    return d == 3 ? volume_fp32k_d3 : volume_fp32k_d2;
}
inline VolumeFn32 volume_mixed_fn(int d, int flux) {
    if (flux == kFluxEulerCh) return d == 3 ? volume_mixed_d3_ch : volume_mixed_d2_ch;
    return d == 3 ? volume_mixed_d3 : volume_mixed_d2;
}

// Generic Hadamard product of the Fig. 1 experiment (sfh_fig1.cu); D is the
// n x n Gauss-Lobatto derivative, row-major.
cudaError_t fig1_hadamard(int n, bool dense, const double *c, double *y, int64_t n_elem, const double *D,
                          cudaStream_t stream);

// Surface Hadamard product (sfh_surface.cu): quadrature weights and the rows
// interpolating to xi = -1 (side 0) and +1 (side 1), e[side][b] = l_b(-+1).
struct SurfTab {
    double w[NMAX];
    double e[2][NMAX];
};
cudaError_t surface_hadamard(int d, int n, int flux, const double *u, const double *u_face, const double *nJ,
                             double *r_vol, double *r_face, int64_t n_elem, const SurfTab &tab, int *err,
                             cudaStream_t stream);

// Entropy-identity defect per element (sfh_entropy.cu); r in FP32 or FP64.
cudaError_t entropy_identity(int d, int n, int flux, const double *u, const double *Ja, const void *r, bool r_fp32,
                             double *out, int64_t n_elem, const OpTab<double> &tab, int *err, cudaStream_t stream);

#define SFH_DECL_VJP(name)                                                                          \
    cudaError_t name(int n, int flux, const double *u, const double *Ja, const double *lam, double *g, \
                     int64_t n_elem, const OpTab<double> &tab, int *err, cudaStream_t stream);
SFH_DECL_VJP(vjp_d2)
SFH_DECL_VJP(vjp_d3)
SFH_DECL_VJP(vjp_d2_ch)
SFH_DECL_VJP(vjp_d3_ch)
#undef SFH_DECL_VJP

#define SFH_DECL_VJP_MODAL(name)                                                                    \
    cudaError_t name(int n, int flux, const double *u, const double *Ja, const double *lam, double *g, \
                     int64_t n_elem, const OpTab<double> &tab, const BasisTab<double> &bt, int *err,   \
                     cudaStream_t stream);
SFH_DECL_VJP_MODAL(vjp_d2_modal)
SFH_DECL_VJP_MODAL(vjp_d3_modal)
SFH_DECL_VJP_MODAL(vjp_d2_ch_modal)
SFH_DECL_VJP_MODAL(vjp_d3_ch_modal)
#undef SFH_DECL_VJP_MODAL

inline cudaError_t (*vjp_modal_fn(int d, int flux))(int, int, const double *, const double *, const double *,
                                                    double *, int64_t, const OpTab<double> &,
                                                    const BasisTab<double> &, int *, cudaStream_t) {
    if (flux == kFluxEulerCh) return d == 3 ? vjp_d3_ch_modal : vjp_d2_ch_modal;
    return d == 3 ? vjp_d3_modal : vjp_d2_modal;
}

inline cudaError_t (*vjp_fn(int d, int flux))(int, int, const double *, const double *, const double *, double *,
                                              int64_t, const OpTab<double> &, int *, cudaStream_t) {
    if (flux == kFluxEulerCh) return d == 3 ? vjp_d3_ch : vjp_d2_ch;
    return d == 3 ? vjp_d3 : vjp_d2;
}

// Operator tables of degree p on node set `nodes` (SFH_NODES_*): w and
// Q1 = diag(w) D (Eq. 5), each entry rounded once from the long-double
// construction to the table's type.  False for p or nodes out of range.
// Shared by the contexts and the context-free entry points, so that both
// compute with the same FP32 and FP64 values.
bool op_tables(int p, int nodes, OpTab<double> &tab_d, OpTab<float> &tab_f);

// Status of a nonzero device error word (kErr* bits), with the calling
// thread's message set: a timeout gives SFH_ETIMEOUT, a bad state or an
// out-of-range metric term SFH_EDOMAIN.  Returns an sfh_status value.
int err_word_status(int h);

// Set the calling thread's message returned by sfh_last_error().
void set_error_message(const char *msg);

}  // namespace sfh
