// sfh_entropy.cu -- the entropy identity of the volume term, evaluated on the
// GPU in FP64 for a residual computed in any precision.
//
// For r = sum_m (Q_m o F_m) 1 with Q_m 1 = 0 (Eq. 3 with the operators of
// Eq. 5) and a symmetric entropy-conservative two-point flux (Tadmor's
// condition (w_i - w_j).F_ij = (psi_i - psi_j).(J_i + J_j)), summation by
// parts gives, per element,
//   w^T r = sum_m [ 1/2 sum_ij E_ij w_i.F_ij - 1/2 sum_i (E 1)_i psi_i.J_i
//                   - 1/2 psi^T E J + psi^T Q J ],   E = Q_m + Q_m^T, J = Ja^m,
// with w the entropy variables and psi the entropy potential (Euler:
// w = ((g - s)/(g - 1) - rho|v|^2/(2p), rho v/p, -rho/p), s = ln p - g ln rho,
// psi = rho v; Burgers: w = u, psi_k = u^3/6).  For diagonal E (Gauss-Lobatto)
// this is the boundary entropy flux of the element.  The kernel returns per
// element |lhs - rhs| / scale with scale = sum_m sum_ij |Q_ij| |w_i . F_ij|
// (componentwise), so that the defect of a residual computed in FP64 sits at
// FP64 round-off and that of an FP32 residual at FP32 round-off.
//
// One CTA per element; a thread per grid line (all directions), node data in
// shared memory, the line's pairs evaluated with the FP64 flux of the volume
// kernels; sums reduced in a fixed order (deterministic).
#include <cuda_runtime.h>

#include "sfh_device.cuh"
#include "sfh_internal.h"
#include "sfh_volume.cuh"

namespace sfh {

constexpr int kEntThreads = 128;

template <int D, int N, int FLUX>
struct EntShape {
    static constexpr int NN = ipow(N, D), NLINE = ipow(N, D - 1);
    static constexpr int NVAR = is_euler(FLUX) ? D + 2 : 1;
    // per node: flux state (rho, v/2 [D], p, beta, FP32 copies of rho and beta
    // in one word) | u ; entropy variables w [NVAR]; potential psi [D]
    static constexpr int NS = is_euler(FLUX) ? D + 4 : 1;
    static constexpr int PER_NODE = NS + NVAR + D;
    static constexpr size_t SMEM = (size_t)PER_NODE * NN * sizeof(double);
};

template <int D, int N, int FLUX, typename TR>
__global__ void __launch_bounds__(kEntThreads)
entropy_identity_kernel(const double *__restrict__ u, const double *__restrict__ Ja, const TR *__restrict__ r,
                        double *__restrict__ out, int64_t n_elem, const __grid_constant__ OpTab<double> tab,
                        int *__restrict__ err) {
    using S = EntShape<D, N, FLUX>;
    constexpr int NN = S::NN, NLINE = S::NLINE, NVAR = S::NVAR, NS = S::NS;
    extern __shared__ __align__(16) double sm[];
    const auto sS = SFH_BP(sm, NS * NN, err);                             // [NS][NN]
    const auto sW = SFH_BP(sm + NS * NN, NVAR * NN, err);                 // [NVAR][NN]
    const auto sPsi = SFH_BP(sm + (NS + NVAR) * NN, D * NN, err);         // [D][NN]
    __shared__ double red[3][kEntThreads];

    const int64_t e = blockIdx.x;
    const int tid = threadIdx.x;
    const auto ue = SFH_BP(u, n_elem * NVAR * NN, err) + e * NVAR * NN;
    const auto re = SFH_BP(r, n_elem * NVAR * NN, err) + e * NVAR * NN;
    const auto Je = SFH_BP(Ja, n_elem * D * D * NN, err) + e * D * D * NN;

    // ---- node pass: states, entropy variables, potentials; w^T r
    double lhs = 0.0, rhs = 0.0, scale = 0.0;
    bool bad = false;
    for (int i = tid; i < NN; i += kEntThreads) {
        if constexpr (is_euler(FLUX)) {
            const double rho = ue[i], E = ue[(D + 1) * NN + i];
            double v[D], v2 = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) { v[k] = ue[(1 + k) * NN + i] / rho; v2 += v[k] * v[k]; }
            const double p = (kGamma - 1.0) * (E - 0.5 * rho * v2);
            const double beta = rho / p;
            bad |= !(rho > 0.0 && p > 0.0);
            sS[i] = rho;
#pragma unroll
            for (int k = 0; k < D; ++k) sS[(1 + k) * NN + i] = 0.5 * v[k];
            sS[(D + 1) * NN + i] = p;
            sS[(D + 2) * NN + i] = beta;
            const float2 rb = make_float2(d2f_int(rho), d2f_int(beta));
            sS[(D + 3) * NN + i] = __longlong_as_double(*reinterpret_cast<const long long *>(&rb));
            const double s = log(p) - kGamma * log(rho);
            double w[D + 2];
            w[0] = (kGamma - s) / (kGamma - 1.0) - 0.5 * rho * v2 / p;
#pragma unroll
            for (int k = 0; k < D; ++k) w[1 + k] = beta * v[k];
            w[D + 1] = -beta;
#pragma unroll
            for (int q = 0; q < D + 2; ++q) {
                sW[q * NN + i] = w[q];
                lhs = fma(w[q], (double)re[q * NN + i], lhs);
            }
#pragma unroll
            for (int k = 0; k < D; ++k) sPsi[k * NN + i] = rho * v[k];
        } else {
            const double uu = ue[i];
            sS[i] = uu;
            sW[i] = uu;
#pragma unroll
            for (int k = 0; k < D; ++k) sPsi[k * NN + i] = uu * uu * uu / 6.0;
            lhs = fma(uu, (double)re[i], lhs);
        }
    }
    if (bad) atomicOr(err, kErrDomain);
    __syncthreads();

    // ---- line pass: the identity's right-hand side and the scale
    for (int L = tid; L < D * NLINE; L += kEntThreads) {
        const int m = L / NLINE, l = L - m * NLINE;
        int base;
        double omega;
        if constexpr (D == 3) {
            const int o0 = l % N, o1 = l / N;
            base = m == 0 ? N * l : (m == 1 ? o0 + N * N * o1 : l);
            omega = tab.w[o0] * tab.w[o1];
        } else {
            base = m == 0 ? N * l : l;
            omega = tab.w[l];
        }
        const int stride = m == 0 ? 1 : (m == 1 ? N : N * N);
        const auto Jm = Je + m * D * NN;   // Ja^m_k(i) = Jm[k * NN + i]
        double t1 = 0.0;
        // the psi terms: -1/2 sum_a (E 1)_a psi_a.J_a - 1/2 sum_ab E_ab psi_a.J_b + sum_ab Q_ab psi_a.J_b
        double tpsi = 0.0;
#pragma unroll 1
        for (int a = 0; a < N; ++a) {
            const int ia = base + a * stride;
            double e1 = 0.0;
#pragma unroll 1
            for (int b = 0; b < N; ++b) {
                const int ib = base + b * stride;
                const double qab = omega * tab.Q1[a * N + b], qba = omega * tab.Q1[b * N + a];
                const double eab = qab + qba;
                e1 += eab;
                double pj = 0.0;
#pragma unroll
                for (int k = 0; k < D; ++k) pj = fma(sPsi[k * NN + ia], Jm[k * NN + ib], pj);
                tpsi += (qab - 0.5 * eab) * pj;
            }
            double pja = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) pja = fma(sPsi[k * NN + ia], Jm[k * NN + ia], pja);
            tpsi -= 0.5 * e1 * pja;
        }
        // the flux terms, each unordered pair once, and the diagonal
#pragma unroll 1
        for (int a = 0; a < N; ++a) {
            const int ia = base + a * stride;
#pragma unroll 1
            for (int b = a; b < N; ++b) {
                const int ib = base + b * stride;
                const double qab = omega * tab.Q1[a * N + b], qba = omega * tab.Q1[b * N + a];
                if (b == a && qab == 0.0) continue;
                double F[NVAR];
                if constexpr (is_euler(FLUX)) {
                    auto node = [&](int i) {
                        EulerNodeD<D> nd;
                        nd.rho = sS[i];
#pragma unroll
                        for (int k = 0; k < D; ++k) nd.hv[k] = sS[(1 + k) * NN + i];
                        nd.p = sS[(D + 1) * NN + i];
                        nd.beta = sS[(D + 2) * NN + i];
#pragma unroll
                        for (int k = 0; k < D; ++k) nd.J[k] = Jm[k * NN + i];
                        const long long bits = __double_as_longlong(sS[(D + 3) * NN + i]);
                        nd.rf = __int_as_float((int)(bits & 0xffffffffll));
                        nd.bf = __int_as_float((int)(bits >> 32));
                        return nd;
                    };
                    const EulerNodeD<D> A = node(ia);
                    if (b == a) {
                        euler_diag_flux_f64<D>(A, F);
                    } else {
                        const EulerNodeD<D> B = node(ib);
                        euler_pair_flux_f64<D, FLUX>(A, B, F);
                    }
                } else {
                    double Sj = 0.0;
#pragma unroll
                    for (int k = 0; k < D; ++k) Sj += Jm[k * NN + ia] + Jm[k * NN + ib];
                    const double ua = sS[ia], ub = sS[ib];
                    F[0] = (ua * ua + ua * ub + ub * ub) * (1.0 / 6.0) * Sj;
                }
                double wfa = 0.0, wfb = 0.0, afa = 0.0, afb = 0.0;
#pragma unroll
                for (int q = 0; q < NVAR; ++q) {
                    const double xa = sW[q * NN + ia] * F[q], xb = sW[q * NN + ib] * F[q];
                    wfa += xa;
                    wfb += xb;
                    afa += fabs(xa);
                    afb += fabs(xb);
                }
                if (b == a) {
                    t1 += 2.0 * qab * wfa;
                    scale += fabs(qab) * afa;
                } else {
                    t1 += (qab + qba) * (wfa + wfb);
                    scale += fabs(qab) * afa + fabs(qba) * afb;
                }
            }
        }
        rhs += 0.5 * t1 + tpsi;
    }

    // ---- fixed-order reduction over the CTA
    red[0][tid] = lhs;
    red[1][tid] = rhs;
    red[2][tid] = scale;
    __syncthreads();
    for (int h = kEntThreads / 2; h > 0; h >>= 1) {
        if (tid < h) {
#pragma unroll
            for (int q = 0; q < 3; ++q) red[q][tid] += red[q][tid + h];
        }
        __syncthreads();
    }
    if (tid == 0) SFH_BP(out, n_elem, err)[e] = fabs(red[0][0] - red[1][0]) / red[2][0];
}

template <int D, int N, int FLUX, typename TR>
static cudaError_t launch_entropy(const double *u, const double *Ja, const void *r, double *out, int64_t n_elem,
                                  const OpTab<double> &tab, int *err, cudaStream_t stream) {
    using S = EntShape<D, N, FLUX>;
    auto kern = entropy_identity_kernel<D, N, FLUX, TR>;
    static_assert(S::SMEM <= 200 * 1024, "shared memory");
    if (S::SMEM > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        if (e != cudaSuccess) return e;
    }
    kern<<<(unsigned)n_elem, kEntThreads, S::SMEM, stream>>>(u, Ja, static_cast<const TR *>(r), out, n_elem, tab, err);
    return cudaGetLastError();
}

template <int D, int FLUX, typename TR>
static cudaError_t dispatch_n(int n, const double *u, const double *Ja, const void *r, double *out, int64_t n_elem,
                              const OpTab<double> &tab, int *err, cudaStream_t stream) {
    switch (n) {
#define SFH_ECASE(N) \
    case N: return launch_entropy<D, N, FLUX, TR>(u, Ja, r, out, n_elem, tab, err, stream);
        SFH_ECASE(2) SFH_ECASE(3) SFH_ECASE(4) SFH_ECASE(5) SFH_ECASE(6) SFH_ECASE(7) SFH_ECASE(8) SFH_ECASE(9)
#undef SFH_ECASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t entropy_identity(int d, int n, int flux, const double *u, const double *Ja, const void *r, bool r_fp32,
                             double *out, int64_t n_elem, const OpTab<double> &tab, int *err, cudaStream_t stream) {
    if (d == 3) {
        if (flux == kFluxEuler)
            return r_fp32 ? dispatch_n<3, kFluxEuler, float>(n, u, Ja, r, out, n_elem, tab, err, stream)
                          : dispatch_n<3, kFluxEuler, double>(n, u, Ja, r, out, n_elem, tab, err, stream);
        if (flux == kFluxEulerCh)
            return r_fp32 ? dispatch_n<3, kFluxEulerCh, float>(n, u, Ja, r, out, n_elem, tab, err, stream)
                          : dispatch_n<3, kFluxEulerCh, double>(n, u, Ja, r, out, n_elem, tab, err, stream);
        return r_fp32 ? dispatch_n<3, kFluxBurgers, float>(n, u, Ja, r, out, n_elem, tab, err, stream)
                      : dispatch_n<3, kFluxBurgers, double>(n, u, Ja, r, out, n_elem, tab, err, stream);
    }
    if (flux == kFluxEuler)
        return r_fp32 ? dispatch_n<2, kFluxEuler, float>(n, u, Ja, r, out, n_elem, tab, err, stream)
                      : dispatch_n<2, kFluxEuler, double>(n, u, Ja, r, out, n_elem, tab, err, stream);
    if (flux == kFluxEulerCh)
        return r_fp32 ? dispatch_n<2, kFluxEulerCh, float>(n, u, Ja, r, out, n_elem, tab, err, stream)
                      : dispatch_n<2, kFluxEulerCh, double>(n, u, Ja, r, out, n_elem, tab, err, stream);
    return r_fp32 ? dispatch_n<2, kFluxBurgers, float>(n, u, Ja, r, out, n_elem, tab, err, stream)
                  : dispatch_n<2, kFluxBurgers, double>(n, u, Ja, r, out, n_elem, tab, err, stream);
}

}  // namespace sfh
