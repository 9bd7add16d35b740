// sfh_surface.cu -- the surface Hadamard product of each element's faces
// (Remark 1: the theorem's operator with alpha = 0 on the facet cubature;
// "one-dimensional basis matrices of size m x n"), FP64.
//
// Face (m, side) has the facet cubature of the other directions' nodes
// (n^{d-1} points f, lower axis fastest, weight w_f = prod w[b_k]); the
// interpolation to it is E = e (x) I (x) I with e[b] = l_b(-1 or +1) in
// position m, so face node f couples only to the n volume nodes j on its
// normal line (one of them for Gauss-Lobatto nodes, where e is a selector).
// With H[f][j] = w_f E[f][j] fsharp(u~_f, u_j) . nJ_f:
//   r_vol[j]  = sum over faces, sum_f H[f][j],   r_face[f] = sum_j H[f][j].
// One thread per (element, face node) of one face at a time; the faces of an
// element block are taken in turn (each volume node meets one face node per
// face, so the volume sums need no atomics), the volume state's primitives
// and the volume sums in shared memory.
#include <cuda_runtime.h>

#include "../../include/sfhad.h"
#include "sfh_internal.h"
#include "sfh_volume.cuh"

namespace sfh {

template <int D, int N, int FLUX>
struct SurfShape {
    static constexpr int NN = ipow(N, D), NF = ipow(N, D - 1);
    static constexpr int NVAR = is_euler(FLUX) ? D + 2 : 1;
    // per volume node: rho, v/2 [D], p, beta, FP32 copies of rho and beta in
    // one word | u
    static constexpr int NS = is_euler(FLUX) ? D + 4 : 1;
    static constexpr int NODE_BYTES = 8 * (NS + NVAR);
    static constexpr int EPB_THREADS = 256 / NF > 0 ? 256 / NF : 1;
    static constexpr int EPB_SMEM = (96 * 1024) / (NN * NODE_BYTES) > 0 ? (96 * 1024) / (NN * NODE_BYTES) : 1;
    static constexpr int EPB = EPB_THREADS < EPB_SMEM ? EPB_THREADS : EPB_SMEM;
    static constexpr int THREADS = ((EPB * NF + 31) / 32) * 32;
    static constexpr size_t SMEM = (size_t)EPB * NN * NODE_BYTES;
};

template <int D>
__device__ __forceinline__ EulerNodeD<D> euler_node_from_u(BPtr<const double> u, int stride, bool &bad) {
    EulerNodeD<D> nd;
    const double rho = u[0], E = u[(D + 1) * stride], irho = rcp_nr(rho);
    double ke = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const double mk = u[(1 + k) * stride], vk = mk * irho;
        nd.hv[k] = 0.5 * vk;
        ke = fma(mk, vk, ke);
    }
    const double p = (kGamma - 1.0) * fma(-0.5, ke, E), ip = rcp_nr(p);
    double bt = rho * ip;
    bt = fma(ip, fma(-p, bt, rho), bt);
    nd.rho = rho;
    nd.p = p;
    nd.beta = bt;
    nd.rf = d2f_int(rho);
    nd.bf = d2f_int(bt);
    bad |= !(rho > 0.0 && p > 0.0);
    return nd;
}

template <int D, int N, int FLUX>
__global__ void __launch_bounds__(SurfShape<D, N, FLUX>::THREADS)
surface_kernel(const double *__restrict__ u, const double *__restrict__ u_face, const double *__restrict__ nJ,
               double *__restrict__ r_vol, double *__restrict__ r_face, int64_t n_elem,
               const __grid_constant__ SurfTab tab, int *__restrict__ err) {
    using S = SurfShape<D, N, FLUX>;
    constexpr int NN = S::NN, NF = S::NF, NVAR = S::NVAR, NS = S::NS, EPB = S::EPB;
    extern __shared__ __align__(16) double sm[];
    const auto sS = SFH_BP(sm, EPB * NS * NN, err);                    // [EPB][NS][NN]
    const auto sR = SFH_BP(sm + EPB * NS * NN, EPB * NVAR * NN, err);  // [EPB][NVAR][NN]
    // the inputs and outputs over their whole extents
    const auto gu = SFH_BP(u, n_elem * NVAR * NN, err);
    const auto guf = SFH_BP(u_face, n_elem * 2 * D * NVAR * NF, err);
    const auto gnJ = SFH_BP(nJ, n_elem * 2 * D * D * NF, err);
    const auto grv = SFH_BP(r_vol, n_elem * NVAR * NN, err);
    const auto grf = SFH_BP(r_face, n_elem * 2 * D * NVAR * NF, err);
    const int64_t e0 = (int64_t)blockIdx.x * EPB;
    const int ne = (int)((n_elem - e0) < EPB ? (n_elem - e0) : EPB);
    const int tid = threadIdx.x;
    bool bad = false;

    // ---- volume primitives, zero the volume sums
    for (int s = tid; s < ne * NN; s += blockDim.x) {
        const int el = s / NN, i = s - el * NN;
        const auto ue = gu + (e0 + el) * NVAR * NN + i;
        const auto se = sS + el * NS * NN + i;
        if constexpr (is_euler(FLUX)) {
            const EulerNodeD<D> nd = euler_node_from_u<D>(ue, NN, bad);
            se[0] = nd.rho;
#pragma unroll
            for (int k = 0; k < D; ++k) se[(1 + k) * NN] = nd.hv[k];
            se[(D + 1) * NN] = nd.p;
            se[(D + 2) * NN] = nd.beta;
            const float2 rb = make_float2(nd.rf, nd.bf);
            se[(D + 3) * NN] = __longlong_as_double(*reinterpret_cast<const long long *>(&rb));
        } else {
            se[0] = ue[0];
        }
#pragma unroll
        for (int v = 0; v < NVAR; ++v) sR[(el * NVAR + v) * NN + i] = 0.0;
    }
    __syncthreads();

    // ---- the faces in turn
#pragma unroll 1
    for (int face = 0; face < 2 * D; ++face) {
        const int m = face >> 1, side = face & 1;
        const int stride = m == 0 ? 1 : (m == 1 ? N : N * N);
        if (tid < ne * NF) {
            const int el = tid / NF, f = tid - el * NF;
            // the face node's indices in the other directions, lower first
            const int b0 = f % N, b1 = f / N;
            int base;   // volume node of the line at a_m = 0
            double wf;
            if constexpr (D == 3) {
                base = m == 0 ? N * b0 + N * N * b1 : (m == 1 ? b0 + N * N * b1 : b0 + N * b1);
                wf = tab.w[b0] * tab.w[b1];
            } else {
                base = m == 0 ? N * b0 : b0;
                wf = tab.w[b0];
            }
            const int64_t fo = ((e0 + el) * 2 * D + face);
            const auto uf = guf + fo * NVAR * NF + f;
            const auto nf = gnJ + fo * D * NF + f;
            double acc[NVAR];
#pragma unroll
            for (int v = 0; v < NVAR; ++v) acc[v] = 0.0;
            BPtr<const double> se = sS + el * NS * NN;
            const auto re = sR + el * NVAR * NN;
            if constexpr (is_euler(FLUX)) {
                EulerNodeD<D> A = euler_node_from_u<D>(uf, NF, bad);
#pragma unroll
                for (int k = 0; k < D; ++k) A.J[k] = nf[k * NF];
#pragma unroll
                for (int b = 0; b < N; ++b) {
                    const double eb = tab.e[side][b];
                    if (eb == 0.0) continue;
                    const int j = base + b * stride;
                    EulerNodeD<D> B;
                    B.rho = se[j];
#pragma unroll
                    for (int k = 0; k < D; ++k) { B.hv[k] = se[(1 + k) * NN + j]; B.J[k] = 0.0; }
                    B.p = se[(D + 1) * NN + j];
                    B.beta = se[(D + 2) * NN + j];
                    const long long bits = __double_as_longlong(se[(D + 3) * NN + j]);
                    B.rf = __int_as_float((int)(bits & 0xffffffffll));
                    B.bf = __int_as_float((int)(bits >> 32));
                    double F[D + 2];
                    euler_pair_flux_f64<D, FLUX>(A, B, F);   // n = nJ_f + 0
                    const double q = wf * eb;
#pragma unroll
                    for (int v = 0; v < NVAR; ++v) {
                        const double h = q * F[v];
                        acc[v] += h;
                        re[v * NN + j] += h;
                    }
                }
            } else {
                const double a = uf[0];
                double sn = nf[0];
#pragma unroll
                for (int k = 1; k < D; ++k) sn += nf[k * NF];
#pragma unroll
                for (int b = 0; b < N; ++b) {
                    const double eb = tab.e[side][b];
                    if (eb == 0.0) continue;
                    const int j = base + b * stride;
                    const double c = se[j];
                    const double h = wf * eb * ((a * a + a * c + c * c) * (1.0 / 6.0) * sn);
                    acc[0] += h;
                    re[j] += h;
                }
            }
            const auto rf = grf + fo * NVAR * NF + f;
#pragma unroll
            for (int v = 0; v < NVAR; ++v) rf[v * NF] = acc[v];
        }
        __syncthreads();
    }
    if (bad) atomicOr(err, kErrDomain);

    // ---- write the volume sums
    const auto rb = grv + e0 * NVAR * NN;
    for (int s = tid; s < ne * NVAR * NN; s += blockDim.x) rb[s] = sR[s];
}

template <int D, int N, int FLUX>
static cudaError_t launch_surface(const double *u, const double *u_face, const double *nJ, double *r_vol,
                                  double *r_face, int64_t n_elem, const SurfTab &tab, int *err, cudaStream_t stream) {
    using S = SurfShape<D, N, FLUX>;
    auto kern = surface_kernel<D, N, FLUX>;
    static_assert(S::SMEM <= 227 * 1024, "shared memory");
    if (S::SMEM > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        if (e != cudaSuccess) return e;
    }
    const int64_t blocks = (n_elem + S::EPB - 1) / S::EPB;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    kern<<<(unsigned)blocks, S::THREADS, S::SMEM, stream>>>(u, u_face, nJ, r_vol, r_face, n_elem, tab, err);
    return cudaGetLastError();
}

template <int D, int FLUX>
static cudaError_t dispatch_surface(int n, const double *u, const double *u_face, const double *nJ, double *r_vol,
                                    double *r_face, int64_t n_elem, const SurfTab &tab, int *err,
                                    cudaStream_t stream) {
    switch (n) {
#define SFH_SCASE(N) \
    case N: return launch_surface<D, N, FLUX>(u, u_face, nJ, r_vol, r_face, n_elem, tab, err, stream);
        SFH_SCASE(2) SFH_SCASE(3) SFH_SCASE(4) SFH_SCASE(5) SFH_SCASE(6) SFH_SCASE(7) SFH_SCASE(8) SFH_SCASE(9)
#undef SFH_SCASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t surface_hadamard(int d, int n, int flux, const double *u, const double *u_face, const double *nJ,
                             double *r_vol, double *r_face, int64_t n_elem, const SurfTab &tab, int *err,
                             cudaStream_t stream) {
    if (d == 3) {
        if (flux == kFluxEuler) return dispatch_surface<3, kFluxEuler>(n, u, u_face, nJ, r_vol, r_face, n_elem, tab, err, stream);
        if (flux == kFluxEulerCh) return dispatch_surface<3, kFluxEulerCh>(n, u, u_face, nJ, r_vol, r_face, n_elem, tab, err, stream);
        return dispatch_surface<3, kFluxBurgers>(n, u, u_face, nJ, r_vol, r_face, n_elem, tab, err, stream);
    }
    if (flux == kFluxEuler) return dispatch_surface<2, kFluxEuler>(n, u, u_face, nJ, r_vol, r_face, n_elem, tab, err, stream);
    if (flux == kFluxEulerCh) return dispatch_surface<2, kFluxEulerCh>(n, u, u_face, nJ, r_vol, r_face, n_elem, tab, err, stream);
    return dispatch_surface<2, kFluxBurgers>(n, u, u_face, nJ, r_vol, r_face, n_elem, tab, err, stream);
}

}  // namespace sfh
