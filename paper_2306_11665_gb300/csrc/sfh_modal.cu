// sfh_modal.cu -- the basis transforms of the modal / uncollocated residual
// as kernels of their own (3D, FP32 state).
//
// The modal residual of Section 2 (the theorem on uncollocated bases) is
// r_hat = V^T r_v(V u_hat): the nodal residual of the nodal values V u_hat,
// tested against the basis.  With V = V1 (x) V1 (x) V1 both transforms are
// sum-factorized, three one-dimensional passes each.  For 3D Euler at
// n = 3..8 the FP32 modes' nodal residual runs on the warp-specialized kernel
// (or the row kernel), which holds no room for the transforms, so their modal
// residual is
//   modal_xform_kernel<forward>  u_hat -> u_v   (scratch)
//   nodal residual                u_v   -> r_v   (scratch)
//   modal_xform_kernel<backward>  r_v   -> r_hat
// with each pass's arithmetic that of the fused kernels (basis_pass_f: the
// same FMA order, the constant part of an orthonormal Legendre basis taken
// out of the forward sums and added back at the end).  Blocks are small
// (two 24 KB buffers) so that several CTAs per SM overlap their loads,
// passes and stores.
#include "sfh_internal.h"
#include "sfh_volume_tma.cuh"

namespace sfh {

template <int N>
struct XformShape {
    static constexpr int D = 3, NVAR = 5;
    static constexpr int NN = N * N * N, EL = NVAR * NN;       // floats per element
    static constexpr int THREADS = 256;
    static constexpr int BUDGET = 24 * 1024;                   // two buffers of EPB elements (several CTAs per SM)
    static constexpr int EPB = BUDGET / (2 * 4 * EL) > 0 ? BUDGET / (2 * 4 * EL) : 1;
    static constexpr size_t SMEM = (size_t)2 * 4 * EPB * EL;
};

// The block's ne elements of `in` into shared memory A.  A full block issues
// every load before its first store (a compile-time trip count, the values
// held in registers in between), as 16-byte loads when the array starts on a
// 16-byte boundary (the block then does too: its offset is a multiple of
// TOT floats, TOT a multiple of 4); the last, partial block and unaligned
// arrays take a plain loop.
template <class S>
__device__ __forceinline__ void xform_load(unsigned char *sm, BPtr<float> A, const float *in, int64_t n_elem,
                                           int64_t e0, int ne, int tid, int *err) {
    constexpr int TOT = S::EPB * S::EL;
    const auto gin = SFH_BP(in, n_elem * S::EL, err) + e0 * S::EL;
    if (ne == S::EPB) {
        if constexpr (TOT % 4 == 0) {
            if ((reinterpret_cast<uintptr_t>(in) & 15) == 0) {
                constexpr int TOT4 = TOT / 4, IT = (TOT4 + S::THREADS - 1) / S::THREADS;
                const auto g4 = SFH_BP(reinterpret_cast<const float4 *>(in), n_elem * S::EL / 4, err) + e0 * S::EL / 4;
                const auto A4 = SFH_BP(reinterpret_cast<float4 *>(sm), TOT4, err);
                float4 v[IT];
#pragma unroll
                for (int k = 0; k < IT; ++k) {
                    const int s = tid + k * S::THREADS;
                    if (s < TOT4) v[k] = g4[s];
                }
#pragma unroll
                for (int k = 0; k < IT; ++k) {
                    const int s = tid + k * S::THREADS;
                    if (s < TOT4) A4[s] = v[k];
                }
                return;
            }
        }
        constexpr int IT = (TOT + S::THREADS - 1) / S::THREADS;
        float v[IT];
#pragma unroll
        for (int k = 0; k < IT; ++k) {
            const int s = tid + k * S::THREADS;
            if (s < TOT) v[k] = gin[s];
        }
#pragma unroll
        for (int k = 0; k < IT; ++k) {
            const int s = tid + k * S::THREADS;
            if (s < TOT) A[s] = v[k];
        }
        return;
    }
    for (int s = tid; s < ne * S::EL; s += S::THREADS) A[s] = gin[s];
}

// One CTA per EPB elements: the block's values are loaded with coalesced
// reads, transformed pass by pass in shared memory, and the last pass writes
// the output.  BACKWARD: r_v -> V^T r_v; else u_hat -> V u_hat.
template <int N, bool BACKWARD>
__global__ void __launch_bounds__(XformShape<N>::THREADS)
modal_xform_kernel(const float *__restrict__ in, float *__restrict__ out, int64_t n_elem,
                   const __grid_constant__ BasisTab<float> bt, int *__restrict__ err) {
    using S = XformShape<N>;
    extern __shared__ __align__(128) unsigned char sm[];
    const auto A = SFH_BP(reinterpret_cast<float *>(sm), S::EPB * S::EL, err);
    const auto B = SFH_BP(reinterpret_cast<float *>(sm) + S::EPB * S::EL, S::EPB * S::EL, err);
    const int64_t e0 = (int64_t)blockIdx.x * S::EPB;
    const int ne = (int)((n_elem - e0) < S::EPB ? (n_elem - e0) : S::EPB);
    const auto gin = SFH_BP(in, n_elem * S::EL, err) + e0 * S::EL;
    const auto gout = SFH_BP(out, n_elem * S::EL, err) + e0 * S::EL;
    const int tid = threadIdx.x, nq = ne * S::NVAR;
    xform_load<S>(sm, A, in, n_elem, e0, ne, tid, err);
    __syncthreads();
    if constexpr (BACKWARD) {
        basis_pass_f<3, N, true>(A, B, 0, nq, bt, tid, S::THREADS);
        __syncthreads();
        basis_pass_f<3, N, true>(B, A, 1, nq, bt, tid, S::THREADS);
        __syncthreads();
        basis_pass_f<3, N, true>(A, gout, 2, nq, bt, tid, S::THREADS);
    } else {
        basis_pass_f<3, N, false, kPassFirst>(A, B, 0, nq, bt, tid, S::THREADS);
        __syncthreads();
        basis_pass_f<3, N, false>(B, A, 1, nq, bt, tid, S::THREADS);
        __syncthreads();
        // the last pass reads its input from A, which now holds pass 1's
        // output; the constant coefficients come from the global input
        basis_pass_f<3, N, false, kPassLast>(A, gout, 2, nq, bt, tid, S::THREADS, gin);
    }
}

template <int N, bool BACKWARD>
static cudaError_t launch_xform(const float *in, float *out, int64_t n_elem, const BasisTab<float> &bt, int *err,
                                cudaStream_t stream) {
    using S = XformShape<N>;
    auto kern = modal_xform_kernel<N, BACKWARD>;
    static_assert(S::SMEM <= 227 * 1024, "shared memory");
    if (S::SMEM > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        if (e != cudaSuccess) return e;
    }
    const int64_t blocks = (n_elem + S::EPB - 1) / S::EPB;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    kern<<<(unsigned)blocks, S::THREADS, S::SMEM, stream>>>(in, out, n_elem, bt, err);
    return cudaGetLastError();
}

cudaError_t modal_xform_3d(int n, bool backward, const float *in, float *out, int64_t n_elem,
                           const BasisTab<float> &bt, int *err, cudaStream_t stream) {
#define SFH_XCASE(N)                                                                                   \
    case N:                                                                                            \
        return backward ? launch_xform<N, true>(in, out, n_elem, bt, err, stream)                      \
                        : launch_xform<N, false>(in, out, n_elem, bt, err, stream);
    switch (n) {
        SFH_XCASE(3) SFH_XCASE(4) SFH_XCASE(5) SFH_XCASE(6) SFH_XCASE(7) SFH_XCASE(8)
        default: return cudaErrorInvalidValue;
    }
#undef SFH_XCASE
}

}  // namespace sfh
