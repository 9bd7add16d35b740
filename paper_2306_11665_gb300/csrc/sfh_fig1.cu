// sfh_fig1.cu -- the generic Hadamard product of the paper's timing
// experiment (Section 3, Fig. 1) on the GPU:
//   y = sum_{m=1..3} (D_m o C) 1,   C = c c^T,
// D_m the derivative of the collocated Lagrange basis along direction m on
// Gauss-Lobatto nodes (D (x) I (x) I with the factor's position naming the
// direction, Eq. 5 without the weights), for one tensor-product element of
// n^3 nodes (x fastest), many elements at once.
//   * sum-factorized: y_i = c_i sum_m sum_b D[a_m(i)][b] c_{j_m(i, b)}, the
//     O(n^{d+1}) evaluation of Section 2;
//   * dense: y_i = c_i sum_j sum_m D_m[i][j] c_j over all n^3 columns j, the
//     entries of D_m formed from the multi-indices of i and j (zero off the
//     line), the O(n^{2d}) evaluation the paper compares against.
// One thread per (element, node); FP64.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/sfhad.h"
#include "sfh_internal.h"

namespace sfh {

constexpr int kFig1MaxN = 16;   // p <= 15

struct Fig1Tab {
    double D[kFig1MaxN * kFig1MaxN];
};

template <int N>
__global__ void __launch_bounds__(256) fig1_sf_kernel(const double *__restrict__ c, double *__restrict__ y,
                                                      int64_t n_elem, const __grid_constant__ Fig1Tab tab) {
    constexpr int NN = N * N * N;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_elem * NN) return;
    const int64_t e = t / NN;
    const int i = (int)(t - e * NN);
    const int a0 = i % N, a1 = (i / N) % N, a2 = i / (N * N);
    const double *ce = c + e * NN;
    double s = 0.0;
#pragma unroll 4
    for (int b = 0; b < N; ++b) {
        s = fma(tab.D[a0 * N + b], ce[b + N * a1 + N * N * a2], s);
        s = fma(tab.D[a1 * N + b], ce[a0 + N * b + N * N * a2], s);
        s = fma(tab.D[a2 * N + b], ce[a0 + N * a1 + N * N * b], s);
    }
    y[t] = ce[i] * s;
}

template <int N>
__global__ void __launch_bounds__(256) fig1_dense_kernel(const double *__restrict__ c, double *__restrict__ y,
                                                         int64_t n_elem, const __grid_constant__ Fig1Tab tab) {
    constexpr int NN = N * N * N;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_elem * NN) return;
    const int64_t e = t / NN;
    const int i = (int)(t - e * NN);
    const int a0 = i % N, a1 = (i / N) % N, a2 = i / (N * N);
    const double *ce = c + e * NN;
    double s = 0.0;
#pragma unroll 1
    for (int j = 0; j < NN; ++j) {
        const int b0 = j % N, b1 = (j / N) % N, b2 = j / (N * N);
        // D_m[i][j]: D[a_m][b_m] where the other two indices agree, else 0
        const double q0 = (a1 == b1 && a2 == b2) ? tab.D[a0 * N + b0] : 0.0;
        const double q1 = (a0 == b0 && a2 == b2) ? tab.D[a1 * N + b1] : 0.0;
        const double q2 = (a0 == b0 && a1 == b1) ? tab.D[a2 * N + b2] : 0.0;
        s = fma((q0 + q1) + q2, ce[j], s);
    }
    y[t] = ce[i] * s;
}

template <int N>
static cudaError_t launch_fig1(bool dense, const double *c, double *y, int64_t n_elem, const Fig1Tab &tab,
                               cudaStream_t stream) {
    const int64_t threads = n_elem * N * N * N;
    const int64_t blocks = (threads + 255) / 256;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (dense) fig1_dense_kernel<N><<<(unsigned)blocks, 256, 0, stream>>>(c, y, n_elem, tab);
    else fig1_sf_kernel<N><<<(unsigned)blocks, 256, 0, stream>>>(c, y, n_elem, tab);
    return cudaGetLastError();
}

cudaError_t fig1_hadamard(int n, bool dense, const double *c, double *y, int64_t n_elem, const double *D,
                          cudaStream_t stream) {
    Fig1Tab tab;
    for (int k = 0; k < kFig1MaxN * kFig1MaxN; ++k) tab.D[k] = k < n * n ? D[k] : 0.0;
    switch (n) {
#define SFH_FCASE(N) \
    case N: return launch_fig1<N>(dense, c, y, n_elem, tab, stream);
        SFH_FCASE(2) SFH_FCASE(3) SFH_FCASE(4) SFH_FCASE(5) SFH_FCASE(6) SFH_FCASE(7) SFH_FCASE(8) SFH_FCASE(9)
        SFH_FCASE(10) SFH_FCASE(11) SFH_FCASE(12) SFH_FCASE(13) SFH_FCASE(14) SFH_FCASE(15) SFH_FCASE(16)
#undef SFH_FCASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sfh
