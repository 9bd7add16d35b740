// sfh_vjp.cuh -- adjoint of the volume residual (FP64).
//
// From r_i = sum_m sum_j Q_m,ij F_m(u_i, u_j) (Eq. 3) with F_m symmetric in
// its two states, the cotangent lambda pulls back to
//   g_l = sum_m sum_{j on the m-line of l} c_lj^T d1F_m(u_l, u_j),
//   c_lj = Q_m,lj lambda_l + Q_m,jl lambda_j   (= c_jl),
// so each unordered line pair (a, b) needs the gradient of the single scalar
// phi = c_ab^T F(u_a, u_b) with respect to both states.  The kernel evaluates
// it in reverse mode through the flux formula, accumulates the adjoints of
// the node primitives (rho, v, p, beta) in shared memory over all pairs and
// directions, and applies the primitive -> conservative chain rule once per
// node at the end.  Q_m,ab = omega Q1[a][b] with omega constant on the line,
// so lambda is pre-scaled by omega.
#pragma once

#include "sfh_device.cuh"

namespace sfh {

// LINES: target line tasks per tile (128 for the standalone kernel; the
// serving kernel asks for tiles that fill its 256 threads); BUDGET: shared
// memory of one tile.
template <int D, int N, int FLUX, int BUDGET = 96 * 1024, int LINES = 128>
struct VjpShape {
    static constexpr int NN = ipow(N, D);
    static constexpr int NLINE = ipow(N, D - 1);
    static constexpr int NVAR = is_euler(FLUX) ? D + 2 : 1;
    static constexpr int NP = is_euler(FLUX) ? D + 3 : 1;
    static constexpr int NODE_BYTES = 8 * (2 * NP + NVAR + D);
    static constexpr int EPB_SMEM = BUDGET / (NN * NODE_BYTES) > 0 ? BUDGET / (NN * NODE_BYTES) : 1;
    static constexpr int EPB_LINES = LINES / NLINE > 0 ? LINES / NLINE : 1;
    static constexpr int EPB = EPB_SMEM < EPB_LINES ? EPB_SMEM : EPB_LINES;
    static constexpr int THREADS = ((EPB * NLINE + 31) / 32) * 32;
    static constexpr size_t SMEM = (size_t)EPB * NN * NODE_BYTES;
};

// Reverse mode of the contracted Euler flux (Ranocha's, or Chandrashekar's
// with pressure average pt = (rho_a + rho_b) / (beta_a + beta_b)): adds
// d(c^T F)/d(prim) of both states.  prim order: rho, v[0..D-1], p, beta.
template <int D, int FLUX>
__device__ __forceinline__ void euler_pair_vjp(const double *PA, const double *PB, const double *n,
                                               const double *c, double *ga, double *gb) {
    const double ra = PA[0], rb = PB[0], pa = PA[D + 1], pb = PB[D + 1];
    double vna = PA[1] * n[0], vnb = PB[1] * n[0], vv = PA[1] * PB[1];
#pragma unroll
    for (int k = 1; k < D; ++k) {
        vna = fma(PA[1 + k], n[k], vna);
        vnb = fma(PB[1 + k], n[k], vnb);
        vv = fma(PA[1 + k], PB[1 + k], vv);
    }
    // {rho}_ln and M = 1/{beta}_ln with their partial derivatives (band tests
    // on FP32 copies made by integer conversion)
    double Lr, Lra, Lrb, M, Ma, Mb;
    ln_mean_grad_f64(ra, rb, d2f_int(ra), d2f_int(rb), Lr, Lra, Lrb);
    inv_ln_mean_grad_f64(PA[D + 2], PB[D + 2], d2f_int(PA[D + 2]), d2f_int(PB[D + 2]), M, Ma, Mb);
    const double h = 0.5 * (vna + vnb);
    const double frho = Lr * h;
    const double K = fma(0.5, vv, M * (1.0 / (kGamma - 1.0)));
    const double cE = c[D + 1];
    double frho_bar = fma(cE, K, c[0]), pavg_bar = 0.0;
#pragma unroll
    for (int l = 0; l < D; ++l) {
        const double vavg = 0.5 * (PA[1 + l] + PB[1 + l]);
        frho_bar = fma(c[1 + l], vavg, frho_bar);
        pavg_bar = fma(c[1 + l], n[l], pavg_bar);
        const double hvavg_bar = 0.5 * c[1 + l] * frho;
        ga[1 + l] += hvavg_bar;
        gb[1 + l] += hvavg_bar;
    }
    const double hK_bar = 0.5 * cE * frho;
    const double Lr_bar = frho_bar * h, h_bar = frho_bar * Lr;
    double vna_bar, vnb_bar;
    if constexpr (FLUX == kFluxEulerCh) {
        // F_m += pt n, F_E += pt h: pt's adjoint goes to rho and beta of both
        const double sr = ra + rb, sb = PA[D + 2] + PB[D + 2], isb = rcp_nr(sb);
        double pt = sr * isb;
        pt = fma(isb, fma(-sb, pt, sr), pt);
        const double pt_bar = fma(cE, h, pavg_bar);
        const double sr_bar = pt_bar * isb, sb_bar = -sr_bar * pt;
        ga[0] += sr_bar;
        gb[0] += sr_bar;
        ga[D + 2] += sb_bar;
        gb[D + 2] += sb_bar;
        vna_bar = vnb_bar = 0.5 * fma(cE, pt, h_bar);
    } else {
        // F_m += {p} n, F_E += (p_a v_b + p_b v_a).n / 2
        vna_bar = 0.5 * fma(cE, pb, h_bar);
        vnb_bar = 0.5 * fma(cE, pa, h_bar);
        ga[D + 1] += 0.5 * fma(cE, vnb, pavg_bar);
        gb[D + 1] += 0.5 * fma(cE, vna, pavg_bar);
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
        ga[1 + k] += fma(hK_bar, PB[1 + k], vna_bar * n[k]);
        gb[1 + k] += fma(hK_bar, PA[1 + k], vnb_bar * n[k]);
    }
    ga[0] = fma(Lr_bar, Lra, ga[0]);
    gb[0] = fma(Lr_bar, Lrb, gb[0]);
    const double M_bar = cE * frho * (1.0 / (kGamma - 1.0));
    ga[D + 2] = fma(M_bar, Ma, ga[D + 2]);
    gb[D + 2] = fma(M_bar, Mb, gb[D + 2]);
}

// One tile of ne (<= EPB) elements from e0, processed by the whole CTA.
// MODAL: u and lambda hold basis coefficients (bt the basis on the cubature
// nodes) and g receives V^T J^T V lambda_hat, the VJP of the modal residual
// V^T r_v(V u_hat): the transforms run in shared memory (the primitive,
// adjoint and lambda buffers serve as scratch).
template <int D, int N, int FLUX, class S = VjpShape<D, N, FLUX>, bool MODAL = false>
__device__ __forceinline__ void vjp_tile(BPtr<const double> SFH_RESTRICT u, BPtr<const double> SFH_RESTRICT Ja,
                                         BPtr<const double> SFH_RESTRICT lam, BPtr<double> SFH_RESTRICT g, int64_t e0, int ne,
                                         const OpTab<double> &tab, int *__restrict__ err, unsigned char *smem_raw,
                                         const BasisTab<double> *bt = nullptr) {
    constexpr int NN = S::NN, NLINE = S::NLINE, NVAR = S::NVAR, NP = S::NP, EPB = S::EPB;
    double *const s0 = reinterpret_cast<double *>(smem_raw);
    const auto sP = SFH_BP(s0, EPB * NP * NN, err);                                    // [EPB][NP][NN]
    const auto sA = SFH_BP(s0 + EPB * NP * NN, EPB * NP * NN, err);                    // adjoints of primitives
    const auto sL = SFH_BP(s0 + 2 * EPB * NP * NN, EPB * NVAR * NN, err);              // [EPB][NVAR][NN] lambda
    const auto sJ = SFH_BP(s0 + 2 * EPB * NP * NN + EPB * NVAR * NN, EPB * D * NN, err);   // [EPB][D][NN]

    BPtr<const double> ub = u + e0 * NVAR * NN;
    const auto lb = lam + e0 * NVAR * NN;
    if constexpr (MODAL) {
        // lambda_v = V lambda_hat into sL, then u_v = V u_hat into sA ([el][var][i])
        const int nq = ne * NVAR, t = threadIdx.x, nt = blockDim.x;
        if constexpr (D == 3) {
            basis_pass<double, D, N, false, kPassFirst>(lb, sL, 0, nq, *bt, t, nt);
            __syncthreads();
            basis_pass<double, D, N, false>(sL, sP, 1, nq, *bt, t, nt);
            __syncthreads();
            basis_pass<double, D, N, false, kPassLast>(sP, sL, 2, nq, *bt, t, nt, lb);
            __syncthreads();
            basis_pass<double, D, N, false, kPassFirst>(ub, sA, 0, nq, *bt, t, nt);
            __syncthreads();
            basis_pass<double, D, N, false>(sA, sP, 1, nq, *bt, t, nt);
            __syncthreads();
            basis_pass<double, D, N, false, kPassLast>(sP, sA, 2, nq, *bt, t, nt, ub);
        } else {
            basis_pass<double, D, N, false, kPassFirst>(lb, sP, 0, nq, *bt, t, nt);
            __syncthreads();
            basis_pass<double, D, N, false, kPassLast>(sP, sL, 1, nq, *bt, t, nt, lb);
            __syncthreads();
            basis_pass<double, D, N, false, kPassFirst>(ub, sP, 0, nq, *bt, t, nt);
            __syncthreads();
            basis_pass<double, D, N, false, kPassLast>(sP, sA, 1, nq, *bt, t, nt, ub);
        }
        __syncthreads();
        ub = sA;
    }

    bool bad = false;
    for (int s = threadIdx.x; s < ne * NN; s += blockDim.x) {
        const int el = s / NN, i = s - el * NN;
        const auto ue = ub + (int64_t)el * NVAR * NN + i;
        const auto pe = sP + el * NP * NN + i;
        if constexpr (is_euler(FLUX)) {
            const double rho = ue[0], E = ue[(D + 1) * NN], irho = rcp_nr(rho);
            double ke = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const double mk = ue[(1 + k) * NN], vk = mk * irho;
                pe[(1 + k) * NN] = vk;
                ke = fma(mk, vk, ke);
            }
            const double p = (kGamma - 1.0) * fma(-0.5, ke, E);
            const double ip = rcp_nr(p);
            double bt = rho * ip;
            bt = fma(ip, fma(-p, bt, rho), bt);   // rho / p to within about half an ulp
            pe[0] = rho;
            pe[(D + 1) * NN] = p;
            pe[(D + 2) * NN] = bt;
            bad |= !(rho > 0.0 && p > 0.0);
        } else {
            pe[0] = ue[0];
        }
        if constexpr (!MODAL) {
#pragma unroll
            for (int q = 0; q < NP; ++q) sA[(el * NP + q) * NN + i] = 0.0;
#pragma unroll
            for (int v = 0; v < NVAR; ++v) sL[(el * NVAR + v) * NN + i] = lb[((int64_t)el * NVAR + v) * NN + i];
        }
    }
    if (bad) atomicOr(err, 1);
    if constexpr (MODAL) {
        // u_v sat in sA with the [el][var][i] layout: zero the adjoints only
        // once every node has read its state
        __syncthreads();
        for (int s2 = threadIdx.x; s2 < ne * NP * NN; s2 += blockDim.x) sA[s2] = 0.0;
    }

    const auto Jb = Ja + e0 * D * D * NN;
    uint32_t hmax = 0;   // largest |Ja| high word: Inf and NaN are refused
#pragma unroll 1
    for (int m = 0; m < D; ++m) {
        __syncthreads();
        for (int s = threadIdx.x; s < ne * D * NN; s += blockDim.x) {
            const int el = s / (D * NN), rem = s - el * D * NN;
            const double j = Jb[((int64_t)el * D * D + m * D) * NN + rem];
            hmax = max(hmax, abs_hi(j));
            sJ[s] = j;
        }
        if (m == D - 1 && hmax >= kMetricHiFp64) atomicOr(err, kErrMetric);
        __syncthreads();
        const int stride = m == 0 ? 1 : (m == 1 ? N : N * N);
        for (int L = threadIdx.x; L < ne * NLINE; L += blockDim.x) {
            const int el = L / NLINE, l = L - el * NLINE;
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
#pragma unroll 1
            for (int a = 0; a < N; ++a) {
                const int ia = base + a * stride;
                double PA[NP], JA[D], LA[NVAR], GA[NP];
#pragma unroll
                for (int q = 0; q < NP; ++q) { PA[q] = sP[(el * NP + q) * NN + ia]; GA[q] = 0.0; }
#pragma unroll
                for (int k = 0; k < D; ++k) JA[k] = sJ[(el * D + k) * NN + ia];
#pragma unroll
                for (int v = 0; v < NVAR; ++v) LA[v] = omega * sL[(el * NVAR + v) * NN + ia];
#pragma unroll 1
                for (int b = a; b < N; ++b) {
                    const int ib = base + b * stride;
                    const double qab = tab.Q1[a * N + b], qba = tab.Q1[b * N + a];
                    if (b == a && qab == 0.0) continue;
                    double PB[NP], n[D], c[NVAR], GB[NP];
#pragma unroll
                    for (int q = 0; q < NP; ++q) { PB[q] = sP[(el * NP + q) * NN + ib]; GB[q] = 0.0; }
#pragma unroll
                    for (int k = 0; k < D; ++k) n[k] = JA[k] + sJ[(el * D + k) * NN + ib];
                    if (b == a) {
#pragma unroll
                        for (int v = 0; v < NVAR; ++v) c[v] = qab * LA[v];
                    } else {
                        const double qbw = qba * omega;
#pragma unroll
                        for (int v = 0; v < NVAR; ++v) c[v] = fma(qbw, sL[(el * NVAR + v) * NN + ib], qab * LA[v]);
                    }
                    if constexpr (is_euler(FLUX)) {
                        euler_pair_vjp<D, FLUX>(PA, PB, n, c, GA, GB);
                    } else {
                        double S = 0.0;
#pragma unroll
                        for (int k = 0; k < D; ++k) S += n[k];
                        GA[0] += c[0] * (2.0 * PA[0] + PB[0]) * (1.0 / 6.0) * S;
                        GB[0] += c[0] * (PA[0] + 2.0 * PB[0]) * (1.0 / 6.0) * S;
                    }
                    // the diagonal pair depends on u_a through both arguments
#pragma unroll
                    for (int q = 0; q < NP; ++q) sA[(el * NP + q) * NN + ib] += GB[q];
                }
#pragma unroll
                for (int q = 0; q < NP; ++q) sA[(el * NP + q) * NN + ia] += GA[q];
            }
        }
    }
    __syncthreads();

    // ---- 3. primitive adjoints -> conservative adjoints; write g (modal:
    //      g_v into sL, then g_hat = V^T g_v)
    const auto gbp = g + e0 * NVAR * NN;
    const auto gdst = MODAL ? sL : gbp;
    for (int s = threadIdx.x; s < ne * NN; s += blockDim.x) {
        const int el = s / NN, i = s - el * NN;
        const auto pe = sP + el * NP * NN + i;
        const auto ae = sA + el * NP * NN + i;
        const auto ge = gdst + (int64_t)el * NVAR * NN + i;
        if constexpr (is_euler(FLUX)) {
            const double rho = pe[0], p = pe[(D + 1) * NN], beta = pe[(D + 2) * NN];
            const double irho = rcp_nr(rho), ip = rcp_nr(p);
            const double bbar = ae[(D + 2) * NN];
            const double rbar = fma(bbar, ip, ae[0]);            // d beta / d rho = 1/p
            const double pbar = fma(-bbar * beta, ip, ae[(D + 1) * NN]);   // d beta / d p = -beta/p
            double g0 = rbar, v2 = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const double vk = pe[(1 + k) * NN], vbar = ae[(1 + k) * NN];
                const double vbr = vbar * irho;
                g0 = fma(-vbr, vk, g0);
                v2 = fma(vk, vk, v2);
                ge[(1 + k) * NN] = fma(-pbar * (kGamma - 1.0), vk, vbr);
            }
            ge[0] = g0 + pbar * (kGamma - 1.0) * 0.5 * v2;
            ge[(D + 1) * NN] = pbar * (kGamma - 1.0);
        } else {
            ge[0] = ae[0];
        }
    }
    if constexpr (MODAL) {
        const int nq = ne * NVAR, t = threadIdx.x, nt = blockDim.x;
        __syncthreads();
        if constexpr (D == 3) {
            basis_pass<double, D, N, true>(sL, sP, 0, nq, *bt, t, nt);
            __syncthreads();
            basis_pass<double, D, N, true>(sP, sL, 1, nq, *bt, t, nt);
            __syncthreads();
            basis_pass<double, D, N, true>(sL, gbp, 2, nq, *bt, t, nt);
        } else {
            basis_pass<double, D, N, true>(sL, sP, 0, nq, *bt, t, nt);
            __syncthreads();
            basis_pass<double, D, N, true>(sP, gbp, 1, nq, *bt, t, nt);
        }
    }
}

template <int D, int N, int FLUX, class S>
__global__ void __launch_bounds__(S::THREADS)
vjp_modal_kernel(const double *__restrict__ u, const double *__restrict__ Ja, const double *__restrict__ lam,
                 double *__restrict__ g, int64_t n_elem, const __grid_constant__ OpTab<double> tab,
                 int *__restrict__ err, const __grid_constant__ BasisTab<double> bt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t e0 = (int64_t)blockIdx.x * S::EPB;
    const int ne = (int)((n_elem - e0) < S::EPB ? (n_elem - e0) : S::EPB);
    const int64_t nu = n_elem * S::NVAR * S::NN;
    vjp_tile<D, N, FLUX, S, true>(SFH_BP(u, nu, err), SFH_BP(Ja, n_elem * D * D * S::NN, err), SFH_BP(lam, nu, err), SFH_BP(g, nu, err),
                                  e0, ne, tab, err, smem_raw, &bt);
}

template <int D, int N, int FLUX>
cudaError_t launch_vjp_modal(const double *u, const double *Ja, const double *lam, double *g, int64_t n_elem,
                             const OpTab<double> &tab, const BasisTab<double> &bt, int *err, cudaStream_t stream) {
    using S = VjpShape<D, N, FLUX>;
    auto kern = vjp_modal_kernel<D, N, FLUX, S>;
    static_assert(S::SMEM <= 227 * 1024, "shared memory");
    if (S::SMEM > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        if (e != cudaSuccess) return e;
    }
    const int64_t blocks = (n_elem + S::EPB - 1) / S::EPB;
    kern<<<(unsigned)blocks, S::THREADS, S::SMEM, stream>>>(u, Ja, lam, g, n_elem, tab, err, bt);
    return cudaGetLastError();
}

template <int D, int N, int FLUX, class S>
__global__ void __launch_bounds__(S::THREADS)
vjp_kernel(const double *__restrict__ u, const double *__restrict__ Ja, const double *__restrict__ lam,
           double *__restrict__ g, int64_t n_elem, const __grid_constant__ OpTab<double> tab,
           int *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t e0 = (int64_t)blockIdx.x * S::EPB;
    const int ne = (int)((n_elem - e0) < S::EPB ? (n_elem - e0) : S::EPB);
    const int64_t nu = n_elem * S::NVAR * S::NN;
    vjp_tile<D, N, FLUX, S>(SFH_BP(u, nu, err), SFH_BP(Ja, n_elem * D * D * S::NN, err), SFH_BP(lam, nu, err), SFH_BP(g, nu, err), e0,
                            ne, tab, err, smem_raw);
}

template <int D, int N, int FLUX, class S>
cudaError_t launch_vjp_shape(const double *u, const double *Ja, const double *lam, double *g, int64_t n_elem,
                             const OpTab<double> &tab, int *err, cudaStream_t stream) {
    auto kern = vjp_kernel<D, N, FLUX, S>;
    static_assert(S::SMEM <= 227 * 1024, "shared memory");
    if (S::SMEM > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        if (e != cudaSuccess) return e;
    }
    const int64_t blocks = (n_elem + S::EPB - 1) / S::EPB;
    kern<<<(unsigned)blocks, S::THREADS, S::SMEM, stream>>>(u, Ja, lam, g, n_elem, tab, err);
    return cudaGetLastError();
}

template <int D, int N, int FLUX>
cudaError_t launch_vjp(const double *u, const double *Ja, const double *lam, double *g, int64_t n_elem,
                       const OpTab<double> &tab, int *err, cudaStream_t stream) {
    return launch_vjp_shape<D, N, FLUX, VjpShape<D, N, FLUX>>(u, Ja, lam, g, n_elem, tab, err, stream);
}

}  // namespace sfh
