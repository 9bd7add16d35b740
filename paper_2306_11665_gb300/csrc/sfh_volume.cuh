// sfh_volume.cuh -- the volume-residual kernel (forward), all precisions.
//
// r_i = sum_m omega_m(i) sum_{j on the m-line of i} Q1[a_m(i)][a_m(j)] F_m(u_i, u_j),
// F_m(u_i, u_j) = sum_k fsharp_k(u_i, u_j) (Ja^m_k(i) + Ja^m_k(j)),
// i.e. Eq. 3 with the Eq. 5 operators: per element and direction, n^{d-1}
// independent lines, each a dense n x n Hadamard product of Q1 with the line's
// two-point-flux matrix.  The paper stores both factors as n^d x n arrays
// (its sparsity-pattern and basis-assembly listings); here neither is stored:
// the pattern is index arithmetic, the basis entry is a kernel-parameter
// constant, and the flux matrix lives in registers for one line at a time.
//
// Work decomposition (one CTA = EPB consecutive elements):
//   1. stage: every node's conservative state -> primitives (rho, v, p,
//      beta = rho/p) in shared memory, coalesced global reads; domain check;
//   2. for each direction m: stage the metric row Ja^m of every node, then
//      one thread per grid line loads its n nodes into registers and forms
//      each unordered pair's flux once (F is symmetric), adding Q1[a][b] F to
//      node a and Q1[b][a] F to node b; diagonal terms only where Q1[a][a] != 0;
//      the line sums are scaled by omega (constant along the line) and added
//      to the node's residual in shared memory;
//   3. write r with coalesced stores.
#pragma once

#include "sfh_device.cuh"
#include "sfh_tma.cuh"

namespace sfh {

template <typename T, typename TJ, int D>
struct EulerNode {
    T rho, v[D], p, beta;
    TJ J[D];
    double beta_d;   // mixed mode only (FP64 copy of rho / p)
};

template <typename T, typename TJ, int D>
struct BurgersNode {
    T u;
    TJ S;            // sum_k Ja^m_k
};

// Two-point Euler flux contracted with n = Ja^m(a) + Ja^m(b): Ranocha's
//   f_rho = {rho}_ln {v.n},  f_m = f_rho {v} + {p} n,
//   f_E = f_rho (v_a.v_b / 2 + 1/((g-1){beta}_ln)) + (p_a v_b + p_b v_a).n / 2,
// or Chandrashekar's, which takes pt = {rho}/{beta} = (rho_a + rho_b) /
// (beta_a + beta_b) for {p} and pt {v}.n for the pressure work.
template <class M, int D, int FLUX>
__device__ __forceinline__ void euler_pair_flux(const EulerNode<typename M::T, typename M::TJ, D> &A,
                                                const EulerNode<typename M::T, typename M::TJ, D> &B,
                                                typename M::T F[D + 2]) {
    using T = typename M::T;
    T n[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        // TJ sum, then rounded to T (an FP64 sum rounded by integer
        // conversion, off the FP64 pipe)
        if constexpr (sizeof(typename M::TJ) == 8 && sizeof(T) == 4) n[k] = d2f_int(A.J[k] + B.J[k]);
        else n[k] = (T)(A.J[k] + B.J[k]);
    }
    T vna = A.v[0] * n[0], vnb = B.v[0] * n[0], vv = A.v[0] * B.v[0];
#pragma unroll
    for (int k = 1; k < D; ++k) { vna += A.v[k] * n[k]; vnb += B.v[k] * n[k]; vv += A.v[k] * B.v[k]; }
    T Lr, iLb;
    if constexpr (M::mixed) {
        // FP64 logarithmic mean inside the near-equal band (band test on the
        // FP32 values; FP64 arithmetic to the accuracy an FP32 result needs),
        // FP32 outside; widening by integer conversion keeps the FP64 pipe
        // for the arithmetic
        const float dr = A.rho - B.rho, sr = A.rho + B.rho;
        if (dr * dr < (float)kLnBand * (sr * sr)) Lr = d2f_int(ln_mean_mix(f2d_int(A.rho), f2d_int(B.rho), A.rho, B.rho));
        else Lr = ln_mean(A.rho, B.rho);
        const float db = A.beta - B.beta, sb = A.beta + B.beta;
        if (db * db < (float)kLnBand * (sb * sb)) iLb = d2f_int(inv_ln_mean_mix(A.beta_d, B.beta_d, A.beta, B.beta));
        else iLb = inv_ln_mean(A.beta, B.beta);
    } else {
        Lr = ln_mean(A.rho, B.rho);
        iLb = inv_ln_mean(A.beta, B.beta);
    }
    const T half = (T)0.5;
    const T frho = Lr * (half * (vna + vnb));
    T pavg;
    if constexpr (FLUX == kFluxEulerCh) {
        // (rho_a + rho_b) / (beta_a + beta_b) to within about half an ulp
        const T sr = A.rho + B.rho, sb = A.beta + B.beta;
        T isb;
        if constexpr (sizeof(T) == 8) {
            isb = rcp_nr(sb);
        } else {
            isb = rcp_approx(sb);
            isb = fma(isb, fma(-sb, isb, (T)1), isb);
        }
        pavg = sr * isb;
        pavg = fma(isb, fma(-sb, pavg, sr), pavg);
    } else {
        pavg = half * (A.p + B.p);
    }
    F[0] = frho;
#pragma unroll
    for (int l = 0; l < D; ++l) F[1 + l] = frho * (half * (A.v[l] + B.v[l])) + pavg * n[l];
    const T work = FLUX == kFluxEulerCh ? pavg * (half * (vna + vnb)) : half * (A.p * vnb + B.p * vna);
    F[D + 1] = frho * (half * vv + iLb * (T)(1.0 / (kGamma - 1.0))) + work;
}

// FP64 pair flux: the node carries v/2 (hv) and FP32 copies of rho and beta
// (rf, bf) for the band tests; see euler_pair_flux for the formula.
template <int D>
struct EulerNodeD {
    double rho, hv[D], p, beta;
    double J[D];
    float rf, bf;
};

template <int D, int FLUX = kFluxEuler>
__device__ __forceinline__ void euler_pair_flux_f64(const EulerNodeD<D> &A, const EulerNodeD<D> &B, double F[D + 2]) {
    double n[D];
#pragma unroll
    for (int k = 0; k < D; ++k) n[k] = A.J[k] + B.J[k];
    double hna = A.hv[0] * n[0], hnb = B.hv[0] * n[0], hvv = A.hv[0] * B.hv[0];
#pragma unroll
    for (int k = 1; k < D; ++k) {
        hna = fma(A.hv[k], n[k], hna);
        hnb = fma(B.hv[k], n[k], hnb);
        hvv = fma(A.hv[k], B.hv[k], hvv);
    }
    const double Lr = ln_mean_f64(A.rho, B.rho, A.rf, B.rf);
    const double iLb = inv_ln_mean_f64(A.beta, B.beta, A.bf, B.bf);
    const double frho = Lr * (hna + hnb);              // {rho}_ln {v.n}
    double pavg;
    if constexpr (FLUX == kFluxEulerCh) {
        // {rho}/{beta} to within about half an ulp (Newton reciprocal, one
        // residual correction)
        const double sr = A.rho + B.rho, sb = A.beta + B.beta, isb = rcp_nr(sb);
        pavg = sr * isb;
        pavg = fma(isb, fma(-sb, pavg, sr), pavg);
    } else {
        pavg = 0.5 * (A.p + B.p);
    }
    F[0] = frho;
#pragma unroll
    for (int k = 0; k < D; ++k) F[1 + k] = fma(frho, A.hv[k] + B.hv[k], pavg * n[k]);
    const double K = fma(2.0, hvv, iLb * (1.0 / (kGamma - 1.0)));
    if constexpr (FLUX == kFluxEulerCh) F[D + 1] = fma(frho, K, pavg * (hna + hnb));
    else F[D + 1] = fma(frho, K, fma(A.p, hnb, B.p * hna));
}

template <int D>
__device__ __forceinline__ void euler_diag_flux_f64(const EulerNodeD<D> &A, double F[D + 2]) {
    double n[D];
#pragma unroll
    for (int k = 0; k < D; ++k) n[k] = 2.0 * A.J[k];
    double hn = A.hv[0] * n[0], hv2 = A.hv[0] * A.hv[0];
#pragma unroll
    for (int k = 1; k < D; ++k) { hn = fma(A.hv[k], n[k], hn); hv2 = fma(A.hv[k], A.hv[k], hv2); }
    const double frho = 2.0 * A.rho * hn;
    F[0] = frho;
#pragma unroll
    for (int k = 0; k < D; ++k) F[1 + k] = fma(2.0 * frho, A.hv[k], A.p * n[k]);
    F[D + 1] = fma(frho, 2.0 * hv2, 2.0 * A.p * hn * (kGamma / (kGamma - 1.0)));
}

// Physical Euler flux f(u_a) . (2 Ja^m(a)) = the two-point flux at (u_a, u_a).
template <class M, int D>
__device__ __forceinline__ void euler_diag_flux(const EulerNode<typename M::T, typename M::TJ, D> &A,
                                                typename M::T F[D + 2]) {
    using T = typename M::T;
    T n[D];
#pragma unroll
    for (int k = 0; k < D; ++k) n[k] = (T)(A.J[k] + A.J[k]);
    T vn = A.v[0] * n[0], v2 = A.v[0] * A.v[0];
#pragma unroll
    for (int k = 1; k < D; ++k) { vn += A.v[k] * n[k]; v2 += A.v[k] * A.v[k]; }
    const T frho = A.rho * vn;
    F[0] = frho;
#pragma unroll
    for (int l = 0; l < D; ++l) F[1 + l] = frho * A.v[l] + A.p * n[l];
    // (E + p) v.n = rho v.n (|v|^2/2 + p/((gamma-1) rho)) + p v.n
    F[D + 1] = frho * ((T)0.5 * v2) + A.p * vn * (T)(kGamma / (kGamma - 1.0));
}

// One tile: the ne (<= EPB) consecutive elements starting at e0, processed by
// the whole CTA (any blockDim; every thread must call it).  smem_raw holds
// Shape::SMEM bytes.  Used by volume_kernel (one tile per CTA) and by the
// persistent serving kernel (tiles of many requests).
// MODAL: u holds basis coefficients (bt the basis on the cubature nodes); the
// nodal values V u_hat are formed in shared memory before the node pass and
// r receives V^T r_v (the residual and primitive buffers serve as scratch).
template <int D, int N, int FLUX, class M, class S = Shape<D, N, FLUX, M>, bool MODAL = false>
__device__ __forceinline__ void volume_tile(BPtr<const typename M::T> SFH_RESTRICT u, BPtr<const double> SFH_RESTRICT Ja,
                                            BPtr<typename M::T> SFH_RESTRICT r, int64_t e0, int ne,
                                            const OpTab<typename M::T> &tab, int *__restrict__ err,
                                            unsigned char *smem_raw,
                                            const BasisTab<typename M::T> *bt = nullptr) {
    using T = typename M::T;
    using TJ = typename M::TJ;
    using Acc = typename AccOf<M>::type;
    constexpr int NN = S::NN, NLINE = S::NLINE, NVAR = S::NVAR, NP = S::NP, EPB = S::EPB;

    // layout: [beta_d (mixed)] [J: EPB][D][NN] TJ  [P: EPB][NP][NN] T  [R: EPB][NVAR][NN] T
    //         (FP64 Euler: [rho_f: EPB][NN] [beta_f: EPB][NN] float in place of beta_d)
    constexpr bool F64E = S::F64E;
    constexpr int BD_COUNT = ((M::mixed || F64E) && is_euler(FLUX)) ? EPB * NN : 0;
    const auto sBd = SFH_BP(reinterpret_cast<double *>(smem_raw), BD_COUNT, err);
    const auto sRF = SFH_BP(reinterpret_cast<float *>(smem_raw), 2 * BD_COUNT, err);
    const auto sJ = SFH_BP(reinterpret_cast<TJ *>(smem_raw + sizeof(double) * BD_COUNT), EPB * D * NN, err);
    const auto sP = SFH_BP(reinterpret_cast<T *>(smem_raw + sizeof(double) * BD_COUNT + sizeof(TJ) * EPB * D * NN),
                       EPB * NP * NN, err);
    const auto sR = SFH_BP(reinterpret_cast<T *>(smem_raw + sizeof(double) * BD_COUNT + sizeof(TJ) * EPB * D * NN) +
                           EPB * NP * NN,
                       EPB * NVAR * NN, err);

    BPtr<const T> ub = u + e0 * NVAR * NN;
    if constexpr (MODAL) {
        // nodal values u_v = V u_hat, ending in sR ([el][var][i])
        if constexpr (D == 3) {
            basis_pass<T, D, N, false, kPassFirst>(ub, sR, 0, ne * NVAR, *bt, threadIdx.x, blockDim.x);
            __syncthreads();
            basis_pass<T, D, N, false>(sR, sP, 1, ne * NVAR, *bt, threadIdx.x, blockDim.x);
            __syncthreads();
            basis_pass<T, D, N, false, kPassLast>(sP, sR, 2, ne * NVAR, *bt, threadIdx.x, blockDim.x, ub);
        } else {
            basis_pass<T, D, N, false, kPassFirst>(ub, sP, 0, ne * NVAR, *bt, threadIdx.x, blockDim.x);
            __syncthreads();
            basis_pass<T, D, N, false, kPassLast>(sP, sR, 1, ne * NVAR, *bt, threadIdx.x, blockDim.x, ub);
        }
        __syncthreads();
        ub = sR;
    }

    // ---- 1. stage primitives, zero the residual (each node's thread reads
    //      its state before zeroing the same slots, also when it sits in sR)
    bool bad = false;
    for (int s = threadIdx.x; s < ne * NN; s += blockDim.x) {
        const int el = s / NN, i = s - el * NN;
        const auto ue = ub + (int64_t)el * NVAR * NN + i;
        const auto pe = sP + el * NP * NN + i;
        if constexpr (is_euler(FLUX)) {
            // reciprocals refined by Newton steps instead of IEEE divisions
            // (FP64: rcp_nr; FP32: hardware seed + one step); beta = rho / p
            // to within about half an ulp by one residual correction, and in
            // FP32 v = m / rho too (FP64 keeps m (1/rho), within an ulp)
            const T rho = ue[0];
            const T E = ue[(D + 1) * NN];
            T irho;
            if constexpr (sizeof(T) == 8) {
                irho = rcp_nr(rho);
            } else {
                irho = rcp_approx(rho);
                irho = fmaf(irho, fmaf(-rho, irho, 1.0f), irho);
            }
            T ke = (T)0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const T mk = ue[(1 + k) * NN];
                T vk = mk * irho;
                if constexpr (sizeof(T) == 4) vk = fma(irho, fma(-rho, vk, mk), vk);
                pe[(1 + k) * NN] = F64E ? (T)0.5 * vk : vk;   // FP64 keeps v/2
                ke = fma(mk, vk, ke);
            }
            const T p = (T)(kGamma - 1.0) * fma((T)-0.5, ke, E);
            T ip;
            if constexpr (sizeof(T) == 8) {
                ip = rcp_nr(p);
            } else {
                ip = rcp_approx(p);
                ip = fmaf(ip, fmaf(-p, ip, 1.0f), ip);
            }
            T bt = rho * ip;
            bt = fma(ip, fma(-p, bt, rho), bt);
            pe[0] = rho;
            pe[(D + 1) * NN] = p;
            pe[(D + 2) * NN] = bt;
            if constexpr (M::mixed) {
                // FP64 beta = rho / p to within about half an ulp (Newton
                // reciprocal, product, one residual correction)
                const double rd = f2d_int((float)rho), pd = f2d_int((float)p), ip = rcp_nr(pd);
                double bt = rd * ip;
                sBd[el * NN + i] = fma(ip, fma(-pd, bt, rd), bt);
            }
            if constexpr (F64E) {
                sRF[el * NN + i] = d2f_int((double)rho);
                sRF[EPB * NN + el * NN + i] = d2f_int((double)bt);
            }
            bad |= !(rho > (T)0 && p > (T)0);
        } else {
            pe[0] = ue[0];
        }
#pragma unroll
        for (int v = 0; v < NVAR; ++v) sR[(el * NVAR + v) * NN + i] = (T)0;
    }
    if (bad) atomicOr(err, 1);

    const auto Jb = Ja + e0 * D * D * NN;
    uint32_t hmax = 0;   // largest |Ja| high word (range check: FP32 modes 2^126, FP64 finite)
#pragma unroll 1
    for (int m = 0; m < D; ++m) {
        // ---- 2a. stage the metric row of direction m: Ja[e][m][k][i] -> sJ[el][k][i]
        __syncthreads();
        for (int s = threadIdx.x; s < ne * D * NN; s += blockDim.x) {
            const int el = s / (D * NN), rem = s - el * D * NN;
            const double j = Jb[((int64_t)el * D * D + m * D) * NN + rem];
            hmax = max(hmax, abs_hi(j));
            sJ[s] = (TJ)j;
        }
        if (m == D - 1 && hmax >= (sizeof(T) == 4 ? kMetricHiFp32 : kMetricHiFp64)) atomicOr(err, kErrMetric);
        __syncthreads();

        // ---- 2b. line sweeps
        const int stride = m == 0 ? 1 : (m == 1 ? N : N * N);
        for (int L = threadIdx.x; L < ne * NLINE; L += blockDim.x) {
            const int el = L / NLINE, l = L - el * NLINE;
            int base;
            T omega;
            if constexpr (D == 3) {
                const int o0 = l % N, o1 = l / N;   // the two other indices, lower axis first
                base = m == 0 ? N * l : (m == 1 ? o0 + N * N * o1 : l);
                omega = tab.w[o0] * tab.w[o1];
            } else {
                base = m == 0 ? N * l : l;
                omega = tab.w[l];
            }
            const int nb = el * NN + base;

            Acc acc[N][NVAR];
#pragma unroll
            for (int a = 0; a < N; ++a)
#pragma unroll
                for (int v = 0; v < NVAR; ++v) acc[a][v].zero();

            if constexpr (F64E) {
                EulerNodeD<D> nd[N];
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    const int i = nb + a * stride;
                    const auto pe = sP + el * NP * NN + (base + a * stride);
                    nd[a].rho = pe[0];
#pragma unroll
                    for (int k = 0; k < D; ++k) nd[a].hv[k] = pe[(1 + k) * NN];
                    nd[a].p = pe[(D + 1) * NN];
                    nd[a].beta = pe[(D + 2) * NN];
#pragma unroll
                    for (int k = 0; k < D; ++k) nd[a].J[k] = sJ[(el * D + k) * NN + base + a * stride];
                    nd[a].rf = sRF[i];
                    nd[a].bf = sRF[EPB * NN + i];
                }
#pragma unroll
                for (int a = 0; a < N; ++a) {
#pragma unroll
                    for (int b = a + 1; b < N; ++b) {
                        double F[D + 2];
                        euler_pair_flux_f64<D, FLUX>(nd[a], nd[b], F);
                        const double qab = tab.Q1[a * N + b], qba = tab.Q1[b * N + a];
#pragma unroll
                        for (int v = 0; v < NVAR; ++v) { acc[a][v].add_prod(qab, F[v]); acc[b][v].add_prod(qba, F[v]); }
                    }
                    const double qaa = tab.Q1[a * N + a];
                    if (qaa != 0.0) {
                        double F[D + 2];
                        euler_diag_flux_f64<D>(nd[a], F);
#pragma unroll
                        for (int v = 0; v < NVAR; ++v) acc[a][v].add_prod(qaa, F[v]);
                    }
                }
            } else if constexpr (is_euler(FLUX)) {
                EulerNode<T, TJ, D> nd[N];
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    const int i = nb + a * stride;
                    const auto pe = sP + el * NP * NN + (base + a * stride);
                    nd[a].rho = pe[0];
#pragma unroll
                    for (int k = 0; k < D; ++k) nd[a].v[k] = pe[(1 + k) * NN];
                    nd[a].p = pe[(D + 1) * NN];
                    nd[a].beta = pe[(D + 2) * NN];
#pragma unroll
                    for (int k = 0; k < D; ++k) nd[a].J[k] = sJ[(el * D + k) * NN + base + a * stride];
                    if constexpr (M::mixed) nd[a].beta_d = sBd[i];
                    else nd[a].beta_d = 0.0;
                }
#pragma unroll
                for (int a = 0; a < N; ++a) {
#pragma unroll
                    for (int b = a + 1; b < N; ++b) {
                        T F[D + 2];
                        euler_pair_flux<M, D, FLUX>(nd[a], nd[b], F);
                        const T qab = tab.Q1[a * N + b], qba = tab.Q1[b * N + a];
#pragma unroll
                        for (int v = 0; v < NVAR; ++v) { acc[a][v].add_prod(qab, F[v]); acc[b][v].add_prod(qba, F[v]); }
                    }
                    const T qaa = tab.Q1[a * N + a];
                    if (qaa != (T)0) {
                        T F[D + 2];
                        euler_diag_flux<M, D>(nd[a], F);
#pragma unroll
                        for (int v = 0; v < NVAR; ++v) acc[a][v].add_prod(qaa, F[v]);
                    }
                }
            } else {
                BurgersNode<T, TJ, D> nd[N];
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    nd[a].u = sP[el * NN + base + a * stride];
                    TJ S = sJ[(el * D + 0) * NN + base + a * stride];
#pragma unroll
                    for (int k = 1; k < D; ++k) S += sJ[(el * D + k) * NN + base + a * stride];
                    nd[a].S = S;
                }
#pragma unroll
                for (int a = 0; a < N; ++a) {
#pragma unroll
                    for (int b = a + 1; b < N; ++b) {
                        const T ua = nd[a].u, ub2 = nd[b].u;
                        const T F = (ua * ua + ua * ub2 + ub2 * ub2) * (T)(1.0 / 6.0) * (T)(nd[a].S + nd[b].S);
                        acc[a][0].add_prod(tab.Q1[a * N + b], F);
                        acc[b][0].add_prod(tab.Q1[b * N + a], F);
                    }
                    const T qaa = tab.Q1[a * N + a];
                    if (qaa != (T)0) {
                        const T ua = nd[a].u;
                        acc[a][0].add_prod(qaa, ua * ua * (T)nd[a].S);
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < N; ++a)
#pragma unroll
                for (int v = 0; v < NVAR; ++v) sR[(el * NVAR + v) * NN + base + a * stride] += omega * acc[a][v].value();
        }
    }
    __syncthreads();

    // ---- 3. write r (layout [el][v][i] matches the global layout); modal:
    //      r_hat = V^T r_v
    const auto rb = r + e0 * NVAR * NN;
    if constexpr (MODAL) {
        if constexpr (D == 3) {
            basis_pass<T, D, N, true>(sR, sP, 0, ne * NVAR, *bt, threadIdx.x, blockDim.x);
            __syncthreads();
            basis_pass<T, D, N, true>(sP, sR, 1, ne * NVAR, *bt, threadIdx.x, blockDim.x);
            __syncthreads();
            basis_pass<T, D, N, true>(sR, rb, 2, ne * NVAR, *bt, threadIdx.x, blockDim.x);
        } else {
            basis_pass<T, D, N, true>(sR, sP, 0, ne * NVAR, *bt, threadIdx.x, blockDim.x);
            __syncthreads();
            basis_pass<T, D, N, true>(sP, rb, 1, ne * NVAR, *bt, threadIdx.x, blockDim.x);
        }
    } else {
        for (int s = threadIdx.x; s < ne * NVAR * NN; s += blockDim.x) rb[s] = sR[s];
    }
}

template <int D, int N, int FLUX, class M, class S = Shape<D, N, FLUX, M>>
__global__ void __launch_bounds__(S::THREADS, S::MINB)
volume_kernel(const typename M::T *__restrict__ u, const double *__restrict__ Ja,
              typename M::T *__restrict__ r, int64_t n_elem,
              const __grid_constant__ OpTab<typename M::T> tab, int *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t e0 = (int64_t)blockIdx.x * S::EPB;
    const int ne = (int)((n_elem - e0) < S::EPB ? (n_elem - e0) : S::EPB);
    volume_tile<D, N, FLUX, M, S>(SFH_BP(u, n_elem * S::NVAR * S::NN, err), SFH_BP(Ja, n_elem * D * D * S::NN, err),
                                  SFH_BP(r, n_elem * S::NVAR * S::NN, err), e0, ne, tab, err, smem_raw);
}

template <int D, int N, int FLUX, class M, class S>
__global__ void __launch_bounds__(S::THREADS)
volume_modal_kernel(const typename M::T *__restrict__ u, const double *__restrict__ Ja,
                    typename M::T *__restrict__ r, int64_t n_elem,
                    const __grid_constant__ OpTab<typename M::T> tab, int *__restrict__ err,
                    const __grid_constant__ BasisTab<typename M::T> bt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t e0 = (int64_t)blockIdx.x * S::EPB;
    const int ne = (int)((n_elem - e0) < S::EPB ? (n_elem - e0) : S::EPB);
    volume_tile<D, N, FLUX, M, S, true>(SFH_BP(u, n_elem * S::NVAR * S::NN, err), SFH_BP(Ja, n_elem * D * D * S::NN, err),
                                        SFH_BP(r, n_elem * S::NVAR * S::NN, err), e0, ne, tab, err, smem_raw, &bt);
}

template <int D, int N, int FLUX, class M, class S = Shape<D, N, FLUX, M>>
cudaError_t launch_volume_modal(const void *u, const double *Ja, void *r, int64_t n_elem,
                                const OpTab<typename M::T> &tab, const BasisTab<typename M::T> &bt, int *err,
                                cudaStream_t stream) {
    auto kern = volume_modal_kernel<D, N, FLUX, M, S>;
    static_assert(S::SMEM <= 227 * 1024, "shared memory");
    if (S::SMEM > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        if (e != cudaSuccess) return e;
    }
    const int64_t blocks = (n_elem + S::EPB - 1) / S::EPB;
    kern<<<(unsigned)blocks, S::THREADS, S::SMEM, stream>>>(
        static_cast<const typename M::T *>(u), Ja, static_cast<typename M::T *>(r), n_elem, tab, err, bt);
    return cudaGetLastError();
}

// Host-side launcher for one (D, N, FLUX, mode) instance and tile shape.
template <int D, int N, int FLUX, class M, class S = Shape<D, N, FLUX, M>>
cudaError_t launch_volume(const void *u, const double *Ja, void *r, int64_t n_elem,
                          const OpTab<typename M::T> &tab, int *err, cudaStream_t stream) {
    auto kern = volume_kernel<D, N, FLUX, M, S>;
    static_assert(S::SMEM <= 227 * 1024, "shared memory");
    if (S::SMEM > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        if (e != cudaSuccess) return e;
    }
    const int64_t blocks = (n_elem + S::EPB - 1) / S::EPB;
    kern<<<(unsigned)blocks, S::THREADS, S::SMEM, stream>>>(
        static_cast<const typename M::T *>(u), Ja, static_cast<typename M::T *>(r), n_elem, tab, err);
    return cudaGetLastError();
}

}  // namespace sfh
