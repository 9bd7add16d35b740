// sfh_volume_tma.cuh -- persistent FP32 (Kahan) volume-residual kernel with
// TMA bulk staging.
//
// Same arithmetic as volume_kernel (Eq. 3 with the Eq. 5 operators, one
// unordered line pair per flux evaluation, compensated line sums), organised
// for GB300:
//   * persistent CTAs walk element blocks blk = blockIdx.x, + gridDim.x, ...;
//   * the raw u (FP32) and Ja (FP64) of a block arrive in shared memory by
//     two 1D bulk copies (cp.async.bulk + mbarrier), issued by one thread;
//     a block whose start is not 16-byte aligned is fetched through a wider
//     aligned window and indexed from the remainder;
//   * as soon as a block's raw data has been converted (primitives, and Ja to
//     FP32 with integer field arithmetic -- an FP64->FP32 conversion
//     instruction would run on the narrow FP64 pipe), the next block's bulk
//     copies are issued into the same raw buffers, so the HBM traffic of
//     block k+1 overlaps the line sweeps of block k;
//   * the d directions are swept concurrently (one thread per line and
//     direction), each direction writing its own residual slice, summed in a
//     fixed order afterwards (deterministic);
//   * r leaves by a bulk store when the block is 16-byte aligned, else by
//     coalesced stores.
// Waits are bounded: a bulk copy that does not arrive within 2 s sets the
// timeout bit of the error word and the CTA leaves after draining its copies.
#pragma once

#include "sfh_device.cuh"
#include "sfh_tma.cuh"

namespace sfh {

// Residency.  Each of the four sub-partitions of an SM holds its warps'
// registers in its own 16K-register file, so CPS resident CTAs of W warps
// each fit only if CPS * ceil(W/4) * regs * 32 <= 16384: the register cap is
// 512 / (CPS * WPS) with WPS = ceil(W/4).  Two CTAs per SM let one CTA's
// per-node phases and barriers overlap the other's line sweeps (measured on
// the 3D n=5 shape: 202 us against 221 us with one CTA); the pairs below
// follow the register counts ptxas reports for each line body (about 55, 64,
// 80, 96, 125, 150, 205, 230 registers for 3D Euler n = 2..9).
template <int D, int N, int FLUX>
constexpr int tma_cps() {
    if (!is_euler(FLUX)) return 2;
    return N <= (D == 3 ? 6 : 7) ? 2 : 1;
}
template <int D, int N, int FLUX>
constexpr int tma_wps() {
    if (!is_euler(FLUX)) return 3;
    if (D == 3) return N <= 3 ? 4 : (N == 4 ? 3 : 2);
    return N <= 4 ? 4 : (N <= 7 ? 2 : 3);
}

template <int D, int N, int FLUX>
struct TmaShape {
    static constexpr int CPS = tma_cps<D, N, FLUX>();
    static constexpr int WPS = tma_wps<D, N, FLUX>();   // per CTA
    static constexpr int NN = ipow(N, D);
    static constexpr int NLINE = ipow(N, D - 1);
    static constexpr int NVAR = is_euler(FLUX) ? D + 2 : 1;
    static constexpr int NP = is_euler(FLUX) ? D + 3 : 1;      // rho, v/2 [D], p, beta | u
    static constexpr int NJ = is_euler(FLUX) ? D * D : D;       // FP32 metric values kept per node
    // Euler keeps the FP32 metric rows line-major per direction,
    // [el][m][line][a][k], so that a line's values sit at constant offsets
    // from one base; LJ = floats per line, odd so that the lines of
    // consecutive lanes fall in different banks
    static constexpr int LJ = (N * D) % 2 == 0 ? N * D + 1 : N * D;
    static constexpr int JF_EL = is_euler(FLUX) ? D * NLINE * LJ : D * NN;   // floats per element
    static constexpr int U_EL = NVAR * NN;                          // floats of u (and r) per element
    static constexpr int J_EL = D * D * NN;                         // doubles of Ja per element
    static constexpr int EL_BYTES = 4 * U_EL + 8 * J_EL + 4 * NP * NN + 4 * JF_EL + 4 * D * U_EL;
    static constexpr int BUDGET = (CPS == 1 ? 200 : 108) * 1024;
    static constexpr int MAX_THREADS = 128 * WPS;
    static constexpr int epb_by_smem() { return BUDGET / EL_BYTES > 0 ? BUDGET / EL_BYTES : 1; }
    // largest EPB whose D * EPB * NLINE line tasks fit the thread budget
    static constexpr int epb_by_threads() {
        int e = 1;
        while (D * (e + 1) * NLINE <= MAX_THREADS) ++e;
        return e;
    }
    static constexpr int epb_raw() { return epb_by_smem() < epb_by_threads() ? epb_by_smem() : epb_by_threads(); }
    static constexpr bool aligned_blocks(int e) { return (e * U_EL * 4) % 16 == 0; }
    // prefer a block whose r slice is a whole number of 16-byte units (bulk store)
    static constexpr int pick_epb() {
        for (int e = epb_raw(); e >= 1 && 4 * e >= 3 * epb_raw(); --e)
            if (aligned_blocks(e)) return e;
        return epb_raw();
    }
    static constexpr int EPB = pick_epb();
    static constexpr int THREADS = ((D * EPB * NLINE + 31) / 32) * 32;
    static constexpr int MAXREG = (512 / (WPS * CPS)) / 8 * 8 < 255 ? (512 / (WPS * CPS)) / 8 * 8 : 255;
    static_assert(THREADS <= MAX_THREADS, "line tasks exceed the CTA");
    static constexpr int RAWU_BYTES = ((EPB * U_EL * 4 + 16) + 15) / 16 * 16;   // + window slack
    static constexpr int RAWJ_BYTES = ((EPB * J_EL * 8 + 16) + 15) / 16 * 16;
    static constexpr int OFF_U = 16;                                             // [0,16): mbarrier
    static constexpr int OFF_J = OFF_U + RAWU_BYTES;
    static constexpr int OFF_P = OFF_J + RAWJ_BYTES;
    static constexpr int up16(int x) { return (x + 15) / 16 * 16; }
    static constexpr int OFF_JF = up16(OFF_P + EPB * NP * NN * 4);
    static constexpr int OFF_R = up16(OFF_JF + EPB * JF_EL * 4);   // bulk-store source: 16-byte aligned
    static constexpr size_t SMEM = OFF_R + (size_t)D * EPB * U_EL * 4;
    static_assert(OFF_U % 16 == 0 && OFF_J % 16 == 0 && OFF_R % 16 == 0, "bulk-copy buffers must be 16-byte aligned");
};

struct BlockPlan {
    int64_t e0;
    int ne;
    bool tma;
    uint32_t offU, offJ;          // element offsets of the block inside the raw windows
    const char *srcU, *srcJ;
    uint32_t bytesU, bytesJ;
};

template <class S, typename TU>
__device__ __forceinline__ BlockPlan plan_block(int64_t blk, int64_t n_elem, const TU *u, const double *Ja,
                                                bool aligned_bases) {
    constexpr uintptr_t ESZ = sizeof(TU);
    BlockPlan pl;
    pl.e0 = blk * S::EPB;
    pl.ne = (int)((n_elem - pl.e0) < S::EPB ? (n_elem - pl.e0) : S::EPB);
    const uintptr_t aU = reinterpret_cast<uintptr_t>(u + pl.e0 * S::U_EL);
    const uintptr_t eU = reinterpret_cast<uintptr_t>(u + n_elem * S::U_EL);
    const uintptr_t loU = aU & ~uintptr_t(15), hiU = (aU + (uintptr_t)pl.ne * S::U_EL * ESZ + 15) & ~uintptr_t(15);
    const uintptr_t aJ = reinterpret_cast<uintptr_t>(Ja + pl.e0 * S::J_EL);
    const uintptr_t eJ = reinterpret_cast<uintptr_t>(Ja + n_elem * S::J_EL);
    const uintptr_t loJ = aJ & ~uintptr_t(15), hiJ = (aJ + (uintptr_t)pl.ne * S::J_EL * 8 + 15) & ~uintptr_t(15);
    pl.tma = aligned_bases && hiU <= eU && hiJ <= eJ;   // never read past the end of either array
    pl.offU = (uint32_t)((aU - loU) / ESZ);
    pl.offJ = (uint32_t)((aJ - loJ) / 8);
    pl.srcU = reinterpret_cast<const char *>(loU);
    pl.srcJ = reinterpret_cast<const char *>(loJ);
    pl.bytesU = (uint32_t)(hiU - loU);
    pl.bytesJ = (uint32_t)(hiJ - loJ);
    if (!pl.tma) { pl.offU = 0; pl.offJ = 0; }
    return pl;
}

// Geometry of one grid line of an element block: first node, node stride
// along direction m, and omega_m (the product of the other directions'
// weights, constant along the line).
template <int D, int N>
__device__ __forceinline__ void line_geometry(int m, int l, const OpTab<float> &tab, int &base, float &omega) {
    if constexpr (D == 3) {
        const int o0 = l % N, o1 = l / N;
        base = m == 0 ? N * l : (m == 1 ? o0 + N * N * o1 : l);
        omega = tab.w[o0] * tab.w[o1];
    } else {
        base = m == 0 ? N * l : l;
        omega = tab.w[l];
    }
}

// 3D Euler with Ranocha's flux: the node pass stores p/2 in place of p, so
// that the mean pressure of a pair is one addition, and the line sweep forms
// the energy flux and its compensated sum at half scale (the pressure work
// with p/2, the inverse beta mean from the series with halved coefficients,
// v_a.v_b/2 in place of 2 (v_a/2).(v_b/2)).  Every such step is an exact
// power-of-two scaling, so the energy sum is exactly half of the full-scale
// one; the store multiplies it by 2 omega.
template <int D, int FLUX>
constexpr bool kHalfP = D == 3 && FLUX == kFluxEuler;

// One Euler line from scratch, with the logarithm for pairs outside the
// series band.  Kept out of line (one copy per kernel) because it runs only
// for states with large jumps along a line; the arithmetic is that of the
// fast path otherwise.
template <int D, int N, int NN, int NP, int FLUX>
__device__ __noinline__ void euler_line_general(BPtr<const float> pe, BPtr<const float> jl, BPtr<float> re, int stride,
                                                float omega, const OpTab<float> &tab) {
    constexpr int NVAR = D + 2;
#pragma unroll 1
    for (int a = 0; a < N; ++a) {
        KahanF acc[NVAR];
#pragma unroll
        for (int v = 0; v < NVAR; ++v) acc[v].zero();
        constexpr float ps = kHalfP<D, FLUX> ? 2.0f : 1.0f;   // p from the stored p/2 (exact)
        const float ra = pe[a * stride], pa = ps * pe[(D + 1) * NN + a * stride], ba = pe[(D + 2) * NN + a * stride];
        float hva[D];
#pragma unroll
        for (int k = 0; k < D; ++k) hva[k] = pe[(1 + k) * NN + a * stride];
#pragma unroll 1
        for (int b = 0; b < N; ++b) {
            const float q = tab.Q1[a * N + b];
            if (q == 0.0f) continue;
            const float rb = pe[b * stride], pb = ps * pe[(D + 1) * NN + b * stride], bb = pe[(D + 2) * NN + b * stride];
            float hvb[D], n[D];
#pragma unroll
            for (int k = 0; k < D; ++k) {
                hvb[k] = pe[(1 + k) * NN + b * stride];
                n[k] = jl[a * D + k] + jl[b * D + k];
            }
            float hna = 0.0f, hnb = 0.0f, hvv = 0.0f;
#pragma unroll
            for (int k = 0; k < D; ++k) { hna = fmaf(hva[k], n[k], hna); hnb = fmaf(hvb[k], n[k], hnb); hvv = fmaf(hva[k], hvb[k], hvv); }
            const float Lr = ln_mean(ra, rb), iLb = inv_ln_mean(ba, bb);
            float F[D + 2];
            const float frho = Lr * (hna + hnb);
            // Chandrashekar: {rho}/{beta} and its work {rho}/{beta} {v}.n
            const float pavg = FLUX == kFluxEulerCh ? (ra + rb) * rcp_approx(ba + bb) : 0.5f * (pa + pb);
            const float work = FLUX == kFluxEulerCh ? pavg * (hna + hnb) : fmaf(pa, hnb, pb * hna);
            F[0] = frho;
#pragma unroll
            for (int k = 0; k < D; ++k) F[1 + k] = fmaf(frho, hva[k] + hvb[k], pavg * n[k]);
            F[D + 1] = fmaf(frho, fmaf(2.0f, hvv, iLb * (float)(1.0 / (kGamma - 1.0))), work);
#pragma unroll
            for (int v = 0; v < NVAR; ++v) acc[v].add_prod(q, F[v]);
        }
#pragma unroll
        for (int v = 0; v < NVAR; ++v) re[v * NN + a * stride] = omega * acc[v].value();
    }
}

// ---------------------------------------------------------------------------
// The phases of one element block, shared by the persistent kernel and the
// serving kernel's FP32 tiles.  S supplies the block geometry (NN, NLINE,
// NVAR, NP, U_EL, J_EL, LJ, JF_EL, EPB).
// ---------------------------------------------------------------------------

// Primitives and FP32 metric rows of ne elements from U ([el][var][i] floats)
// and J ([el][m][k][i] doubles), in shared or global memory; returns the
// error bits this thread found: kErrDomain (rho <= 0 or p <= 0, or NaN),
// kErrMetric (a metric term outside the FP32 modes' range).
template <class S, int D, int N, int FLUX>
__device__ __forceinline__ int fp32_block_convert(BPtr<const float> U, BPtr<const double> J, int ne, BPtr<float> sP,
                                                  BPtr<float> sJF, int tid, int nthreads) {
    constexpr int NN = S::NN, NLINE = S::NLINE, NP = S::NP, U_EL = S::U_EL, J_EL = S::J_EL;
    bool bad = false;
    uint32_t hmax = 0;
    for (int s = tid; s < ne * NN; s += nthreads) {
        const int el = s / NN, i = s - el * NN;
        const auto ue = U + el * U_EL + i;
        const auto pe = sP + el * NP * NN + i;
        if constexpr (is_euler(FLUX)) {
            // per-node divisions to within about half an ulp: with the
            // residual's cancellation, per-node errors act like
            // perturbations of the input state.  q = m / rho is formed as
            // m r (r: reciprocal seed plus one Newton step) followed by one
            // residual correction q += r (m - rho q), each a fused op.
            const float rho = ue[0], E = ue[(D + 1) * NN];
            float ir = rcp_approx(rho);
            ir = fmaf(ir, fmaf(-rho, ir, 1.0f), ir);
            float ke = 0.0f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const float mk = ue[(1 + k) * NN];
                float vk = mk * ir;
                vk = fmaf(ir, fmaf(-rho, vk, mk), vk);
                pe[(1 + k) * NN] = 0.5f * vk;
                ke = fmaf(mk, vk, ke);
            }
            const float p = (float)(kGamma - 1.0) * fmaf(-0.5f, ke, E);
            float ip = rcp_approx(p);
            ip = fmaf(ip, fmaf(-p, ip, 1.0f), ip);
            float bt = rho * ip;
            bt = fmaf(ip, fmaf(-p, bt, rho), bt);
            pe[0] = rho;
            pe[(D + 1) * NN] = kHalfP<D, FLUX> ? 0.5f * p : p;   // exact
            pe[(D + 2) * NN] = bt;
            bad |= !(rho > 0.0f && p > 0.0f);
            // the node's d*d metric values, FP64 -> FP32, into the line of
            // each direction through it: (line, position) = (i / N, i0),
            // (i0 + N i2, i1), (i0 + N i1, i2) in 3D; (i1, i0), (i0, i1) in 2D
            const auto je = J + el * J_EL + i;
            const auto jl = sJF + el * S::JF_EL;
            const int i0 = i % N;
#pragma unroll
            for (int m = 0; m < D; ++m) {
                int line, pos;
                if constexpr (D == 3) {
                    const int i1 = (i / N) % N, i2 = i / (N * N);
                    line = m == 0 ? i / N : (m == 1 ? i0 + N * i2 : i0 + N * i1);
                    pos = m == 0 ? i0 : (m == 1 ? i1 : i2);
                } else {
                    line = m == 0 ? i / N : i0;
                    pos = m == 0 ? i0 : i / N;
                }
                const auto dst = jl + (m * NLINE + line) * S::LJ + pos * D;
#pragma unroll
                for (int k = 0; k < D; ++k) dst[k] = d2f_int_track(je[(m * D + k) * NN], hmax);
            }
        } else {
            pe[0] = ue[0];
        }
    }
    if constexpr (!is_euler(FLUX)) {
        for (int s = tid; s < ne * D * NN; s += nthreads) {
            const int el = s / (D * NN), rem = s - el * D * NN, m = rem / NN, i = rem - m * NN;
            const auto jm = J + ((el * D + m) * D) * NN + i;
            static_assert(is_euler(FLUX) || S::JF_EL == D * NN, "Burgers metric sums are node-major");
            float acc = d2f_int_track(jm[0], hmax);
#pragma unroll
            for (int k = 1; k < D; ++k) acc += d2f_int_track(jm[k * NN], hmax);
            sJF[s] = acc;
        }
    }
    return (bad ? kErrDomain : 0) | (hmax >= kMetricHiFp32 ? kErrMetric : 0);
}

// Line sweeps of all directions at once: thread tid < D * EPB * NLINE owns one
// (direction, element, line) and writes its direction's residual slice of sR
// ([m][el][var][i]).
template <class S, int D, int N, int FLUX>
__device__ __forceinline__ void fp32_block_sweep(int tid, int ne, BPtr<const float> sP, BPtr<const float> sJF,
                                                 BPtr<float> sR, const OpTab<float> &tab) {
    constexpr int NN = S::NN, NLINE = S::NLINE, NVAR = S::NVAR, NP = S::NP, EPB = S::EPB, U_EL = S::U_EL;
    if (tid < D * EPB * NLINE) {
        const int m = tid / (EPB * NLINE);
        const int L = tid - m * (EPB * NLINE);
        const int el = L / NLINE, l = L - el * NLINE;
        if (el < ne) {
            const int stride = m == 0 ? 1 : (m == 1 ? N : N * N);
            int base;
            float omega;
            if constexpr (D == 3) {
                const int o0 = l % N, o1 = l / N;
                base = m == 0 ? N * l : (m == 1 ? o0 + N * N * o1 : l);
                omega = tab.w[o0] * tab.w[o1];
            } else {
                base = m == 0 ? N * l : l;
                omega = tab.w[l];
            }
            const auto pe = sP + el * NP * NN + base;
            float umax = 0.0f;   // largest u_rho + u_beta of the line's pairs
            if constexpr (is_euler(FLUX)) {
                // Euler: variables accumulate in packed pairs (0,1), (2,3) [, 4]
                constexpr int NPAIR = NVAR / 2;
                KahanF2 accp[N][NPAIR];
                KahanF acc4[N];
#pragma unroll
                for (int a = 0; a < N; ++a) {
#pragma unroll
                    for (int v = 0; v < NPAIR; ++v) accp[a][v].zero();
                    acc4[a].zero();
                }
                const auto jl = sJF + el * S::JF_EL + (m * NLINE + l) * S::LJ;   // this line's metric rows
                float2 rb[N];          // (rho, beta)
                float hv[N][D], p[N];
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    rb[a] = f2(pe[a * stride], pe[(D + 2) * NN + a * stride]);
#pragma unroll
                    for (int k = 0; k < D; ++k) hv[a][k] = pe[(1 + k) * NN + a * stride];
                    p[a] = pe[(D + 1) * NN + a * stride];
                }
                // S(u)/2 (rho mean) and P(u) 2/(gamma-1) (inverse beta mean; with the
                // stored p/2, half of it) as one packed Horner chain
                constexpr bool PH = kHalfP<D, FLUX>;
                const float cg = (float)((PH ? 1.0 : 2.0) / (kGamma - 1.0));
                const float2 c0 = f2(0.5f, cg), c1 = f2(0.5f * (-1.0f / 3.0f), cg * (1.0f / 3.0f));
                const float2 c2 = f2(0.5f * (-4.0f / 45.0f), cg * (1.0f / 5.0f));
                const float2 c3 = f2(0.5f * (-44.0f / 945.0f), cg * (1.0f / 7.0f));
#pragma unroll
                for (int a = 0; a < N; ++a) {
#pragma unroll
                    for (int b = a + 1; b < N; ++b) {
                        float n[D];
#pragma unroll
                        for (int k = 0; k < D; ++k) n[k] = jl[a * D + k] + jl[b * D + k];
                        float hna = hv[a][0] * n[0], hnb = hv[b][0] * n[0], hvv = hv[a][0] * hv[b][0];
#pragma unroll
                        for (int k = 1; k < D; ++k) {
                            hna = fmaf(hv[a][k], n[k], hna);
                            hnb = fmaf(hv[b][k], n[k], hnb);
                            hvv = fmaf(hv[a][k], hv[b][k], hvv);
                        }
                        // both logarithmic means at once (.x: rho, .y: beta), by the series
                        // in u = ((a-b)/(a+b))^2.  1/(a+b) is the hardware reciprocal
                        // (at most 1 ulp off): it scales the inverse mean directly, an
                        // error of the order of the FP32 rounding of the other factors.
                        // The line leaves for the general routine if any pair has
                        // u_rho + u_beta >= 1e-2 (which covers both u < 1e-2).
                        const float2 d2 = sub2(rb[a], rb[b]), s2 = add2(rb[a], rb[b]);
                        const float2 r2 = f2(rcp_approx(s2.x), rcp_approx(s2.y));
                        const float2 t2 = mul2(d2, r2);
                        const float2 u2 = mul2(t2, t2);
                        float2 h = fma2(u2, c3, c2);
                        h = fma2(u2, h, c1);
                        h = fma2(u2, h, c0);
                        umax = fmaxf(umax, u2.x + u2.y);
                        const float2 m2 = mul2(f2(s2.x, r2.y), h);   // ({rho}_ln, 1/((g-1){beta}_ln))
                        const float frho = m2.x * (hna + hnb);      // {rho}_ln {v.n}
                        // pressure average: {p} (Ranocha) or {rho}/{beta}
                        // (Chandrashekar), the latter from the sums and
                        // reciprocals of the log means
                        const float pavg = FLUX == kFluxEulerCh ? s2.x * r2.y : (PH ? p[a] + p[b] : 0.5f * (p[a] + p[b]));
                        const float work = FLUX == kFluxEulerCh ? pavg * (hna + hnb) : fmaf(p[a], hnb, p[b] * hna);
                        float2 F01, F23;
                        F01.x = frho;
                        F01.y = fmaf(frho, hv[a][0] + hv[b][0], pavg * n[0]);
                        float FE;
                        const float K = PH ? hvv + m2.y : fmaf(2.0f, hvv, m2.y);
                        if constexpr (D == 3) {
                            F23.x = fmaf(frho, hv[a][1] + hv[b][1], pavg * n[1]);
                            F23.y = fmaf(frho, hv[a][2] + hv[b][2], pavg * n[2]);
                            FE = fmaf(frho, K, work);
                        } else {
                            F23.x = fmaf(frho, hv[a][1] + hv[b][1], pavg * n[1]);
                            F23.y = fmaf(frho, K, work);
                            FE = 0.0f;
                        }
                        const float qab = tab.Q1[a * N + b], qba = tab.Q1[b * N + a];
                        const float2 qa2 = f2s(qab), qb2 = f2s(qba);
                        accp[a][0].add_prod(qa2, F01);
                        accp[b][0].add_prod(qb2, F01);
                        accp[a][1].add_prod(qa2, F23);
                        accp[b][1].add_prod(qb2, F23);
                        if constexpr (D == 3) {
                            acc4[a].add_prod(qab, FE);
                            acc4[b].add_prod(qba, FE);
                        }
                    }
                    const float qaa = tab.Q1[a * N + a];
                    if (qaa != 0.0f) {
                        // physical flux f(u_a) . (2 Ja^m(a))
                        float n[D];
#pragma unroll
                        for (int k = 0; k < D; ++k) n[k] = 2.0f * jl[a * D + k];
                        float hn = hv[a][0] * n[0], hv2 = hv[a][0] * hv[a][0];
#pragma unroll
                        for (int k = 1; k < D; ++k) { hn = fmaf(hv[a][k], n[k], hn); hv2 = fmaf(hv[a][k], hv[a][k], hv2); }
                        float F[D + 2];
                        const float frho = 2.0f * rb[a].x * hn;
                        const float pf = PH ? p[a] + p[a] : p[a];
                        F[0] = frho;
#pragma unroll
                        for (int k = 0; k < D; ++k) F[1 + k] = fmaf(2.0f * frho, hv[a][k], pf * n[k]);
                        if constexpr (PH) F[D + 1] = fmaf(frho, hv2, pf * hn * (float)(kGamma / (kGamma - 1.0)));
                        else F[D + 1] = fmaf(frho, 2.0f * hv2, 2.0f * pf * hn * (float)(kGamma / (kGamma - 1.0)));
                        const float2 qq = f2s(qaa);
                        accp[a][0].add_prod(qq, f2(F[0], F[1]));
                        accp[a][1].add_prod(qq, f2(F[2], F[3]));
                        if constexpr (D == 3) acc4[a].add_prod(qaa, F[4]);
                    }
                }
                const auto re = sR + (size_t)m * EPB * U_EL + el * U_EL + base;
                // also false for a NaN maximum (fmaxf drops NaN operands; the
                // domain flag of the node pass reports the state)
                if (__builtin_expect(!(umax < 1e-2f), 0)) {
                    // rare: redo the whole line with logarithms where needed
                    euler_line_general<D, N, NN, NP, FLUX>(pe, jl, re, stride, omega, tab);
                } else {
#pragma unroll
                    for (int a = 0; a < N; ++a) {
                        const float2 v01 = accp[a][0].value(), v23 = accp[a][1].value();
                        re[0 * NN + a * stride] = omega * v01.x;
                        re[1 * NN + a * stride] = omega * v01.y;
                        re[2 * NN + a * stride] = omega * v23.x;
                        re[3 * NN + a * stride] = omega * v23.y;
                        if constexpr (D == 3) re[4 * NN + a * stride] = (PH ? omega + omega : omega) * acc4[a].value();
                    }
                }
            } else {
                KahanF acc[N][NVAR];
#pragma unroll
                for (int a = 0; a < N; ++a) acc[a][0].zero();
                const auto je = sJF + (el * D + m) * NN + base;
                float uu[N], Sm[N];
#pragma unroll
                for (int a = 0; a < N; ++a) { uu[a] = pe[a * stride]; Sm[a] = je[a * stride]; }
#pragma unroll
                for (int a = 0; a < N; ++a) {
#pragma unroll
                    for (int b = a + 1; b < N; ++b) {
                        const float F = (uu[a] * uu[a] + uu[a] * uu[b] + uu[b] * uu[b]) * (1.0f / 6.0f) * (Sm[a] + Sm[b]);
                        acc[a][0].add_prod(tab.Q1[a * N + b], F);
                        acc[b][0].add_prod(tab.Q1[b * N + a], F);
                    }
                    const float qaa = tab.Q1[a * N + a];
                    if (qaa != 0.0f) acc[a][0].add_prod(qaa, uu[a] * uu[a] * Sm[a]);
                }
                const auto re = sR + (size_t)m * EPB * U_EL + el * U_EL + base;
#pragma unroll
                for (int a = 0; a < N; ++a) re[a * stride] = omega * acc[a][0].value();
            }
        }
    }
}

// The directions' slices summed in a fixed order into r (coalesced).
template <class S, int D>
__device__ __forceinline__ void fp32_block_store(BPtr<const float> sR, BPtr<float> gR, int ne, int tid, int nthreads) {
    constexpr int EPB = S::EPB, U_EL = S::U_EL;
    for (int s2 = tid; s2 < ne * U_EL; s2 += nthreads) {
        float t = sR[s2] + sR[EPB * U_EL + s2];
        if constexpr (D == 3) t += sR[2 * EPB * U_EL + s2];
        gR[s2] = t;
    }
}

// FP32 basis-transform pass of the persistent kernel: basis_pass with, for
// NSUM > 1 (backward pass 0), the input summed in a fixed order over NSUM
// slices `slice` floats apart (the directions' residuals, in the order of the
// nodal store).  (Packing two element-variables into FP32x2 lanes measured
// 6 % slower at p = 4.)
template <int D, int N, bool TRANSPOSE, int ROLE = kPassPlain, int NSUM = 1>
__device__ __forceinline__ void basis_pass_f(BPtr<const float> in, BPtr<float> out, int m, int nq,
                                             const BasisTab<float> &bt, int tid, int nthreads,
                                             BPtr<const float> coef = nullptr, int slice = 0) {
    constexpr int NN = ipow(N, D), NLINE = ipow(N, D - 1);
    const int stride = m == 0 ? 1 : (m == 1 ? N : N * N);
    for (int t = tid; t < nq * NLINE; t += nthreads) {
        const int q = t / NLINE, l = t - q * NLINE;
        int base;
        if constexpr (D == 3) base = m == 0 ? N * l : (m == 1 ? l % N + N * N * (l / N) : l);
        else base = m == 0 ? N * l : l;
        const auto src = in + q * NN + base;
        float x[N];
#pragma unroll
        for (int b = 0; b < N; ++b) {
            float a = src[b * stride];
#pragma unroll
            for (int k = 1; k < NSUM; ++k) a += src[k * slice + b * stride];
            x[b] = a;
        }
        if constexpr (ROLE == kPassFirst) {
            if (bt.const_mode && base == 0) x[0] = 0.0f;
        }
        float c = 0.0f;
        if constexpr (ROLE == kPassLast) {
            if (bt.const_mode) c = coef[q * NN] * bt.c0;
        }
        const auto dst = out + q * NN + base;
#pragma unroll
        for (int a = 0; a < N; ++a) {
            float acc = 0.0f;
#pragma unroll
            for (int b = 0; b < N; ++b) acc = fmaf(TRANSPOSE ? bt.V[b * N + a] : bt.V[a * N + b], x[b], acc);
            if constexpr (ROLE == kPassLast) acc += c;
            dst[a * stride] = acc;
        }
    }
}

// The persistent kernel's body.  MODAL: u holds basis coefficients and r
// receives V^T r_v; the transforms run in shared memory (the directions'
// residual slices serve as scratch), so HBM traffic is that of the nodal
// residual.
template <int D, int N, int FLUX, bool MODAL>
__device__ __forceinline__ void fp32_tma_body(const float *__restrict__ u, const double *__restrict__ Ja,
                                              float *__restrict__ r, int64_t n_elem, const OpTab<float> &tab,
                                              int *__restrict__ err, int aligned_bases, const BasisTab<float> *bt) {
    using S = TmaShape<D, N, FLUX>;
    constexpr int NN = S::NN, NLINE = S::NLINE, NVAR = S::NVAR, NP = S::NP, NJ = S::NJ, EPB = S::EPB;
    constexpr int U_EL = S::U_EL, J_EL = S::J_EL;
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    const auto rawU = SFH_BP(reinterpret_cast<float *>(sm + S::OFF_U), S::RAWU_BYTES / 4, err);
    const auto rawJ = SFH_BP(reinterpret_cast<double *>(sm + S::OFF_J), S::RAWJ_BYTES / 8, err);
    const auto sP = SFH_BP(reinterpret_cast<float *>(sm + S::OFF_P), EPB * NP * NN, err);
    const auto sJF = SFH_BP(reinterpret_cast<float *>(sm + S::OFF_JF), EPB * S::JF_EL, err);
    const auto sR = SFH_BP(reinterpret_cast<float *>(sm + S::OFF_R), D * EPB * U_EL, err);
    // u, Ja and r over their whole extents (bytes of u and Ja for the bulk copies)
    const auto gu = SFH_BP(u, n_elem * U_EL, err);
    const auto gJ = SFH_BP(Ja, n_elem * J_EL, err);
    const auto gr = SFH_BP(r, n_elem * U_EL, err);
    const auto gUb = SFH_BP(reinterpret_cast<const char *>(u), n_elem * U_EL * 4, err);
    const auto gJb = SFH_BP(reinterpret_cast<const char *>(Ja), n_elem * J_EL * 8, err);
    __shared__ int s_abort;

    const int tid = threadIdx.x;
    const int64_t nblk = (n_elem + EPB - 1) / EPB;
    if ((int64_t)blockIdx.x >= nblk) return;
    if (tid == 0) {
        mbar_init(bar, 1);
        s_abort = 0;
        fence_proxy_async_smem();
    }
    __syncthreads();

    uint32_t phase = 0;
    int64_t blk = blockIdx.x;
    BlockPlan cur = plan_block<S>(blk, n_elem, u, Ja, aligned_bases != 0);
    if (tid == 0 && cur.tma) {
        mbar_arrive_expect_tx(bar, cur.bytesU + cur.bytesJ);
        bulk_load_ck(rawU, bp_at(gUb, cur.srcU), cur.bytesU, bar);
        bulk_load_ck(rawJ, bp_at(gJb, cur.srcJ), cur.bytesJ, bar);
    }

    for (; blk < nblk; blk += gridDim.x) {
        const int ne = cur.ne;
        // ---- 1. raw data of this block
        if (cur.tma) {
            if (!mbar_wait_bounded(bar, phase, 2000000000ull)) s_abort = 1;
            phase ^= 1u;
        } else {
            const auto gU = gu + cur.e0 * U_EL;
            const auto gJe = gJ + cur.e0 * J_EL;
            for (int s = tid; s < ne * U_EL; s += blockDim.x) rawU[s] = gU[s];
            for (int s = tid; s < ne * J_EL; s += blockDim.x) rawJ[s] = gJe[s];
        }
        __syncthreads();
        if (s_abort) {
            if (tid == 0) {
                atomicOr(err, kErrTimeout);
                mbar_wait_bounded(bar, phase ^ 1u, 1000000000ull);
                bulk_wait_all();
            }
            return;
        }

        // ---- 2. (modal: nodal values u_v = V u_hat into the last residual
        //      slice) primitives and FP32 metrics
        BPtr<const float> uin = rawU + cur.offU;
        if constexpr (MODAL) {
            const auto s0 = sR, s1 = sR + EPB * U_EL, s2 = sR + 2 * EPB * U_EL;
            basis_pass_f<D, N, false, kPassFirst>(uin, s0, 0, ne * NVAR, *bt, tid, S::THREADS);
            __syncthreads();
            if constexpr (D == 3) {
                basis_pass_f<D, N, false>(s0, s1, 1, ne * NVAR, *bt, tid, S::THREADS);
                __syncthreads();
                basis_pass_f<D, N, false, kPassLast>(s1, s2, 2, ne * NVAR, *bt, tid, S::THREADS, uin);
            } else {
                basis_pass_f<D, N, false, kPassLast>(s0, s1, 1, ne * NVAR, *bt, tid, S::THREADS, uin);
            }
            __syncthreads();
            uin = D == 3 ? s2 : s1;
        }
        const int bad = fp32_block_convert<S, D, N, FLUX>(uin, rawJ + cur.offJ, ne, sP, sJF, tid, S::THREADS);
        if (bad) atomicOr(err, bad);
        __syncthreads();

        // ---- 3. prefetch the next block into the raw buffers
        const int64_t nxt = blk + gridDim.x;
        BlockPlan nx = cur;
        if (nxt < nblk) nx = plan_block<S>(nxt, n_elem, u, Ja, aligned_bases != 0);
        if (tid == 0 && nxt < nblk && nx.tma) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, nx.bytesU + nx.bytesJ);
            bulk_load_ck(rawU, bp_at(gUb, nx.srcU), nx.bytesU, bar);
            bulk_load_ck(rawJ, bp_at(gJb, nx.srcJ), nx.bytesJ, bar);
        }

        // ---- 4. line sweeps, all directions at once
        fp32_block_sweep<S, D, N, FLUX>(tid, ne, sP, sJF, sR, tab);
        __syncthreads();

        // ---- 5. sum the directions in a fixed order and store r (modal:
        //      r_v into slice 0, then r_hat = V^T r_v pass by pass)
        if constexpr (MODAL) {
            // pass 0 sums the directions' slices (same order as the nodal
            // store) into the free primitive buffer
            const auto s0 = sR;
            const auto gR = gr + cur.e0 * U_EL;
            basis_pass_f<D, N, true, kPassPlain, D>(sR, sP, 0, ne * NVAR, *bt, tid, S::THREADS, nullptr,
                                                     EPB * U_EL);
            __syncthreads();
            if constexpr (D == 3) {
                basis_pass_f<D, N, true>(sP, s0, 1, ne * NVAR, *bt, tid, S::THREADS);
                __syncthreads();
                basis_pass_f<D, N, true>(s0, gR, 2, ne * NVAR, *bt, tid, S::THREADS);
            } else {
                basis_pass_f<D, N, true>(sP, gR, 1, ne * NVAR, *bt, tid, S::THREADS);
            }
        } else {
            fp32_block_store<S, D>(sR, gr + cur.e0 * U_EL, ne, tid, S::THREADS);
        }
        cur = nx;
    }
}

template <int D, int N, int FLUX>
__global__ void __launch_bounds__(TmaShape<D, N, FLUX>::THREADS) __maxnreg__((TmaShape<D, N, FLUX>::MAXREG))
volume_fp32_tma_kernel(const float *__restrict__ u, const double *__restrict__ Ja, float *__restrict__ r,
                       int64_t n_elem, const __grid_constant__ OpTab<float> tab, int *__restrict__ err,
                       int aligned_bases) {
    fp32_tma_body<D, N, FLUX, false>(u, Ja, r, n_elem, tab, err, aligned_bases, nullptr);
}

template <int D, int N, int FLUX>
__global__ void __launch_bounds__(TmaShape<D, N, FLUX>::THREADS) __maxnreg__((TmaShape<D, N, FLUX>::MAXREG))
volume_fp32_tma_modal_kernel(const float *__restrict__ u, const double *__restrict__ Ja, float *__restrict__ r,
                             int64_t n_elem, const __grid_constant__ OpTab<float> tab, int *__restrict__ err,
                             int aligned_bases, const __grid_constant__ BasisTab<float> bt) {
    fp32_tma_body<D, N, FLUX, true>(u, Ja, r, n_elem, tab, err, aligned_bases, &bt);
}

// grid: one resident CTA per SM slot (persistent); occupancy is queried once
// per device.  bt != nullptr selects the modal kernel.
template <int D, int N, int FLUX, bool MODAL = false>
cudaError_t launch_volume_fp32_tma(const void *u, const double *Ja, void *r, int64_t n_elem, const OpTab<float> &tab,
                                   int *err, cudaStream_t stream, const BasisTab<float> *bt = nullptr) {
    using S = TmaShape<D, N, FLUX>;
    static_assert(S::SMEM <= 227 * 1024, "shared memory");
    static LaunchCache cache;
    int per_sm = 0, sms = 0;
    const int aligned = ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(Ja) |
                          reinterpret_cast<uintptr_t>(r)) & 15) == 0;
    const int64_t nblk = (n_elem + S::EPB - 1) / S::EPB;
    if constexpr (MODAL) {
        auto kern = volume_fp32_tma_modal_kernel<D, N, FLUX>;
        const cudaError_t e0 = persistent_slots(kern, S::THREADS, S::SMEM, cache, per_sm, sms);
        if (e0 != cudaSuccess) return e0;
        const int64_t grid = nblk < (int64_t)sms * per_sm ? nblk : (int64_t)sms * per_sm;
        kern<<<(unsigned)grid, S::THREADS, S::SMEM, stream>>>(static_cast<const float *>(u), Ja,
                                                             static_cast<float *>(r), n_elem, tab, err, aligned, *bt);
    } else {
        auto kern = volume_fp32_tma_kernel<D, N, FLUX>;
        const cudaError_t e0 = persistent_slots(kern, S::THREADS, S::SMEM, cache, per_sm, sms);
        if (e0 != cudaSuccess) return e0;
        const int64_t grid = nblk < (int64_t)sms * per_sm ? nblk : (int64_t)sms * per_sm;
        kern<<<(unsigned)grid, S::THREADS, S::SMEM, stream>>>(static_cast<const float *>(u), Ja,
                                                             static_cast<float *>(r), n_elem, tab, err, aligned);
    }
    return cudaGetLastError();
}

}  // namespace sfh
