// sfh_volume_ws.cuh -- warp-specialized persistent FP32 volume residual of
// the 3D Euler fluxes: FP32-Kahan and the mixed mode at n = 3..8.
//
// The arithmetic is that of the persistent line kernel (Eq. 3 with the Eq. 5
// operators: one unordered line pair per flux evaluation, scattered to both
// endpoints with Q1[a][b] and Q1[b][a], compensated line sums, directions
// summed in a fixed order), so the two produce the same bits.  What differs
// is how the work is laid out on an SM:
//   * one CTA per SM, two roles.  Sweep warps (up to twelve) own one
//     (direction, element, line) each and run the pair loops; four service
//     warps (two at n >= 7) stage the element blocks (1D bulk copies,
//     mbarrier completion), compute the primitives of every node and store
//     the residual;
//   * FP32-Kahan at n = 3..6 splits the registers between the roles
//     (setmaxnreg): the service warpgroup gives back registers it does not
//     need and the three sweep warpgroups take them, 152 a thread at n = 5, 6
//     and 144 at n = 3, 4 instead of the 128 that sixteen warps leave;
//   * element blocks rotate through two sets of buffers (raw u and Ja,
//     primitives, the directions' residual slices; one residual buffer at
//     n >= 7), and the roles hand
//     blocks to each other through mbarriers: the service warps prepare
//     block k + 1 and store block k - 1 while the sweep warps work on block
//     k, so neither role waits at a CTA-wide barrier;
//   * the block size is picked so that the line tasks fill the sweep warps
//     (375 of 384 lanes at n = 5, all 384 at n = 4);
//   * each sweep thread converts its line's FP64 metric rows to FP32 itself
//     (integer field arithmetic on the staged FP64 values), so the metric
//     never makes a second trip through shared memory.  Metric values
//     outside the FP32 modes' range (non-finite, or |Ja| >= 2^126) set the
//     metric bit of the error word.
// Every wait is bounded (2 s, or sooner once another thread has given up);
// a wait that gives up sets the timeout bit and the CTA leaves after the
// copies it issued have landed.
#pragma once

#include "sfh_volume_tma.cuh"

namespace sfh {

// FP32-Kahan: n = 3..8.  At n = 6 the line body fits the 152 registers of
// the split (it spilled under the 128 of sixteen warps: 273 against 310 us
// on 32^3 elements, 330 us on the thread-per-line kernel).  At n = 7 two elements per
// block with ten sweep warps and two service warps beat the row kernel at
// every mesh size (604 against 877 us on 32^3 elements, 104 against 119 us
// on 16^3).  At n = 8 (one element per block) the row kernel stays faster
// for Ranocha's flux on small meshes (146 against 168 us on 16^3 Gauss
// elements; 1.075 against 1.062 ms on 32^3), so it keeps n = 8; Chandrashekar's
// flux has no row kernel and takes this one.  Mixed mode: n = 3..8 (at n = 7,
// 8 its line body spills, and is still 2.6x faster than the thread-per-line
// kernel: 0.71 against 1.82 ms at n = 8 on 16^3 Gauss elements).
template <int D, int N, int FLUX>
constexpr bool use_ws_kernel() {
    return D == 3 && is_euler(FLUX) && N >= 3 && N <= 8;
}

template <int D, int N, int FLUX>
constexpr bool use_ws_mixed() {
    return D == 3 && is_euler(FLUX) && N >= 3 && N <= 8;
}

template <int D, int N, int FLUX, bool MIX = false>
struct WsShape {
    static constexpr int NN = ipow(N, D);
    static constexpr int NLINE = ipow(N, D - 1);
    static constexpr int NVAR = D + 2;
    static constexpr int U_EL = NVAR * NN;   // floats of u (and r) per element
    static constexpr int J_EL = D * D * NN;  // doubles of Ja per element
    // primitives as three float2 per node: (rho, beta), (v0/2, v1/2), (v2/2, p)
    // (FP32-Kahan with Ranocha's flux: (v2/2, p/2), see ws_line_sweep)
    static constexpr int P2_EL = 3 * NN;
    static constexpr int TASKS_EL = D * NLINE;
    // twelve sweep warps (three per sub-partition) also in the mixed mode:
    // its FP64 chains are latency-bound, and more warps beat more registers
    // per warp (653 against 763 us at p = 4 with eight warps of 168 registers)
    static constexpr int SVC_WARPS = N >= 7 ? 2 : 4, MAX_SWEEP_WARPS = 12;
    // residual buffers: two (the sweep of block k + 1 overlaps the store of
    // block k), one at n >= 7, where the shared memory it frees holds a second
    // element per block at n = 7; with two service warps the ten sweep warps
    // of that block keep 168 registers (n = 7 on 32^3 elements: 604 against
    // 767 us with one element per block and four service warps)
    static constexpr int RB = N >= 7 ? 1 : 2;
    static constexpr int SVC_THREADS = 32 * SVC_WARPS;
    static constexpr int RAW_EL = 4 * U_EL + 8 * J_EL;
    // double-buffered raw staging, primitives and residual slices (the mixed
    // mode adds an FP64 beta = rho / p per node)
    static constexpr int EL_BYTES = 2 * RAW_EL + 2 * 8 * P2_EL + RB * 4 * D * U_EL + (MIX ? 2 * 8 * NN : 0);
    static constexpr int HDR = 128;                       // mbarriers
    static constexpr int SMEM_MAX = 227 * 1024;
    static constexpr int SLACK = 4 * 48;                  // aligned-window slack of the four raw arrays
    static constexpr int epb_smem() { return (SMEM_MAX - HDR - SLACK) / EL_BYTES; }
    static constexpr int epb_lanes() { return 32 * MAX_SWEEP_WARPS / TASKS_EL; }
    static constexpr int EPB = epb_smem() < epb_lanes() ? epb_smem() : epb_lanes();
    static_assert(EPB >= 1, "one element must fit");
    static constexpr int TASKS = EPB * TASKS_EL;
    // register split between the roles (FP32-Kahan with four service warps
    // and at most twelve sweep warps; sweep warps padded to whole warpgroups,
    // the unit of setmaxnreg).  The shares add up to at most the registers
    // the CTA is launched with, MAXREG a thread, so neither role can wait on
    // registers that do not exist; the launch checks that the compiled
    // kernel has MAXREG.  Measured on 32^3 elements (same bits): n = 5 131.5
    // (64/144: 133.3) against 135.9 us unsplit; n = 6 272.8 (277.9) against
    // 309.7 us; n = 4 67.8 with 64/144 (74.0 with 56/152) against 70.6 us.
    // The mixed mode gains nothing from it (650 against 653 us at n = 5).
    static constexpr bool SPLIT = !MIX && SVC_WARPS == 4 && (TASKS + 127) / 128 == 3;
    static constexpr int SWEEP_WARPS = SPLIT ? 12 : (TASKS + 31) / 32;
    static constexpr int SWEEP_THREADS = 32 * SWEEP_WARPS;
    static constexpr int THREADS = SWEEP_THREADS + SVC_THREADS;
    // registers per thread: each of the SM's four sub-partitions holds the
    // registers of its warps (a quarter of the CTA's, rounded up) in its own
    // 16K-entry file; in units of 8
    static constexpr int WARPS_PER_SUB = (THREADS / 32 + 3) / 4;
    static constexpr int MAXREG = (16384 / (32 * WARPS_PER_SUB)) / 8 * 8 < 255 ? (16384 / (32 * WARPS_PER_SUB)) / 8 * 8 : 255;
    static constexpr int SVC_REG = N >= 5 ? 56 : 64, SWEEP_REG = N >= 5 ? 152 : 144;
    static_assert(!SPLIT || (MAXREG == 128 && SVC_REG % 8 == 0 && SWEEP_REG % 8 == 0 &&
                             SVC_REG * SVC_THREADS + SWEEP_REG * SWEEP_THREADS <= MAXREG * THREADS &&
                             SVC_REG * 32 + SWEEP_REG * 96 <= 16384),
                  "register split within the launch's registers (per CTA and per sub-partition)");
    static constexpr int up16(int x) { return (x + 15) / 16 * 16; }
    static constexpr int RAWU_BYTES = up16(EPB * U_EL * 4 + 16);   // + aligned-window slack
    static constexpr int RAWJ_BYTES = up16(EPB * J_EL * 8 + 16);
    static constexpr int RAW_BYTES = RAWU_BYTES + RAWJ_BYTES;
    static constexpr int OFF_RAW = HDR;                                   // raw[b]: u, then Ja
    static constexpr int OFF_P2 = OFF_RAW + 2 * RAW_BYTES;                 // P2[b]
    static constexpr int P2_BYTES = EPB * P2_EL * 8;
    static constexpr int OFF_R = up16(OFF_P2 + 2 * P2_BYTES);              // R[b]: [m][el][var][i]
    static constexpr int R_SLICE = EPB * U_EL;   // floats of one direction's residual slice
    static constexpr int R_BYTES = D * R_SLICE * 4;
    static constexpr int OFF_B64 = up16(OFF_R + RB * R_BYTES);              // B64[b]: [el][i] (mixed)
    static constexpr int B64_BYTES = MIX ? EPB * NN * 8 : 0;
    static constexpr size_t SMEM = (size_t)OFF_B64 + 2 * (size_t)B64_BYTES;
    static_assert(SMEM <= (size_t)SMEM_MAX, "shared memory");
    static_assert(OFF_RAW % 16 == 0 && RAWU_BYTES % 16 == 0 && RAW_BYTES % 16 == 0, "bulk-copy destinations");
};

// Completed phases of the barriers a raw buffer is published on (full[b]
// for bulk copies, copied[b] for plain loads): both roles replay the same
// block plans, so their counts agree.
struct RawPhases {
    uint32_t n[4] = {0, 0, 0, 0};   // [b * 2 + plain]
    __device__ __forceinline__ uint32_t next(int b, bool plain) {
        const int i = b * 2 + (plain ? 1 : 0);
        uint32_t v = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j == i) v = n[j]++;
        return v & 1u;
    }
};

// Bounded mbarrier wait that also gives up as soon as another thread of the
// CTA has set *abort.  A waiting thread sleeps in try_wait (20 us hint; it
// wakes when the phase completes), so waiting costs almost no issue slots;
// the limit and the abort flag are checked every 16 tries (at most ~0.3 ms
// apart).
__device__ __forceinline__ bool ws_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 0; it < (1u << 28); ++it) {
        if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
        if ((it & 15u) == 15u && (*abort || global_timer_ns() - t0 > 2000000000ull)) return false;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// One Euler line from scratch, with the logarithm for pairs outside the
// series band (primitives as float2 triples, p halved as in ws_line_sweep for
// Ranocha's flux; metric rows re-read from the
// staged FP64 values).  Out of line: it runs only for states with large
// jumps along a line.
template <int D, int N, int NN, int FLUX>
__device__ __noinline__ void ws_euler_line_general(BPtr<const float2> pe, BPtr<const double> je, BPtr<float> re,
                                                   int stride, float omega, const OpTab<float> &tab) {
    constexpr int NVAR = D + 2;
    static_assert(D == 3, "3D only");
    uint32_t hmax = 0;
#pragma unroll 1
    for (int a = 0; a < N; ++a) {
        KahanF acc[NVAR];
#pragma unroll
        for (int v = 0; v < NVAR; ++v) acc[v].zero();
        const float2 rba = pe[a * stride], h01a = pe[NN + a * stride], h2pa = pe[2 * NN + a * stride];
        const float hva[3] = {h01a.x, h01a.y, h2pa.x};
        float ja[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) ja[k] = d2f_int_track(je[k * NN + a * stride], hmax);
#pragma unroll 1
        for (int b = 0; b < N; ++b) {
            const float q = tab.Q1[a * N + b];
            if (q == 0.0f) continue;
            const float2 rbb = pe[b * stride], h01b = pe[NN + b * stride], h2pb = pe[2 * NN + b * stride];
            const float hvb[3] = {h01b.x, h01b.y, h2pb.x};
            float n[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) n[k] = ja[k] + d2f_int_track(je[k * NN + b * stride], hmax);
            float hna = 0.0f, hnb = 0.0f, hvv = 0.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k) { hna = fmaf(hva[k], n[k], hna); hnb = fmaf(hvb[k], n[k], hnb); hvv = fmaf(hva[k], hvb[k], hvv); }
            const float ra = rba.x, rb = rbb.x;
            const float pa = FLUX == kFluxEuler ? 2.0f * h2pa.y : h2pa.y, pb = FLUX == kFluxEuler ? 2.0f * h2pb.y : h2pb.y;
            const float Lr = ln_mean(ra, rb), iLb = inv_ln_mean(rba.y, rbb.y);
            float F[NVAR];
            const float frho = Lr * (hna + hnb);
            const float pavg = FLUX == kFluxEulerCh ? (ra + rb) * rcp_approx(rba.y + rbb.y) : 0.5f * (pa + pb);
            const float work = FLUX == kFluxEulerCh ? pavg * (hna + hnb) : fmaf(pa, hnb, pb * hna);
            F[0] = frho;
#pragma unroll
            for (int k = 0; k < 3; ++k) F[1 + k] = fmaf(frho, hva[k] + hvb[k], pavg * n[k]);
            F[4] = fmaf(frho, fmaf(2.0f, hvv, iLb * (float)(1.0 / (kGamma - 1.0))), work);
#pragma unroll
            for (int v = 0; v < NVAR; ++v) acc[v].add_prod(q, F[v]);
        }
#pragma unroll
        for (int v = 0; v < NVAR; ++v) re[v * NN + a * stride] = omega * acc[v].value();
    }
}

// The line sweep of one (direction m, element, line l): pair loop over the
// line's nodes with compensated sums, results scaled by omega_m into the
// direction's residual slice.  pe: the element's primitives (float2 triples,
// [3][NN]); je: the element's staged FP64 metric, [m][k][NN].  Returns the
// largest high word of the metric magnitudes met (range check).
template <int D, int N, int FLUX>
__device__ __forceinline__ uint32_t ws_line_sweep(int m, int l, BPtr<const float2> pe0, BPtr<const double> je0,
                                                  BPtr<float> re0, const OpTab<float> &tab) {
    constexpr int NN = ipow(N, D), NLINE = ipow(N, D - 1), NVAR = D + 2;
    static_assert(D == 3 && NLINE == N * N, "3D only");
    const int stride = m == 0 ? 1 : (m == 1 ? N : N * N);
    const int o0 = l % N, o1 = l / N;
    const int base = m == 0 ? N * l : (m == 1 ? o0 + N * N * o1 : l);
    const float omega = tab.w[o0] * tab.w[o1];
    const auto pe = pe0 + base;
    const auto je = je0 + m * D * NN + base;
    const auto re = re0 + base;

    uint32_t hmax = 0;
    // node data in FP32x2 lanes where the pair arithmetic pairs them:
    // (rho, beta), (v0/2, v1/2), and the metric row (Ja_0, Ja_1) of direction m
    float2 rb[N], h01[N], j01[N];
    float h2[N], p[N], j2[N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
        rb[a] = pe[a * stride];
        h01[a] = pe[NN + a * stride];
        const float2 h2p = pe[2 * NN + a * stride];
        h2[a] = h2p.x;
        p[a] = h2p.y;
        j01[a].x = d2f_int_track(je[0 * NN + a * stride], hmax);
        j01[a].y = d2f_int_track(je[1 * NN + a * stride], hmax);
        j2[a] = d2f_int_track(je[2 * NN + a * stride], hmax);
    }
    // compensated sums per node: (m0, m1) and (m2, E) flux pairs packed,
    // the density flux alone
    constexpr int NPAIR = NVAR / 2;
    KahanF2 accp[N][NPAIR];
    KahanF acc4[N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
#pragma unroll
        for (int v = 0; v < NPAIR; ++v) accp[a][v].zero();
        acc4[a].zero();
    }
    // Ranocha's flux: the node pass stores p/2, so that the mean {p} is one
    // addition.  The energy flux is then formed at half scale: the pressure
    // work with p/2 in place of p, the inverse beta mean from the series
    // with halved coefficients, and v_a.v_b / 2 in place of 2 (v_a/2).(v_b/2).
    // Each step is an exact power-of-two scaling of the full-scale
    // arithmetic, so the energy sum is exactly half of the full-scale one;
    // the store scales it by 2 omega.
    constexpr bool PH = FLUX == kFluxEuler;
    float umax = 0.0f;   // largest u_rho + u_beta of the line's pairs
    // S(u)/2 (rho mean) and P(u) 2/(gamma-1) (inverse beta mean; PH: half of
    // it) as one packed Horner chain
    const float cg = (float)((PH ? 1.0 : 2.0) / (kGamma - 1.0));
    const float2 c0 = f2(0.5f, cg), c1 = f2(0.5f * (-1.0f / 3.0f), cg * (1.0f / 3.0f));
    const float2 c2 = f2(0.5f * (-4.0f / 45.0f), cg * (1.0f / 5.0f));
    const float2 c3 = f2(0.5f * (-44.0f / 945.0f), cg * (1.0f / 7.0f));
#pragma unroll
    for (int a = 0; a < N; ++a) {
#pragma unroll
        for (int b = a + 1; b < N; ++b) {
            // metric sum Ja^m(a) + Ja^m(b) and velocity sums, two lanes at once
            const float2 n01 = add2(j01[a], j01[b]);
            const float n2 = j2[a] + j2[b];
            const float2 hs01 = add2(h01[a], h01[b]);
            float hna = h01[a].x * n01.x, hnb = h01[b].x * n01.x, hvv = h01[a].x * h01[b].x;
            hna = fmaf(h01[a].y, n01.y, hna);
            hnb = fmaf(h01[b].y, n01.y, hnb);
            hvv = fmaf(h01[a].y, h01[b].y, hvv);
            hna = fmaf(h2[a], n2, hna);
            hnb = fmaf(h2[b], n2, hnb);
            hvv = fmaf(h2[a], h2[b], hvv);
            // both logarithmic means at once (.x: rho, .y: beta) by the series
            // in u = ((a-b)/(a+b))^2 with the hardware reciprocal of a + b
            const float2 d2 = sub2(rb[a], rb[b]), s2 = add2(rb[a], rb[b]);
            const float2 r2 = f2(rcp_approx(s2.x), rcp_approx(s2.y));
            const float2 t2 = mul2(d2, r2);
            const float2 u2 = mul2(t2, t2);
            float2 h = fma2(u2, c3, c2);
            h = fma2(u2, h, c1);
            h = fma2(u2, h, c0);
            umax = fmaxf(umax, u2.x + u2.y);
            const float2 m2 = mul2(f2(s2.x, r2.y), h);   // ({rho}_ln, 1/((g-1){beta}_ln))
            const float frho = m2.x * (hna + hnb);
            const float pavg = FLUX == kFluxEulerCh ? s2.x * r2.y : (PH ? p[a] + p[b] : 0.5f * (p[a] + p[b]));
            const float work = FLUX == kFluxEulerCh ? pavg * (hna + hnb) : fmaf(p[a], hnb, p[b] * hna);
            const float2 F12 = fma2(f2s(frho), hs01, mul2(f2s(pavg), n01));
            const float F3 = fmaf(frho, h2[a] + h2[b], pavg * n2);
            const float K = PH ? hvv + m2.y : fmaf(2.0f, hvv, m2.y);
            const float FE = fmaf(frho, K, work);
            const float2 F34 = f2(F3, FE);
            const float qab = tab.Q1[a * N + b], qba = tab.Q1[b * N + a];
            const float2 qa2 = f2s(qab), qb2 = f2s(qba);
            accp[a][0].add_prod(qa2, F12);
            accp[b][0].add_prod(qb2, F12);
            accp[a][1].add_prod(qa2, F34);
            accp[b][1].add_prod(qb2, F34);
            acc4[a].add_prod(qab, frho);
            acc4[b].add_prod(qba, frho);
        }
        const float qaa = tab.Q1[a * N + a];
        if (qaa != 0.0f) {
            // physical flux f(u_a) . (2 Ja^m(a))
            const float n[D] = {2.0f * j01[a].x, 2.0f * j01[a].y, 2.0f * j2[a]};
            const float hva[D] = {h01[a].x, h01[a].y, h2[a]};
            float hn = hva[0] * n[0], hv2 = hva[0] * hva[0];
#pragma unroll
            for (int k = 1; k < D; ++k) { hn = fmaf(hva[k], n[k], hn); hv2 = fmaf(hva[k], hva[k], hv2); }
            float F[D + 2];
            const float frho = 2.0f * rb[a].x * hn;
            const float pf = PH ? p[a] + p[a] : p[a];
            F[0] = frho;
#pragma unroll
            for (int k = 0; k < D; ++k) F[1 + k] = fmaf(2.0f * frho, hva[k], pf * n[k]);
            if constexpr (PH) F[D + 1] = fmaf(frho, hv2, pf * hn * (float)(kGamma / (kGamma - 1.0)));
            else F[D + 1] = fmaf(frho, 2.0f * hv2, 2.0f * pf * hn * (float)(kGamma / (kGamma - 1.0)));
            const float2 qq = f2s(qaa);
            accp[a][0].add_prod(qq, f2(F[1], F[2]));
            accp[a][1].add_prod(qq, f2(F[3], F[4]));
            acc4[a].add_prod(qaa, F[0]);
        }
    }
    // also false for a NaN maximum (fmaxf drops NaN operands; the domain
    // flag of the node pass reports the state)
    if (__builtin_expect(!(umax < 1e-2f), 0)) {
        ws_euler_line_general<D, N, NN, FLUX>(pe, je, re, stride, omega, tab);
    } else {
#pragma unroll
        for (int a = 0; a < N; ++a) {
            const float2 v12 = accp[a][0].value(), v34 = accp[a][1].value();
            re[0 * NN + a * stride] = omega * acc4[a].value();
            re[1 * NN + a * stride] = omega * v12.x;
            re[2 * NN + a * stride] = omega * v12.y;
            re[3 * NN + a * stride] = omega * v34.x;
            re[4 * NN + a * stride] = (PH ? omega + omega : omega) * v34.y;
        }
    }
    return hmax;
}

// One Euler line from scratch in the mixed mode, with the logarithm (FP32)
// for pairs outside the series band: metric pair sums in FP64 as in the fast
// path; inside the band the means of ws_mix_means.  Out of line (rare).
template <int D, int N, int NN, int FLUX>
__device__ __noinline__ void ws_mix_line_general(BPtr<const float2> pe, BPtr<const double> je, BPtr<const double> be,
                                                 BPtr<float> re, int stride, float omega, const OpTab<float> &tab);

// The two logarithmic means of a pair in the mixed mode (inside the series
// band): FP64 where FP32 would lose accuracy, FP32 where it cannot.
//   {rho}_ln = (s/2) S(u): s = rho_a + rho_b summed in FP64 (exact for FP32
//     rho) and the product (s/2) S formed in FP64;
//   1/((g-1){beta}_ln) = (2/(g-1)) P(u) / s: s = beta_a + beta_b from the FP64
//     betas, 1/s from the FP32 hardware seed and one FP64 Newton step (error
//     about 2^-46), the product with P formed in FP64.
// The series S and P and their argument u = ((a-b)/(a+b))^2 stay in FP32:
// S, P lie in [0.99, 1.01] inside the band, so a relative error e in u moves
// them by at most u e / 3 < 1e-2 e -- the FP32 rounding of u (a few ulp) and
// of the FP32 betas entering it (an ulp of beta against |beta_a - beta_b|,
// which enters u squared) stay far below an FP32 ulp of the results.
// h: (S/2, P 2/(g-1)) from the FP32 Horner chain; r2y: FP32 seed of 1/s_beta.
__device__ __forceinline__ float2 ws_mix_means(float rho_a, float rho_b, double beta_a, double beta_b, float2 h,
                                               float r2y) {
    const double sr = f2d_pos(rho_a) + f2d_pos(rho_b);
    const double sb = beta_a + beta_b;
    const double r0 = f2d_pos(r2y);
    const double rb = fma(r0, fma(-sb, r0, 1.0), r0);
    return f2(d2f_pos(sr * f2d_pos(h.x)), d2f_pos(rb * f2d_pos(h.y)));
}

// The mixed-mode line sweep (precision mode "fp32 with FP64 islands"): the
// arithmetic of ws_line_sweep with the metric pair sums Ja^m(a) + Ja^m(b)
// formed in FP64 (then rounded to FP32) and the logarithmic means of
// ws_mix_means.  be0: the element's FP64 betas [NN].
template <int D, int N, int FLUX>
__device__ __forceinline__ uint32_t ws_line_sweep_mix(int m, int l, BPtr<const float2> pe0, BPtr<const double> je0,
                                                      BPtr<const double> be0, BPtr<float> re0,
                                                      const OpTab<float> &tab) {
    constexpr int NN = ipow(N, D), NLINE = ipow(N, D - 1), NVAR = D + 2;
    static_assert(D == 3 && NLINE == N * N, "3D only");
    const int stride = m == 0 ? 1 : (m == 1 ? N : N * N);
    const int o0 = l % N, o1 = l / N;
    const int base = m == 0 ? N * l : (m == 1 ? o0 + N * N * o1 : l);
    const float omega = tab.w[o0] * tab.w[o1];
    const auto pe = pe0 + base;
    const auto je = je0 + m * D * NN + base;
    const auto be = be0 + base;
    const auto re = re0 + base;

    uint32_t hmax = 0;
    float2 rb[N], h01[N];
    float h2[N], p[N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
        rb[a] = pe[a * stride];
        h01[a] = pe[NN + a * stride];
        const float2 h2p = pe[2 * NN + a * stride];
        h2[a] = h2p.x;
        p[a] = h2p.y;
#pragma unroll
        for (int k = 0; k < D; ++k) hmax = max(hmax, abs_hi(je[k * NN + a * stride]));
    }
    constexpr int NPAIR = NVAR / 2;
    KahanF2 accp[N][NPAIR];
    KahanF acc4[N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
#pragma unroll
        for (int v = 0; v < NPAIR; ++v) accp[a][v].zero();
        acc4[a].zero();
    }
    float umax = 0.0f;
    const float cg = (float)(2.0 / (kGamma - 1.0));
    const float2 c0 = f2(0.5f, cg), c1 = f2(0.5f * (-1.0f / 3.0f), cg * (1.0f / 3.0f));
    const float2 c2 = f2(0.5f * (-4.0f / 45.0f), cg * (1.0f / 5.0f));
    const float2 c3 = f2(0.5f * (-44.0f / 945.0f), cg * (1.0f / 7.0f));
#pragma unroll
    for (int a = 0; a < N; ++a) {
        const double ja0 = je[a * stride], ja1 = je[NN + a * stride], ja2 = je[2 * NN + a * stride];
        const double ba = be[a * stride];
        // the FP64 island of row a first, for every partner b > a: the FP64
        // pipe is narrow, so its chains of all of a row's pairs are issued
        // together and overlap (the FP32 series feeding them are cheap)
        float2 nb01[N], mb[N];
        float nb2[N], pb[N];
#pragma unroll
        for (int b = a + 1; b < N; ++b) {
            nb01[b] = f2(d2f_int(ja0 + je[b * stride]), d2f_int(ja1 + je[NN + b * stride]));
            nb2[b] = d2f_int(ja2 + je[2 * NN + b * stride]);
            const float2 d2 = sub2(rb[a], rb[b]), s2 = add2(rb[a], rb[b]);
            const float2 r2 = f2(rcp_approx(s2.x), rcp_approx(s2.y));
            const float2 t2 = mul2(d2, r2);
            const float2 u2 = mul2(t2, t2);
            float2 h = fma2(u2, c3, c2);
            h = fma2(u2, h, c1);
            h = fma2(u2, h, c0);
            umax = fmaxf(umax, u2.x + u2.y);
            mb[b] = ws_mix_means(rb[a].x, rb[b].x, ba, be[b * stride], h, r2.y);
            pb[b] = FLUX == kFluxEulerCh ? s2.x * r2.y : 0.5f * (p[a] + p[b]);
        }
#pragma unroll
        for (int b = a + 1; b < N; ++b) {
            const float2 n01 = nb01[b];
            const float n2 = nb2[b];
            const float2 hs01 = add2(h01[a], h01[b]);
            float hna = h01[a].x * n01.x, hnb = h01[b].x * n01.x, hvv = h01[a].x * h01[b].x;
            hna = fmaf(h01[a].y, n01.y, hna);
            hnb = fmaf(h01[b].y, n01.y, hnb);
            hvv = fmaf(h01[a].y, h01[b].y, hvv);
            hna = fmaf(h2[a], n2, hna);
            hnb = fmaf(h2[b], n2, hnb);
            hvv = fmaf(h2[a], h2[b], hvv);
            const float2 m2 = mb[b];
            const float frho = m2.x * (hna + hnb);
            const float pavg = pb[b];
            const float work = FLUX == kFluxEulerCh ? pavg * (hna + hnb) : fmaf(p[a], hnb, p[b] * hna);
            float2 F01, F23;
            F01.x = frho;
            F01.y = fmaf(frho, hs01.x, pavg * n01.x);
            F23.x = fmaf(frho, hs01.y, pavg * n01.y);
            F23.y = fmaf(frho, h2[a] + h2[b], pavg * n2);
            const float K = fmaf(2.0f, hvv, m2.y);
            const float FE = fmaf(frho, K, work);
            const float qab = tab.Q1[a * N + b], qba = tab.Q1[b * N + a];
            const float2 qa2 = f2s(qab), qb2 = f2s(qba);
            accp[a][0].add_prod(qa2, F01);
            accp[b][0].add_prod(qb2, F01);
            accp[a][1].add_prod(qa2, F23);
            accp[b][1].add_prod(qb2, F23);
            acc4[a].add_prod(qab, FE);
            acc4[b].add_prod(qba, FE);
        }
        const float qaa = tab.Q1[a * N + a];
        if (qaa != 0.0f) {
            // physical flux f(u_a) . (2 Ja^m(a)): fl32(2 Ja) = 2 fl32(Ja) exactly
            const float n[D] = {2.0f * d2f_int(ja0), 2.0f * d2f_int(ja1), 2.0f * d2f_int(ja2)};
            const float hva[D] = {h01[a].x, h01[a].y, h2[a]};
            float hn = hva[0] * n[0], hv2 = hva[0] * hva[0];
#pragma unroll
            for (int k = 1; k < D; ++k) { hn = fmaf(hva[k], n[k], hn); hv2 = fmaf(hva[k], hva[k], hv2); }
            float F[D + 2];
            const float frho = 2.0f * rb[a].x * hn;
            F[0] = frho;
#pragma unroll
            for (int k = 0; k < D; ++k) F[1 + k] = fmaf(2.0f * frho, hva[k], p[a] * n[k]);
            F[D + 1] = fmaf(frho, 2.0f * hv2, 2.0f * p[a] * hn * (float)(kGamma / (kGamma - 1.0)));
            const float2 qq = f2s(qaa);
            accp[a][0].add_prod(qq, f2(F[0], F[1]));
            accp[a][1].add_prod(qq, f2(F[2], F[3]));
            acc4[a].add_prod(qaa, F[4]);
        }
    }
    if (__builtin_expect(!(umax < 1e-2f), 0)) {
        ws_mix_line_general<D, N, NN, FLUX>(pe, je, be, re, stride, omega, tab);
    } else {
#pragma unroll
        for (int a = 0; a < N; ++a) {
            const float2 v01 = accp[a][0].value(), v23 = accp[a][1].value();
            re[0 * NN + a * stride] = omega * v01.x;
            re[1 * NN + a * stride] = omega * v01.y;
            re[2 * NN + a * stride] = omega * v23.x;
            re[3 * NN + a * stride] = omega * v23.y;
            re[4 * NN + a * stride] = omega * acc4[a].value();
        }
    }
    return hmax;
}

template <int D, int N, int NN, int FLUX>
__device__ __noinline__ void ws_mix_line_general(BPtr<const float2> pe, BPtr<const double> je, BPtr<const double> be,
                                                 BPtr<float> re, int stride, float omega, const OpTab<float> &tab) {
    constexpr int NVAR = D + 2;
    static_assert(D == 3, "3D only");
    const float cg = (float)(2.0 / (kGamma - 1.0));
#pragma unroll 1
    for (int a = 0; a < N; ++a) {
        KahanF acc[NVAR];
#pragma unroll
        for (int v = 0; v < NVAR; ++v) acc[v].zero();
        const float2 rba = pe[a * stride], h01a = pe[NN + a * stride], h2pa = pe[2 * NN + a * stride];
        const float hva[3] = {h01a.x, h01a.y, h2pa.x};
#pragma unroll 1
        for (int b = 0; b < N; ++b) {
            const float q = tab.Q1[a * N + b];
            if (q == 0.0f) continue;
            const float2 rbb = pe[b * stride], h01b = pe[NN + b * stride], h2pb = pe[2 * NN + b * stride];
            const float hvb[3] = {h01b.x, h01b.y, h2pb.x};
            float n[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) n[k] = d2f_int(je[k * NN + a * stride] + je[k * NN + b * stride]);
            float hna = 0.0f, hnb = 0.0f, hvv = 0.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k) { hna = fmaf(hva[k], n[k], hna); hnb = fmaf(hvb[k], n[k], hnb); hvv = fmaf(hva[k], hvb[k], hvv); }
            const float ra = rba.x, rb = rbb.x, pa = h2pa.y, pb = h2pb.y;
            // each mean by the mixed series inside the band, by FP32 logarithms outside
            const float dr = ra - rb, sr = ra + rb, dbt = rba.y - rbb.y, sbt = rba.y + rbb.y;
            float Lr, iK;
            if (dr * dr < (float)kLnBand * (sr * sr)) {
                const float t = dr * rcp_approx(sr);
                Lr = d2f_pos((f2d_pos(ra) + f2d_pos(rb)) * f2d_pos(0.5f * series_S(t * t)));
            } else {
                Lr = ln_mean(ra, rb);
            }
            if (dbt * dbt < (float)kLnBand * (sbt * sbt)) {
                const float r0f = rcp_approx(sbt), t = dbt * r0f;
                const double sb = be[a * stride] + be[b * stride], r0 = f2d_pos(r0f);
                const double r1 = fma(r0, fma(-sb, r0, 1.0), r0);
                iK = d2f_pos(r1 * f2d_pos(cg * series_P(t * t)));
            } else {
                iK = inv_ln_mean(rba.y, rbb.y) * (float)(1.0 / (kGamma - 1.0));
            }
            float F[NVAR];
            const float frho = Lr * (hna + hnb);
            const float pavg = FLUX == kFluxEulerCh ? (ra + rb) * rcp_approx(rba.y + rbb.y) : 0.5f * (pa + pb);
            const float work = FLUX == kFluxEulerCh ? pavg * (hna + hnb) : fmaf(pa, hnb, pb * hna);
            F[0] = frho;
#pragma unroll
            for (int k = 0; k < 3; ++k) F[1 + k] = fmaf(frho, hva[k] + hvb[k], pavg * n[k]);
            F[4] = fmaf(frho, fmaf(2.0f, hvv, iK), work);
#pragma unroll
            for (int v = 0; v < NVAR; ++v) acc[v].add_prod(q, F[v]);
        }
#pragma unroll
        for (int v = 0; v < NVAR; ++v) re[v * NN + a * stride] = omega * acc[v].value();
    }
}

// Primitives of node items [s0, s_end) step `step` of a block (u layout
// [el][var][i]) into float2 triples [el][3][i]; returns whether any node had
// rho <= 0 or p <= 0 (or NaN).  Same arithmetic as fp32_block_convert; PH
// stores p/2 in place of p (exact).
template <class S, int D, bool PH = false>
__device__ __forceinline__ bool ws_primitives(BPtr<const float> U, BPtr<float2> P2, int ne, int s0, int step,
                                              BPtr<double> B64 = nullptr) {
    constexpr int NN = S::NN, U_EL = S::U_EL;
    bool bad = false;
    for (int s = s0; s < ne * NN; s += step) {
        const int el = s / NN, i = s - el * NN;
        const auto ue = U + el * U_EL + i;
        const float rho = ue[0], E = ue[(D + 1) * NN];
        float ir = rcp_approx(rho);
        ir = fmaf(ir, fmaf(-rho, ir, 1.0f), ir);
        float ke = 0.0f, hv[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const float mk = ue[(1 + k) * NN];
            float vk = mk * ir;
            vk = fmaf(ir, fmaf(-rho, vk, mk), vk);
            hv[k] = 0.5f * vk;
            ke = fmaf(mk, vk, ke);
        }
        const float p = (float)(kGamma - 1.0) * fmaf(-0.5f, ke, E);
        float ip = rcp_approx(p);
        ip = fmaf(ip, fmaf(-p, ip, 1.0f), ip);
        float bt = rho * ip;
        bt = fmaf(ip, fmaf(-p, bt, rho), bt);
        const auto pe = P2 + el * 3 * NN + i;
        pe[0] = f2(rho, bt);
        pe[NN] = f2(hv[0], hv[1]);
        pe[2 * NN] = f2(hv[2], PH ? 0.5f * p : p);
        if (raw(B64)) {
            // mixed mode: beta = rho / p in FP64 (exact FP32 rho and p, the
            // FP32 reciprocal seed refined by one FP64 Newton step: ~2^-46)
            const double pd = f2d_pos(p), r0 = f2d_pos(ip);
            B64[el * NN + i] = f2d_pos(rho) * fma(r0, fma(-pd, r0, 1.0), r0);
        }
        bad |= !(rho > 0.0f && p > 0.0f);
    }
    return bad;
}

template <int D, int N, int FLUX, bool MIX>
__global__ void __launch_bounds__(WsShape<D, N, FLUX, MIX>::THREADS, 1) __maxnreg__((WsShape<D, N, FLUX, MIX>::MAXREG))
volume_fp32_ws_kernel(const float *__restrict__ u, const double *__restrict__ Ja, float *__restrict__ r,
                      int64_t n_elem, const __grid_constant__ OpTab<float> tab, int *__restrict__ err,
                      int aligned_bases) {
    using S = WsShape<D, N, FLUX, MIX>;
    constexpr int EPB = S::EPB, NLINE = S::NLINE, U_EL = S::U_EL, J_EL = S::J_EL;
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *full = reinterpret_cast<uint64_t *>(sm);   // raw[b] landed (bulk copy)
    uint64_t *ready = full + 2;                          // P2[b] holds the block's primitives
    uint64_t *swept = full + 4;                          // R[b] written, raw[b] and P2[b] read
    uint64_t *stored = full + 6;                         // R[b] stored (one buffer: stored[0] only)
    uint64_t *copied = full + 8;                         // raw[b] filled by plain loads instead
    __shared__ int s_abort;
    volatile int *abort = &s_abort;

    const int tid = threadIdx.x;
    const int64_t nblk = (n_elem + EPB - 1) / EPB;
    if ((int64_t)blockIdx.x >= nblk) return;
    const int nloc = (int)((nblk - 1 - (int64_t)blockIdx.x) / gridDim.x + 1);   // blocks of this CTA
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(full + b, 1);
            mbar_init(ready + b, S::SVC_THREADS);
            mbar_init(swept + b, S::SWEEP_THREADS);
            mbar_init(stored + b, S::SVC_THREADS);
            mbar_init(copied + b, S::SVC_THREADS);
        }
        s_abort = 0;
        fence_proxy_async_smem();
    }
    __syncthreads();
    const bool al = aligned_bases != 0;
    // the carve-outs of buffer b, each checked against its own extent
    auto rawU = [&](int b) {
        return SFH_BP(reinterpret_cast<float *>(sm + S::OFF_RAW + b * S::RAW_BYTES), S::RAWU_BYTES / 4, err);
    };
    auto rawJ = [&](int b) {
        return SFH_BP(reinterpret_cast<double *>(sm + S::OFF_RAW + b * S::RAW_BYTES + S::RAWU_BYTES),
                      (S::RAW_BYTES - S::RAWU_BYTES) / 8, err);
    };
    auto P2 = [&](int b) {
        return SFH_BP(reinterpret_cast<float2 *>(sm + S::OFF_P2 + b * S::P2_BYTES), S::P2_BYTES / 8, err);
    };
    auto R = [&](int b) {
        return SFH_BP(reinterpret_cast<float *>(sm + S::OFF_R + (S::RB == 2 ? b : 0) * S::R_BYTES), S::R_BYTES / 4,
                      err);
    };
    auto B64 = [&](int b) {
        return SFH_BP(reinterpret_cast<double *>(sm + S::OFF_B64 + b * S::B64_BYTES), S::B64_BYTES / 8, err);
    };
    // u, Ja and r over their whole extents (bytes of u and Ja for the bulk copies)
    const auto gu = SFH_BP(u, n_elem * U_EL, err);
    const auto gJ = SFH_BP(Ja, n_elem * J_EL, err);
    const auto gr = SFH_BP(r, n_elem * U_EL, err);
    const auto gUb = SFH_BP(reinterpret_cast<const char *>(u), n_elem * U_EL * 4, err);
    const auto gJb = SFH_BP(reinterpret_cast<const char *>(Ja), n_elem * J_EL * 8, err);
    auto plan = [&](int k) {
        return plan_block<S>((int64_t)blockIdx.x + (int64_t)k * gridDim.x, n_elem, u, Ja, al);
    };
    auto give_up = [&]() {
        if (atomicExch(const_cast<int *>(abort), 1) == 0) atomicOr(err, kErrTimeout);
    };

    if (tid >= S::SWEEP_THREADS) {
        // ------------------------------------------------------------ service
        if constexpr (S::SPLIT) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(S::SVC_REG));
        const int st = tid - S::SWEEP_THREADS;
        int issued = 0, landed = 0;   // TMA blocks issued / waited for (thread st == 0)
        auto issue = [&](int k) {
            const BlockPlan pl = plan(k);
            if (!pl.tma) return;
            const int b = k & 1;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(full + b, pl.bytesU + pl.bytesJ);
            bulk_load_ck(rawU(b), bp_at(gUb, pl.srcU), pl.bytesU, full + b);
            bulk_load_ck(rawJ(b), bp_at(gJb, pl.srcJ), pl.bytesJ, full + b);
            issued = k + 1;
        };
        auto store = [&](int k) {
            // the directions' slices summed in a fixed order, (m0 + m1) + m2
            const BlockPlan pl = plan(k);
            const auto R0 = R(k & 1);
            const auto gR = gr + pl.e0 * U_EL;
            // unrolled: independent loads of several outputs in flight per thread
#pragma unroll 8
            for (int s = st; s < pl.ne * U_EL; s += S::SVC_THREADS) {
                float t = R0[s] + R0[S::R_SLICE + s];
                t += R0[2 * S::R_SLICE + s];
                gR[s] = t;
            }
        };
        if (st == 0) {
            issue(0);
            if (nloc > 1) issue(1);
        }
        bool bad = false, ok = true;
        RawPhases ph;
        for (int k = 0; k < nloc && ok; ++k) {
            const int b = k & 1;
            const BlockPlan cur = plan(k);
            // 1. raw data of block k (its buffer was released by the sweep of
            //    block k - 2, waited for in the previous iteration)
            if (cur.tma) {
                if (!ws_wait(full + b, ph.next(b, false), abort)) { give_up(); ok = false; break; }
                if (st == 0) landed = k + 1;
            } else {
                // a block whose aligned window would leave the arrays (or
                // unaligned bases): plain loads, published on copied[b]
                const auto gU = gu + cur.e0 * U_EL;
                const auto gJe = gJ + cur.e0 * J_EL;
                const auto dU = rawU(b);
                const auto dJ = rawJ(b);
                for (int s = st; s < cur.ne * U_EL; s += S::SVC_THREADS) dU[s] = gU[s];
                for (int s = st; s < cur.ne * J_EL; s += S::SVC_THREADS) dJ[s] = gJe[s];
                mbar_arrive(copied + b);
                if (!ws_wait(copied + b, ph.next(b, true), abort)) { give_up(); ok = false; break; }
            }
            // 2. primitives of block k, handed to the sweep warps
            bad |= ws_primitives<S, D, !MIX && FLUX == kFluxEuler>(rawU(b) + cur.offU, P2(b), cur.ne, st, S::SVC_THREADS,
                                       MIX ? B64(b) : BPtr<double>(nullptr));
            mbar_arrive(ready + b);
            // 3. block k - 1: once swept, its raw buffer takes block k + 1 and
            //    its residual is stored
            if (k >= 1) {
                if (!ws_wait(swept + (b ^ 1), ((k - 1) >> 1) & 1, abort)) { give_up(); ok = false; break; }
                if (st == 0 && k + 1 < nloc) issue(k + 1);
                store(k - 1);
                mbar_arrive(stored + (S::RB == 2 ? (b ^ 1) : 0));
            }
        }
        if (ok) {
            const int k = nloc - 1;
            if (ws_wait(swept + (k & 1), (k >> 1) & 1, abort)) store(k);
            else give_up();
        }
        if (bad) atomicOr(err, kErrDomain);
        // never leave with a bulk copy in flight into this CTA's memory
        if (st == 0 && landed < issued) {
            RawPhases dr;   // phases of full[b] up to block `landed`
            for (int k = 0; k < landed; ++k)
                if (plan(k).tma) dr.next(k & 1, false);
            for (int k = landed; k < issued; ++k)
                if (plan(k).tma) mbar_wait_bounded(full + (k & 1), dr.next(k & 1, false), 1000000000ull);
        }
    } else {
        // --------------------------------------------------------------- sweep
        if constexpr (S::SPLIT) asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(S::SWEEP_REG));
        uint32_t hmax = 0;
        RawPhases ph;   // as in the service role
        for (int k = 0; k < nloc; ++k) {
            const int b = k & 1;
            const BlockPlan cur = plan(k);
            // primitives ready; the raw Ja landed (bulk copy or plain loads);
            // the residual buffer free: block k - 2 stored (one buffer: k - 1)
            if (!ws_wait(ready + b, (k >> 1) & 1, abort) || !ws_wait((cur.tma ? full : copied) + b, ph.next(b, !cur.tma), abort) ||
                (S::RB == 2 ? (k >= 2 && !ws_wait(stored + b, ((k - 2) >> 1) & 1, abort))
                            : (k >= 1 && !ws_wait(stored, (k - 1) & 1, abort)))) {
                give_up();
                break;
            }
            if (tid < S::TASKS) {
                const int m = tid / (EPB * NLINE);
                const int L = tid - m * (EPB * NLINE);
                const int el = L / NLINE, l = L - el * NLINE;
                if (el < cur.ne) {
                    const auto re0 = R(b) + m * S::R_SLICE + el * U_EL;
                    const auto je0 = rawJ(b) + cur.offJ + el * J_EL;
                    if constexpr (MIX)
                        hmax = max(hmax, ws_line_sweep_mix<D, N, FLUX>(m, l, P2(b) + el * S::P2_EL, je0,
                                                                        B64(b) + el * S::NN, re0, tab));
                    else
                        hmax = max(hmax, ws_line_sweep<D, N, FLUX>(m, l, P2(b) + el * S::P2_EL, je0, re0, tab));
                }
            }
            mbar_arrive(swept + b);
        }
        if (hmax >= kMetricHiFp32) atomicOr(err, kErrMetric);
    }
}

// grid: one CTA per SM (persistent); occupancy is queried once per device.
// MIX: the mixed precision mode (FP64 metric pair sums and log-mean islands).
template <int D, int N, int FLUX, bool MIX = false>
cudaError_t launch_volume_fp32_ws(const void *u, const double *Ja, void *r, int64_t n_elem, const OpTab<float> &tab,
                                  int *err, cudaStream_t stream) {
    using S = WsShape<D, N, FLUX, MIX>;
    static LaunchCache cache;
    int per_sm = 0, sms = 0;
    const int aligned = ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(Ja) |
                          reinterpret_cast<uintptr_t>(r)) & 15) == 0;
    const int64_t nblk = (n_elem + S::EPB - 1) / S::EPB;
    auto kern = volume_fp32_ws_kernel<D, N, FLUX, MIX>;
    if constexpr (S::SPLIT) {
        // the register split assumes MAXREG registers a thread at launch
        cudaFuncAttributes fa;
        const cudaError_t ea = cudaFuncGetAttributes(&fa, kern);
        if (ea != cudaSuccess) return ea;
        if (fa.numRegs != S::MAXREG) return cudaErrorInvalidKernelImage;
    }
    const cudaError_t e0 = persistent_slots(kern, S::THREADS, S::SMEM, cache, per_sm, sms);
    if (e0 != cudaSuccess) return e0;
    const int64_t grid = nblk < (int64_t)sms * per_sm ? nblk : (int64_t)sms * per_sm;
    kern<<<(unsigned)grid, S::THREADS, S::SMEM, stream>>>(static_cast<const float *>(u), Ja, static_cast<float *>(r),
                                                         n_elem, tab, err, aligned);
    return cudaGetLastError();
}

}  // namespace sfh
