// sfh_volume_row.cuh -- persistent FP32 (Kahan) volume-residual kernel for
// 3D Euler at high degree, one thread per (line, node).
//
// The line kernel (sfh_volume_tma.cuh) gives a whole grid line to one thread,
// which then holds the accumulators and states of all n nodes: about 250
// registers at n = 8, so that only 6-8 warps fit on an SM.  Here the n
// threads of a line each own one node's row of Eq. 3,
//   r_a = omega * sum_b Q1[a][b] F(u_a, u_b),
// and the unordered pairs of the line are dealt out in rounds (a round-robin
// tournament): in round k = 1 .. (n-1)/2 thread a evaluates the pair
// {a, a+k mod n}, adds Q1[a][a+k] F to its own row and passes F by a warp
// shuffle to thread a+k, which adds Q1[a+k][a] F.  Every unordered pair is
// evaluated once; for even n the pairs {a, a+n/2} are evaluated by both
// ends (no shuffle).  A thread holds one node's state and accumulators, about
// 80 registers at any n, so 19-27 warps run per SM.
//
// Staging is that of the line kernel: raw u (FP32) and Ja (FP64) of an
// element block arrive by 1D bulk copies (mbarrier, bounded wait), the next
// block's copies are issued once the current one has been converted, each
// direction writes its own residual slice, and the slices are summed in a
// fixed order into a coalesced store (deterministic).  A line group any of
// whose pairs lies outside the series band of the logarithmic means redoes
// its rows with logarithms (rare for smooth states).
#pragma once

#include "sfh_device.cuh"
#include "sfh_tma.cuh"
#include "sfh_volume_tma.cuh"

namespace sfh {

// warps per CTA and elements per block: a pass covers WARPS * (32 / N) lines,
// and the EPB * 3 N^2 lines of a block take a whole number of passes (or
// nearly so); one CTA per SM
template <int N> struct RowCfg { static constexpr int WARPS = 0, EPB = 0; };
template <> struct RowCfg<5> { static constexpr int WARPS = 25, EPB = 2; };   // 150 lines, 1 pass
template <> struct RowCfg<6> { static constexpr int WARPS = 22, EPB = 2; };   // 216 lines, 2 passes of 110
template <> struct RowCfg<7> { static constexpr int WARPS = 19, EPB = 1; };   // 147 lines, 2 passes of 76
template <> struct RowCfg<8> { static constexpr int WARPS = 24, EPB = 1; };   // 192 lines, 2 passes of 96
template <> struct RowCfg<9> { static constexpr int WARPS = 27, EPB = 1; };   // 243 lines, 3 passes of 81

template <int N>
struct RowShape {
    static constexpr int D = 3;
    static constexpr int NN = N * N * N, NLINE = N * N, NVAR = 5;
    static constexpr int U_EL = NVAR * NN, J_EL = 9 * NN;
    static constexpr int LPE = 3 * NLINE;                 // lines per element
    static constexpr int G = 32 / N;                      // line groups per warp
    static constexpr int WARPS = RowCfg<N>::WARPS, EPB = RowCfg<N>::EPB;
    static constexpr int THREADS = 32 * WARPS;
    static constexpr int SLOTS = WARPS * G;               // lines per pass
    static constexpr int LB = EPB * LPE;                  // lines per block
    static constexpr int PASSES = (LB + SLOTS - 1) / SLOTS;
    static constexpr int R = (N - 1) / 2;                 // shuffled rounds
    // Node slots of the state and metric arrays.  A line's nodes are 1, N or
    // N^2 slots apart; for even N the latter two are multiples of 8 float4
    // (128 bytes), which would put a line group's 16-byte loads in the same
    // banks.  Even N therefore pads every x-row and every xy-plane by one
    // slot: slot(i) = i + i/N + i/N^2, and the strides become 1, N+1,
    // N^2+N+1 (odd).
    static constexpr bool PAD = N % 2 == 0;
    static constexpr int NNP = PAD ? NN + N * N + N : NN;   // slots per element
    __host__ __device__ static constexpr int slot(int i) { return PAD ? i + i / N + i / (N * N) : i; }
    __host__ __device__ static constexpr int slot_stride(int m) {
        return m == 0 ? 1 : (m == 1 ? (PAD ? N + 1 : N) : (PAD ? N * N + N + 1 : N * N));
    }
    static constexpr bool HALF = N % 2 == 0;              // the pairs {a, a + n/2}
    // one CTA per SM: each sub-partition holds ceil(WARPS/4) warps
    static constexpr int MAXREG_RAW = 16384 / (((WARPS + 3) / 4) * 32) / 8 * 8;
    static constexpr int MAXREG = MAXREG_RAW < 255 ? MAXREG_RAW : 255;
    static constexpr int up16(int x) { return (x + 15) / 16 * 16; }
    static constexpr int RAWU_BYTES = up16(EPB * U_EL * 4 + 16);   // + window slack
    static constexpr int RAWJ_BYTES = up16(EPB * J_EL * 8 + 16);
    static constexpr int OFF_U = 16;                                // [0,16): mbarrier
    static constexpr int OFF_J = OFF_U + RAWU_BYTES;
    static constexpr int OFF_A = OFF_J + RAWJ_BYTES;                // float4 (rho, beta, v0/2, v1/2) per node
    static constexpr int OFF_B = OFF_A + EPB * NNP * 16;            // float2 (v2/2, p) per node
    static constexpr int OFF_JF = up16(OFF_B + EPB * NNP * 8);      // float4 (Ja^m_0..2, 0) per (m, node)
    static constexpr int OFF_R = OFF_JF + EPB * 3 * NNP * 16;       // [m][el][var][node], unpadded
    static constexpr size_t SMEM = OFF_R + (size_t)3 * EPB * U_EL * 4;
    static_assert(WARPS > 0 && THREADS <= 1024, "row kernel shape");
    static_assert(SMEM <= 227 * 1024, "row kernel shared memory");
    static_assert(OFF_J % 16 == 0 && OFF_A % 16 == 0 && OFF_JF % 16 == 0, "16-byte alignment");
};

struct RowNode {
    float rho, beta, hv[3], p, J[3];
};

__device__ __forceinline__ RowNode row_node(const float4 A, const float2 B, const float4 J) {
    RowNode n;
    n.rho = A.x; n.beta = A.y; n.hv[0] = A.z; n.hv[1] = A.w; n.hv[2] = B.x; n.p = B.y;
    n.J[0] = J.x; n.J[1] = J.y; n.J[2] = J.z;
    return n;
}

// Ranocha's flux between nodes o and q contracted with Ja^m(o) + Ja^m(q),
// both logarithmic means by the series (same arithmetic as the line kernel);
// umax collects u_rho + u_beta for the band test.
__device__ __forceinline__ void row_pair_flux(const RowNode &o, const RowNode &q, float F[5], float &umax) {
    float n[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) n[k] = o.J[k] + q.J[k];
    float hna = o.hv[0] * n[0], hnb = q.hv[0] * n[0], hvv = o.hv[0] * q.hv[0];
#pragma unroll
    for (int k = 1; k < 3; ++k) {
        hna = fmaf(o.hv[k], n[k], hna);
        hnb = fmaf(q.hv[k], n[k], hnb);
        hvv = fmaf(o.hv[k], q.hv[k], hvv);
    }
    const float cg = (float)(2.0 / (kGamma - 1.0));
    const float2 c0 = f2(0.5f, cg), c1 = f2(0.5f * (-1.0f / 3.0f), cg * (1.0f / 3.0f));
    const float2 c2 = f2(0.5f * (-4.0f / 45.0f), cg * (1.0f / 5.0f));
    const float2 c3 = f2(0.5f * (-44.0f / 945.0f), cg * (1.0f / 7.0f));
    const float2 ro = f2(o.rho, o.beta), rq = f2(q.rho, q.beta);
    const float2 d2 = sub2(ro, rq), s2 = add2(ro, rq);
    const float2 r2 = f2(rcp_approx(s2.x), rcp_approx(s2.y));
    const float2 t2 = mul2(d2, r2);
    const float2 u2 = mul2(t2, t2);
    float2 h = fma2(u2, c3, c2);
    h = fma2(u2, h, c1);
    h = fma2(u2, h, c0);
    umax = fmaxf(umax, u2.x + u2.y);
    const float2 m2 = mul2(f2(s2.x, r2.y), h);   // ({rho}_ln, 1/((g-1){beta}_ln))
    const float frho = m2.x * (hna + hnb);
    const float pavg = 0.5f * (o.p + q.p);
    F[0] = frho;
#pragma unroll
    for (int k = 0; k < 3; ++k) F[1 + k] = fmaf(frho, o.hv[k] + q.hv[k], pavg * n[k]);
    F[4] = fmaf(frho, fmaf(2.0f, hvv, m2.y), fmaf(o.p, hnb, q.p * hna));
}

// physical flux f(u_o) . (2 Ja^m(o)): the diagonal term
__device__ __forceinline__ void row_diag_flux(const RowNode &o, float F[5]) {
    float n[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) n[k] = 2.0f * o.J[k];
    float hn = o.hv[0] * n[0], hv2 = o.hv[0] * o.hv[0];
#pragma unroll
    for (int k = 1; k < 3; ++k) { hn = fmaf(o.hv[k], n[k], hn); hv2 = fmaf(o.hv[k], o.hv[k], hv2); }
    const float frho = 2.0f * o.rho * hn;
    F[0] = frho;
#pragma unroll
    for (int k = 0; k < 3; ++k) F[1 + k] = fmaf(2.0f * frho, o.hv[k], o.p * n[k]);
    F[4] = fmaf(frho, 2.0f * hv2, 2.0f * o.p * hn * (float)(kGamma / (kGamma - 1.0)));
}

struct RowAcc {
    KahanF2 a01, a23;
    KahanF a4;
    __device__ __forceinline__ void zero() { a01.zero(); a23.zero(); a4.zero(); }
    __device__ __forceinline__ void add(float q, const float F[5]) {
        const float2 q2 = f2s(q);
        a01.add_prod(q2, f2(F[0], F[1]));
        a23.add_prod(q2, f2(F[2], F[3]));
        a4.add_prod(q, F[4]);
    }
};

// One node's row from scratch, with logarithms where a pair leaves the
// series band; out of line because it runs only for states with large jumps.
// A, B, Jm, base and stride address node slots; re points at the node's
// residual (unpadded layout).
template <int N>
__device__ __noinline__ void row_general(BPtr<const float4> A, BPtr<const float2> B, BPtr<const float4> Jm, int base,
                                         int stride, int a, float omega, const OpTab<float> &tab, BPtr<float> re) {
    constexpr int NN = N * N * N;
    const int ia = base + a * stride;
    const RowNode o = row_node(A[ia], B[ia], Jm[ia]);
    KahanF acc[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v].zero();
#pragma unroll 1
    for (int b = 0; b < N; ++b) {
        const float q = tab.Q1[a * N + b];
        if (q == 0.0f) continue;
        float F[5];
        if (b == a) {
            row_diag_flux(o, F);
        } else {
            const int ib = base + b * stride;
            const RowNode w = row_node(A[ib], B[ib], Jm[ib]);
            float n[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) n[k] = o.J[k] + w.J[k];
            float hna = 0.0f, hnb = 0.0f, hvv = 0.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k) { hna = fmaf(o.hv[k], n[k], hna); hnb = fmaf(w.hv[k], n[k], hnb); hvv = fmaf(o.hv[k], w.hv[k], hvv); }
            const float Lr = ln_mean(o.rho, w.rho), iLb = inv_ln_mean(o.beta, w.beta);
            const float frho = Lr * (hna + hnb);
            const float pavg = 0.5f * (o.p + w.p);
            F[0] = frho;
#pragma unroll
            for (int k = 0; k < 3; ++k) F[1 + k] = fmaf(frho, o.hv[k] + w.hv[k], pavg * n[k]);
            F[4] = fmaf(frho, fmaf(2.0f, hvv, iLb * (float)(1.0 / (kGamma - 1.0))), fmaf(o.p, hnb, w.p * hna));
        }
#pragma unroll
        for (int v = 0; v < 5; ++v) acc[v].add_prod(q, F[v]);
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) re[v * NN] = omega * acc[v].value();
}

template <int N>
__global__ void __launch_bounds__(RowShape<N>::THREADS) __maxnreg__((RowShape<N>::MAXREG))
volume_fp32_row_kernel(const float *__restrict__ u, const double *__restrict__ Ja, float *__restrict__ r,
                       int64_t n_elem, const __grid_constant__ OpTab<float> tab, int *__restrict__ err,
                       int aligned_bases) {
    using S = RowShape<N>;
    constexpr int NN = S::NN, NLINE = S::NLINE, EPB = S::EPB, U_EL = S::U_EL, J_EL = S::J_EL, G = S::G;
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    const auto rawU = SFH_BP(reinterpret_cast<float *>(sm + S::OFF_U), S::RAWU_BYTES / 4, err);
    const auto rawJ = SFH_BP(reinterpret_cast<double *>(sm + S::OFF_J), S::RAWJ_BYTES / 8, err);
    const auto sA = SFH_BP(reinterpret_cast<float4 *>(sm + S::OFF_A), EPB * S::NNP, err);
    const auto sB = SFH_BP(reinterpret_cast<float2 *>(sm + S::OFF_B), EPB * S::NNP, err);
    const auto sJ = SFH_BP(reinterpret_cast<float4 *>(sm + S::OFF_JF), EPB * 3 * S::NNP, err);
    const auto sR = SFH_BP(reinterpret_cast<float *>(sm + S::OFF_R), 3 * EPB * U_EL, err);
    // u, Ja and r over their whole extents (bytes of u and Ja for the bulk copies)
    const auto gu = SFH_BP(u, n_elem * U_EL, err);
    const auto gJ = SFH_BP(Ja, n_elem * J_EL, err);
    const auto gr = SFH_BP(r, n_elem * U_EL, err);
    const auto gUb = SFH_BP(reinterpret_cast<const char *>(u), n_elem * U_EL * 4, err);
    const auto gJb = SFH_BP(reinterpret_cast<const char *>(Ja), n_elem * J_EL * 8, err);
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // lane role: group g of N lanes owns one line, lane a of the group one
    // node; the 32 - G N spare lanes shadow the last group (their results
    // are discarded) so that every shuffle runs on the full warp
    const bool lane_ok = lane < G * N;
    const int g = lane_ok ? lane / N : G - 1;
    const int a = lane_ok ? lane - g * N : lane - G * N;
    const unsigned gmask = lane_ok ? (((1u << N) - 1u) << (g * N)) : 0u;
    int src[S::R + 1];
    float qo[S::R + 1], qr[S::R + 1];
#pragma unroll
    for (int k = 1; k <= S::R; ++k) {
        const int b = a + k < N ? a + k : a + k - N;
        const int c = a - k >= 0 ? a - k : a - k + N;
        src[k] = lane_ok ? g * N + c : lane;
        qo[k] = tab.Q1[a * N + b];
        qr[k] = tab.Q1[a * N + c];
    }
    const int bh = a + N / 2 < N ? a + N / 2 : a + N / 2 - N;
    const float qh = S::HALF ? tab.Q1[a * N + bh] : 0.0f;
    const float qd = tab.Q1[a * N + a];

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

        // ---- 2. primitives and FP32 metrics, node by node
        const auto U = rawU + cur.offU;
        const auto J = rawJ + cur.offJ;
        bool bad = false;
        uint32_t hmax = 0;   // largest |Ja| high word (range check)
        for (int s = tid; s < ne * NN; s += blockDim.x) {
            const int el = s / NN, i = s - el * NN;
            const auto ue = U + el * U_EL + i;
            const float rho = ue[0], E = ue[4 * NN];
            float ir = rcp_approx(rho);
            ir = fmaf(ir, fmaf(-rho, ir, 1.0f), ir);
            float hv[3], ke = 0.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
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
            const int sl = el * S::NNP + S::slot(i);
            sA[sl] = make_float4(rho, bt, hv[0], hv[1]);
            sB[sl] = make_float2(hv[2], p);
            bad |= !(rho > 0.0f && p > 0.0f);
            const auto je = J + el * J_EL + i;
#pragma unroll
            for (int m = 0; m < 3; ++m)
                sJ[(el * 3 + m) * S::NNP + S::slot(i)] =
                    make_float4(d2f_int_track(je[(3 * m) * NN], hmax), d2f_int_track(je[(3 * m + 1) * NN], hmax),
                                d2f_int_track(je[(3 * m + 2) * NN], hmax), 0.0f);
        }
        if (bad) atomicOr(err, kErrDomain);
        if (hmax >= kMetricHiFp32) atomicOr(err, kErrMetric);
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

        // ---- 4. rows, a pass of SLOTS lines at a time
#pragma unroll 1
        for (int pass = 0; pass < S::PASSES; ++pass) {
            const int Lx = pass * S::SLOTS + warp * G + g;
            bool ok = lane_ok && Lx < S::LB;
            const int Lc = Lx < S::LB ? Lx : S::LB - 1;
            const int m = Lc / (EPB * NLINE);
            const int rem = Lc - m * (EPB * NLINE);
            int el = rem / NLINE;
            const int l = rem - el * NLINE;
            if (el >= ne) { ok = false; el = 0; }
            const int o0 = l % N, o1 = l / N;
            const int base = m == 0 ? N * l : (m == 1 ? o0 + N * N * o1 : l);
            const int stride = m == 0 ? 1 : (m == 1 ? N : N * N);
            const int pbase = S::slot(base), pstride = S::slot_stride(m);
            const float omega = tab.w[o0] * tab.w[o1];
            BPtr<const float4> A = sA + el * S::NNP;
            BPtr<const float2> B = sB + el * S::NNP;
            BPtr<const float4> Jm = sJ + (el * 3 + m) * S::NNP;
            const int ia = base + a * stride, pa = pbase + a * pstride;
            const RowNode o = row_node(A[pa], B[pa], Jm[pa]);

            RowAcc acc;
            acc.zero();
            float umax = 0.0f;
#pragma unroll
            for (int k = 1; k <= S::R; ++k) {
                const int b = a + k < N ? a + k : a + k - N;
                const int pb = pbase + b * pstride;
                const RowNode q = row_node(A[pb], B[pb], Jm[pb]);
                float F[5], Fr[5];
                row_pair_flux(o, q, F, umax);
                acc.add(qo[k], F);
#pragma unroll
                for (int v = 0; v < 5; ++v) Fr[v] = __shfl_sync(0xffffffffu, F[v], src[k]);
                acc.add(qr[k], Fr);
            }
            if constexpr (S::HALF) {
                const int pb = pbase + bh * pstride;
                const RowNode q = row_node(A[pb], B[pb], Jm[pb]);
                float F[5];
                row_pair_flux(o, q, F, umax);
                acc.add(qh, F);
            }
            if (qd != 0.0f) {
                float F[5];
                row_diag_flux(o, F);
                acc.add(qd, F);
            }
            // a pair outside the band anywhere in the line group sends the
            // whole group to the general routine (also for a NaN maximum)
            const unsigned out = __ballot_sync(0xffffffffu, !(umax < 1e-2f));
            const auto re = sR + (size_t)m * EPB * U_EL + el * U_EL + ia;
            if (__builtin_expect((out & gmask) != 0u, 0)) {
                if (ok) row_general<N>(A, B, Jm, pbase, pstride, a, omega, tab, re);
            } else if (ok) {
                const float2 v01 = acc.a01.value(), v23 = acc.a23.value();
                re[0 * NN] = omega * v01.x;
                re[1 * NN] = omega * v01.y;
                re[2 * NN] = omega * v23.x;
                re[3 * NN] = omega * v23.y;
                re[4 * NN] = omega * acc.a4.value();
            }
        }
        __syncthreads();

        // ---- 5. sum the directions in a fixed order and store r
        const auto gR = gr + cur.e0 * U_EL;
        for (int s2 = tid; s2 < ne * U_EL; s2 += blockDim.x)
            gR[s2] = (sR[s2] + sR[EPB * U_EL + s2]) + sR[2 * EPB * U_EL + s2];
        cur = nx;
    }
}

// one CTA per SM (persistent); occupancy is queried once per shape
template <int N>
cudaError_t launch_volume_fp32_row(const void *u, const double *Ja, void *r, int64_t n_elem, const OpTab<float> &tab,
                                   int *err, cudaStream_t stream) {
    using S = RowShape<N>;
    auto kern = volume_fp32_row_kernel<N>;
    static LaunchCache cache;
    int per_sm = 0, sms = 0;
    const cudaError_t e0 = persistent_slots(kern, S::THREADS, S::SMEM, cache, per_sm, sms);
    if (e0 != cudaSuccess) return e0;
    const int64_t nblk = (n_elem + S::EPB - 1) / S::EPB;
    const int64_t grid = nblk < (int64_t)sms * per_sm ? nblk : (int64_t)sms * per_sm;
    const int aligned = ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(Ja) |
                          reinterpret_cast<uintptr_t>(r)) & 15) == 0;
    kern<<<(unsigned)grid, S::THREADS, S::SMEM, stream>>>(static_cast<const float *>(u), Ja, static_cast<float *>(r),
                                                         n_elem, tab, err, aligned);
    return cudaGetLastError();
}

// The row kernel serves 3D Euler (Ranocha's flux) at n = 8, where it
// measured 10-25 % faster than the line kernel and, on small meshes, than
// the warp-specialized kernel (146 against 168 us on 16^3 Gauss elements);
// at n <= 7 the warp-specialized kernel wins, and at n = 9 the 27-lane
// groups of the row kernel lose.
template <int D, int N, int FLUX>
constexpr bool use_row_kernel() { return D == 3 && FLUX == kFluxEuler && N == 8; }

}  // namespace sfh
