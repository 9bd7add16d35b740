// sfh_volume_row64.cuh -- persistent FP64 volume-residual kernel for 3D
// Euler, one thread per (line, node).
//
// FP64 arithmetic binds this path: the FP64 pipe retires about two lanes
// per clock per SM, so one warp instruction holds a sub-partition's FP64
// unit for tens of cycles, and the pipe idles whenever none of the resident
// warps has an FP64 instruction ready (waiting on shared memory, the
// reciprocal seed, a barrier).  A thread-per-line kernel needs ~175
// registers (n nodes' states and sums) and keeps only two warps per
// sub-partition; here the n threads of a line each own one node's row of
// Eq. 3 and deal the line's unordered pairs out in tournament rounds with
// warp shuffles, as in the FP32 row kernel (sfh_volume_row.cuh), so a
// thread holds one node's state and five sums and 9-16 warps run per SM.
// On large meshes the thread-per-line kernel measured 0-17 % faster (its
// states stay in registers); this one serves meshes too small to fill the
// GPU with the former's element blocks.
//
// Every pair is evaluated once (pairs {a, a+n/2} of even n by both ends);
// each logarithmic mean takes the series or the logarithm per pair (band
// test on FP32 copies), so no line needs a second pass.  Staging: raw u and
// Ja of an element block by 1D bulk copies, the next block's copies issued
// once the block has been converted; per-direction residual slices summed in
// a fixed order into a coalesced store.
#pragma once

#include "sfh_device.cuh"
#include "sfh_tma.cuh"
#include "sfh_volume.cuh"
#include "sfh_volume_tma.cuh"

namespace sfh {

template <int N> struct Row64Cfg { static constexpr int WARPS = 0, EPB = 0; };
template <> struct Row64Cfg<2> { static constexpr int WARPS = 12, EPB = 16; };   // 192 lines, 1 pass
template <> struct Row64Cfg<3> { static constexpr int WARPS = 9, EPB = 10; };    // 270 lines, 3 passes of 90
template <> struct Row64Cfg<4> { static constexpr int WARPS = 12, EPB = 2; };    // 96 lines, 1 pass
template <> struct Row64Cfg<5> { static constexpr int WARPS = 13, EPB = 2; };    // 150 lines, 2 passes of 78
template <> struct Row64Cfg<6> { static constexpr int WARPS = 11, EPB = 1; };    // 108 lines, 2 passes of 55
template <> struct Row64Cfg<7> { static constexpr int WARPS = 13, EPB = 1; };    // 147 lines, 3 passes of 52
template <> struct Row64Cfg<8> { static constexpr int WARPS = 16, EPB = 1; };    // 192 lines, 3 passes of 64

template <int N>
struct Row64Shape {
    static constexpr int D = 3;
    static constexpr int NN = N * N * N, NLINE = N * N, NVAR = 5;
    static constexpr int U_EL = NVAR * NN, J_EL = 9 * NN;
    static constexpr int LPE = 3 * NLINE;
    static constexpr int G = 32 / N;
    static constexpr int WARPS = Row64Cfg<N>::WARPS, EPB = Row64Cfg<N>::EPB;
    static constexpr int THREADS = 32 * WARPS;
    static constexpr int SLOTS = WARPS * G;
    static constexpr int LB = EPB * LPE;
    static constexpr int PASSES = (LB + SLOTS - 1) / SLOTS;
    static constexpr int R = (N - 1) / 2;
    static constexpr bool HALF = N % 2 == 0;
    // node slots: every array below holds one 16-byte unit per node, so odd
    // slot strides keep a line group's loads in distinct banks (even N pads
    // every x-row and xy-plane by one slot)
    static constexpr bool PAD = N % 2 == 0;
    static constexpr int NNP = PAD ? NN + N * N + N : NN;
    __host__ __device__ static constexpr int slot(int i) { return PAD ? i + i / N + i / (N * N) : i; }
    __host__ __device__ static constexpr int slot_stride(int m) {
        return m == 0 ? 1 : (m == 1 ? (PAD ? N + 1 : N) : (PAD ? N * N + N + 1 : N * N));
    }
    static constexpr int MAXREG_RAW = 16384 / (((WARPS + 3) / 4) * 32) / 8 * 8;
    static constexpr int MAXREG = MAXREG_RAW < 255 ? MAXREG_RAW : 255;
    static constexpr int up16(int x) { return (x + 15) / 16 * 16; }
    static constexpr int RAWU_BYTES = up16(EPB * U_EL * 8 + 16);
    static constexpr int RAWJ_BYTES = up16(EPB * J_EL * 8 + 16);
    static constexpr int OFF_U = 16;
    static constexpr int OFF_J = OFF_U + RAWU_BYTES;
    static constexpr int OFF_N = OFF_J + RAWJ_BYTES;            // 3 arrays of double2 per slot: (rho, beta), (hv0, hv1), (hv2, p)
    static constexpr int OFF_M = OFF_N + 3 * EPB * NNP * 16;    // per direction 2 arrays: (J0, J1), (J2, [rho_f, beta_f])
    static constexpr int OFF_R = OFF_M + 6 * EPB * NNP * 16;    // [m][el][var][node] FP64, unpadded
    static constexpr size_t SMEM = OFF_R + (size_t)3 * EPB * U_EL * 8;
    static_assert(WARPS > 0 && THREADS <= 1024, "row kernel shape");
    static_assert(SMEM <= 227 * 1024, "row kernel shared memory");
};

template <int N>
__global__ void __launch_bounds__(Row64Shape<N>::THREADS) __maxnreg__((Row64Shape<N>::MAXREG))
volume_fp64_row_kernel(const double *__restrict__ u, const double *__restrict__ Ja, double *__restrict__ r,
                       int64_t n_elem, const __grid_constant__ OpTab<double> tab, int *__restrict__ err,
                       int aligned_bases) {
    using S = Row64Shape<N>;
    constexpr int NN = S::NN, NLINE = S::NLINE, EPB = S::EPB, U_EL = S::U_EL, J_EL = S::J_EL, G = S::G;
    constexpr int NNP = S::NNP;
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    const auto rawU = SFH_BP(reinterpret_cast<double *>(sm + S::OFF_U), S::RAWU_BYTES / 8, err);
    const auto rawJ = SFH_BP(reinterpret_cast<double *>(sm + S::OFF_J), S::RAWJ_BYTES / 8, err);
    const auto sN = SFH_BP(reinterpret_cast<double2 *>(sm + S::OFF_N), 3 * EPB * NNP, err);   // [3][EPB * NNP]
    const auto sM = SFH_BP(reinterpret_cast<double2 *>(sm + S::OFF_M), 6 * EPB * NNP, err);   // [EPB][3 m][2][NNP]
    const auto sR = SFH_BP(reinterpret_cast<double *>(sm + S::OFF_R), 3 * EPB * U_EL, err);
    // u, Ja and r over their whole extents (bytes of u and Ja for the bulk copies)
    const auto gu = SFH_BP(u, n_elem * U_EL, err);
    const auto gJ = SFH_BP(Ja, n_elem * J_EL, err);
    const auto gr = SFH_BP(r, n_elem * U_EL, err);
    const auto gUb = SFH_BP(reinterpret_cast<const char *>(u), n_elem * U_EL * 8, err);
    const auto gJb = SFH_BP(reinterpret_cast<const char *>(Ja), n_elem * J_EL * 8, err);
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool lane_ok = lane < G * N;
    const int g = lane_ok ? lane / N : G - 1;
    const int a = lane_ok ? lane - g * N : lane - G * N;
    int src[S::R + 1];
    double qo[S::R + 1], qr[S::R + 1];
#pragma unroll
    for (int k = 1; k <= S::R; ++k) {
        const int b = a + k < N ? a + k : a + k - N;
        const int c = a - k >= 0 ? a - k : a - k + N;
        src[k] = lane_ok ? g * N + c : lane;
        qo[k] = tab.Q1[a * N + b];
        qr[k] = tab.Q1[a * N + c];
    }
    const int bh = a + N / 2 < N ? a + N / 2 : a + N / 2 - N;
    const double qh = S::HALF ? tab.Q1[a * N + bh] : 0.0;
    const double qd = tab.Q1[a * N + a];

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

        // ---- 2. primitives (v/2, p, beta) and metric rows, node by node
        BPtr<const double> U = rawU + cur.offU;
        BPtr<const double> J = rawJ + cur.offJ;
        bool bad = false;
        uint32_t hmax = 0;   // largest |Ja| high word (range check)
        for (int s = tid; s < ne * NN; s += blockDim.x) {
            const int el = s / NN, i = s - el * NN;
            const auto ue = U + el * U_EL + i;
            const double rho = ue[0], E = ue[4 * NN];
            const double ir = rcp_nr(rho);
            double hv[3], ke = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double mk = ue[(1 + k) * NN];
                const double vk = mk * ir;
                hv[k] = 0.5 * vk;
                ke = fma(mk, vk, ke);
            }
            const double p = (kGamma - 1.0) * fma(-0.5, ke, E);
            // beta = rho / p to within about half an ulp: reciprocal, product,
            // one residual correction
            const double ip = rcp_nr(p);
            double bt = rho * ip;
            bt = fma(ip, fma(-p, bt, rho), bt);
            bad |= !(rho > 0.0 && p > 0.0);
            const int sl = el * NNP + S::slot(i);
            sN[sl] = make_double2(rho, bt);
            sN[EPB * NNP + sl] = make_double2(hv[0], hv[1]);
            sN[2 * EPB * NNP + sl] = make_double2(hv[2], p);
            // FP32 copies of rho and beta for the band tests, in the spare half
            // of the (J2, .) unit
            const float2 rbf = make_float2(d2f_int(rho), d2f_int(bt));
            const double rbd = __longlong_as_double(*reinterpret_cast<const long long *>(&rbf));
            const auto je = J + el * J_EL + i;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const auto mm = sM + ((el * 3 + m) * 2) * NNP + S::slot(i);
                const double j0 = je[(3 * m) * NN], j1 = je[(3 * m + 1) * NN], j2 = je[(3 * m + 2) * NN];
                hmax = max(hmax, max(abs_hi(j0), max(abs_hi(j1), abs_hi(j2))));
                mm[0] = make_double2(j0, j1);
                mm[NNP] = make_double2(j2, rbd);
            }
        }
        if (bad) atomicOr(err, kErrDomain);
        if (hmax >= kMetricHiFp64) atomicOr(err, kErrMetric);
        __syncthreads();

        // ---- 3. prefetch the next block
        const int64_t nxt = blk + gridDim.x;
        BlockPlan nx = cur;
        if (nxt < nblk) nx = plan_block<S>(nxt, n_elem, u, Ja, aligned_bases != 0);
        if (tid == 0 && nxt < nblk && nx.tma) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, nx.bytesU + nx.bytesJ);
            bulk_load_ck(rawU, bp_at(gUb, nx.srcU), nx.bytesU, bar);
            bulk_load_ck(rawJ, bp_at(gJb, nx.srcJ), nx.bytesJ, bar);
        }

        // ---- 4. rows
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
            const double omega = tab.w[o0] * tab.w[o1];
            BPtr<const double2> N0 = sN + el * NNP, N1 = N0 + EPB * NNP, N2 = N1 + EPB * NNP;
            BPtr<const double2> M0 = sM + ((el * 3 + m) * 2) * NNP, M1 = M0 + NNP;
            auto node = [&](int sl) {
                EulerNodeD<3> nd;
                const double2 x0 = N0[sl], x1 = N1[sl], x2 = N2[sl], y0 = M0[sl], y1 = M1[sl];
                nd.rho = x0.x; nd.beta = x0.y; nd.hv[0] = x1.x; nd.hv[1] = x1.y; nd.hv[2] = x2.x; nd.p = x2.y;
                nd.J[0] = y0.x; nd.J[1] = y0.y; nd.J[2] = y1.x;
                const long long bits = __double_as_longlong(y1.y);
                nd.rf = __int_as_float((int)(bits & 0xffffffffll));
                nd.bf = __int_as_float((int)(bits >> 32));
                return nd;
            };
            const int ia = base + a * stride, pa = pbase + a * pstride;
            const EulerNodeD<3> o = node(pa);

            double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int k = 1; k <= S::R; ++k) {
                const int b = a + k < N ? a + k : a + k - N;
                const EulerNodeD<3> q = node(pbase + b * pstride);
                double F[5], Fr[5];
                euler_pair_flux_f64<3>(o, q, F);
#pragma unroll
                for (int v = 0; v < 5; ++v) acc[v] = fma(qo[k], F[v], acc[v]);
#pragma unroll
                for (int v = 0; v < 5; ++v) Fr[v] = __shfl_sync(0xffffffffu, F[v], src[k]);
#pragma unroll
                for (int v = 0; v < 5; ++v) acc[v] = fma(qr[k], Fr[v], acc[v]);
            }
            if constexpr (S::HALF) {
                const EulerNodeD<3> q = node(pbase + bh * pstride);
                double F[5];
                euler_pair_flux_f64<3>(o, q, F);
#pragma unroll
                for (int v = 0; v < 5; ++v) acc[v] = fma(qh, F[v], acc[v]);
            }
            if (qd != 0.0) {
                double F[5];
                euler_diag_flux_f64<3>(o, F);
#pragma unroll
                for (int v = 0; v < 5; ++v) acc[v] = fma(qd, F[v], acc[v]);
            }
            if (ok) {
                const auto re = sR + (size_t)m * EPB * U_EL + el * U_EL + ia;
#pragma unroll
                for (int v = 0; v < 5; ++v) re[v * NN] = omega * acc[v];
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

template <int N>
cudaError_t launch_volume_fp64_row(const void *u, const double *Ja, void *r, int64_t n_elem, const OpTab<double> &tab,
                                   int *err, cudaStream_t stream) {
    using S = Row64Shape<N>;
    auto kern = volume_fp64_row_kernel<N>;
    static LaunchCache cache;
    int per_sm = 0, sms = 0;
    const cudaError_t e0 = persistent_slots(kern, S::THREADS, S::SMEM, cache, per_sm, sms);
    if (e0 != cudaSuccess) return e0;
    const int64_t nblk = (n_elem + S::EPB - 1) / S::EPB;
    const int64_t grid = nblk < (int64_t)sms * per_sm ? nblk : (int64_t)sms * per_sm;
    const int aligned = ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(Ja) |
                          reinterpret_cast<uintptr_t>(r)) & 15) == 0;
    kern<<<(unsigned)grid, S::THREADS, S::SMEM, stream>>>(static_cast<const double *>(u), Ja, static_cast<double *>(r),
                                                         n_elem, tab, err, aligned);
    return cudaGetLastError();
}

// FP64 row kernel: 3D Euler, n = 2 .. 8, for meshes too small to fill the GPU
// with the thread-per-line kernel's blocks (n = 9 needs more shared memory
// than a CTA has)
constexpr int kRow64MinN = 2;
template <int D, int N, int FLUX>
constexpr bool use_row64_kernel() { return D == 3 && FLUX == kFluxEuler && N >= kRow64MinN && N <= 8; }

}  // namespace sfh
