// sfh_serve.cu -- serving runtime: continuous batching of residual and VJP
// requests (3D Euler, Ranocha's or Chandrashekar's flux, p = 2..8, mixed
// precision) through one persistent kernel.
//
// Data path
//   * The host admission thread takes requests FIFO as long as the HBM budget
//     and the in-flight limit allow, writes the request's descriptor into a
//     slot table and one descriptor per element tile into a ring, both in
//     page-locked host memory mapped into the device address space, and
//     publishes them by advancing the ring's tail (release store).
//   * Persistent CTAs (one per SM by default) claim ring entries with a
//     compare-and-swap on a device-side head counter -- only entries below the
//     published tail -- and run the tile with the body of the request's class
//     (kind x precision x degree x flux).  Tiles of requests that arrive while
//     others run are claimed as soon as they are published, so their work
//     interleaves on the GPU.
//   * A per-request tile counter on the device finds the last tile; its CTA
//     publishes the request's completion record (status, sequence number) to
//     host-mapped memory after a system-scope fence.
//   * CTAs that find no work for idle_ns (bounded also by an iteration cap)
//     exit; the host relaunches the kernel whenever work is in flight and the
//     kernel is not running, so a claim can never be stranded.
// All device waits are bounded; no wait can hang the GPU.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/sfhad.h"
#include "sfh_internal.h"
#include "sfh_tma.cuh"
#include "sfh_volume.cuh"
#include "sfh_vjp.cuh"
#include "sfh_volume_tma.cuh"

namespace sfh {
namespace serve {

constexpr int kThreads = 256;
constexpr int kMaxSlots = 256;
constexpr uint64_t kRing = 1ull << 18;
constexpr int kPMin = 2, kPMax = 8;

struct Tile {
    int32_t slot;
    int32_t tile;
};

struct __align__(16) Req {   // written by the host before the request's tiles are published
    int16_t kind, flux;
    int32_t prec, n, nodes;
    const void *u;
    const double *Ja;
    const double *lam;
    void *out;
    int32_t n_elem, epb, ntiles;
    uint32_t seq;
};
static_assert(sizeof(Req) == 64, "descriptor read as four 16-byte words");

struct Done {  // written by the device
    uint32_t seq;
    int32_t status;
    unsigned long long t_start;   // device timer at the start of the request's first tile
};

struct DevCtrl {   // device memory
    unsigned long long head;
    int idle_ctas;     // CTAs that found nothing to claim for the quiet window
    int quit;          // set once every CTA is idle: the whole kernel leaves
    int done_tiles[kMaxSlots];
    int err[kMaxSlots];
    unsigned long long t_start[kMaxSlots];   // earliest tile start of the slot's request (~0: none yet)
    unsigned long long tiles[4], busy_ns[4], claim_ns;   // counters (sfh_serve_stats)
};

struct Args {
    const Tile *ring;                        // mapped
    const Req *reqs;                         // mapped
    Done *done;                              // mapped
    const volatile unsigned long long *tail; // mapped
    const volatile int *stop;                // mapped
    DevCtrl *ctrl;                           // device
    const OpTab<double> *tabd;               // device [2][10] (nodes, n)
    const OpTab<float> *tabf;
    unsigned long long idle_ns;
};

__device__ __forceinline__ unsigned long long ld_acquire_sys_u64(const volatile unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// ---- per-class tile bodies (all 3D Euler) --------------------------------
// tiles sized to give the 256 threads a line each (as far as a 200 KB
// budget allows): one serving CTA per SM must keep all of its warps busy
constexpr int kTileBudget = 200 * 1024;
// FP32-Kahan tiles run the persistent kernel's block phases (packed Kahan
// sums, series log means, line-major FP32 metric rows), all directions at
// once: D * EPB * N^2 line tasks on the 256 threads.
template <int N>
struct ServeF32 {
    static constexpr int D = 3;
    static constexpr int NN = N * N * N, NLINE = N * N, NVAR = 5, NP = 6;
    static constexpr int U_EL = NVAR * NN, J_EL = 9 * NN;
    static constexpr int LJ = (N * D) % 2 == 0 ? N * D + 1 : N * D;
    static constexpr int JF_EL = D * NLINE * LJ;
    static constexpr int EL_BYTES = 4 * NP * NN + 4 * JF_EL + 4 * D * U_EL + 4 * U_EL + 8 * J_EL;
    static constexpr int EPB_T = kThreads / (D * NLINE) > 0 ? kThreads / (D * NLINE) : 1;
    static constexpr int EPB_S = kTileBudget / EL_BYTES > 0 ? kTileBudget / EL_BYTES : 1;
    static constexpr int EPB = EPB_T < EPB_S ? EPB_T : EPB_S;   // elements per sub-block
    // sub-blocks per tile: a tile should carry about 1024 lines per direction.
    // Claims are serialized on the ring's head (about 0.6 us each with all
    // SMs claiming); FP32 tiles of 256 lines kept the CTAs claiming for 3/4
    // of their time (measured with sfh_serve_stats)
    static constexpr int SUB = (1024 / NLINE + EPB / 2) / EPB > 0 ? (1024 / NLINE + EPB / 2) / EPB : 1;
    static constexpr int TILE = SUB * EPB;                       // elements per tile
    static constexpr int up16(int x) { return (x + 15) / 16 * 16; }
    static constexpr int OFF_JF = up16(EPB * NP * NN * 4);
    static constexpr int OFF_R = up16(OFF_JF + EPB * JF_EL * 4);
    static constexpr int OFF_RU = up16(OFF_R + D * EPB * U_EL * 4);   // raw u of the next sub-block
    static constexpr int OFF_RJ = up16(OFF_RU + EPB * U_EL * 4);      // raw Ja of the next sub-block
    static constexpr size_t SMEM = OFF_RJ + (size_t)EPB * J_EL * 8;
    static_assert(D * EPB * NLINE <= kThreads, "one thread per line task");
};

template <int N, int FLUX = kFluxEuler> struct Cls {
    using F64 = Shape<3, N, FLUX, ModeFP64, kTileBudget, kThreads>;
    using F32 = ServeF32<N>;   // tiles of F32::TILE elements
    using MIX = Shape<3, N, FLUX, ModeMixed, kTileBudget, kThreads>;
    using VJP = VjpShape<3, N, FLUX, kTileBudget, kThreads>;
};
// both Euler fluxes have the same node data, so a class's tiles do not
// depend on the flux (tile_epb takes none)
template <int N> constexpr bool same_tiles() {
    using R = Cls<N, kFluxEuler>;
    using C = Cls<N, kFluxEulerCh>;
    return R::F64::EPB == C::F64::EPB && R::F64::SMEM == C::F64::SMEM && R::MIX::EPB == C::MIX::EPB &&
           R::MIX::SMEM == C::MIX::SMEM && R::VJP::EPB == C::VJP::EPB && R::VJP::SMEM == C::VJP::SMEM &&
           R::VJP::THREADS == C::VJP::THREADS && R::F64::THREADS == C::F64::THREADS &&
           R::MIX::THREADS == C::MIX::THREADS;
}
static_assert(same_tiles<3>() && same_tiles<4>() && same_tiles<5>() && same_tiles<6>() && same_tiles<7>() &&
                  same_tiles<8>() && same_tiles<9>(),
              "tiles independent of the Euler flux");

template <int N> constexpr size_t cls_smem() {
    size_t a = Cls<N>::F64::SMEM, b = Cls<N>::F32::SMEM, c = Cls<N>::MIX::SMEM, d = Cls<N>::VJP::SMEM;
    size_t m = a > b ? a : b;
    m = m > c ? m : c;
    return m > d ? m : d;
}
constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kSmem = cmax(cmax(cmax(cls_smem<3>(), cls_smem<4>()), cmax(cls_smem<5>(), cls_smem<6>())),
                              cmax(cmax(cls_smem<7>(), cls_smem<8>()), cls_smem<9>()));
static_assert(kSmem <= 200 * 1024, "serving shared memory");

// elements per tile of a class (host and device agree through this function)
__host__ __device__ inline int tile_epb(int kind, int prec, int n) {
#define SFH_EPB_CASE(N)                                                    \
    case N:                                                                \
        if (kind == SFH_REQ_VJP) return Cls<N>::VJP::EPB;                  \
        if (prec == SFH_FP64) return Cls<N>::F64::EPB;                     \
        if (prec == SFH_FP32_KAHAN) return Cls<N>::F32::TILE;              \
        return Cls<N>::MIX::EPB;
    switch (n) {
        SFH_EPB_CASE(3) SFH_EPB_CASE(4) SFH_EPB_CASE(5) SFH_EPB_CASE(6) SFH_EPB_CASE(7) SFH_EPB_CASE(8)
        SFH_EPB_CASE(9)
    }
#undef SFH_EPB_CASE
    return 1;
}

// One out-of-line body per class, so that each gets its own register
// allocation (a body that shares a function with the others inherits their
// register pressure and spills in its inner loops).
template <int N, int FLUX>
__device__ __noinline__ void run_vjp(const Req &q, int64_t e0, int ne, const OpTab<double> &td, int *err,
                                     unsigned char *smem) {
    const int64_t nu = (int64_t)q.n_elem * 5 * N * N * N, nj = (int64_t)q.n_elem * 9 * N * N * N;
    vjp_tile<3, N, FLUX, typename Cls<N, FLUX>::VJP>(SFH_BP(static_cast<const double *>(q.u), nu, err), SFH_BP(q.Ja, nj, err),
                                                     SFH_BP(q.lam, nu, err), SFH_BP(static_cast<double *>(q.out), nu, err), e0,
                                                     ne, td, err, smem);
}
template <int N, int FLUX>
__device__ __noinline__ void run_f64(const Req &q, int64_t e0, int ne, const OpTab<double> &td, int *err,
                                     unsigned char *smem) {
    const int64_t nu = (int64_t)q.n_elem * 5 * N * N * N, nj = (int64_t)q.n_elem * 9 * N * N * N;
    volume_tile<3, N, FLUX, ModeFP64, typename Cls<N, FLUX>::F64>(SFH_BP(static_cast<const double *>(q.u), nu, err),
                                                                  SFH_BP(q.Ja, nj, err),
                                                                  SFH_BP(static_cast<double *>(q.out), nu, err), e0, ne,
                                                                  td, err, smem);
}
template <int N, int FLUX>
__device__ __noinline__ void run_f32(const Req &q, int64_t e0, int ne, const OpTab<float> &tf, int *err,
                                     unsigned char *smem) {
    using S = ServeF32<N>;
    const auto sP = SFH_BP(reinterpret_cast<float *>(smem), S::EPB * S::NP * S::NN, err);
    const auto sJF = SFH_BP(reinterpret_cast<float *>(smem + S::OFF_JF), S::EPB * S::JF_EL, err);
    const auto sR = SFH_BP(reinterpret_cast<float *>(smem + S::OFF_R), S::D * S::EPB * S::U_EL, err);
    const auto rawU = SFH_BP(reinterpret_cast<float *>(smem + S::OFF_RU), S::EPB * S::U_EL, err);
    const auto rawJ = SFH_BP(reinterpret_cast<double *>(smem + S::OFF_RJ), S::EPB * S::J_EL, err);
    // the raw u and Ja of a sub-block arrive by per-thread asynchronous copies,
    // issued while the previous sub-block is swept
    auto fetch = [&](int b0) {
        const int nb = ne - b0 < S::EPB ? ne - b0 : S::EPB;
        const auto U = SFH_BP(static_cast<const float *>(q.u), (int64_t)q.n_elem * S::U_EL, err) + (e0 + b0) * S::U_EL;
        const auto J = SFH_BP(q.Ja, (int64_t)q.n_elem * S::J_EL, err) + (e0 + b0) * S::J_EL;
        for (int s = threadIdx.x; s < nb * S::U_EL; s += kThreads) cp_async4_ck(rawU + s, U + s);
        for (int s = threadIdx.x; s < nb * S::J_EL; s += kThreads) cp_async8_ck(rawJ + s, J + s);
        cp_async_commit();
    };
    int bad = 0;
    fetch(0);
    for (int b0 = 0; b0 < ne; b0 += S::EPB) {
        const int nb = ne - b0 < S::EPB ? ne - b0 : S::EPB;
        cp_async_wait_all();
        __syncthreads();
        bad |= fp32_block_convert<S, 3, N, FLUX>(rawU, rawJ, nb, sP, sJF, threadIdx.x, kThreads);
        __syncthreads();
        if (b0 + S::EPB < ne) fetch(b0 + S::EPB);
        fp32_block_sweep<S, 3, N, FLUX>(threadIdx.x, nb, sP, sJF, sR, tf);
        __syncthreads();
        fp32_block_store<S, 3>(sR, SFH_BP(static_cast<float *>(q.out), (int64_t)q.n_elem * S::U_EL, err) + (e0 + b0) * S::U_EL,
                               nb, threadIdx.x, kThreads);
        __syncthreads();
    }
    if (bad) atomicOr(err, bad);
}
template <int N, int FLUX>
__device__ __noinline__ void run_mix(const Req &q, int64_t e0, int ne, const OpTab<float> &tf, int *err,
                                     unsigned char *smem) {
    const int64_t nu = (int64_t)q.n_elem * 5 * N * N * N, nj = (int64_t)q.n_elem * 9 * N * N * N;
    volume_tile<3, N, FLUX, ModeMixed, typename Cls<N, FLUX>::MIX>(SFH_BP(static_cast<const float *>(q.u), nu, err),
                                                                   SFH_BP(q.Ja, nj, err),
                                                                   SFH_BP(static_cast<float *>(q.out), nu, err), e0, ne,
                                                                   tf, err, smem);
}

template <int N, int FLUX>
__device__ __forceinline__ void run_tile_f(const Req &q, int64_t e0, int ne, const OpTab<double> &td,
                                           const OpTab<float> &tf, int *err, unsigned char *smem) {
    if (q.kind == SFH_REQ_VJP) run_vjp<N, FLUX>(q, e0, ne, td, err, smem);
    else if (q.prec == SFH_FP64) run_f64<N, FLUX>(q, e0, ne, td, err, smem);
    else if (q.prec == SFH_FP32_KAHAN) run_f32<N, FLUX>(q, e0, ne, tf, err, smem);
    else run_mix<N, FLUX>(q, e0, ne, tf, err, smem);
}
template <int N>
__device__ __forceinline__ void run_tile(const Req &q, int64_t e0, int ne, const OpTab<double> &td,
                                         const OpTab<float> &tf, int *err, unsigned char *smem) {
    if (q.flux == kFluxEulerCh) run_tile_f<N, kFluxEulerCh>(q, e0, ne, td, tf, err, smem);
    else run_tile_f<N, kFluxEuler>(q, e0, ne, td, tf, err, smem);
}

__global__ void __launch_bounds__(kThreads, 1) serve_kernel(const __grid_constant__ Args a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Req s_req;
    __shared__ int s_tile, s_slot, s_exit;
    __shared__ OpTab<double> s_td;
    __shared__ OpTab<float> s_tf;

    // Idle exit is all-or-nothing: a CTA that found nothing to claim for idle_ns
    // counts itself idle (and uncounts itself when work appears); the kernel
    // leaves only when every CTA is idle, so a lull never thins out the CTAs
    // of a kernel that keeps running.  The host relaunches it for new work.
    unsigned long long last_tail = 0, known_tail = 0;   // known_tail: last tail read (acquire)
    uint64_t quiet_since = global_timer_ns();
    bool counted_idle = false;
    for (;;) {
        uint64_t t_claim = 0;
        if (threadIdx.x == 0) {
            t_claim = global_timer_ns();
            s_exit = 1;
            for (uint32_t it = 0; it < (1u << 28); ++it) {
                const unsigned long long h = *reinterpret_cast<volatile unsigned long long *>(&a.ctrl->head);
                // the host-mapped tail is read (system-scope acquire) only when
                // the head has caught up with the last value seen: entries
                // below a tail that was acquired are published
                if (h >= known_tail) known_tail = ld_acquire_sys_u64(a.tail);
                const unsigned long long t = known_tail;
                if (t != last_tail) {
                    last_tail = t;
                    quiet_since = global_timer_ns();
                }
                if (h < t) {
                    if (counted_idle) {
                        atomicSub(&a.ctrl->idle_ctas, 1);
                        counted_idle = false;
                    }
                    if (atomicCAS(&a.ctrl->head, h, h + 1) == h) {
                        const volatile Tile *te = a.ring + (h % kRing);
                        const int slot = te->slot;
                        s_tile = te->tile;
                        // the 64-byte descriptor in four 16-byte volatile loads
                        const volatile uint4 *src = reinterpret_cast<const volatile uint4 *>(a.reqs + slot);
                        uint4 *dst = reinterpret_cast<uint4 *>(&s_req);
#pragma unroll
                        for (int w = 0; w < 4; ++w) {
                            uint4 v;
                            v.x = src[w].x; v.y = src[w].y; v.z = src[w].z; v.w = src[w].w;
                            dst[w] = v;
                        }
                        s_slot = slot;
                        s_exit = 0;
                        break;
                    }
                    continue;
                }
                if (*a.stop || *reinterpret_cast<volatile int *>(&a.ctrl->quit)) break;
                if ((it & 15u) == 15u) {
                    if (!counted_idle && global_timer_ns() - quiet_since > a.idle_ns) {
                        atomicAdd(&a.ctrl->idle_ctas, 1);
                        counted_idle = true;
                    }
                    if (counted_idle && *reinterpret_cast<volatile int *>(&a.ctrl->idle_ctas) >= (int)gridDim.x) {
                        atomicExch(&a.ctrl->quit, 1);
                        break;
                    }
                }
                __nanosleep(256);
            }
        }
        __syncthreads();
        if (s_exit) return;
        const Req &q = s_req;
        const int slot = s_slot;
        const int tabi = q.nodes * 10 + q.n;
        // debug build: a descriptor whose slot or operator-table index leaves
        // its array is skipped, with kErrBounds latched in slot 0's error word
        // (the skipped request never completes and times out on the host)
        if (kDebugBuild && !dbg_require((unsigned)slot < (unsigned)kMaxSlots && (unsigned)tabi < 20u, &a.ctrl->err[0])) {
            __syncthreads();
            continue;
        }
        for (int i = threadIdx.x; i < (int)(sizeof(OpTab<double>) / 8); i += blockDim.x)
            reinterpret_cast<double *>(&s_td)[i] = reinterpret_cast<const double *>(a.tabd + tabi)[i];
        for (int i = threadIdx.x; i < (int)(sizeof(OpTab<float>) / 4); i += blockDim.x)
            reinterpret_cast<float *>(&s_tf)[i] = reinterpret_cast<const float *>(a.tabf + tabi)[i];
        __syncthreads();
        uint64_t t_run = 0;
        if (threadIdx.x == 0) {
            t_run = global_timer_ns();
            atomicAdd(&a.ctrl->claim_ns, (unsigned long long)(t_run - t_claim));
            atomicMin(&a.ctrl->t_start[s_slot], (unsigned long long)t_run);
        }
        const int64_t e0 = (int64_t)s_tile * q.epb;
        const int ne = (int)((q.n_elem - e0) < q.epb ? (q.n_elem - e0) : q.epb);
        int *err = &a.ctrl->err[slot];
        switch (q.n) {
            case 3: run_tile<3>(q, e0, ne, s_td, s_tf, err, smem); break;
            case 4: run_tile<4>(q, e0, ne, s_td, s_tf, err, smem); break;
            case 5: run_tile<5>(q, e0, ne, s_td, s_tf, err, smem); break;
            case 6: run_tile<6>(q, e0, ne, s_td, s_tf, err, smem); break;
            case 7: run_tile<7>(q, e0, ne, s_td, s_tf, err, smem); break;
            case 8: run_tile<8>(q, e0, ne, s_td, s_tf, err, smem); break;
            case 9: run_tile<9>(q, e0, ne, s_td, s_tf, err, smem); break;
            default: break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int cls = q.kind == SFH_REQ_VJP ? 3 : (q.prec == SFH_FP64 ? 0 : (q.prec == SFH_FP32_KAHAN ? 1 : 2));
            atomicAdd(&a.ctrl->tiles[cls], 1ull);
            atomicAdd(&a.ctrl->busy_ns[cls], (unsigned long long)(global_timer_ns() - t_run));
            __threadfence();   // this tile's output before the count
            const int done = atomicAdd(&a.ctrl->done_tiles[slot], 1) + 1;
            if (done == q.ntiles) {
                __threadfence();
                const int st = atomicExch(&a.ctrl->err[slot], 0);
                const unsigned long long ts = atomicExch(&a.ctrl->t_start[slot], ~0ull);
                a.ctrl->done_tiles[slot] = 0;
                __threadfence_system();
                volatile Done *dn = a.done + slot;
                dn->status = st ? ((kDebugBuild && (st & kErrBounds)) ? SFH_EBOUNDS
                                                                      : (st & kErrTimeout ? SFH_ETIMEOUT : SFH_EDOMAIN))
                                : SFH_OK;
                dn->t_start = ts;
                __threadfence_system();
                dn->seq = q.seq;
            }
        }
        __syncthreads();
    }
}

// Device timer read into mapped host memory (clock calibration).
__global__ void read_timer_kernel(volatile unsigned long long *out) {
    if (threadIdx.x == 0) {
        *out = global_timer_ns();
        __threadfence_system();
    }
}

}  // namespace serve
}  // namespace sfh

// ---------------------------------------------------------------------------
// host runtime
// ---------------------------------------------------------------------------
using namespace sfh::serve;

namespace {

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Pending {
    uint64_t ticket;
    sfh_request req;
    size_t bytes;
    int epb, ntiles;
    uint64_t t_submit;
};

struct Inflight {
    uint64_t ticket;
    size_t bytes;
    int ntiles;
    uint32_t seq;
    uint64_t t_submit, t_admit;
    bool abandoned;   // reported SFH_ETIMEOUT to the caller; slot and budget held until the device finishes
};

// Test-only fault injection (sfh_serve_inject_fault): host-side faults only.
std::atomic<int> g_fail_alloc{0};   // the next server creation fails at this allocation (1-based; 0 off)

size_t req_bytes(const sfh_request &r) {
    const size_t nn = (size_t)(r.p + 1) * (r.p + 1) * (r.p + 1);
    const size_t esz = (r.kind == SFH_REQ_VJP || r.prec == SFH_FP64) ? 8 : 4;
    size_t b = (size_t)r.n_elem * nn * (2 * 5 * esz + 9 * sizeof(double));
    if (r.kind == SFH_REQ_VJP) b += (size_t)r.n_elem * nn * 5 * sizeof(double);
    return b;
}

}  // namespace

struct sfh_server {
    sfh_server_opts opts;
    int device;
    int n_workers;
    // mapped host memory
    Tile *ring_h;
    Req *reqs_h;
    Done *done_h;
    volatile unsigned long long *tail_h;
    volatile int *stop_h;
    Args args;
    DevCtrl *ctrl_d;
    sfh::OpTab<double> *tabd_d;
    sfh::OpTab<float> *tabf_d;
    cudaStream_t stream;
    // host state
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Pending> pending;
    Inflight slots[kMaxSlots];
    bool slot_busy[kMaxSlots];
    uint32_t slot_seq[kMaxSlots];
    int inflight = 0;
    int abandoned = 0;   // in flight but already reported SFH_ETIMEOUT
    size_t used_bytes = 0;
    uint64_t tiles_live = 0;
    uint64_t tail = 0;
    uint64_t next_ticket = 1;
    std::unordered_map<uint64_t, sfh_result> results;
    std::unordered_map<uint64_t, int> where;   // 0 pending, 1 inflight, 2 done
    bool quit = false;
    bool kernel_error = false;
    std::thread worker;
    int64_t clk_offset = 0;       // host steady clock - device timer (ns)
    int inject_drop_tile = 0;     // test hook: publish all but the last tile of the next N admitted requests
    int inject_stall_ms = 0;      // test hook: the admission thread sleeps this long once
    bool give_up = false;         // destroy after a failed drain: stop relaunching, leave the loop
};

namespace {

sfh_status launch(sfh_server *s) {
    // a fresh kernel starts with no idle CTAs and no exit decision
    if (cudaMemsetAsync(&s->ctrl_d->idle_ctas, 0, 2 * sizeof(int), s->stream) != cudaSuccess) return SFH_ECUDA;
    serve_kernel<<<s->n_workers, kThreads, kSmem, s->stream>>>(s->args);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SFH_OK : SFH_ECUDA;
}

void admission_loop(sfh_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        // completions
        if (s->inject_stall_ms > 0) {   // test hook: a stalled admission thread
            const int ms = s->inject_stall_ms;
            s->inject_stall_ms = 0;
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::milliseconds(ms));
            lk.lock();
        }
        const uint64_t t_now = now_ns();
        for (int k = 0; k < s->opts.max_inflight; ++k) {
            if (!s->slot_busy[k]) continue;
            const volatile Done *dn = s->done_h + k;
            if (dn->seq != s->slots[k].seq) {
                // watchdog: a request in flight for longer than timeout_ms is
                // reported SFH_ETIMEOUT; its slot and budget stay held until
                // the device finishes it (it may still read its arrays)
                if (!s->slots[k].abandoned &&
                    t_now - s->slots[k].t_admit > (uint64_t)s->opts.timeout_ms * 1000000ull) {
                    s->slots[k].abandoned = true;
                    sfh_result r = {SFH_ETIMEOUT, s->slots[k].t_submit, s->slots[k].t_admit, 0, t_now};
                    s->results[s->slots[k].ticket] = r;
                    s->where[s->slots[k].ticket] = 2;
                    ++s->abandoned;
                    s->cv.notify_all();
                }
                continue;
            }
            std::atomic_thread_fence(std::memory_order_acquire);
            if (s->slots[k].abandoned) {
                --s->abandoned;   // already reported; only the resources come back
            } else {
                sfh_result r;
                r.status = dn->status;
                r.t_submit_ns = s->slots[k].t_submit;
                r.t_admit_ns = s->slots[k].t_admit;
                const unsigned long long ts = dn->t_start;
                r.t_start_ns = ts == ~0ull ? 0 : (uint64_t)((int64_t)ts + s->clk_offset);
                r.t_done_ns = now_ns();
                s->results[s->slots[k].ticket] = r;
                s->where[s->slots[k].ticket] = 2;
            }
            s->slot_busy[k] = false;
            s->used_bytes -= s->slots[k].bytes;
            s->tiles_live -= (uint64_t)s->slots[k].ntiles;
            --s->inflight;
            s->cv.notify_all();
        }
        // admissions, FIFO
        while (!s->pending.empty() && s->inflight < s->opts.max_inflight) {
            Pending &pq = s->pending.front();
            if (s->used_bytes + pq.bytes > s->opts.hbm_budget_bytes) break;
            if (s->tiles_live + (uint64_t)pq.ntiles > kRing) break;
            int k = 0;
            while (s->slot_busy[k]) ++k;
            const uint32_t seq = ++s->slot_seq[k];
            Req &q = s->reqs_h[k];
            q.kind = (int16_t)pq.req.kind;
            q.flux = (int16_t)pq.req.flux;
            q.prec = pq.req.kind == SFH_REQ_VJP ? SFH_FP64 : pq.req.prec;
            q.n = pq.req.p + 1;
            q.nodes = pq.req.nodes;
            q.n_elem = (int32_t)pq.req.n_elem;
            q.u = pq.req.u;
            q.Ja = pq.req.Ja;
            q.lam = pq.req.lambda;
            q.out = pq.req.out;
            q.epb = pq.epb;
            q.ntiles = pq.ntiles;
            q.seq = seq;
            int publish = pq.ntiles;
            if (s->inject_drop_tile > 0 && pq.ntiles > 0) {   // test hook: a tile that is never published
                --s->inject_drop_tile;
                --publish;
            }
            for (int t = 0; t < publish; ++t) {
                Tile &te = s->ring_h[(s->tail + t) % kRing];
                te.slot = k;
                te.tile = t;
            }
            std::atomic_thread_fence(std::memory_order_release);
            s->tail += (uint64_t)publish;
            *s->tail_h = s->tail;
            Inflight &f = s->slots[k];
            f.ticket = pq.ticket;
            f.bytes = pq.bytes;
            f.ntiles = pq.ntiles;
            f.seq = seq;
            f.t_submit = pq.t_submit;
            f.t_admit = now_ns();
            f.abandoned = false;
            s->slot_busy[k] = true;
            s->where[pq.ticket] = 1;
            s->used_bytes += pq.bytes;
            s->tiles_live += (uint64_t)pq.ntiles;
            ++s->inflight;
            s->pending.pop_front();
        }
        // keep the persistent kernel alive while work is in flight (a
        // request whose tiles will never all arrive keeps it relaunching at
        // the idle interval until the server is destroyed)
        if (s->inflight > 0 && !s->kernel_error && !s->give_up) {
            const cudaError_t q = cudaStreamQuery(s->stream);
            if (q == cudaSuccess) {
                if (launch(s) != SFH_OK) s->kernel_error = true;
            } else if (q != cudaErrorNotReady) {
                s->kernel_error = true;
            }
        }
        if (s->kernel_error) {
            // fail everything in flight: the device cannot be trusted to finish it
            for (int k = 0; k < s->opts.max_inflight; ++k) {
                if (!s->slot_busy[k]) continue;
                if (!s->slots[k].abandoned) {
                    sfh_result r = {SFH_ECUDA, s->slots[k].t_submit, s->slots[k].t_admit, 0, now_ns()};
                    s->results[s->slots[k].ticket] = r;
                    s->where[s->slots[k].ticket] = 2;
                } else {
                    --s->abandoned;
                }
                s->slot_busy[k] = false;
                s->used_bytes -= s->slots[k].bytes;
                s->tiles_live -= (uint64_t)s->slots[k].ntiles;
                --s->inflight;
            }
            s->cv.notify_all();
        }
        if (s->quit && ((s->pending.empty() && s->inflight == 0) || s->give_up)) break;
        if (s->inflight == 0 && s->pending.empty()) {
            s->cv.wait_for(lk, std::chrono::milliseconds(2));
        } else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

}  // namespace

namespace {

// Allocation step k (1-based) of a server creation: fails with `e` when the
// test hook asked for it, else performs `op`.
template <class Op>
cudaError_t alloc_step(int k, Op op) {
    int want = g_fail_alloc.load();
    if (want == k && g_fail_alloc.compare_exchange_strong(want, 0)) return cudaErrorMemoryAllocation;
    return op();
}

// Host steady clock minus device timer, from the tightest of a few
// launch-and-wait brackets around one read of the device timer.
cudaError_t calibrate_clock(cudaStream_t st, volatile unsigned long long *h, unsigned long long *d, int64_t *out) {
    int64_t best_w = INT64_MAX, best = 0;
    for (int it = 0; it < 5; ++it) {
        *h = 0;
        const uint64_t t0 = now_ns();
        read_timer_kernel<<<1, 32, 0, st>>>(d);
        cudaError_t e = cudaStreamSynchronize(st);
        const uint64_t t1 = now_ns();
        if (e != cudaSuccess) return e;
        if ((int64_t)(t1 - t0) < best_w) {
            best_w = (int64_t)(t1 - t0);
            best = (int64_t)((t0 + t1) / 2) - (int64_t)*h;
        }
    }
    *out = best;
    return cudaSuccess;
}

}  // namespace

extern "C" sfh_status sfh_server_create(const sfh_server_opts *opts, sfh_server **out) {
    if (!out) return SFH_EINVAL;
    *out = nullptr;
    if (!opts || opts->max_inflight < 1 || opts->max_inflight > kMaxSlots || opts->timeout_ms < 1 ||
        opts->hbm_budget_bytes == 0 || opts->n_workers < 0)
        return SFH_EINVAL;
    sfh_server *s = new (std::nothrow) sfh_server();
    if (!s) return SFH_ENOMEM;
    s->opts = *opts;
    cudaError_t e = cudaGetDevice(&s->device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e != cudaSuccess) { delete s; return SFH_ECUDA; }
    s->n_workers = opts->n_workers > 0 ? opts->n_workers : sms;
    memset(s->slot_busy, 0, sizeof s->slot_busy);
    memset(s->slot_seq, 0, sizeof s->slot_seq);
    // mapped host memory for the ring, descriptors, completions, control words
    // and the clock-calibration word
    const size_t hbytes = sizeof(Tile) * kRing + sizeof(Req) * kMaxSlots + sizeof(Done) * kMaxSlots + 128;
    void *h = nullptr;
    if ((e = alloc_step(1, [&] { return cudaHostAlloc(&h, hbytes, cudaHostAllocMapped); })) != cudaSuccess) {
        delete s;
        return SFH_ENOMEM;
    }
    memset(h, 0, hbytes);
    char *hc = static_cast<char *>(h);
    s->ring_h = reinterpret_cast<Tile *>(hc);
    s->reqs_h = reinterpret_cast<Req *>(hc + sizeof(Tile) * kRing);
    s->done_h = reinterpret_cast<Done *>(hc + sizeof(Tile) * kRing + sizeof(Req) * kMaxSlots);
    s->tail_h = reinterpret_cast<volatile unsigned long long *>(hc + hbytes - 128);
    s->stop_h = reinterpret_cast<volatile int *>(hc + hbytes - 96);
    volatile unsigned long long *clk_h = reinterpret_cast<volatile unsigned long long *>(hc + hbytes - 64);
    void *dh = nullptr;
    if ((e = cudaHostGetDevicePointer(&dh, h, 0)) != cudaSuccess) { cudaFreeHost(h); delete s; return SFH_ECUDA; }
    char *dc = static_cast<char *>(dh);
    s->args.ring = reinterpret_cast<const Tile *>(dc);
    s->args.reqs = reinterpret_cast<const Req *>(dc + sizeof(Tile) * kRing);
    s->args.done = reinterpret_cast<Done *>(dc + sizeof(Tile) * kRing + sizeof(Req) * kMaxSlots);
    s->args.tail = reinterpret_cast<const volatile unsigned long long *>(dc + hbytes - 128);
    s->args.stop = reinterpret_cast<const volatile int *>(dc + hbytes - 96);
    unsigned long long *clk_d = reinterpret_cast<unsigned long long *>(dc + hbytes - 64);
    s->args.idle_ns = 2000000ull;   // 2 ms without work: CTAs leave, the host relaunches on demand
    // device: control block and operator tables for every (node set, n)
    s->ctrl_d = nullptr;
    s->tabd_d = nullptr;
    s->tabf_d = nullptr;
    if ((e = alloc_step(2, [&] { return cudaMalloc(&s->ctrl_d, sizeof(DevCtrl)); })) != cudaSuccess ||
        (e = alloc_step(3, [&] { return cudaMalloc(&s->tabd_d, sizeof(sfh::OpTab<double>) * 20); })) != cudaSuccess ||
        (e = alloc_step(4, [&] { return cudaMalloc(&s->tabf_d, sizeof(sfh::OpTab<float>) * 20); })) != cudaSuccess) {
        cudaFree(s->ctrl_d); cudaFree(s->tabd_d); cudaFreeHost(h); delete s; return SFH_ENOMEM;
    }
    cudaMemset(s->ctrl_d, 0, sizeof(DevCtrl));
    cudaMemset(&s->ctrl_d->t_start, 0xff, sizeof(DevCtrl::t_start));   // no tile started yet
    std::vector<sfh::OpTab<double>> td(20);
    std::vector<sfh::OpTab<float>> tf(20);
    memset(td.data(), 0, sizeof(sfh::OpTab<double>) * 20);
    memset(tf.data(), 0, sizeof(sfh::OpTab<float>) * 20);
    for (int nodes = 0; nodes < 2; ++nodes)
        for (int p = kPMin; p <= kPMax; ++p) sfh::op_tables(p, nodes, td[nodes * 10 + p + 1], tf[nodes * 10 + p + 1]);
    cudaMemcpy(s->tabd_d, td.data(), sizeof(sfh::OpTab<double>) * 20, cudaMemcpyHostToDevice);
    cudaMemcpy(s->tabf_d, tf.data(), sizeof(sfh::OpTab<float>) * 20, cudaMemcpyHostToDevice);
    s->args.ctrl = s->ctrl_d;
    s->args.tabd = s->tabd_d;
    s->args.tabf = s->tabf_d;
    if ((e = cudaFuncSetAttribute(serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess) {
        cudaFree(s->ctrl_d); cudaFree(s->tabd_d); cudaFree(s->tabf_d); cudaFreeHost(h); delete s; return SFH_ECUDA;
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess ||
        (e = calibrate_clock(s->stream, clk_h, clk_d, &s->clk_offset)) != cudaSuccess) {
        cudaStreamDestroy(s->stream); cudaFree(s->ctrl_d); cudaFree(s->tabd_d); cudaFree(s->tabf_d);
        cudaFreeHost(h); delete s; return SFH_ECUDA;
    }
    s->worker = std::thread(admission_loop, s);
    *out = s;
    return SFH_OK;
}

extern "C" sfh_status sfh_serve_inject_fault(sfh_server *s, int kind, int arg) {
    if (kind == SFH_FAULT_CREATE_ALLOC) {
        if (arg < 0 || arg > 4) return SFH_EINVAL;
        g_fail_alloc.store(arg);
        return SFH_OK;
    }
    if (!s || arg < 0) return SFH_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (kind == SFH_FAULT_DROP_TILE) s->inject_drop_tile = arg;
    else if (kind == SFH_FAULT_STALL_ADMISSION) s->inject_stall_ms = arg;
    else return SFH_EINVAL;
    s->cv.notify_all();
    return SFH_OK;
}

extern "C" sfh_status sfh_serve_submit(sfh_server *s, const sfh_request *r, uint64_t *ticket) {
    if (!s || !r || !ticket) return SFH_EINVAL;
    if (r->kind != SFH_REQ_RESIDUAL && r->kind != SFH_REQ_VJP) return SFH_EINVAL;
    if (r->p < kPMin || r->p > kPMax || (r->nodes != SFH_NODES_GLL && r->nodes != SFH_NODES_GAUSS)) return SFH_EINVAL;
    if (r->flux != SFH_FLUX_EULER_RANOCHA && r->flux != SFH_FLUX_EULER_CHANDRASHEKAR) return SFH_EINVAL;
    if (r->kind == SFH_REQ_RESIDUAL && r->prec != SFH_FP64 && r->prec != SFH_FP32_KAHAN && r->prec != SFH_FP32_MIXED)
        return SFH_EINVAL;
    if (r->n_elem < 1 || r->n_elem > (int64_t)1 << 30 || !r->u || !r->Ja || !r->out || (r->kind == SFH_REQ_VJP && !r->lambda)) return SFH_EINVAL;
    const bool f64 = r->kind == SFH_REQ_VJP || r->prec == SFH_FP64;
    const uintptr_t al = f64 ? 8 : 4;
    if (((uintptr_t)r->u | (uintptr_t)r->out) % al || (uintptr_t)r->Ja % 8 ||
        (r->kind == SFH_REQ_VJP && (uintptr_t)r->lambda % 8))
        return SFH_EINVAL;
    Pending pq;
    pq.req = *r;
    pq.bytes = req_bytes(*r);
    if (pq.bytes > s->opts.hbm_budget_bytes) return SFH_ENOMEM;
    pq.epb = tile_epb(r->kind, r->kind == SFH_REQ_VJP ? SFH_FP64 : r->prec, r->p + 1);
    const int64_t nt = (r->n_elem + pq.epb - 1) / pq.epb;
    if (nt > (int64_t)kRing) return SFH_ENOMEM;
    pq.ntiles = (int)nt;
    pq.t_submit = now_ns();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->quit) return SFH_EBUSY;
    pq.ticket = s->next_ticket++;
    s->where[pq.ticket] = 0;
    s->pending.push_back(pq);
    *ticket = pq.ticket;
    s->cv.notify_all();
    return SFH_OK;
}

extern "C" sfh_status sfh_serve_poll(sfh_server *s, uint64_t ticket, sfh_result *out) {
    if (!s || !out) return SFH_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto w = s->where.find(ticket);
    if (w == s->where.end()) return SFH_EINVAL;
    if (w->second != 2) return SFH_ENOTREADY;
    *out = s->results[ticket];
    s->results.erase(ticket);
    s->where.erase(w);
    return SFH_OK;
}

extern "C" sfh_status sfh_serve_stats(sfh_server *s, sfh_serve_stats_t *out) {
    if (!s || !out) return SFH_EINVAL;
    DevCtrl c;
    cudaError_t e = cudaSetDevice(s->device);
    if (e == cudaSuccess) e = cudaMemcpy(&c, s->ctrl_d, sizeof c, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return SFH_ECUDA;
    for (int k = 0; k < 4; ++k) {
        out->tiles[k] = c.tiles[k];
        out->busy_ns[k] = c.busy_ns[k];
    }
    out->claim_ns = c.claim_ns;
    return SFH_OK;
}

extern "C" sfh_status sfh_serve_drain(sfh_server *s, int timeout_ms) {
    if (!s) return SFH_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                   [s] { return s->pending.empty() && s->inflight == 0; });
    return ok ? SFH_OK : SFH_ETIMEOUT;
}

extern "C" sfh_status sfh_server_destroy(sfh_server *s) {
    if (!s) return SFH_OK;
    sfh_status st = sfh_serve_drain(s, s->opts.timeout_ms);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->quit = true;
        if (st != SFH_OK) {
            // give up on what is left: nothing more is admitted or relaunched;
            // requests still in flight (never completed) stay unreported
            s->pending.clear();
            s->give_up = true;
        }
        s->cv.notify_all();
    }
    *s->stop_h = 1;
    // the admission thread leaves once nothing is in flight, or at once after
    // a failed drain; every wait of its loop is short, so the join is bounded
    s->worker.join();
    // the persistent kernel leaves on the stop word (a CTA finishes the tile it
    // runs first); wait for it, bounded.  Only then can nothing on the device
    // touch the server's memory.
    const uint64_t t1 = now_ns();
    while (cudaStreamQuery(s->stream) == cudaErrorNotReady) {
        if (now_ns() - t1 > (uint64_t)s->opts.timeout_ms * 1000000ull) return SFH_ETIMEOUT;   // cannot free safely
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
    cudaStreamDestroy(s->stream);
    cudaFree(s->ctrl_d);
    cudaFree(s->tabd_d);
    cudaFree(s->tabf_d);
    cudaFreeHost(s->ring_h);   // base of the mapped allocation
    delete s;
    return st;
}

extern "C" sfh_status sfh_serve_replay(sfh_server *s, int n, const sfh_request *reqs, const double *arrival_s,
                                       sfh_result *results, int timeout_ms) {
    if (!s || n < 0 || (n > 0 && (!reqs || !arrival_s || !results)) || timeout_ms < 1) return SFH_EINVAL;
    std::vector<uint64_t> tickets((size_t)n, 0);
    std::vector<int> open;            // submitted, not yet done
    open.reserve((size_t)n);
    int n_done = 0, next = 0;
    const uint64_t t0 = now_ns();
    for (int i = 0; i < n; ++i) results[i].status = SFH_ENOTREADY;
    while (n_done < n) {
        const uint64_t now = now_ns();
        // submit everything whose arrival time has come
        while (next < n && now >= t0 + (uint64_t)(arrival_s[next] * 1e9)) {
            const sfh_status st = sfh_serve_submit(s, &reqs[next], &tickets[next]);
            if (st != SFH_OK) {
                results[next] = sfh_result{st, now, now, 0, now};
                ++n_done;
            } else {
                open.push_back(next);
            }
            ++next;
        }
        // collect completions under one lock acquisition per sweep
        if (!open.empty()) {
            std::lock_guard<std::mutex> lk(s->mu);
            size_t w = 0;
            for (size_t k = 0; k < open.size(); ++k) {
                const int i = open[k];
                auto it = s->where.find(tickets[i]);
                if (it != s->where.end() && it->second == 2) {
                    results[i] = s->results[tickets[i]];
                    s->results.erase(tickets[i]);
                    s->where.erase(it);
                    ++n_done;
                } else {
                    open[w++] = i;
                }
            }
            open.resize(w);
        }
        if (now_ns() - t0 > (uint64_t)timeout_ms * 1000000ull) return SFH_ETIMEOUT;
        const uint64_t due = next < n ? t0 + (uint64_t)(arrival_s[next] * 1e9) : UINT64_MAX;
        const uint64_t t = now_ns();
        if (due > t + 30000) std::this_thread::sleep_for(std::chrono::microseconds(10));
    }
    return SFH_OK;
}

// ---------------------------------------------------------------------------
// serving baseline: the same stream as plain single-request launches, FIFO on
// one stream, each enqueued at its arrival time (queueing included)
// ---------------------------------------------------------------------------
extern "C" sfh_status sfh_serial_replay(int n, const sfh_request *reqs, const double *arrival_s,
                                        sfh_result *results, int timeout_ms) {
    if (n < 0 || (n > 0 && (!reqs || !arrival_s || !results)) || timeout_ms < 1) return SFH_EINVAL;
    for (int i = 0; i < n; ++i) {
        const sfh_request &r = reqs[i];
        if ((r.kind != SFH_REQ_RESIDUAL && r.kind != SFH_REQ_VJP) || r.p < kPMin || r.p > kPMax ||
            (r.nodes != SFH_NODES_GLL && r.nodes != SFH_NODES_GAUSS) ||
            (r.flux != SFH_FLUX_EULER_RANOCHA && r.flux != SFH_FLUX_EULER_CHANDRASHEKAR) || r.n_elem < 1 ||
            (i > 0 && arrival_s[i] < arrival_s[i - 1]))
            return SFH_EINVAL;
        results[i] = sfh_result{SFH_ENOTREADY, 0, 0, 0, 0};
    }
    sfh_ctx *ctx[2][2][kPMax + 1] = {};   // [nodes][flux == Chandrashekar][p]
    cudaStream_t st = nullptr;
    std::vector<cudaEvent_t> ev((size_t)n, nullptr);
    std::vector<char> launched((size_t)n, 0);
    sfh_status ret = SFH_OK;
    auto cleanup = [&]() {
        if (st) cudaStreamSynchronize(st);   // every launch is a bounded kernel
        for (int nd = 0; nd < 2; ++nd)
            for (int fl = 0; fl < 2; ++fl)
                for (int p = 0; p <= kPMax; ++p)
                    if (ctx[nd][fl][p]) {
                        if (ret == SFH_OK && sfh_check(ctx[nd][fl][p], st) != SFH_OK) ret = SFH_EDOMAIN;
                        sfh_destroy(ctx[nd][fl][p]);
                    }
        for (auto &x : ev)
            if (x) cudaEventDestroy(x);
        if (st) cudaStreamDestroy(st);
    };
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return SFH_ECUDA;
    for (int i = 0; i < n; ++i)
        if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) {
            ret = SFH_ECUDA;
            cleanup();
            return ret;
        }
    int next = 0, head = 0, n_done = 0;
    uint64_t prev_done = 0;
    const uint64_t t0 = now_ns();
    while (n_done < n) {
        // enqueue every request whose arrival time has come
        while (next < n && now_ns() >= t0 + (uint64_t)(arrival_s[next] * 1e9)) {
            const sfh_request &r = reqs[next];
            sfh_ctx *&c = ctx[r.nodes][r.flux == SFH_FLUX_EULER_CHANDRASHEKAR ? 1 : 0][r.p];
            sfh_status s1 = SFH_OK;
            if (!c) s1 = sfh_create(3, r.p, (sfh_nodes)r.nodes, 5, (sfh_flux)r.flux, &c);
            const uint64_t t = now_ns();
            if (s1 == SFH_OK)
                s1 = r.kind == SFH_REQ_VJP
                         ? sfh_vjp(c, r.n_elem, static_cast<const double *>(r.u), r.Ja, r.lambda,
                                   static_cast<double *>(r.out), st)
                         : sfh_volume_residual(c, r.n_elem, r.u, r.Ja, r.out, (sfh_prec)r.prec, st);
            results[next] = sfh_result{s1, t, t, 0, t};
            if (s1 == SFH_OK && cudaEventRecord(ev[next], st) == cudaSuccess) {
                launched[next] = 1;
                results[next].status = SFH_ENOTREADY;
            } else {
                if (s1 == SFH_OK) results[next].status = SFH_ECUDA;
                ++n_done;
            }
            ++next;
        }
        // completions, in FIFO order
        while (head < next) {
            if (!launched[head]) { ++head; continue; }
            const cudaError_t q = cudaEventQuery(ev[head]);
            if (q == cudaErrorNotReady) break;
            const uint64_t t = now_ns();
            sfh_result &r = results[head];
            r.t_start_ns = r.t_admit_ns > prev_done ? r.t_admit_ns : prev_done;
            r.t_done_ns = t;
            r.status = q == cudaSuccess ? SFH_OK : SFH_ECUDA;
            prev_done = t;
            ++n_done;
            ++head;
        }
        if (now_ns() - t0 > (uint64_t)timeout_ms * 1000000ull) {
            ret = SFH_ETIMEOUT;
            break;
        }
        const uint64_t due = next < n ? t0 + (uint64_t)(arrival_s[next] * 1e9) : UINT64_MAX;
        if (due > now_ns() + 30000) std::this_thread::sleep_for(std::chrono::microseconds(10));
    }
    cleanup();
    return ret;
}
