// sfh_tma.cuh -- bulk asynchronous copies (TMA, sm_90+ / sm_103a) and
// mbarrier helpers in inline PTX, with bounded waits.
//
// Every wait here gives up after a time limit (globaltimer) or an iteration
// cap, whichever comes first; the caller then records an error instead of
// spinning forever.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace sfh {

constexpr int kMaxDevices = 64;  // launch facts are cached per device index below this
constexpr int kErrDomain = 1;    // density or pressure <= 0 (or NaN)
constexpr int kErrTimeout = 2;   // a bounded wait gave up
constexpr int kErrMetric = 4;    // a metric term outside the accepted range (see below)
constexpr int kErrBounds = 8;    // debug build: an index outside its buffer (access not made)

// Accepted metric terms, compared on the high word of |Ja| (sign cleared):
// FP32 modes take |Ja| < 2^126, so that its FP32 value and the sum of two of
// them stay finite; FP64 takes any finite value.  Inf and NaN are refused
// everywhere.
constexpr uint32_t kMetricHiFp32 = 0x47d00000u;   // high word of 2^126
constexpr uint32_t kMetricHiFp64 = 0x7ff00000u;   // Inf / NaN exponent
__device__ __forceinline__ uint32_t abs_hi(double x) {
    return static_cast<uint32_t>(static_cast<unsigned long long>(__double_as_longlong(x)) >> 32) & 0x7fffffffu;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// make generic-proxy shared-memory writes visible to the async proxy (TMA)
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// try_wait with a suspend-time hint: a thread whose phase is not complete
// sleeps until it completes or about hint_ns pass, instead of spinning (a
// spinning warp takes issue slots from the warps doing the work).
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the barrier; false if the limit was reached.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && global_timer_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// 1D bulk copy global -> shared, completion counted on `bar` (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// 1D bulk copy shared -> global (bytes % 16 == 0, 16-byte aligned), tracked by
// the issuing thread's bulk group.
__device__ __forceinline__ void bulk_store(void *dst_gmem, const void *src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
                 "r"(smem_addr(src_smem)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared-memory source of every committed bulk store has been read
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed bulk store has completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// SM count of the current device and resident CTAs per SM of a persistent
// kernel, asked of the runtime once per device (the kernel's dynamic
// shared-memory limit is raised on that device at the same time) and cached
// per device.  Both numbers live in one atomic word, (sms << 8) | per_sm,
// published with a release store and read with an acquire load, so that a
// thread that sees the word also sees both numbers (the host may be a weakly
// ordered Arm machine).  Two threads that race on the first call both ask the
// runtime and store the same word.
struct LaunchCache {
    std::atomic<int> packed[kMaxDevices];
};

template <typename Kern>
inline cudaError_t persistent_slots(Kern kern, int threads, size_t smem, LaunchCache &cache, int &per_sm, int &sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    int word = cache.packed[dev].load(std::memory_order_acquire);
    if (word == 0) {
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        int n = 0, k = 0;
        if ((e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, kern, threads, smem)) != cudaSuccess) return e;
        if (k < 1 || k > 255 || n < 1 || n > (1 << 22)) return cudaErrorInvalidConfiguration;
        word = (n << 8) | k;
        cache.packed[dev].store(word, std::memory_order_release);
    }
    per_sm = word & 255;
    sms = word >> 8;
    return cudaSuccess;
}

// Per-thread asynchronous global -> shared copies (cp.async, sm_80+): each
// thread waits only for its own copies, so a wait always ends.
__device__ __forceinline__ void cp_async4(void *dst_smem, const void *src_gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst_smem)), "l"(src_gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst_smem, const void *src_gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst_smem)), "l"(src_gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// FP64 -> FP32 by integer operations (IEEE-754 field arithmetic), so that the
// conversion does not occupy the FP64 pipe.  On the magnitude m (sign removed):
// adding 2^28 rounds the 29 discarded mantissa bits half away from zero (the
// carry may ripple into the exponent, which is the correct rounding), the
// funnel shift by 3 lines the exponent up with bit 23 of the high word, and
// subtracting 896 << 23 re-biases it (1023 -> 127; the modular arithmetic is
// exact because the FP32 exponent fits 8 bits).  Magnitudes below the FP32
// normal range give a signed zero; inputs must stay below 2^128 (metric
// terms are O(h^{d-1})).
__device__ __forceinline__ float d2f_int(double x) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned long long mag = (b & 0x7fffffffffffffffull) + (1ull << 28);
    const uint32_t hi = static_cast<uint32_t>(mag >> 32), lo = static_cast<uint32_t>(mag);
    uint32_t f = __funnelshift_l(lo, hi, 3) - 0xc0000000u;   // (896 << 23) mod 2^32
    f = hi < 0x38100000u ? 0u : f;
    return __uint_as_float(f | (static_cast<uint32_t>(b >> 32) & 0x80000000u));
}

// d2f_int that also keeps the largest high word of the rounded magnitude
// seen (hmax), for the range check against kMetricHiFp32.
__device__ __forceinline__ float d2f_int_track(double x, uint32_t &hmax) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned long long mag = (b & 0x7fffffffffffffffull) + (1ull << 28);
    const uint32_t hi = static_cast<uint32_t>(mag >> 32), lo = static_cast<uint32_t>(mag);
    hmax = max(hmax, hi);
    uint32_t f = __funnelshift_l(lo, hi, 3) - 0xc0000000u;
    f = hi < 0x38100000u ? 0u : f;
    return __uint_as_float(f | (static_cast<uint32_t>(b >> 32) & 0x80000000u));
}

// FP32 -> FP64 by integer operations (exact for normal x; zero and
// subnormal x are not handled), so that the widening does not occupy the
// FP64 pipe: the exponent field moves from bit 23 to bit 52 (of the high
// word: bit 20) and is re-biased by 1023 - 127 = 896.
__device__ __forceinline__ double f2d_int(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t hi = (b & 0x80000000u) | (((b & 0x7fffffffu) >> 3) + (896u << 20));
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(b << 29));
}

// Exact FP32 -> FP64 of a positive normal x by integer operations (three:
// the exponent moves from bit 23 to bit 52 and is re-biased by 896).
__device__ __forceinline__ double f2d_pos(float x) {
    const uint32_t b = __float_as_uint(x);
    return __hiloint2double(static_cast<int>((b >> 3) + (896u << 20)), static_cast<int>(b << 29));
}

// FP64 -> FP32 of a positive value inside the FP32 normal range, rounded half
// away from zero, by integer operations (four: the rounding add with carry,
// the funnel shift and the re-bias of d2f_int, without its sign and
// underflow handling).
__device__ __forceinline__ float d2f_pos(double x) {
    const unsigned long long mag = static_cast<unsigned long long>(__double_as_longlong(x)) + (1ull << 28);
    const uint32_t hi = static_cast<uint32_t>(mag >> 32), lo = static_cast<uint32_t>(mag);
    return __uint_as_float(__funnelshift_l(lo, hi, 3) - 0xc0000000u);
}

// Hardware reciprocal approximation (PTX rcp.approx.ftz.f32: at most 1 ulp
// from 1/x for normal x; subnormal inputs and results flush to zero).
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------------------
// Packed FP32x2 arithmetic (sm_100+): one instruction performs the same
// operation on two independent FP32 lanes (here: two grid lines).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long x = *reinterpret_cast<unsigned long long *>(&a), y = *reinterpret_cast<unsigned long long *>(&b), d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x), "l"(y));
    return *reinterpret_cast<float2 *>(&d);
}

// Kahan accumulation of two lanes at once, with the compensation kept negated
// (cn = -c) so that every step is one packed instruction:
//   y = q f + cn, t = s + y, cn = y - (t - s), s = t;   value = s + cn.
struct KahanF2 {
    float2 s, cn;
    __device__ __forceinline__ void zero() { s = f2s(0.0f); cn = f2s(0.0f); }
    __device__ __forceinline__ void add_prod(float2 q, float2 f) {
        const float2 y = fma2(q, f, cn);
        const float2 t = add2(s, y);
        cn = sub2(y, sub2(t, s));
        s = t;
    }
    __device__ __forceinline__ float2 value() const { return add2(s, cn); }
};

}  // namespace sfh
