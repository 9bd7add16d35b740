// sfh_debug.cuh -- bounds checks of the debug build (-DSFH_DEBUG).
//
// The kernels address global and shared memory through BPtr<T>.  Without
// SFH_DEBUG, BPtr<T> is T* and every helper below is the identity, so the
// release kernels are the same code.  With SFH_DEBUG, a BPtr also carries the
// extent [lo, hi) that it may address and the call's error word: an access
// that would leave the extent latches kErrBounds and goes to a scratch word
// instead (a load reads whatever is there, a store is lost).  No thread leaves
// a kernel early and nothing traps, so every barrier still completes and the
// host reads the error with the next status check.  Bulk copies check their
// source and destination ranges the same way; a refused bulk load still
// completes its transaction count on the mbarrier, so its waiters do not wait
// for bytes that never come.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <type_traits>

#include "sfh_tma.cuh"

namespace sfh {

#ifdef SFH_DEBUG

constexpr bool kDebugBuild = true;
#define SFH_RESTRICT

// where a refused access goes (its contents mean nothing; any number of
// threads may use it at once)
static __device__ __align__(16) unsigned char g_dbg_sink[256];

__device__ __forceinline__ bool dbg_inside(const void *q, uint64_t bytes, const void *lo, const void *hi) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(q);
    return a >= reinterpret_cast<uintptr_t>(lo) && a <= reinterpret_cast<uintptr_t>(hi) &&
           bytes <= reinterpret_cast<uintptr_t>(hi) - a;
}

template <class T>
struct BPtr {
    T *p;          // position
    T *lo, *hi;    // the extent it may address, [lo, hi) in bytes
    int *err;      // the call's error word

    __device__ __forceinline__ BPtr() : p(nullptr), lo(nullptr), hi(nullptr), err(nullptr) {}
    __device__ __forceinline__ BPtr(std::nullptr_t) : p(nullptr), lo(nullptr), hi(nullptr), err(nullptr) {}
    __device__ __forceinline__ BPtr(T *p_, T *lo_, T *hi_, int *e) : p(p_), lo(lo_), hi(hi_), err(e) {}
    template <class U, class = std::enable_if_t<std::is_convertible<U *, T *>::value>>
    __device__ __forceinline__ BPtr(const BPtr<U> &o) : p(o.p), lo(o.lo), hi(o.hi), err(o.err) {}

    __device__ __forceinline__ T &at(T *q) const {
        static_assert(sizeof(T) <= sizeof(g_dbg_sink), "scratch too small");
        if (dbg_inside(q, sizeof(T), lo, hi)) return *q;
        atomicOr(err, kErrBounds);
        return *reinterpret_cast<T *>(g_dbg_sink);
    }
    __device__ __forceinline__ T &operator[](int64_t i) const { return at(p + i); }
    __device__ __forceinline__ T &operator*() const { return at(p); }
    __device__ __forceinline__ BPtr operator+(int64_t i) const { return BPtr(p + i, lo, hi, err); }
    __device__ __forceinline__ BPtr operator-(int64_t i) const { return BPtr(p - i, lo, hi, err); }
    __device__ __forceinline__ BPtr &operator+=(int64_t i) {
        p += i;
        return *this;
    }
};

// a checked pointer to the count elements at base
template <class T>
__device__ __forceinline__ BPtr<T> bp(T *base, int64_t count, int *err) {
    return BPtr<T>(base, base, base + count, err);
}
// the same extent seen as another element type
template <class U, class T>
__device__ __forceinline__ BPtr<U> bp_cast(const BPtr<T> &q) {
    return BPtr<U>(reinterpret_cast<U *>(q.p), reinterpret_cast<U *>(q.lo), reinterpret_cast<U *>(q.hi), q.err);
}
// q, computed by address arithmetic, checked against the extent of ext
template <class T>
__device__ __forceinline__ BPtr<T> bp_at(const BPtr<T> &ext, T *q) {
    return BPtr<T>(q, ext.lo, ext.hi, ext.err);
}
// the plain pointer, for inline PTX (the caller checks the range it covers)
template <class T>
__device__ __forceinline__ T *raw(const BPtr<T> &q) {
    return q.p;
}
// true when [q, q + bytes) lies inside q's extent; otherwise latches kErrBounds
template <class T>
__device__ __forceinline__ bool range_ok(const BPtr<T> &q, uint64_t bytes) {
    if (dbg_inside(q.p, bytes, q.lo, q.hi)) return true;
    atomicOr(q.err, kErrBounds);
    return false;
}
// a condition the caller's indexing relies on (an element range inside the
// buffer, a count inside a capacity); false latches kErrBounds
__device__ __forceinline__ bool dbg_require(bool ok, int *err) {
    if (!ok) atomicOr(err, kErrBounds);
    return ok;
}

// bp() for use inside a lambda: the release form does not name err, whose
// capture would change the release code
#define SFH_BP(ptr, count, err) ::sfh::bp((ptr), (count), (err))

#else

constexpr bool kDebugBuild = false;
#define SFH_BP(ptr, count, err) (ptr)
#define SFH_RESTRICT __restrict__

template <class T>
using BPtr = T *;
template <class T>
__device__ __forceinline__ T *bp(T *base, int64_t, int *) {
    return base;
}
template <class U, class T>
__device__ __forceinline__ U *bp_cast(T *q) {
    return reinterpret_cast<U *>(q);
}
template <class T>
__device__ __forceinline__ T *bp_at(T *, T *q) {
    return q;
}
template <class T>
__device__ __forceinline__ T *raw(T *q) {
    return q;
}
template <class T>
__device__ __forceinline__ bool range_ok(T *, uint64_t) {
    return true;
}
__device__ __forceinline__ bool dbg_require(bool ok, int *) { return ok; }

#endif

// Release the transaction count of a bulk load that was not issued.
__device__ __forceinline__ void mbar_complete_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// Bulk copies through checked pointers: in the debug build a copy whose
// source or destination range leaves its extent is not issued (a load then
// completes its bytes on the mbarrier itself).
template <class TD, class TS>
__device__ __forceinline__ void bulk_load_ck(BPtr<TD> dst, BPtr<TS> src, uint32_t bytes, uint64_t *bar) {
    if (kDebugBuild && !(range_ok(dst, bytes) && range_ok(src, bytes))) {
        mbar_complete_tx(bar, bytes);
        return;
    }
    bulk_load(raw(dst), raw(src), bytes, bar);
}
template <class TD, class TS>
__device__ __forceinline__ void bulk_store_ck(BPtr<TD> dst, BPtr<TS> src, uint32_t bytes) {
    if (kDebugBuild && !(range_ok(dst, bytes) && range_ok(src, bytes))) return;
    bulk_store(raw(dst), raw(src), bytes);
}
template <class TD, class TS>
__device__ __forceinline__ void cp_async4_ck(BPtr<TD> dst, BPtr<TS> src) {
    if (kDebugBuild && !(range_ok(dst, 4) && range_ok(src, 4))) return;
    cp_async4(raw(dst), raw(src));
}
template <class TD, class TS>
__device__ __forceinline__ void cp_async8_ck(BPtr<TD> dst, BPtr<TS> src) {
    if (kDebugBuild && !(range_ok(dst, 8) && range_ok(src, 8))) return;
    cp_async8(raw(dst), raw(src));
}

}  // namespace sfh
