// sfh_noalloc.cu -- the volume residual for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: a host application embedding this
// library inside a process whose device memory is owned by another allocator
// (a framework's caching allocator, a memory pool with a fixed budget, or a
// sandbox that forbids runtime allocations after start-up).  They still have
// host buffers and a stream.  This entry point stages u, Ja and r through one
// file-scope device array of fixed size, so it needs neither a context nor an
// allocation: operator tables are built on the host stack, the device error
// word lives at the start of the same array.
//
// The array (SFH_NOALLOC_SCRATCH_BYTES) is part of the library image: every
// GPU that loads the library holds it until the process exits.  Every call
// shares it and it keeps the last call's contents, so the error word is
// cleared at the start of each call, and calls that overlap on the GPU (two
// host threads, or two streams) race on it: callers must serialize them.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/sfhad.h"
#include "sfh_internal.h"

#define SFH_NOALLOC_SCRATCH_BYTES (64u << 20)
#define SFH_NOALLOC_MAX_DEVICES 64

// [0, 256): error word; then u, Ja and r staging, each 256-byte aligned
static __device__ __align__(256) unsigned char g_noalloc_scratch[SFH_NOALLOC_SCRATCH_BYTES];

namespace {

sfh_status na_fail(sfh_status st, const char *fmt, ...) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    sfh::set_error_message(msg);
    return st;
}

std::mutex g_mu;
unsigned char *g_scratch_addr[SFH_NOALLOC_MAX_DEVICES];

// Device address of the scratch array on the current device.  The symbol's
// name is a host-side stand-in in host code, never a device address: the
// address is asked of the runtime once per device, with that device current.
sfh_status scratch_address(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return na_fail(SFH_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return SFH_OK;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" sfh_status sfh_volume_residual_host_noalloc(int d, int p, sfh_nodes nodes, sfh_flux flux, int64_t n_elem,
                                                       const void *u_host, const double *Ja_host, void *r_host,
                                                       sfh_prec prec, sfh_stream_t stream) {
    sfh::set_error_message("");
    if (d != 2 && d != 3) return na_fail(SFH_EINVAL, "d must be 2 or 3, got %d", d);
    if (p < 1 || p > sfh::NMAX - 1) return na_fail(SFH_EINVAL, "p must be in [1, %d], got %d", sfh::NMAX - 1, p);
    if (flux != SFH_FLUX_BURGERS && flux != SFH_FLUX_EULER_RANOCHA && flux != SFH_FLUX_EULER_CHANDRASHEKAR)
        return na_fail(SFH_EINVAL, "bad flux %d", (int)flux);
    if (prec != SFH_FP64 && prec != SFH_FP32_KAHAN && prec != SFH_FP32_MIXED)
        return na_fail(SFH_EINVAL, "bad precision mode %d", (int)prec);
    if (n_elem < 0) return na_fail(SFH_EINVAL, "n_elem must be >= 0");
    if (n_elem == 0) return SFH_OK;
    if (!u_host || !Ja_host || !r_host) return na_fail(SFH_EINVAL, "null array pointer");

    const int n = p + 1, nvar = flux == SFH_FLUX_BURGERS ? 1 : d + 2;
    const size_t nn = (size_t)sfh::ipow(n, d);
    const size_t esz = prec == SFH_FP64 ? 8 : 4;
    // bytes per element (u and r, plus Ja) and the largest element count that
    // fits, found before any product with n_elem so that no size can wrap
    const size_t per_elem = 2 * nvar * nn * esz + d * d * nn * sizeof(double);
    const int64_t max_elem = (int64_t)((SFH_NOALLOC_SCRATCH_BYTES - 256 - 3 * 255) / per_elem);
    if (n_elem > max_elem)
        return na_fail(SFH_EINVAL,
                       "n_elem %lld exceeds the no-allocation entry point's staging array of %u bytes "
                       "(at most %lld elements of this type)",
                       (long long)n_elem, SFH_NOALLOC_SCRATCH_BYTES, (long long)max_elem);
    const size_t ub = (size_t)n_elem * nvar * nn * esz, jb = (size_t)n_elem * d * d * nn * sizeof(double);
    const size_t need = 256 + 2 * up256(ub) + up256(jb);
    if (need > SFH_NOALLOC_SCRATCH_BYTES)   // cannot happen after the element cap; kept as a guard
        return na_fail(SFH_EINVAL, "n_elem %lld needs %zu bytes of device staging; the array holds %u",
                       (long long)n_elem, need, SFH_NOALLOC_SCRATCH_BYTES);

    // operator tables on the host stack (no context), rounded as a context
    // rounds them
    sfh::OpTab<double> tab_d;
    sfh::OpTab<float> tab_f;
    if (!sfh::op_tables(p, nodes, tab_d, tab_f)) return na_fail(SFH_EINVAL, "bad node set %d", (int)nodes);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(SFH_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= SFH_NOALLOC_MAX_DEVICES) return na_fail(SFH_EUNSUPPORTED, "device index %d", dev);
    unsigned char *base = nullptr;
    const sfh_status st = scratch_address(dev, &base);
    if (st != SFH_OK) return st;
    int *d_err = reinterpret_cast<int *>(base);
    unsigned char *du = base + 256;
    unsigned char *dj = du + up256(ub);
    unsigned char *dr = dj + up256(jb);
    cudaStream_t s = (cudaStream_t)stream;

    // the array keeps the previous call's contents: the error word starts at zero
    if ((e = cudaMemsetAsync(d_err, 0, sizeof(int), s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(du, u_host, ub, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dj, Ja_host, jb, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return na_fail(SFH_ECUDA, "staging copy: %s", cudaGetErrorString(e));
    if (prec == SFH_FP64)
        e = sfh::volume_fp64_fn(d, flux)(n, flux, du, (const double *)dj, dr, n_elem, tab_d, d_err, s);
    else if (prec == SFH_FP32_KAHAN)
        e = sfh::volume_fp32k_fn(d, flux)(n, flux, du, (const double *)dj, dr, n_elem, tab_f, d_err, s);
    else
        e = sfh::volume_mixed_fn(d, flux)(n, flux, du, (const double *)dj, dr, n_elem, tab_f, d_err, s);
    if (e != cudaSuccess) return na_fail(SFH_ECUDA, "volume kernel launch: %s", cudaGetErrorString(e));
    int h_err = 0;
    if ((e = cudaMemcpyAsync(r_host, dr, ub, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return na_fail(SFH_ECUDA, "result copy: %s", cudaGetErrorString(e));
    if (h_err) return (sfh_status)sfh::err_word_status(h_err);
    return SFH_OK;
}
