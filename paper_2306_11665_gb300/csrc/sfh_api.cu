// sfh_api.cu -- host side of libsfhad: operator tables, contexts, argument
// validation, launches, the host-buffer pipeline and the peak benchmarks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "../../include/sfhad.h"
#include "sfh_internal.h"
#include "sfh_tma.cuh"

// ---------------------------------------------------------------------------
// thread-local error message
// ---------------------------------------------------------------------------
static thread_local char g_err[512];

static sfh_status fail(sfh_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}
static sfh_status cuda_fail(cudaError_t e, const char *what) {
    return fail(SFH_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}
static void clear_err() { g_err[0] = '\0'; }

extern "C" const char *sfh_last_error(void) { return g_err; }

void sfh::set_error_message(const char *msg) { snprintf(g_err, sizeof g_err, "%s", msg); }
extern "C" int sfh_version(void) { return 10000; }

// ---------------------------------------------------------------------------
// 1D operator tables (Eq. 5 needs the collocated Lagrange basis on the nodes).
// Long-double Newton iterations:
//   Gauss-Legendre: roots of P_n, derivative P_n' = n (x P_n - P_{n-1}) / (x^2 - 1);
//   Gauss-Lobatto:  interior roots of P_{p+1} - P_{p-1} (whose roots are +-1 and
//                   the zeros of P_p'), derivative (2p + 1) P_p.
// Weights: 2 / ((1 - x^2) P_n'(x)^2) and 2 / (p (p+1) P_p(x)^2).
// D_ij = l_j'(x_i) = (c_i / c_j) / (x_i - x_j), c_i = prod_{k != i} (x_i - x_k),
// D_ii = sum_{k != i} 1 / (x_i - x_k).
// ---------------------------------------------------------------------------
namespace {

void legendre2(int k, long double x, long double &Pk, long double &Pkm1) {
    long double a = 1.0L, b = x;   // P_0, P_1
    if (k == 0) { Pk = 1.0L; Pkm1 = 0.0L; return; }
    for (int j = 1; j < k; ++j) {
        long double c = ((2 * j + 1) * x * b - j * a) / (j + 1);
        a = b;
        b = c;
    }
    Pk = b;
    Pkm1 = a;
}

bool make_tables(int p, int kind, long double *x, long double *w, long double *D, int pmax = sfh::NMAX - 1) {
    const int n = p + 1;
    const long double PI = 3.141592653589793238462643383279502884L;
    if (p < 1 || p > pmax) return false;
    if (kind == SFH_NODES_GAUSS) {
        for (int j = 0; j < n; ++j) {
            long double xx = -cosl(PI * (4 * j + 3) / (4 * n + 2));
            for (int it = 0; it < 64; ++it) {
                long double P, Pm;
                legendre2(n, xx, P, Pm);
                const long double dP = n * (xx * P - Pm) / (xx * xx - 1.0L);
                const long double step = P / dP;
                xx -= step;
                if (fabsl(step) < 1e-21L) break;
            }
            long double P, Pm;
            legendre2(n, xx, P, Pm);
            const long double dP = n * (xx * P - Pm) / (xx * xx - 1.0L);
            x[j] = xx;
            w[j] = 2.0L / ((1.0L - xx * xx) * dP * dP);
        }
    } else {
        x[0] = -1.0L;
        x[p] = 1.0L;
        for (int j = 1; j < p; ++j) {
            long double xx = -cosl(PI * j / p);
            for (int it = 0; it < 64; ++it) {
                long double Pp1, Pp, Ppm1, tmp;
                legendre2(p + 1, xx, Pp1, Pp);
                legendre2(p - 1, xx, Ppm1, tmp);
                const long double q = Pp1 - Ppm1, dq = (2 * p + 1) * Pp;
                const long double step = q / dq;
                xx -= step;
                if (fabsl(step) < 1e-21L) break;
            }
            x[j] = xx;
        }
        for (int j = 0; j < n; ++j) {
            long double P, Pm;
            legendre2(p, x[j], P, Pm);
            w[j] = 2.0L / ((long double)p * (p + 1) * P * P);
        }
    }
    std::sort(x, x + n);   // Gauss guesses run from -1 up already; keep ascending in any case
    // both node sets are symmetric about 0: enforce it exactly (the middle
    // node of an odd set becomes exactly 0)
    for (int j = 0; j < n / 2; ++j) {
        const long double h = 0.5L * (x[n - 1 - j] - x[j]);
        x[j] = -h;
        x[n - 1 - j] = h;
        const long double wh = 0.5L * (w[j] + w[n - 1 - j]);
        w[j] = wh;
        w[n - 1 - j] = wh;
    }
    if (n % 2) x[n / 2] = 0.0L;
    for (int i = 0; i < n; ++i) {
        long double ci = 1.0L, dii = 0.0L;
        for (int k = 0; k < n; ++k)
            if (k != i) { ci *= (x[i] - x[k]); dii += 1.0L / (x[i] - x[k]); }
        for (int j = 0; j < n; ++j) {
            if (j == i) {
                // Gauss-Lobatto interior nodes and the middle node of an odd
                // symmetric set have D_ii = 0 exactly; keep it exact so that the
                // kernels can skip zero diagonal entries
                const bool zero = (n % 2 && i == n / 2) ||
                                  (kind == SFH_NODES_GLL && i > 0 && i < n - 1);
                D[i * n + j] = zero ? 0.0L : dii;
                continue;
            }
            long double cj = 1.0L;
            for (int k = 0; k < n; ++k)
                if (k != j) cj *= (x[j] - x[k]);
            D[i * n + j] = (ci / cj) / (x[i] - x[j]);
        }
    }
    return true;
}

// Solution basis on the cubature nodes x of a context (Section 2, the
// uncollocated case): V[a*n + k] = chi_k(x_a) with chi_k the orthonormal
// Legendre polynomial sqrt((2k + 1)/2) P_k, or the Lagrange polynomial of the
// k-th Gauss-Lobatto / Gauss solution node (product formula).
bool make_basis(int p, const long double *x, int basis, long double *V) {
    const int n = p + 1;
    if (basis == SFH_BASIS_LEGENDRE) {
        for (int a = 0; a < n; ++a)
            for (int k = 0; k < n; ++k) {
                long double P, Pm;
                legendre2(k, x[a], P, Pm);
                V[a * n + k] = sqrtl((2.0L * k + 1.0L) / 2.0L) * P;
            }
        return true;
    }
    if (basis != SFH_BASIS_LAGRANGE_GLL && basis != SFH_BASIS_LAGRANGE_GAUSS) return false;
    long double s[sfh::NMAX], sw[sfh::NMAX], sD[sfh::NMAX * sfh::NMAX];
    if (!make_tables(p, basis == SFH_BASIS_LAGRANGE_GLL ? SFH_NODES_GLL : SFH_NODES_GAUSS, s, sw, sD)) return false;
    for (int a = 0; a < n; ++a)
        for (int k = 0; k < n; ++k) {
            long double l = 1.0L;
            bool same = false;
            for (int j = 0; j < n; ++j) {
                if (j == k) continue;
                l *= (x[a] - s[j]) / (s[k] - s[j]);
            }
            // a solution node that coincides with a cubature node: exact 0/1
            for (int j = 0; j < n; ++j) same |= (x[a] == s[j]);
            if (same) l = (x[a] == s[k]) ? 1.0L : 0.0L;
            V[a * n + k] = l;
        }
    return true;
}

}  // namespace

extern "C" sfh_status sfh_basis_table(int p, sfh_nodes nodes, sfh_basis basis, double *V) {
    clear_err();
    if (p < 1 || p > sfh::NMAX - 1) return fail(SFH_EINVAL, "p must be in [1, %d], got %d", sfh::NMAX - 1, p);
    if (nodes != SFH_NODES_GLL && nodes != SFH_NODES_GAUSS) return fail(SFH_EINVAL, "bad node set %d", (int)nodes);
    if (!V) return fail(SFH_EINVAL, "V is NULL");
    long double x[sfh::NMAX], ww[sfh::NMAX], DD[sfh::NMAX * sfh::NMAX], VV[sfh::NMAX * sfh::NMAX];
    if (!make_tables(p, nodes, x, ww, DD) || !make_basis(p, x, basis, VV))
        return fail(SFH_EINVAL, "bad basis %d", (int)basis);
    for (int k = 0; k < (p + 1) * (p + 1); ++k) V[k] = (double)VV[k];
    return SFH_OK;
}

extern "C" sfh_status sfh_operator_tables(int p, sfh_nodes nodes, double *xi, double *w, double *D,
                                          double *Q1) {
    clear_err();
    if (p < 1 || p > sfh::NMAX - 1) return fail(SFH_EINVAL, "p must be in [1, %d], got %d", sfh::NMAX - 1, p);
    if (nodes != SFH_NODES_GLL && nodes != SFH_NODES_GAUSS) return fail(SFH_EINVAL, "bad node set %d", (int)nodes);
    long double x[sfh::NMAX], ww[sfh::NMAX], DD[sfh::NMAX * sfh::NMAX];
    if (!make_tables(p, nodes, x, ww, DD)) return fail(SFH_EINVAL, "table construction failed");
    const int n = p + 1;
    for (int i = 0; i < n; ++i) {
        if (xi) xi[i] = (double)x[i];
        if (w) w[i] = (double)ww[i];
        for (int j = 0; j < n; ++j) {
            if (D) D[i * n + j] = (double)DD[i * n + j];
            if (Q1) Q1[i * n + j] = (double)(ww[i] * DD[i * n + j]);
        }
    }
    return SFH_OK;
}

namespace sfh {
bool op_tables(int p, int nodes, OpTab<double> &tab_d, OpTab<float> &tab_f) {
    memset(&tab_d, 0, sizeof tab_d);
    memset(&tab_f, 0, sizeof tab_f);
    if (p < 1 || p > NMAX - 1 || (nodes != SFH_NODES_GLL && nodes != SFH_NODES_GAUSS)) return false;
    long double x[NMAX], ww[NMAX], DD[NMAX * NMAX];
    if (!make_tables(p, nodes, x, ww, DD)) return false;
    const int n = p + 1;
    for (int a = 0; a < n; ++a) {
        tab_d.w[a] = (double)ww[a];
        tab_f.w[a] = (float)ww[a];
        for (int b = 0; b < n; ++b) {
            const long double q = ww[a] * DD[a * n + b];
            tab_d.Q1[a * n + b] = (double)q;
            tab_f.Q1[a * n + b] = (float)q;
        }
    }
    return true;
}
}  // namespace sfh

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
// Host-buffer pipeline: chunks of about kHostChunkBytes (u + Ja + r) rotate
// over kHostStages streams and device staging buffers, so that the copies of
// one chunk overlap the kernel and the result copy of the others.
constexpr int kHostStages = 2;
constexpr size_t kHostChunkBytes = 48u << 20;
// Pipeline of the bound-metric residual: chunks of about kBoundChunkBytes of
// u rotate over kBoundStages streams, H2D(u) -> kernel -> D2H(r) on each.
// With four stages the next chunk's copy in never waits for a copy out on
// the same stream, so both copy directions stay busy; the chunks are small
// enough that the first copy in and the last copy out (the pipeline's
// unoverlapped ends) stay short.
constexpr int kBoundStages = 4;
constexpr size_t kBoundChunkBytes = 4u << 20;

struct sfh_ctx {
    int d, p, n, nodes, nvar, flux, device;
    int *d_err;
    sfh::OpTab<double> tab_d;
    sfh::OpTab<float> tab_f;
    // solution bases on the cubature nodes (indexed by sfh_basis)
    sfh::BasisTab<double> basis_d[3];
    sfh::BasisTab<float> basis_f[3];
    // weights and face-interpolation rows of the surface Hadamard product
    sfh::SurfTab surf;
    // staging of the host-buffer entry point
    std::mutex host_mu;
    cudaStream_t hs[kHostStages];
    void *stage[kHostStages];
    size_t stage_bytes;
    // metric terms bound to the context (sfh_bind_metric): device copy, its
    // element count and capacity in bytes
    double *d_ja;
    int64_t ja_elems;
    size_t ja_bytes;
    // streams and staging buffers of the bound-metric pipeline
    cudaStream_t bs[kBoundStages];
    void *bstage[kBoundStages];
    size_t bstage_bytes;
    // stream-ordered scratch of the modal residual (nullptr: the fused
    // modal kernels serve every call)
    cudaMemPool_t pool;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int mode_of(sfh_prec prec) { return (int)prec; }
size_t elem_size(sfh_prec prec) { return prec == SFH_FP64 ? sizeof(double) : sizeof(float); }

bool overlap(const void *a, size_t na, const void *b, size_t nb) {
    const char *pa = (const char *)a, *pb = (const char *)b;
    return pa < pb + nb && pb < pa + na;
}

cudaError_t launch_volume(sfh_ctx *c, sfh_prec prec, int64_t n_elem, const void *u, const double *Ja, void *r,
                          cudaStream_t s) {
    using namespace sfh;
    if (prec == SFH_FP64) return volume_fp64_fn(c->d, c->flux)(c->n, c->flux, u, Ja, r, n_elem, c->tab_d, c->d_err, s);
    if (prec == SFH_FP32_KAHAN)
        return volume_fp32k_fn(c->d, c->flux)(c->n, c->flux, u, Ja, r, n_elem, c->tab_f, c->d_err, s);
    return volume_mixed_fn(c->d, c->flux)(c->n, c->flux, u, Ja, r, n_elem, c->tab_f, c->d_err, s);
}

}  // namespace

extern "C" sfh_status sfh_create(int d, int p, sfh_nodes nodes, int nvar, sfh_flux flux, sfh_ctx **out) {
    clear_err();
    if (!out) return fail(SFH_EINVAL, "out is NULL");
    *out = nullptr;
    if (d != 2 && d != 3) return fail(SFH_EINVAL, "d must be 2 or 3, got %d", d);
    if (p < 1 || p > sfh::NMAX - 1) return fail(SFH_EINVAL, "p must be in [1, %d], got %d", sfh::NMAX - 1, p);
    if (nodes != SFH_NODES_GLL && nodes != SFH_NODES_GAUSS) return fail(SFH_EINVAL, "bad node set %d", (int)nodes);
    if (flux != SFH_FLUX_BURGERS && flux != SFH_FLUX_EULER_RANOCHA && flux != SFH_FLUX_EULER_CHANDRASHEKAR)
        return fail(SFH_EINVAL, "bad flux %d", (int)flux);
    const int want = flux == SFH_FLUX_BURGERS ? 1 : d + 2;
    if (nvar != want) return fail(SFH_EINVAL, "nvar must be %d for this flux and d = %d, got %d", want, d, nvar);

    double xi[sfh::NMAX], w[sfh::NMAX], D[sfh::NMAX * sfh::NMAX], Q1[sfh::NMAX * sfh::NMAX];
    sfh_status st = sfh_operator_tables(p, nodes, xi, w, D, Q1);
    if (st != SFH_OK) return st;

    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) return fail(SFH_EUNSUPPORTED, "no CUDA device: %s", cudaGetErrorString(e));
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");

    sfh_ctx *c = new (std::nothrow) sfh_ctx();
    if (!c) return fail(SFH_ENOMEM, "host allocation failed");
    c->d = d; c->p = p; c->n = p + 1; c->nodes = nodes; c->nvar = nvar; c->flux = flux; c->device = dev;
    for (int k = 0; k < kHostStages; ++k) {
        c->hs[k] = nullptr;
        c->stage[k] = nullptr;
    }
    c->stage_bytes = 0;
    c->d_ja = nullptr;
    c->ja_elems = 0;
    c->ja_bytes = 0;
    for (int k = 0; k < kBoundStages; ++k) {
        c->bs[k] = nullptr;
        c->bstage[k] = nullptr;
    }
    c->bstage_bytes = 0;
    c->pool = nullptr;
    {
        // a pool of this context's own, so that stream-ordered scratch of
        // concurrent calls never races and freed blocks are kept for reuse
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if (cudaMemPoolCreate(&c->pool, &props) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            if (cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
                cudaMemPoolDestroy(c->pool);
                c->pool = nullptr;
            }
        } else {
            c->pool = nullptr;
            cudaGetLastError();
        }
    }
    const int n = p + 1;
    sfh::op_tables(p, nodes, c->tab_d, c->tab_f);
    long double x[sfh::NMAX], ww[sfh::NMAX], DD[sfh::NMAX * sfh::NMAX];
    make_tables(p, nodes, x, ww, DD);
    for (int b = 0; b < 3; ++b) {
        long double VV[sfh::NMAX * sfh::NMAX];
        memset(&c->basis_d[b], 0, sizeof c->basis_d[b]);
        memset(&c->basis_f[b], 0, sizeof c->basis_f[b]);
        make_basis(p, x, b, VV);
        for (int k = 0; k < n * n; ++k) {
            c->basis_d[b].V[k] = (double)VV[k];
            c->basis_f[b].V[k] = (float)VV[k];
        }
        // chi_0 of the orthonormal Legendre basis is the constant 2^(-1/2)
        const bool cm = b == SFH_BASIS_LEGENDRE;
        const long double c0 = powl(2.0L, -0.5L * d);
        c->basis_d[b].const_mode = c->basis_f[b].const_mode = cm ? 1 : 0;
        c->basis_d[b].c0 = cm ? (double)c0 : 0.0;
        c->basis_f[b].c0 = cm ? (float)c0 : 0.0f;
    }
    memset(&c->surf, 0, sizeof c->surf);
    for (int a = 0; a < n; ++a) {
        c->surf.w[a] = (double)ww[a];
        for (int side = 0; side < 2; ++side) {
            // l_a(-1) / l_a(+1) by the product formula; exactly 0 or 1 where a
            // node sits at the end point (Gauss-Lobatto)
            const long double xe = side ? 1.0L : -1.0L;
            long double l = 1.0L;
            for (int j = 0; j < n; ++j)
                if (j != a) l *= (xe - x[j]) / (x[a] - x[j]);
            c->surf.e[side][a] = (double)l;
        }
    }
    if ((e = cudaMalloc(&c->d_err, sizeof(int))) != cudaSuccess) { delete c; return cuda_fail(e, "cudaMalloc(error word)"); }
    if ((e = cudaMemset(c->d_err, 0, sizeof(int))) != cudaSuccess) {
        cudaFree(c->d_err); delete c; return cuda_fail(e, "cudaMemset(error word)");
    }
    *out = c;
    return SFH_OK;
}

extern "C" sfh_status sfh_destroy(sfh_ctx *c) {
    clear_err();
    if (!c) return SFH_OK;
    DeviceGuard g(c->device);
    for (int k = 0; k < kHostStages; ++k) {
        if (c->hs[k]) { cudaStreamSynchronize(c->hs[k]); cudaStreamDestroy(c->hs[k]); }
        if (c->stage[k]) cudaFree(c->stage[k]);
    }
    if (c->d_err) cudaFree(c->d_err);
    if (c->d_ja) cudaFree(c->d_ja);
    if (c->pool) cudaMemPoolDestroy(c->pool);   // released once no scratch of it is outstanding
    for (int k = 0; k < kBoundStages; ++k) {
        if (c->bs[k]) { cudaStreamSynchronize(c->bs[k]); cudaStreamDestroy(c->bs[k]); }
        if (c->bstage[k]) cudaFree(c->bstage[k]);
    }
    delete c;
    return SFH_OK;
}

extern "C" sfh_status sfh_ctx_info(const sfh_ctx *c, int *d, int *p, int *nodes, int *nvar, int *flux, int *n_nodes) {
    clear_err();
    if (!c) return fail(SFH_EINVAL, "ctx is NULL");
    if (d) *d = c->d;
    if (p) *p = c->p;
    if (nodes) *nodes = c->nodes;
    if (nvar) *nvar = c->nvar;
    if (flux) *flux = c->flux;
    if (n_nodes) *n_nodes = sfh::ipow(c->n, c->d);
    return SFH_OK;
}

static sfh_status check_common(const sfh_ctx *c, int64_t n_elem, const void *u, const double *Ja, const void *out,
                               size_t esz) {
    if (!c) return fail(SFH_EINVAL, "ctx is NULL");
    if (n_elem < 0) return fail(SFH_EINVAL, "n_elem must be >= 0, got %lld", (long long)n_elem);
    if (n_elem == 0) return SFH_OK;
    if (!u || !Ja || !out) return fail(SFH_EINVAL, "null array pointer");
    if (((uintptr_t)u % esz) || ((uintptr_t)out % esz) || ((uintptr_t)Ja % sizeof(double)))
        return fail(SFH_EINVAL, "misaligned array pointer");
    const int64_t nn = sfh::ipow(c->n, c->d);
    if (n_elem > (int64_t)1 << 40) return fail(SFH_EINVAL, "n_elem too large");
    const size_t ub = (size_t)(n_elem * c->nvar * nn) * esz;
    const size_t jb = (size_t)(n_elem * c->d * c->d * nn) * sizeof(double);
    if (overlap(out, ub, u, ub) || overlap(out, ub, Ja, jb)) return fail(SFH_EINVAL, "output overlaps an input");
    return SFH_OK;
}

extern "C" sfh_status sfh_fig1_hadamard(int p, int64_t n_elem, const double *c, double *y, int dense,
                                        sfh_stream_t stream) {
    clear_err();
    constexpr int kPMax = 15;
    if (p < 1 || p > kPMax) return fail(SFH_EINVAL, "p must be in [1, %d], got %d", kPMax, p);
    if (n_elem < 0) return fail(SFH_EINVAL, "n_elem must be >= 0");
    if (n_elem == 0) return SFH_OK;
    if (!c || !y) return fail(SFH_EINVAL, "null array pointer");
    if (((uintptr_t)c | (uintptr_t)y) % sizeof(double)) return fail(SFH_EINVAL, "misaligned array pointer");
    const int n = p + 1;
    const size_t bytes = (size_t)n_elem * n * n * n * sizeof(double);
    if (overlap(y, bytes, c, bytes)) return fail(SFH_EINVAL, "output overlaps the input");
    long double x[kPMax + 1], ww[kPMax + 1], DD[(kPMax + 1) * (kPMax + 1)];
    if (!make_tables(p, SFH_NODES_GLL, x, ww, DD, kPMax)) return fail(SFH_EINVAL, "table construction failed");
    double D[(kPMax + 1) * (kPMax + 1)];
    for (int k = 0; k < n * n; ++k) D[k] = (double)DD[k];
    const cudaError_t e = sfh::fig1_hadamard(n, dense != 0, c, y, n_elem, D, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "Hadamard kernel launch");
    return SFH_OK;
}

extern "C" sfh_status sfh_entropy_residual(sfh_ctx *c, int64_t n_elem, const double *u, const double *Ja,
                                           const void *r, sfh_prec r_prec, double *out, sfh_stream_t stream) {
    clear_err();
    if (r_prec != SFH_FP64 && r_prec != SFH_FP32_KAHAN && r_prec != SFH_FP32_MIXED)
        return fail(SFH_EINVAL, "bad precision mode %d", (int)r_prec);
    if (!c) return fail(SFH_EINVAL, "ctx is NULL");
    if (n_elem < 0) return fail(SFH_EINVAL, "n_elem must be >= 0, got %lld", (long long)n_elem);
    if (n_elem == 0) return SFH_OK;
    if (n_elem > ((int64_t)1 << 31) - 1) return fail(SFH_EINVAL, "n_elem must be below 2^31 (one CTA per element)");
    if (!u || !Ja || !r || !out) return fail(SFH_EINVAL, "null array pointer");
    const size_t resz = elem_size(r_prec);
    if (((uintptr_t)u | (uintptr_t)Ja | (uintptr_t)out) % sizeof(double) || (uintptr_t)r % resz)
        return fail(SFH_EINVAL, "misaligned array pointer");
    const size_t nn = (size_t)sfh::ipow(c->n, c->d);
    const size_t ub = (size_t)n_elem * c->nvar * nn * sizeof(double), rb = (size_t)n_elem * c->nvar * nn * resz;
    const size_t jb = (size_t)n_elem * c->d * c->d * nn * sizeof(double), ob = (size_t)n_elem * sizeof(double);
    if (overlap(out, ob, u, ub) || overlap(out, ob, Ja, jb) || overlap(out, ob, r, rb))
        return fail(SFH_EINVAL, "output overlaps an input");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(SFH_ECUDA, "cannot select the context's device");
    const cudaError_t e = sfh::entropy_identity(c->d, c->n, c->flux, u, Ja, r, r_prec != SFH_FP64, out, n_elem,
                                                c->tab_d, c->d_err, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "entropy identity kernel launch");
    return SFH_OK;
}

extern "C" sfh_status sfh_volume_residual(sfh_ctx *c, int64_t n_elem, const void *u, const double *Ja, void *r,
                                          sfh_prec prec, sfh_stream_t stream) {
    clear_err();
    if (prec != SFH_FP64 && prec != SFH_FP32_KAHAN && prec != SFH_FP32_MIXED)
        return fail(SFH_EINVAL, "bad precision mode %d", (int)prec);
    sfh_status st = check_common(c, n_elem, u, Ja, r, elem_size(prec));
    if (st != SFH_OK || n_elem == 0) return st;
    DeviceGuard g(c->device);
    if (!g.ok) return fail(SFH_ECUDA, "cannot select the context's device");
    cudaError_t e = launch_volume(c, prec, n_elem, u, Ja, r, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "volume kernel launch");
    (void)mode_of;
    return SFH_OK;
}

extern "C" sfh_status sfh_volume_residual_modal(sfh_ctx *c, sfh_basis basis, int64_t n_elem, const void *u_hat,
                                                const double *Ja, void *r_hat, sfh_prec prec, sfh_stream_t stream) {
    clear_err();
    if (prec != SFH_FP64 && prec != SFH_FP32_KAHAN && prec != SFH_FP32_MIXED)
        return fail(SFH_EINVAL, "bad precision mode %d", (int)prec);
    if (basis != SFH_BASIS_LEGENDRE && basis != SFH_BASIS_LAGRANGE_GLL && basis != SFH_BASIS_LAGRANGE_GAUSS)
        return fail(SFH_EINVAL, "bad basis %d", (int)basis);
    sfh_status st = check_common(c, n_elem, u_hat, Ja, r_hat, elem_size(prec));
    if (st != SFH_OK || n_elem == 0) return st;
    DeviceGuard g(c->device);
    if (!g.ok) return fail(SFH_ECUDA, "cannot select the context's device");
    using namespace sfh;
    const cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if ((prec == SFH_FP32_MIXED || prec == SFH_FP32_KAHAN) && c->d == 3 && c->flux != kFluxBurgers && c->n >= 3 &&
        c->n <= 8 && c->pool) {
        // 3D Euler at n = 3..8 in the FP32 modes: the transforms as kernels
        // of their own around the nodal kernel (warp-specialized, or the row
        // kernel of Ranocha's flux at n = 8), through stream-ordered scratch
        // for V u_hat and r_v (sfh_modal.cu).  The same arithmetic in the same
        // order as the fused kernels, so the same bits.  At n = 5 on 32^3
        // elements: mixed mode 0.78 against 1.88 ms for the fused
        // thread-per-line kernel; FP32-Kahan 0.235 against 0.241 ms for the
        // fused line kernel.
        const size_t bytes = (size_t)n_elem * c->nvar * sfh::ipow(c->n, 3) * sizeof(float);
        float *uv = nullptr;
        if ((e = cudaMallocFromPoolAsync((void **)&uv, 2 * bytes, c->pool, s)) != cudaSuccess)
            return fail(SFH_ENOMEM, "modal scratch of %zu bytes: %s", 2 * bytes, cudaGetErrorString(e));
        float *rv = uv + bytes / sizeof(float);
        e = modal_xform_3d(c->n, false, (const float *)u_hat, uv, n_elem, c->basis_f[basis], c->d_err, s);
        if (e == cudaSuccess) e = launch_volume(c, prec, n_elem, uv, Ja, rv, s);
        if (e == cudaSuccess)
            e = modal_xform_3d(c->n, true, rv, (float *)r_hat, n_elem, c->basis_f[basis], c->d_err, s);
        const cudaError_t ef = cudaFreeAsync(uv, s);
        if (e != cudaSuccess) return cuda_fail(e, "modal volume kernel launch");
        if (ef != cudaSuccess) return cuda_fail(ef, "modal scratch release");
        return SFH_OK;
    }
    if (prec == SFH_FP64)
        e = modal_fp64_fn(c->d, c->flux)(c->n, c->flux, u_hat, Ja, r_hat, n_elem, c->tab_d, c->basis_d[basis],
                                         c->d_err, s);
    else if (prec == SFH_FP32_KAHAN)
        e = modal_fp32k_fn(c->d, c->flux)(c->n, c->flux, u_hat, Ja, r_hat, n_elem, c->tab_f, c->basis_f[basis],
                                          c->d_err, s);
    else
        e = modal_mixed_fn(c->d, c->flux)(c->n, c->flux, u_hat, Ja, r_hat, n_elem, c->tab_f, c->basis_f[basis],
                                          c->d_err, s);
    if (e != cudaSuccess) return cuda_fail(e, "modal volume kernel launch");
    return SFH_OK;
}

extern "C" sfh_status sfh_surface_hadamard(sfh_ctx *c, int64_t n_elem, const double *u, const double *u_face,
                                           const double *nJ_face, double *r_vol, double *r_face,
                                           sfh_stream_t stream) {
    clear_err();
    if (!c) return fail(SFH_EINVAL, "ctx is NULL");
    if (n_elem < 0) return fail(SFH_EINVAL, "n_elem must be >= 0, got %lld", (long long)n_elem);
    if (n_elem == 0) return SFH_OK;
    if (n_elem > (int64_t)1 << 36) return fail(SFH_EINVAL, "n_elem too large");
    if (!u || !u_face || !nJ_face || !r_vol || !r_face) return fail(SFH_EINVAL, "null array pointer");
    if (((uintptr_t)u | (uintptr_t)u_face | (uintptr_t)nJ_face | (uintptr_t)r_vol | (uintptr_t)r_face) % sizeof(double))
        return fail(SFH_EINVAL, "misaligned array pointer");
    const size_t nn = (size_t)sfh::ipow(c->n, c->d), nf = (size_t)sfh::ipow(c->n, c->d - 1);
    const size_t ub = (size_t)n_elem * c->nvar * nn * sizeof(double);
    const size_t fb = (size_t)n_elem * 2 * c->d * c->nvar * nf * sizeof(double);
    const size_t jb = (size_t)n_elem * 2 * c->d * c->d * nf * sizeof(double);
    if (overlap(r_vol, ub, u, ub) || overlap(r_vol, ub, u_face, fb) || overlap(r_vol, ub, nJ_face, jb) ||
        overlap(r_face, fb, u, ub) || overlap(r_face, fb, u_face, fb) || overlap(r_face, fb, nJ_face, jb) ||
        overlap(r_vol, ub, r_face, fb))
        return fail(SFH_EINVAL, "an output overlaps an input or the other output");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(SFH_ECUDA, "cannot select the context's device");
    const cudaError_t e = sfh::surface_hadamard(c->d, c->n, c->flux, u, u_face, nJ_face, r_vol, r_face, n_elem,
                                                c->surf, c->d_err, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "surface kernel launch");
    return SFH_OK;
}

extern "C" sfh_status sfh_vjp_modal(sfh_ctx *c, sfh_basis basis, int64_t n_elem, const double *u_hat,
                                    const double *Ja, const double *lambda_hat, double *grad_hat,
                                    sfh_stream_t stream) {
    clear_err();
    if (basis != SFH_BASIS_LEGENDRE && basis != SFH_BASIS_LAGRANGE_GLL && basis != SFH_BASIS_LAGRANGE_GAUSS)
        return fail(SFH_EINVAL, "bad basis %d", (int)basis);
    sfh_status st = check_common(c, n_elem, u_hat, Ja, grad_hat, sizeof(double));
    if (st != SFH_OK || n_elem == 0) return st;
    if (!lambda_hat) return fail(SFH_EINVAL, "lambda_hat is NULL");
    if ((uintptr_t)lambda_hat % sizeof(double)) return fail(SFH_EINVAL, "misaligned lambda_hat");
    const size_t ub = (size_t)(n_elem * c->nvar * sfh::ipow(c->n, c->d)) * sizeof(double);
    if (overlap(grad_hat, ub, lambda_hat, ub)) return fail(SFH_EINVAL, "grad_hat overlaps lambda_hat");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(SFH_ECUDA, "cannot select the context's device");
    cudaError_t e = sfh::vjp_modal_fn(c->d, c->flux)(c->n, c->flux, u_hat, Ja, lambda_hat, grad_hat, n_elem,
                                                    c->tab_d, c->basis_d[basis], c->d_err, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "modal vjp kernel launch");
    return SFH_OK;
}

extern "C" sfh_status sfh_vjp(sfh_ctx *c, int64_t n_elem, const double *u, const double *Ja, const double *lambda,
                              double *grad_u, sfh_stream_t stream) {
    clear_err();
    sfh_status st = check_common(c, n_elem, u, Ja, grad_u, sizeof(double));
    if (st != SFH_OK || n_elem == 0) return st;
    if (!lambda) return fail(SFH_EINVAL, "lambda is NULL");
    if ((uintptr_t)lambda % sizeof(double)) return fail(SFH_EINVAL, "misaligned lambda");
    const size_t ub = (size_t)(n_elem * c->nvar * sfh::ipow(c->n, c->d)) * sizeof(double);
    if (overlap(grad_u, ub, lambda, ub)) return fail(SFH_EINVAL, "grad_u overlaps lambda");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(SFH_ECUDA, "cannot select the context's device");
    cudaError_t e = sfh::vjp_fn(c->d, c->flux)(c->n, c->flux, u, Ja, lambda, grad_u, n_elem, c->tab_d, c->d_err,
                                              (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "vjp kernel launch");
    return SFH_OK;
}

extern "C" sfh_status sfh_check(sfh_ctx *c, sfh_stream_t stream) {
    clear_err();
    if (!c) return fail(SFH_EINVAL, "ctx is NULL");
    DeviceGuard g(c->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    int h = 0;
    if ((e = cudaMemcpy(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(e, "read error word");
    if (h) {
        if ((e = cudaMemset(c->d_err, 0, sizeof(int))) != cudaSuccess) return cuda_fail(e, "clear error word");
        return (sfh_status)sfh::err_word_status(h);
    }
    return SFH_OK;
}

namespace sfh {
int err_word_status(int h) {
    if (h & kErrBounds)
        return fail(SFH_EBOUNDS, "debug build: a kernel index left its buffer (the access was not made)");
    if (h & kErrTimeout) return fail(SFH_ETIMEOUT, "a bounded device wait gave up");
    if ((h & kErrDomain) && (h & kErrMetric))
        return fail(SFH_EDOMAIN, "density or pressure <= 0 (or NaN) in the state, and a metric term out of range "
                                 "(Inf, NaN, or |Ja| >= 2^126 in an FP32 mode)");
    if (h & kErrMetric)
        return fail(SFH_EDOMAIN, "metric term out of range (Inf, NaN, or |Ja| >= 2^126 in an FP32 mode)");
    return fail(SFH_EDOMAIN, "density or pressure <= 0 (or NaN) in the state");
}
}  // namespace sfh

// ---------------------------------------------------------------------------
// host-buffer pipeline: chunks alternate between two streams; on each stream
// H2D(u, Ja) -> kernel -> D2H(r), so the copies of one chunk overlap the
// kernel of the other.
// ---------------------------------------------------------------------------
extern "C" sfh_status sfh_volume_residual_host(sfh_ctx *c, int64_t n_elem, const void *u_host,
                                               const double *Ja_host, void *r_host, sfh_prec prec) {
    clear_err();
    if (prec != SFH_FP64 && prec != SFH_FP32_KAHAN && prec != SFH_FP32_MIXED)
        return fail(SFH_EINVAL, "bad precision mode %d", (int)prec);
    const size_t esz = elem_size(prec);
    sfh_status st = check_common(c, n_elem, u_host, Ja_host, r_host, esz);
    if (st != SFH_OK || n_elem == 0) return st;
    std::lock_guard<std::mutex> lk(c->host_mu);
    DeviceGuard g(c->device);
    if (!g.ok) return fail(SFH_ECUDA, "cannot select the context's device");
    const size_t nn = (size_t)sfh::ipow(c->n, c->d);
    const size_t ub_e = c->nvar * nn * esz, jb_e = (size_t)c->d * c->d * nn * sizeof(double);
    const size_t per_elem = 2 * ub_e + jb_e;
    int64_t chunk = std::max<int64_t>(64, (int64_t)(kHostChunkBytes / per_elem));
    chunk = std::min<int64_t>(chunk, n_elem);
    const size_t need = (size_t)chunk * per_elem + 3 * 256;   // three 256-byte-aligned sub-buffers
    cudaError_t e;
    for (int k = 0; k < kHostStages; ++k) {
        if (!c->hs[k] && (e = cudaStreamCreateWithFlags(&c->hs[k], cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamCreate");
    }
    if (c->stage_bytes < need) {
        for (int k = 0; k < kHostStages; ++k) {
            if (c->stage[k]) { cudaFree(c->stage[k]); c->stage[k] = nullptr; }
        }
        c->stage_bytes = 0;
        for (int k = 0; k < kHostStages; ++k)
            if ((e = cudaMalloc(&c->stage[k], need)) != cudaSuccess) {
                for (int j = 0; j < k; ++j) { cudaFree(c->stage[j]); c->stage[j] = nullptr; }
                return fail(SFH_ENOMEM, "staging allocation of %zu bytes failed", need);
            }
        c->stage_bytes = need;
    }
    const char *uh = (const char *)u_host;
    const char *jh = (const char *)Ja_host;
    char *rh = (char *)r_host;
    int64_t k = 0;
    for (int64_t e0 = 0; e0 < n_elem; e0 += chunk, ++k) {
        const int64_t ne = std::min<int64_t>(chunk, n_elem - e0);
        const int b = (int)(k % kHostStages);
        cudaStream_t s = c->hs[b];
        char *base = (char *)c->stage[b];
        char *du = base;
        char *dj = base + ((ne * ub_e + 255) / 256) * 256;
        char *dr = dj + ((ne * jb_e + 255) / 256) * 256;
        if ((e = cudaMemcpyAsync(du, uh + e0 * ub_e, ne * ub_e, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(dj, jh + e0 * jb_e, ne * jb_e, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return cuda_fail(e, "host-to-device copy");
        if ((e = launch_volume(c, prec, ne, du, (const double *)dj, dr, s)) != cudaSuccess) return cuda_fail(e, "volume kernel launch");
        if ((e = cudaMemcpyAsync(rh + e0 * ub_e, dr, ne * ub_e, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_fail(e, "device-to-host copy");
    }
    for (int b = 0; b < kHostStages; ++b)
        if ((e = cudaStreamSynchronize(c->hs[b])) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return sfh_check(c, c->hs[0]);
}

// ---------------------------------------------------------------------------
// bound metric: Ja uploaded once per mesh, then only u and r travel per call
// ---------------------------------------------------------------------------
extern "C" sfh_status sfh_bind_metric(sfh_ctx *c, int64_t n_elem, const double *Ja_host) {
    clear_err();
    if (!c) return fail(SFH_EINVAL, "ctx is NULL");
    if (n_elem < 0 || n_elem > (int64_t)1 << 40) return fail(SFH_EINVAL, "n_elem out of range: %lld", (long long)n_elem);
    if (n_elem > 0 && !Ja_host) return fail(SFH_EINVAL, "Ja_host is NULL");
    if ((uintptr_t)Ja_host % sizeof(double)) return fail(SFH_EINVAL, "misaligned Ja_host");
    std::lock_guard<std::mutex> lk(c->host_mu);
    DeviceGuard g(c->device);
    if (!g.ok) return fail(SFH_ECUDA, "cannot select the context's device");
    const size_t jb = (size_t)n_elem * c->d * c->d * sfh::ipow(c->n, c->d) * sizeof(double);
    cudaError_t e;
    c->ja_elems = 0;   // no metric is bound while the copy is incomplete
    if (c->ja_bytes < jb) {
        if (c->d_ja) { cudaFree(c->d_ja); c->d_ja = nullptr; c->ja_bytes = 0; }
        if ((e = cudaMalloc(&c->d_ja, jb)) != cudaSuccess) {
            c->d_ja = nullptr;
            return fail(SFH_ENOMEM, "metric allocation of %zu bytes failed", jb);
        }
        c->ja_bytes = jb;
    }
    if (jb && (e = cudaMemcpy(c->d_ja, Ja_host, jb, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "metric copy");
    c->ja_elems = n_elem;
    return SFH_OK;
}


extern "C" sfh_status sfh_volume_residual_host_bound(sfh_ctx *c, int64_t n_elem, const void *u_host, void *r_host,
                                                     sfh_prec prec) {
    clear_err();
    if (prec != SFH_FP64 && prec != SFH_FP32_KAHAN && prec != SFH_FP32_MIXED)
        return fail(SFH_EINVAL, "bad precision mode %d", (int)prec);
    if (!c) return fail(SFH_EINVAL, "ctx is NULL");
    if (n_elem < 0) return fail(SFH_EINVAL, "n_elem must be >= 0, got %lld", (long long)n_elem);
    if (n_elem == 0) return SFH_OK;
    const size_t esz = elem_size(prec);
    if (!u_host || !r_host) return fail(SFH_EINVAL, "null array pointer");
    if (((uintptr_t)u_host % esz) || ((uintptr_t)r_host % esz)) return fail(SFH_EINVAL, "misaligned array pointer");
    std::lock_guard<std::mutex> lk(c->host_mu);
    if (n_elem > c->ja_elems)
        return fail(SFH_EINVAL, "%lld elements requested, %lld bound by sfh_bind_metric", (long long)n_elem,
                    (long long)c->ja_elems);
    const size_t nn = (size_t)sfh::ipow(c->n, c->d);
    const size_t ub_e = c->nvar * nn * esz, jb_e = (size_t)c->d * c->d * nn * sizeof(double);
    if (overlap(r_host, n_elem * ub_e, u_host, n_elem * ub_e)) return fail(SFH_EINVAL, "output overlaps an input");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(SFH_ECUDA, "cannot select the context's device");
    // a multiple of 16 elements, so that every chunk's slice of the bound
    // metric starts on a 16-byte boundary (the kernels' bulk copies need it)
    int64_t chunk = std::max<int64_t>(64, (int64_t)(kBoundChunkBytes / ub_e) / 16 * 16);
    chunk = std::min<int64_t>(chunk, n_elem);
    const size_t need = 2 * ((size_t)chunk * ub_e + 256);   // u and r, each 256-byte aligned
    cudaError_t e;
    for (int k = 0; k < kBoundStages; ++k) {
        if (!c->bs[k] && (e = cudaStreamCreateWithFlags(&c->bs[k], cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamCreate");
    }
    if (c->bstage_bytes < need) {
        for (int k = 0; k < kBoundStages; ++k) {
            if (c->bstage[k]) { cudaFree(c->bstage[k]); c->bstage[k] = nullptr; }
        }
        c->bstage_bytes = 0;
        for (int k = 0; k < kBoundStages; ++k)
            if ((e = cudaMalloc(&c->bstage[k], need)) != cudaSuccess) {
                for (int j = 0; j < k; ++j) { cudaFree(c->bstage[j]); c->bstage[j] = nullptr; }
                return fail(SFH_ENOMEM, "staging allocation of %zu bytes failed", need);
            }
        c->bstage_bytes = need;
    }
    const char *uh = (const char *)u_host;
    char *rh = (char *)r_host;
    const char *jd = (const char *)c->d_ja;
    int64_t k = 0;
    for (int64_t e0 = 0; e0 < n_elem; e0 += chunk, ++k) {
        const int64_t ne = std::min<int64_t>(chunk, n_elem - e0);
        const int b = (int)(k % kBoundStages);
        cudaStream_t s = c->bs[b];
        char *du = (char *)c->bstage[b];
        char *dr = du + ((ne * ub_e + 255) / 256) * 256;
        if ((e = cudaMemcpyAsync(du, uh + e0 * ub_e, ne * ub_e, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return cuda_fail(e, "host-to-device copy");
        if ((e = launch_volume(c, prec, ne, du, (const double *)(jd + e0 * jb_e), dr, s)) != cudaSuccess)
            return cuda_fail(e, "volume kernel launch");
        if ((e = cudaMemcpyAsync(rh + e0 * ub_e, dr, ne * ub_e, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_fail(e, "device-to-host copy");
    }
    for (int b = 0; b < kBoundStages; ++b)
        if ((e = cudaStreamSynchronize(c->bs[b])) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return sfh_check(c, c->bs[0]);
}

// ---------------------------------------------------------------------------
// bounded-wait self-test: an mbarrier phase that nothing completes
// ---------------------------------------------------------------------------
__global__ void bounded_wait_selftest_kernel(uint64_t limit_ns, int *out) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    sfh::mbar_init(&bar, 1);
    sfh::fence_proxy_async_smem();
    // announce 16 bytes that no copy will deliver: phase 0 never completes
    sfh::mbar_arrive_expect_tx(&bar, 16);
    const uint64_t t0 = sfh::global_timer_ns();
    const bool done = sfh::mbar_wait_bounded(&bar, 0, limit_ns);
    out[0] = done ? 0 : sfh::kErrTimeout;
    out[1] = (int)((sfh::global_timer_ns() - t0) / 1000);
}

extern "C" sfh_status sfh_selftest_bounded_wait(int64_t limit_us, sfh_stream_t stream, double *elapsed_us) {
    clear_err();
    if (limit_us < 1 || limit_us > 10000000) return fail(SFH_EINVAL, "limit_us must be in [1, 1e7], got %lld", (long long)limit_us);
    int *d = nullptr;
    cudaError_t e = cudaMalloc(&d, 2 * sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    cudaStream_t s = (cudaStream_t)stream;
    int h[2] = {-1, 0};
    bounded_wait_selftest_kernel<<<1, 32, 0, s>>>((uint64_t)limit_us * 1000ull, d);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "self-test kernel");
    }
    cudaFree(d);
    if (elapsed_us) *elapsed_us = (double)h[1];
    if (h[0] == sfh::kErrTimeout) return fail(SFH_ETIMEOUT, "bounded wait gave up after %d us (expected)", h[1]);
    return SFH_OK;
}

// ---------------------------------------------------------------------------
// build variant and the debug build's bounds self-test
// ---------------------------------------------------------------------------
extern "C" int sfh_build_flags(void) { return sfh::kDebugBuild ? SFH_BUILD_DEBUG : 0; }

#ifdef SFH_DEBUG
// a checked pointer over buf[0, n) of a 2n-word buffer: word n is read and
// word n + 1 written (both refused: outside the extent, inside the
// allocation), word 0 written (made)
__global__ void bounds_selftest_kernel(int *buf, int n, int *err, int *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const auto p = sfh::bp(buf, n, err);
    out[0] = p[n];
    p[n + 1] = 12345;
    p[0] = 777;
}
#endif

extern "C" sfh_status sfh_selftest_bounds(sfh_stream_t stream) {
    clear_err();
#ifdef SFH_DEBUG
    constexpr int n = 64;
    int *d = nullptr;
    cudaError_t e = cudaMalloc(&d, (2 * n + 2) * sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    cudaStream_t s = (cudaStream_t)stream;
    int h[2 * n + 2];
    int *err = d + 2 * n, *out = d + 2 * n + 1;
    if ((e = cudaMemsetAsync(d, 0, sizeof h, s)) == cudaSuccess) {
        bounds_selftest_kernel<<<1, 32, 0, s>>>(d, n, err, out);
        if ((e = cudaGetLastError()) == cudaSuccess && (e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, s)) == cudaSuccess)
            e = cudaStreamSynchronize(s);
    }
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "bounds self-test kernel");
    const int herr = h[2 * n];
    if ((herr & sfh::kErrBounds) && h[n + 1] == 0 && h[0] == 777) return SFH_OK;
    return fail(SFH_EBOUNDS, "bounds checks did not act as designed (error word %d, word n+1 = %d, word 0 = %d)", herr,
                h[n + 1], h[0]);
#else
    (void)stream;
    return fail(SFH_EUNSUPPORTED, "the release library has no bounds checks (build with debug=True)");
#endif
}

// ---------------------------------------------------------------------------
// peak microbenchmarks: independent FMA chains per thread, every SM busy
// ---------------------------------------------------------------------------
template <typename T>
__global__ void fma_chain_kernel(T *out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;   // contracted to one FMA
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static sfh_status peak_impl(int iters, double *tflops, double *ms) {
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return cuda_fail(e, "attr");
    const int threads = 256, blocks = sms * 8;
    T *out = nullptr;
    if ((e = cudaMalloc(&out, sizeof(T) * threads * blocks)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    fma_chain_kernel<T><<<blocks, threads>>>(out, iters / 8, (T)0.9999999, (T)1e-7);   // warm-up
    cudaEventRecord(t0);
    fma_chain_kernel<T><<<blocks, threads>>>(out, iters, (T)0.9999999, (T)1e-7);
    cudaEventRecord(t1);
    e = cudaEventSynchronize(t1);
    float elapsed = 0.0f;
    cudaEventElapsedTime(&elapsed, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(out);
    if (e != cudaSuccess) return cuda_fail(e, "peak kernel");
    const double fmas = (double)blocks * threads * iters * 8.0;
    if (ms) *ms = elapsed;
    if (tflops) *tflops = 2.0 * fmas / (elapsed * 1e-3) / 1e12;
    return SFH_OK;
}

extern "C" sfh_status sfh_peak_fma(sfh_prec prec, double *tflops, double *ms) {
    clear_err();
    if (prec == SFH_FP64) return peak_impl<double>(1 << 12, tflops, ms);
    if (prec == SFH_FP32_KAHAN) return peak_impl<float>(1 << 16, tflops, ms);
    return fail(SFH_EINVAL, "prec must be SFH_FP64 or SFH_FP32_KAHAN");
}
