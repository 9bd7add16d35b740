/*
 * sfhad.h -- C ABI of libsfhad, a GB300 (sm_103a) library for the
 * sum-factorized Hadamard-product volume term of entropy-conserving flux
 * differencing (Cicchino & Nadarajah, arXiv 2306.11665).
 *
 * What it computes (Section 2, Eq. 3 with the operators of Eq. 5): for every
 * element of a tensor-product mesh with n = p + 1 collocated nodes per
 * direction,
 *
 *     r_i = sum_{m=0}^{d-1} sum_j (Q_m o F_m)_ij,
 *     Q_m = (W (x) .. (x) W D (x) .. (x) W)  with W D in direction m,
 *     F_m,ij = sum_k fsharp_k(u_i, u_j) (Ja^m_k(i) + Ja^m_k(j)),
 *
 * where only node pairs (i, j) on the same grid line along m contribute, so
 * each element costs d n^{d+1} two-point fluxes instead of n^{2d}
 * (Theorem 2.1).  fsharp is Ranocha's entropy-conserving, kinetic-energy-
 * preserving Euler flux (gamma = 1.4) or the Burgers flux (a^2 + ab + b^2)/6.
 *
 * Layouts (all arrays dense, C order, nodes x fastest as in Section 2):
 *   u, r, lambda, grad_u : [n_elem][nvar][n^d]        (i = a_0 + n a_1 + n^2 a_2)
 *   Ja                   : [n_elem][d][d][n^d]        Ja[e][m][k][i] = J dxi_m/dx_k
 *   Euler variables      : (rho, rho v_1, .., rho v_d, E); nvar = d + 2
 *   Burgers              : nvar = 1
 *
 * Ownership: every array is owned by the caller.  Device pointers must stay
 * valid until the work on `stream` has completed; the library keeps none of
 * them after that.  The library owns only what a context allocates (the
 * operator tables and an error word on the device).
 *
 * Errors: no call aborts, traps or hangs.  Argument errors are reported
 * before any device work is issued.  Errors found by the device (a density
 * or pressure <= 0 in the state) are latched in the context's error word and
 * reported by sfh_check().  sfh_last_error() returns a thread-local message
 * for the last failing call of the calling thread.
 *
 * Streams: sfh_stream_t is a cudaStream_t; NULL means the legacy default
 * stream.  Device entry points are asynchronous with respect to the host.
 */
#ifndef SFHAD_H
#define SFHAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *sfh_stream_t;

typedef enum {
    SFH_OK = 0,
    SFH_EINVAL = 1,        /* bad argument (null pointer, size, enum, misalignment) */
    SFH_ENOMEM = 2,        /* allocation failed, or a request exceeds a memory budget */
    SFH_ECUDA = 3,         /* a CUDA runtime call failed (message in sfh_last_error) */
    SFH_EDOMAIN = 4,       /* the device saw a density or pressure <= 0 (or NaN) */
    SFH_EBUSY = 5,         /* the server cannot take the request now */
    SFH_ENOTREADY = 6,     /* a polled request has not completed yet */
    SFH_ETIMEOUT = 7,      /* a bounded wait gave up */
    SFH_EUNSUPPORTED = 8,  /* valid but not provided (e.g. no CUDA device) */
    SFH_EBOUNDS = 9        /* debug build only: a kernel index left its buffer (the access was not made) */
} sfh_status;

typedef enum { SFH_NODES_GLL = 0, SFH_NODES_GAUSS = 1 } sfh_nodes;

typedef enum {
    SFH_FLUX_BURGERS = 0,       /* fsharp_k(a, b) = (a^2 + a b + b^2) / 6 in every direction k */
    SFH_FLUX_EULER_RANOCHA = 1, /* Ranocha EC/KEP flux with logarithmic means, gamma = 1.4:
                                   f_m = f_rho {v} + {p} n, pressure work (p_a v_b + p_b v_a).n / 2 */
    SFH_FLUX_EULER_CHANDRASHEKAR = 2 /* Chandrashekar's EC/KEP flux (named for the TGV runs of
                                   Section 3): as Ranocha's but with the pressure average
                                   {rho}/{beta} (beta = rho/p) and pressure work {rho}/{beta} {v}.n.
                                   Residual, VJP, entropy identity, the host entry points and
                                   the serving runtime */
} sfh_flux;

typedef enum {
    SFH_FP64 = 0,        /* all arithmetic in FP64; u, r are double */
    SFH_FP32_KAHAN = 1,  /* FP32 flux arithmetic, compensated line sums; u, r are float */
    SFH_FP32_MIXED = 2   /* as SFH_FP32_KAHAN, with FP64 metric sums Ja(i)+Ja(j) and an
                            FP64 logarithmic mean in the near-equal band; u, r are float */
} sfh_prec;

/* Solution basis of the modal / uncollocated entry point (Section 2, Eq. 4
 * and the theorem after it), n = p + 1 functions per direction, tensor
 * product, evaluated on the context's cubature nodes. */
typedef enum {
    SFH_BASIS_LEGENDRE = 0,       /* orthonormal Legendre sqrt((2k + 1)/2) P_k(xi) */
    SFH_BASIS_LAGRANGE_GLL = 1,   /* Lagrange polynomials of the p + 1 Gauss-Lobatto nodes */
    SFH_BASIS_LAGRANGE_GAUSS = 2  /* Lagrange polynomials of the p + 1 Gauss-Legendre nodes */
} sfh_basis;

typedef struct sfh_ctx sfh_ctx;

/* Create a context for one element type (Section 2: d directions, n = p + 1
 * nodes on each, collocated Lagrange basis; Eq. 5 operators).
 * d in {2, 3}; p in [1, 8]; nvar must be 1 for SFH_FLUX_BURGERS and d + 2 for
 * the Euler fluxes.  Builds the 1D operator tables (nodes, weights,
 * D, Q1 = W D) on the host and allocates the device error word on the
 * current device.  *out is set only on SFH_OK.
 * Errors: SFH_EINVAL for bad arguments; SFH_ECUDA / SFH_EUNSUPPORTED when no
 * CUDA device can be used; SFH_ENOMEM. */
sfh_status sfh_create(int d, int p, sfh_nodes nodes, int nvar, sfh_flux flux, sfh_ctx **out);

/* Release a context (waits for nothing: the caller must not destroy a context
 * whose work is still in flight).  NULL is accepted. */
sfh_status sfh_destroy(sfh_ctx *ctx);

/* Volume residual r (Eq. 3 with Eq. 5, Section 2, three-step evaluation of
 * the three-dimensional listing): builds each line's two-point fluxes in
 * registers and sums the Hadamard product row by row, r overwritten.
 * u, r: device, [n_elem][nvar][n^d], double for SFH_FP64, float otherwise,
 *       8-byte (double) or 4-byte (float) aligned; r must not overlap u or Ja.
 * Ja:   device, [n_elem][d][d][n^d] double (FP64 in every mode), 8-byte aligned.
 *       Accepted values: finite, and |Ja| < 2^126 in the FP32 modes (their
 *       FP32 copies and pair sums then stay finite); metric terms are
 *       O(h^{d-1}), far inside this range.
 * n_elem >= 0 (0 is a no-op).  Asynchronous on `stream`.
 * Errors: SFH_EINVAL before any launch; SFH_ECUDA if the launch fails;
 * device-detected errors are latched for sfh_check(): SFH_EDOMAIN for a
 * density or pressure <= 0 (or NaN) and for a metric term outside the
 * accepted range (the other elements' results are still computed). */
sfh_status sfh_volume_residual(sfh_ctx *ctx, int64_t n_elem, const void *u, const double *Ja,
                               void *r, sfh_prec prec, sfh_stream_t stream);

/* Modal / uncollocated volume residual (Section 2: Eq. 4, the theorem on
 * general bases and its proof).  The solution is given by coefficients in the
 * basis chi; with V = chi(xi) on the context's n^d cubature nodes (Kronecker
 * product of the 1D table of sfh_basis_table, x fastest),
 *   r_hat = V^T r_v(V u_hat),
 * r_v the collocated volume residual of sfh_volume_residual at the nodal
 * values.  Both transforms are sum-factorized (d n^{d+1} per variable) and
 * fused into the residual kernels (the nodal values never reach HBM), except
 * in the FP32 modes for 3D Euler at n = 3..8: there they run as kernels of
 * their own around the nodal kernel (the same arithmetic in the same order,
 * so the same bits), with scratch for V u_hat and r_v taken
 * in stream order from a memory pool of the context (2 n_elem nvar n^d
 * floats per call, released in stream order; SFH_ENOMEM if the pool cannot
 * provide it).  The
 * entropy projection of the uncollocated scheme, u~ = u(V Pi w(V u_hat)) with
 * Pi = (V^T W V)^{-1} V^T W, is the identity here: V is square and invertible
 * (as many cubature nodes as basis functions), so Pi = V^{-1} and u~ = V u_hat.
 * u_hat, r_hat: device, [n_elem][nvar][n^d] (coefficient index k = k_0 +
 *       n k_1 + n^2 k_2), double for SFH_FP64, float otherwise; Ja: device
 *       [n_elem][d][d][n^d] double on the cubature nodes.
 * r_hat is overwritten and must not overlap the inputs.  Asynchronous.
 * Errors: SFH_EINVAL (bad basis, precision, sizes, alignment, overlap) before
 * any launch; SFH_ENOMEM (FP32-mode scratch); SFH_ECUDA if a launch fails;
 * domain errors of the nodal values are latched for sfh_check(). */
sfh_status sfh_volume_residual_modal(sfh_ctx *ctx, sfh_basis basis, int64_t n_elem, const void *u_hat,
                                     const double *Ja, void *r_hat, sfh_prec prec, sfh_stream_t stream);

/* The 1D basis table of the modal entry point on the cubature nodes of
 * `nodes`: V[a*(p+1) + k] = chi_k(xi_a), host memory of (p+1)^2 doubles,
 * written by the caller-owned pointer.  No device is needed.
 * Errors: SFH_EINVAL for p outside [1, 8], an unknown node set or basis, or
 * V == NULL. */
sfh_status sfh_basis_table(int p, sfh_nodes nodes, sfh_basis basis, double *V);

/* Vector-Jacobian product of the volume residual with respect to u (FP64):
 * grad_u = (dr/du)^T lambda with Ja held fixed, i.e.
 *   g_l = sum_m sum_{j on the m-line of l} (Q_m,lj lambda_l + Q_m,jl lambda_j)^T d1F_m(u_l, u_j),
 * which follows from Eq. 3 and the symmetry of F_m in its two states.
 * u, lambda, grad_u: device double [n_elem][nvar][n^d]; Ja as above.
 * grad_u is overwritten and must not overlap the inputs.  Asynchronous. */
sfh_status sfh_vjp(sfh_ctx *ctx, int64_t n_elem, const double *u, const double *Ja,
                   const double *lambda, double *grad_u, sfh_stream_t stream);

/* Surface Hadamard product of every element's 2d faces (Remark 1: the
 * operator of the theorem on general bases with alpha = 0 on the facet
 * cubature, one-dimensional factors of size 1 x n), FP64.  Face (m, side),
 * side 0 at xi_m = -1 and side 1 at +1, carries the facet cubature of the
 * other directions' nodes (n^{d-1} points f, lower axis fastest, weights
 * w_f = prod w); E = e (x) I (x) I interpolates to it (e[b] = l_b(-+1) in
 * position m), so face node f couples to the n volume nodes j of its normal
 * line only (d n^d two-point fluxes per element and face direction; one per
 * face node on Gauss-Lobatto nodes).  With
 *   H[f][j] = w_f E[f][j] fsharp(u_face_f, u_j) . nJ_f,
 *   r_vol[j] = sum over the faces of sum_f H[f][j],  r_face[f] = sum_j H[f][j]
 * (the volume-to-face coupling of a hybridised SBP discretisation).
 * u, r_vol: device double [n_elem][nvar][n^d]; u_face, r_face: device double
 * [n_elem][2d][nvar][n^{d-1}] (face index 2 m + side); nJ_face: device double
 * [n_elem][2d][d][n^{d-1}], the scaled face normal at each face node, supplied
 * by the caller (its sign and scaling are the caller's).  Outputs are
 * overwritten and must not overlap each other or the inputs.  Asynchronous.
 * Errors: SFH_EINVAL before any launch; SFH_ECUDA; domain errors latched for
 * sfh_check(). */
sfh_status sfh_surface_hadamard(sfh_ctx *ctx, int64_t n_elem, const double *u, const double *u_face,
                                const double *nJ_face, double *r_vol, double *r_face, sfh_stream_t stream);

/* VJP of the modal residual (FP64), Ja fixed: with r_hat = V^T r_v(V u_hat)
 * as in sfh_volume_residual_modal,
 *   grad_hat = V^T (dr_v/du_v)^T V lambda_hat,   u_v = V u_hat,
 * the nodal VJP of sfh_vjp between two sum-factorized transforms, all fused
 * in one kernel.  u_hat, lambda_hat, grad_hat: device double
 * [n_elem][nvar][n^d] (coefficients); Ja as above.  grad_hat is overwritten
 * and must not overlap the inputs.  Asynchronous.  Errors as
 * sfh_volume_residual_modal. */
sfh_status sfh_vjp_modal(sfh_ctx *ctx, sfh_basis basis, int64_t n_elem, const double *u_hat, const double *Ja,
                         const double *lambda_hat, double *grad_hat, sfh_stream_t stream);

/* Entropy identity of the volume term (summation by parts, Tadmor's
 * condition for the symmetric entropy-conservative flux; general SBP form,
 * which for Gauss-Lobatto nodes is the element's boundary entropy flux):
 * per element e, in FP64 on the GPU,
 *   out[e] = |w^T r_e - sum_m [ 1/2 sum_ij E_ij w_i.F_ij - 1/2 sum_i (E 1)_i psi_i.J_i
 *                                - 1/2 psi^T E J + psi^T Q J ]| / sum_m sum_ij |Q_ij| |w_i . F_ij|,
 * E = Q_m + Q_m^T, J = Ja^m, w the entropy variables and psi the entropy
 * potential of the FP64 state u (Eq. 3 operators).  r is a residual of this
 * context's volume term computed in any mode: r_prec SFH_FP64 (double) or
 * SFH_FP32_KAHAN / SFH_FP32_MIXED (float).  A residual of the method sits at
 * the round-off of its precision (FP64 ~1e-16, FP32 ~1e-9).
 * u: device double [n_elem][nvar][n^d]; Ja as above; out: device double
 * [n_elem].  Asynchronous; domain errors latched for sfh_check(). */
sfh_status sfh_entropy_residual(sfh_ctx *ctx, int64_t n_elem, const double *u, const double *Ja, const void *r,
                                sfh_prec r_prec, double *out, sfh_stream_t stream);

/* Synchronize `stream`, then read and clear the context's device error word.
 * Returns SFH_EDOMAIN if any kernel of this context saw rho <= 0 or p <= 0
 * (or a NaN) or a metric term outside the accepted range (see
 * sfh_volume_residual) since the last check, SFH_ETIMEOUT if a bounded device
 * wait gave up, SFH_ECUDA on a CUDA error, else SFH_OK; sfh_last_error()
 * says which. */
sfh_status sfh_check(sfh_ctx *ctx, sfh_stream_t stream);

/* Host-buffer form of sfh_volume_residual: u_host, Ja_host, r_host are host
 * pointers (page-locked memory gives full copy bandwidth; pageable memory
 * works but is staged by the CUDA runtime).  The elements are processed in
 * chunks on two internal streams so that host->device copies, kernels and
 * device->host copies overlap; the device staging buffers belong to the
 * context (allocated on first use, grown when needed, freed by
 * sfh_destroy).  Synchronous: returns when r_host is filled, and also
 * reports device domain errors (as sfh_check would).
 * Errors: SFH_EINVAL, SFH_ENOMEM, SFH_ECUDA, SFH_EDOMAIN. */
sfh_status sfh_volume_residual_host(sfh_ctx *ctx, int64_t n_elem, const void *u_host,
                                    const double *Ja_host, void *r_host, sfh_prec prec);

/* Bind the metric terms of a mesh to the context.  The metric terms Ja of
 * Eq. 3 depend only on the mesh (Section 2), so a solver that evaluates the
 * residual at every stage of every time step can upload them once and then
 * move only u and r per call (sfh_volume_residual_host_bound).  Copies
 * Ja_host ([n_elem][d][d][n^d] double, host memory, pageable or page-locked)
 * into device memory owned by the context: allocated or grown here, kept
 * until the next bind or sfh_destroy.  Synchronous.  n_elem = 0 unbinds.
 * The metric range check of sfh_volume_residual applies when a residual runs.
 * Errors: SFH_EINVAL (NULL or misaligned Ja_host, n_elem < 0 or > 2^40),
 * SFH_ENOMEM, SFH_ECUDA. */
sfh_status sfh_bind_metric(sfh_ctx *ctx, int64_t n_elem, const double *Ja_host);

/* Host-buffer residual on the bound metric: the same result as
 * sfh_volume_residual_host(ctx, n_elem, u_host, Ja, r_host, prec) with the Ja
 * last passed to sfh_bind_metric, but only u travels to the device and r back
 * (for 3D Euler p = 4 in FP32: 5,000 bytes per element instead of 14,000).
 * Elements [0, n_elem) of the bound metric are used; n_elem may not exceed
 * the bound count.  Chunks of u rotate over four internal streams (copy in,
 * kernel, copy out) with staging buffers owned by the context (allocated on
 * first use, freed by sfh_destroy).  Synchronous: returns when r_host is filled, and
 * reports device errors as sfh_check would.
 * Errors: SFH_EINVAL (bad mode, NULL or misaligned pointers, overlapping u
 * and r, n_elem above the bound count), SFH_ENOMEM, SFH_ECUDA, SFH_EDOMAIN,
 * SFH_ETIMEOUT. */
sfh_status sfh_volume_residual_host_bound(sfh_ctx *ctx, int64_t n_elem, const void *u_host, void *r_host,
                                          sfh_prec prec);

/* Volume residual for callers that cannot allocate device memory (no
 * counterpart in the paper: this is a deployment convenience).  Some callers
 * cannot call cudaMalloc -- for instance a host application whose device
 * memory belongs to another allocator with a fixed budget, or one that must
 * not allocate after start-up.  They pass host buffers (layouts as in
 * sfh_volume_residual; pageable or page-locked) and a stream; the library
 * needs no context: it builds the operator tables on the host stack and
 * stages u, Ja and r, plus its device error word, through one fixed device
 * array that is part of the library image (64 MiB; every GPU that loads the
 * library holds it until the process exits).  It calls no cudaMalloc,
 * cudaFree or allocating routine.
 * Limit: 256 + 2 * round256(bytes(u)) + round256(bytes(Ja)) <= 64 MiB (for 3D
 * Euler p = 4: about 4,790 elements in FP32, 3,530 in FP64); larger
 * requests return SFH_EINVAL with the limit in sfh_last_error().  The
 * element count is compared with that limit before any byte count is formed,
 * so no n_elem (up to INT64_MAX) can wrap the size check.
 * The array keeps the last call's contents (the error word is cleared at the
 * start of each call); calls that overlap on the GPU -- from two host threads
 * or on two streams -- race on it and must be serialized by the caller.  The
 * first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any
 * stream capture.  Synchronous: returns when r_host is
 * filled.  Errors: SFH_EINVAL, SFH_ECUDA, SFH_EDOMAIN, SFH_ETIMEOUT. */
sfh_status sfh_volume_residual_host_noalloc(int d, int p, sfh_nodes nodes, sfh_flux flux, int64_t n_elem,
                                            const void *u_host, const double *Ja_host, void *r_host,
                                            sfh_prec prec, sfh_stream_t stream);

/* Describe a context: any output pointer may be NULL.  n_nodes = (p+1)^d. */
sfh_status sfh_ctx_info(const sfh_ctx *ctx, int *d, int *p, int *nodes, int *nvar, int *flux,
                        int *n_nodes);

/* The 1D operator tables of one element type, computed on the host (no
 * device needed): nodes xi[n] (ascending on [-1, 1]), quadrature weights
 * w[n], collocation derivative D[n*n] (D[i*n + j] = l_j'(xi_i)) and the
 * weighted derivative Q1 = W D [n*n] of Eq. 5, n = p + 1, FP64, row-major.
 * Gauss-Lobatto: endpoints and the roots of P_p'; Gauss-Legendre: roots of
 * P_{p+1}.  Any output pointer may be NULL.  Errors: SFH_EINVAL. */
sfh_status sfh_operator_tables(int p, sfh_nodes nodes, double *xi, double *w, double *D, double *Q1);

/* Thread-local message describing the last error of the calling thread
 * ("" if none).  Never NULL. */
const char *sfh_last_error(void);

/* The generic Hadamard product of the paper's timing experiment (Section 3,
 * Fig. 1): for each of n_elem elements of (p+1)^3 Gauss-Lobatto nodes
 * (x fastest), y = sum_{m=1..3} (D_m o C) 1 with C = c c^T and D_m the
 * derivative of the collocated Lagrange basis along direction m (the factor
 * D in the m-th position of D (x) I (x) I, Eq. 5 without weights).
 * dense = 0: the sum-factorized O(n^{d+1}) evaluation (Section 2);
 * dense != 0: the direct O(n^{2d}) evaluation over all columns.
 * p in [1, 15]; c, y: device double [n_elem][(p+1)^3], 8-byte aligned, y
 * must not overlap c.  Asynchronous on `stream`; argument errors
 * (SFH_EINVAL) before any launch, SFH_ECUDA if the launch fails. */
sfh_status sfh_fig1_hadamard(int p, int64_t n_elem, const double *c, double *y, int dense, sfh_stream_t stream);

/* Library version as major * 10000 + minor * 100 + patch. */
int sfh_version(void);

/* ---------------------------------------------------------------------------
 * Arithmetic-peak microbenchmarks (the denominators of the ALU rooflines).
 * Runs a register-resident chain of fused multiply-adds on every SM of the
 * current device and reports the achieved rate.  prec: SFH_FP64 (DFMA) or
 * SFH_FP32_KAHAN (FFMA).  *tflops receives 2 * FMAs / second / 1e12, *ms the
 * measured kernel time.  Synchronous.
 * ------------------------------------------------------------------------- */
sfh_status sfh_peak_fma(sfh_prec prec, double *tflops, double *ms);

/* ---------------------------------------------------------------------------
 * Self-test of the failure path of the kernels' bounded waits (no paper
 * counterpart: failure detection).  Launches one CTA on the current device
 * that waits, with the same bounded wait the volume kernels use for their
 * bulk copies, on a shared-memory barrier phase that nothing completes (a
 * transaction count is announced, no copy is issued).  After limit_us
 * microseconds (1 .. 10^7) the wait gives up, the kernel records the timeout
 * in its error word and returns; no copy is in flight and the context stays
 * usable.  Synchronous on `stream`.
 * Returns SFH_ETIMEOUT when the wait gave up as designed, SFH_OK if it
 * completed (a defect), SFH_EINVAL for a limit out of range, SFH_ECUDA for a
 * CUDA error.  *elapsed_us (optional) receives the device-measured wait.
 * ------------------------------------------------------------------------- */
sfh_status sfh_selftest_bounded_wait(int64_t limit_us, sfh_stream_t stream, double *elapsed_us);

/* ---------------------------------------------------------------------------
 * Build variant (no paper counterpart).  Returns a bit set: SFH_BUILD_DEBUG
 * when this library is the bounds-checked debug build (libsfhad_debug.so,
 * compiled with -DSFH_DEBUG).  In that build every kernel addresses global and
 * shared memory through checked pointers that know their buffer: an index
 * outside it latches a bit in the call's device error word, the access is
 * not made (a load reads a scratch word, a store is dropped, a bulk copy is
 * not issued and its mbarrier bytes are released), no thread leaves early and
 * no barrier is skipped; the next sfh_check (or the synchronous call) returns
 * SFH_EBOUNDS.  The release library (libsfhad.so) has no checks; its kernels
 * are the same code as without the checked pointers.
 * ------------------------------------------------------------------------- */
#define SFH_BUILD_DEBUG 1
int sfh_build_flags(void);

/* ---------------------------------------------------------------------------
 * Self-test of the debug build's bounds checks (no paper counterpart).
 * Launches one thread on the current device with a checked pointer over the
 * first 64 words of a 128-word device buffer (so even an unchecked access
 * would stay inside the allocation): it reads word 64 and writes word 65,
 * both outside the pointer's extent, and writes word 0, inside it.
 * Synchronous on `stream`.
 * Returns SFH_OK when the checks latched the bounds bit, skipped the write
 * outside the extent and made the one inside it; SFH_EBOUNDS if they did not
 * (a defect); SFH_EUNSUPPORTED in the release build (nothing is launched);
 * SFH_ECUDA for a CUDA error.
 * ------------------------------------------------------------------------- */
sfh_status sfh_selftest_bounds(sfh_stream_t stream);

/* ---------------------------------------------------------------------------
 * Serving: batched residual and VJP requests of mixed degree p, node set,
 * flux, element count and precision on one device (3D Euler, Ranocha's or
 * Chandrashekar's flux; nodal form).  Requests are
 * admitted in FIFO order against an HBM budget and a limit on requests in
 * flight; admitted work is cut into element tiles and executed by persistent
 * CTAs that pull tiles from a device queue, so tiles of requests that arrive
 * while others run are interleaved with them on the GPU.
 * ------------------------------------------------------------------------- */
typedef struct sfh_server sfh_server;

typedef struct {
    size_t hbm_budget_bytes;   /* admission budget for resident request data (u, Ja, out, lambda) */
    int max_inflight;          /* requests admitted at once (>= 1) */
    int timeout_ms;            /* bound on every wait of the server (device and host) */
    int n_workers;             /* persistent CTAs; 0 = one per SM */
} sfh_server_opts;

typedef enum { SFH_REQ_RESIDUAL = 0, SFH_REQ_VJP = 1 } sfh_req_kind;

typedef struct {
    int kind;            /* sfh_req_kind */
    int p;               /* 2..8 */
    int nodes;           /* sfh_nodes */
    int prec;            /* sfh_prec for residuals; VJP requests are FP64 */
    int64_t n_elem;
    const void *u;       /* device, resident; double (FP64, VJP) or float (FP32 modes) */
    const double *Ja;    /* device, resident */
    const double *lambda;/* device, VJP only */
    void *out;           /* device: r (residual) or grad_u (VJP), overwritten */
    int flux;            /* sfh_flux: SFH_FLUX_EULER_RANOCHA or SFH_FLUX_EULER_CHANDRASHEKAR
                            (anything else, Burgers included: SFH_EINVAL) */
} sfh_request;

typedef struct {
    int status;          /* sfh_status of the request */
    /* host CLOCK_MONOTONIC timestamps: submitted, admitted (its tiles
     * published), started (the first of its tiles began on the device: the
     * device timer mapped to the host clock by a calibration at server
     * creation, to within a few microseconds; 0 if no tile ran), done (the
     * completion seen by the host) */
    uint64_t t_submit_ns, t_admit_ns, t_start_ns, t_done_ns;
} sfh_result;

/* Create a server on the current device; starts its persistent kernel and
 * its host admission thread.  Errors: SFH_EINVAL, SFH_ENOMEM, SFH_ECUDA. */
sfh_status sfh_server_create(const sfh_server_opts *opts, sfh_server **out);

/* Queue a request (thread-safe).  SFH_ENOMEM if the request alone exceeds
 * the budget, SFH_EINVAL for bad fields; otherwise the request is queued
 * FIFO and *ticket identifies it.  The arrays must stay valid and unchanged
 * until sfh_serve_poll reports the request done.  The server's persistent
 * kernel may start the request at once and is not ordered against the
 * caller's streams: device work that writes u, Ja or lambda, or that still
 * reads or writes out, must be complete before the call. */
sfh_status sfh_serve_submit(sfh_server *srv, const sfh_request *req, uint64_t *ticket);

/* Non-blocking: SFH_OK and *out filled when the request is done (out->status
 * holds its own result), SFH_ENOTREADY while it is pending, SFH_EINVAL for an
 * unknown ticket.  A ticket can be polled done once.  A request still in
 * flight timeout_ms after its admission is reported done with status
 * SFH_ETIMEOUT; the device may still be running it, so its arrays must stay
 * valid until sfh_server_destroy returns. */
sfh_status sfh_serve_poll(sfh_server *srv, uint64_t ticket, sfh_result *out);

/* Replay a request stream: request i is submitted at arrival_s[i] seconds
 * after the call starts (arrival_s ascending), completions are polled while
 * the stream is fed, and results[i] receives request i's result (timestamps
 * included; a request refused at submission carries that status).  Blocks
 * until every request is done (SFH_OK) or timeout_ms passes (SFH_ETIMEOUT).
 * The load generator of the serving benchmark: a native loop keeps up with
 * arrival rates a scripting-language client cannot. */
sfh_status sfh_serve_replay(sfh_server *srv, int n, const sfh_request *reqs, const double *arrival_s,
                            sfh_result *results, int timeout_ms);

/* Baseline of the serving benchmark (no paper counterpart): the same kind of
 * request stream as sfh_serve_replay, run without a server -- each request
 * as one plain launch of sfh_volume_residual (in its own precision) or
 * sfh_vjp, in FIFO order on one stream of the current device, enqueued at
 * its arrival time, so that waiting behind earlier requests is part of its
 * latency.  Requests as for sfh_serve_submit (3D Euler, either flux);
 * contexts are created per node set, flux and degree for the call.  results[i]: t_submit_ns =
 * t_admit_ns = enqueue time; t_start_ns = max(enqueue time, previous
 * request's done time), the start of a FIFO stream; t_done_ns = host time at
 * which its completion was seen (polled every ~10 us).  Blocks until all are
 * done (SFH_OK), or timeout_ms passes (SFH_ETIMEOUT).  A device-detected
 * domain error of any request makes the call return SFH_EDOMAIN (not
 * attributed to a request).  Errors: SFH_EINVAL, SFH_ECUDA. */
sfh_status sfh_serial_replay(int n, const sfh_request *reqs, const double *arrival_s, sfh_result *results,
                             int timeout_ms);

/* Block until every submitted request is done or timeout_ms passes
 * (SFH_ETIMEOUT). */
sfh_status sfh_serve_drain(sfh_server *srv, int timeout_ms);

/* Host-side fault injection, for testing the server's failure detection (no
 * paper counterpart; no device fault is involved):
 *   SFH_FAULT_CREATE_ALLOC (srv may be NULL): the next sfh_server_create
 *     fails at its arg-th allocation (1..4; 0 clears) and returns
 *     SFH_ENOMEM after releasing what it had allocated;
 *   SFH_FAULT_DROP_TILE: the next arg admitted requests publish all but
 *     their last tile, so they never complete.  The server's watchdog reports
 *     each SFH_ETIMEOUT timeout_ms after admission (its slot and budget stay
 *     held), sfh_serve_drain returns SFH_ETIMEOUT, and sfh_server_destroy
 *     stops the kernel, frees the server and returns SFH_ETIMEOUT;
 *   SFH_FAULT_STALL_ADMISSION: the admission thread sleeps arg milliseconds
 *     once (a stalled host thread); the caller's waits stay bounded.
 * Errors: SFH_EINVAL for an unknown kind or argument. */
typedef enum { SFH_FAULT_CREATE_ALLOC = 1, SFH_FAULT_DROP_TILE = 2, SFH_FAULT_STALL_ADMISSION = 3 } sfh_fault;
sfh_status sfh_serve_inject_fault(sfh_server *srv, int kind, int arg);

/* Serving-kernel counters since the server was created (tracing; no paper
 * counterpart), summed over the persistent CTAs from the device timer:
 * per class (0 residual FP64, 1 residual FP32-Kahan, 2 residual mixed,
 * 3 VJP) the tiles run and the nanoseconds spent running them, and the
 * nanoseconds CTAs spent claiming a tile (from the end of one tile to the
 * start of the next, idle waits included).  Call with no request in flight
 * for exact figures (synchronizes with the device). */
typedef struct {
    uint64_t tiles[4];
    uint64_t busy_ns[4];
    uint64_t claim_ns;
} sfh_serve_stats_t;
sfh_status sfh_serve_stats(sfh_server *srv, sfh_serve_stats_t *out);

/* Stop the server: drains (bounded by timeout_ms), stops the persistent
 * kernel, joins the admission thread and frees the server. NULL accepted. */
sfh_status sfh_server_destroy(sfh_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* SFHAD_H */
