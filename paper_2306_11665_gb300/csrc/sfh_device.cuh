// sfh_device.cuh -- device building blocks of libsfhad: element shapes,
// logarithmic means, two-point fluxes and compensated sums.
//
// Notation follows Section 2 of arXiv 2306.11665: n = p + 1 nodes per
// direction, element node i = a_0 + n a_1 + n^2 a_2 (x fastest), Q1 = W D the
// weighted 1D derivative of Eq. 5, and omega_m(i) = prod_{k != m} w[a_k(i)]
// the product of the diagonal factors in Eq. 3.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sfh_debug.cuh"
#include "sfh_tma.cuh"

namespace sfh {

constexpr int NMAX = 9;              // p <= 8
constexpr double kGamma = 1.4;
constexpr int kFluxBurgers = 0;
constexpr int kFluxEuler = 1;     // Ranocha's entropy-conserving, kinetic-energy-preserving flux
constexpr int kFluxEulerCh = 2;   // Chandrashekar's: the same but for the pressure terms
__host__ __device__ constexpr bool is_euler(int flux) { return flux == kFluxEuler || flux == kFluxEulerCh; }

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// 1D operator table passed by value as a kernel parameter: compile-time
// indices then become constant-bank operands of the arithmetic instructions.
template <typename T>
struct OpTab {
    T Q1[NMAX * NMAX];   // packed n x n, row-major, Q1[a*n + b] = w_a D_ab
    T w[NMAX];
};

// 1D basis of a modal / uncollocated solution on the cubature nodes:
// V[a*n + k] = chi_k(xi_a) (node a, basis function k), a kernel parameter.
// const_mode: chi_0 is the constant c0^(1/d) (orthonormal Legendre): the
// forward transform then takes the element's constant part c = u_hat_0 c0
// out of the sums and adds it back at the end, so that the rounding of the
// sums scales with the (small) non-constant part of the state.
template <typename T>
struct BasisTab {
    T V[NMAX * NMAX];
    T c0;             // chi_0^d (const_mode only)
    int const_mode;
};

// Role of a forward pass in the constant-part split (const_mode bases).
constexpr int kPassPlain = 0, kPassFirst = 1, kPassLast = 2;

// One pass of the sum-factorized basis transform (Section 2, the theorem on
// uncollocated bases): along direction m, every line of every
// element-variable q < nq (layout [q][i], NN values each) is multiplied by V
// (node values from coefficients) or, TRANSPOSE, by V^T (tests against chi).
// A thread per (q, line); the line's n inputs in registers, the table indices
// compile-time constants.  ROLE (forward, const_mode): kPassFirst drops the
// constant coefficient u_hat_0 (read from `coef`, the pass-0 input), kPassLast
// adds c = u_hat_0 c0 to every output.
// in, out and coef are pointers or checked pointers (BPtr) to the elements.
template <typename T, int D, int N, bool TRANSPOSE, int ROLE = kPassPlain, typename PI, typename PO,
          typename PC = const T *>
__device__ __forceinline__ void basis_pass(PI in, PO out, int m, int nq, const BasisTab<T> &bt, int tid,
                                           int nthreads, PC coef = nullptr) {
    constexpr int NN = ipow(N, D), NLINE = ipow(N, D - 1);
    const int stride = m == 0 ? 1 : (m == 1 ? N : N * N);
    for (int t = tid; t < nq * NLINE; t += nthreads) {
        const int q = t / NLINE, l = t - q * NLINE;
        int base;
        if constexpr (D == 3) base = m == 0 ? N * l : (m == 1 ? l % N + N * N * (l / N) : l);
        else base = m == 0 ? N * l : l;
        const auto src = in + (size_t)q * NN + base;
        const auto dst = out + (size_t)q * NN + base;
        T x[N];
#pragma unroll
        for (int b = 0; b < N; ++b) x[b] = (T)src[b * stride];
        if constexpr (ROLE == kPassFirst) {
            if (bt.const_mode && base == 0) x[0] = (T)0;   // coefficient (0, .., 0) sits on line 0, b = 0
        }
        T c = (T)0;
        if constexpr (ROLE == kPassLast) {
            if (bt.const_mode) c = (T)coef[(size_t)q * NN] * bt.c0;
        }
#pragma unroll
        for (int a = 0; a < N; ++a) {
            T s = (T)0;
#pragma unroll
            for (int b = 0; b < N; ++b) s = fma(TRANSPOSE ? bt.V[b * N + a] : bt.V[a * N + b], x[b], s);
            if constexpr (ROLE == kPassLast) s += c;
            dst[a * stride] = s;
        }
    }
}

// ---------------------------------------------------------------------------
// Precision modes.
//   T  : type of u, r and the flux arithmetic
//   TJ : type in which the metric sum Ja(i) + Ja(j) is formed
// ---------------------------------------------------------------------------
struct ModeFP64 { using T = double; using TJ = double; static constexpr bool kahan = false; static constexpr bool mixed = false; };
struct ModeFP32K { using T = float; using TJ = float; static constexpr bool kahan = true; static constexpr bool mixed = false; };
struct ModeMixed { using T = float; using TJ = double; static constexpr bool kahan = true; static constexpr bool mixed = true; };

// ---------------------------------------------------------------------------
// Element shape and CTA geometry.  One CTA handles EPB consecutive elements;
// in the line phase one thread owns one grid line of one element.
// Shared memory per node: primitives (NP values of T), the residual
// accumulator (NVAR of T), the metric row of the current direction (D of TJ)
// and, for the mixed mode, an FP64 copy of beta = rho / p.
// ---------------------------------------------------------------------------
// BUDGET: shared-memory budget of one tile; LINES: target line tasks per
// tile (0: 128, or 256 for lines of 48 and more nodes).  The standalone
// kernels use the defaults; the serving kernel asks for tiles that fill its
// 256 threads.
template <int D, int N, int FLUX, class M, int BUDGET = 96 * 1024, int LINES = 0>
struct Shape {
    using T = typename M::T;
    using TJ = typename M::TJ;
    static constexpr int NN = ipow(N, D);
    static constexpr int NLINE = ipow(N, D - 1);
    static constexpr int NVAR = is_euler(FLUX) ? D + 2 : 1;
    static constexpr int NP = is_euler(FLUX) ? D + 3 : 1;   // rho, v[D], p, beta | u
    // FP64 Euler keeps FP32 copies of rho and beta (band tests), the mixed
    // mode an FP64 copy of beta: 8 extra bytes per node either way
    static constexpr bool F64E = sizeof(T) == 8 && is_euler(FLUX);
    static constexpr int NODE_BYTES = (int)sizeof(T) * (NP + NVAR) + (int)sizeof(TJ) * D
                                      + (((M::mixed || F64E) && is_euler(FLUX)) ? 8 : 0);
    static constexpr int SMEM_BUDGET = BUDGET;
    static constexpr int EPB_SMEM = SMEM_BUDGET / (NN * NODE_BYTES) > 0 ? SMEM_BUDGET / (NN * NODE_BYTES) : 1;
    static constexpr int TARGET_LINES = LINES > 0 ? LINES : (NLINE >= 48 ? 256 : 128);
    static constexpr int EPB_LINES = TARGET_LINES / NLINE > 0 ? TARGET_LINES / NLINE : 1;
    static constexpr int EPB = EPB_SMEM < EPB_LINES ? EPB_SMEM : EPB_LINES;
    static constexpr int THREADS = ((EPB * NLINE + 31) / 32) * 32;
    static constexpr size_t SMEM = (size_t)EPB * NN * NODE_BYTES;
    // resident CTAs asked of the compiler: the mixed mode's FP64 log means
    // are latency-bound, so at n <= 5 its line body is held to 128 registers
    // (four warps per sub-partition instead of three)
    static constexpr int MINB = (M::mixed && N <= 5 && THREADS <= 128) ? 65536 / (THREADS * 128) : 1;
};

// ---------------------------------------------------------------------------
// Logarithmic mean {a,b}_ln = (a - b) / (ln a - ln b), a, b > 0.
// With s = a + b, t = (a - b)/s, u = t^2 (so 0 <= u < 1):
//   ln a - ln b = 2 artanh(t) = 2 t sum_k u^k / (2k + 1),
//   {a,b}_ln   = (s / 2) S(u),   S(u) = sqrt(u) / artanh(sqrt(u)),
//   1/{a,b}_ln = (2 / s) P(u),   P(u) = sum_k u^k / (2k + 1).
// The Taylor coefficients of S (1, -1/3, -4/45, -44/945, -428/14175, ...) come
// from inverting the series of P.  Inside the band u < 1e-2 (|a-b| < 0.1 (a+b))
// the truncated series below are accurate to the working precision (FP64:
// 8 and 9 terms, next term < 2e-18; FP32: 4 terms, next term < 1e-9); outside
// it the quotient uses the logarithm of the ratio, whose relative error is
// then at most a few ulp / |ln(a/b)| <= a few ulp / 0.2.
// ---------------------------------------------------------------------------
constexpr double kLnBand = 1e-2;

__device__ __forceinline__ double series_S(double u) {
    return 1.0 + u * (-1.0 / 3.0 + u * (-4.0 / 45.0 + u * (-44.0 / 945.0 + u * (-428.0 / 14175.0
           + u * (-10196.0 / 467775.0 + u * (-10719068.0 / 638512875.0 + u * (-25865068.0 / 1915538625.0)))))));
}
__device__ __forceinline__ double series_dS(double u) {   // S'(u)
    return -1.0 / 3.0 + u * (2.0 * -4.0 / 45.0 + u * (3.0 * -44.0 / 945.0 + u * (4.0 * -428.0 / 14175.0
           + u * (5.0 * -10196.0 / 467775.0 + u * (6.0 * -10719068.0 / 638512875.0
           + u * (7.0 * -25865068.0 / 1915538625.0))))));
}
__device__ __forceinline__ double series_P(double u) {
    return 1.0 + u * (1.0 / 3.0 + u * (1.0 / 5.0 + u * (1.0 / 7.0 + u * (1.0 / 9.0 + u * (1.0 / 11.0
           + u * (1.0 / 13.0 + u * (1.0 / 15.0 + u * (1.0 / 17.0))))))));
}
__device__ __forceinline__ float series_S(float u) {
    return 1.0f + u * (-1.0f / 3.0f + u * (-4.0f / 45.0f + u * (-44.0f / 945.0f)));
}
__device__ __forceinline__ float series_P(float u) {
    return 1.0f + u * (1.0f / 3.0f + u * (1.0f / 5.0f + u * (1.0f / 7.0f)));
}

__device__ __forceinline__ double ln_mean(double a, double b) {
    const double d = a - b, s = a + b;
    if (d * d < kLnBand * (s * s)) {
        const double t = d / s;
        return 0.5 * s * series_S(t * t);
    }
    return d / log(a / b);
}
__device__ __forceinline__ double inv_ln_mean(double a, double b) {
    const double d = a - b, s = a + b;
    if (d * d < kLnBand * (s * s)) {
        const double rs = 1.0 / s;
        const double t = d * rs;
        return 2.0 * rs * series_P(t * t);
    }
    return log(a / b) / d;
}
__device__ __forceinline__ float ln_mean(float a, float b) {
    const float d = a - b, s = a + b;
    if (d * d < (float)kLnBand * (s * s)) {
        const float t = __fdividef(d, s);
        return 0.5f * s * series_S(t * t);
    }
    return __fdividef(d, logf(__fdividef(a, b)));
}
__device__ __forceinline__ float inv_ln_mean(float a, float b) {
    const float d = a - b, s = a + b;
    if (d * d < (float)kLnBand * (s * s)) {
        const float rs = __fdividef(1.0f, s);
        const float t = d * rs;
        return 2.0f * rs * series_P(t * t);
    }
    return __fdividef(logf(__fdividef(a, b)), d);
}

// Reciprocal for the FP64 kernels: the hardware seed of rcp.approx.ftz.f64
// refined by two Newton-Raphson steps r <- r + r (1 - s r) (each step doubles
// the correct bits; four fused multiply-adds instead of a full IEEE division).
// Accurate to about 1 ulp for normal s; subnormal s flushes to zero.
__device__ __forceinline__ double rcp_nr(double s) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(s));
    double e = fma(-s, r, 1.0);
    r = fma(r, e, r);
    e = fma(-s, r, 1.0);
    return fma(r, e, r);
}

// FP64 logarithmic means with the band test taken on FP32 copies of the
// arguments (af, bf), so that it costs no FP64 instruction.  Inside the band
// (u < 1e-2) the series run in FP64 up to u^4; the tail u^5 T(u) is below
// 3e-12 relative and is summed in FP32 (its rounding then weighs < 2e-19),
// which moves three of the eight FP64 steps to the FP32 pipe.
__device__ __forceinline__ double ln_mean_f64(double a, double b, float af, float bf) {
    const double d = a - b, s = a + b;
    if (fabsf(af - bf) < 0.1f * (af + bf)) {
        const double t = d * rcp_nr(s);
        const double u = t * t;
        const float uf = d2f_int(u);
        const float T = fmaf(uf, fmaf(uf, (float)(-25865068.0 / 1915538625.0), (float)(-10719068.0 / 638512875.0)),
                             (float)(-10196.0 / 467775.0));
        double h = fma(u, f2d_int(T), -428.0 / 14175.0);
        h = fma(u, h, -44.0 / 945.0);
        h = fma(u, h, -4.0 / 45.0);
        h = fma(u, h, -1.0 / 3.0);
        return (0.5 * s) * fma(u, h, 1.0);
    }
    return d / log(a / b);
}
__device__ __forceinline__ double inv_ln_mean_f64(double a, double b, float af, float bf) {
    const double d = a - b, s = a + b;
    if (fabsf(af - bf) < 0.1f * (af + bf)) {
        const double rs = rcp_nr(s);
        const double t = d * rs;
        const double u = t * t;
        const float uf = d2f_int(u);
        const float T = fmaf(uf, fmaf(uf, fmaf(uf, (float)(1.0 / 17.0), (float)(1.0 / 15.0)), (float)(1.0 / 13.0)),
                             (float)(1.0 / 11.0));
        double h = fma(u, f2d_int(T), 1.0 / 9.0);
        h = fma(u, h, 1.0 / 7.0);
        h = fma(u, h, 1.0 / 5.0);
        h = fma(u, h, 1.0 / 3.0);
        return (2.0 * rs) * fma(u, h, 1.0);
    }
    return log(a / b) / d;
}

// The mixed mode's FP64 logarithmic means inside the band (the caller has
// tested it on the FP32 values af, bf): their results are rounded to FP32,
// so about 2^-40 relative accuracy suffices, not FP64's 2^-53.  1/(a + b) is
// the FP32 hardware reciprocal refined by one FP64 Newton step (2^-22 ->
// below 2^-43); the series run in FP64 up to u^2, the tail from u^3 in FP32
// (its rounding weighs below u^3 2^-24 / 20 < 1e-14).  Eleven FP64
// operations each instead of fifteen.
__device__ __forceinline__ double ln_mean_mix(double a, double b, float af, float bf) {
    const double d = a - b, s = a + b;
    const double r0 = f2d_int(rcp_approx(af + bf));
    const double rs = fma(r0, fma(-s, r0, 1.0), r0);
    const double t = d * rs;
    const double u = t * t;
    const float uf = d2f_int(u);
    float T = fmaf(uf, (float)(-25865068.0 / 1915538625.0), (float)(-10719068.0 / 638512875.0));
    T = fmaf(uf, T, (float)(-10196.0 / 467775.0));
    T = fmaf(uf, T, (float)(-428.0 / 14175.0));
    T = fmaf(uf, T, (float)(-44.0 / 945.0));
    double h = fma(u, f2d_int(T), -4.0 / 45.0);
    h = fma(u, h, -1.0 / 3.0);
    return (0.5 * s) * fma(u, h, 1.0);
}
__device__ __forceinline__ double inv_ln_mean_mix(double a, double b, float af, float bf) {
    const double d = a - b, s = a + b;
    const double r0 = f2d_int(rcp_approx(af + bf));
    const double rs = fma(r0, fma(-s, r0, 1.0), r0);
    const double t = d * rs;
    const double u = t * t;
    const float uf = d2f_int(u);
    float T = fmaf(uf, 1.0f / 17.0f, 1.0f / 15.0f);
    T = fmaf(uf, T, 1.0f / 13.0f);
    T = fmaf(uf, T, 1.0f / 11.0f);
    T = fmaf(uf, T, 1.0f / 9.0f);
    T = fmaf(uf, T, 1.0f / 7.0f);
    double h = fma(u, f2d_int(T), 1.0 / 5.0);
    h = fma(u, h, 1.0 / 3.0);
    return (2.0 * rs) * fma(u, h, 1.0);
}

// Value and both partial derivatives of {a,b}_ln and of its reciprocal
// (FP64, for the adjoint), with the band test on FP32 copies af, bf and the
// series tails from u^5 in FP32 as in ln_mean_f64.  With s = a + b,
// t = (a - b)/s, u = t^2, du/da = 4 t b / s^2, du/db = -4 t a / s^2:
//   L = (s/2) S(u):       dL/da = S/2 + 2 t b S'(u) / s,   dL/db = S/2 - 2 t a S'(u) / s;
//   M = 1/L = (2/s) P(u): dM/da = (2/s^2)(4 t b P'(u)/s - P), dM/db = -(2/s^2)(4 t a P'(u)/s + P).
// Outside the band (logarithms): dL/da = (1 - L/a)/ln(a/b), dL/db = (L/b - 1)/ln(a/b);
//   dM/da = (1/a - M)/(a - b), dM/db = (M - 1/b)/(a - b).
__device__ __forceinline__ void ln_mean_grad_f64(double a, double b, float af, float bf, double &L, double &La,
                                                 double &Lb) {
    const double d = a - b, s = a + b;
    if (fabsf(af - bf) < 0.1f * (af + bf)) {
        const double rs = rcp_nr(s);
        const double t = d * rs, u = t * t;
        const float uf = d2f_int(u);
        const float T = fmaf(uf, fmaf(uf, (float)(-25865068.0 / 1915538625.0), (float)(-10719068.0 / 638512875.0)),
                             (float)(-10196.0 / 467775.0));
        double h = fma(u, f2d_int(T), -428.0 / 14175.0);
        h = fma(u, h, -44.0 / 945.0);
        h = fma(u, h, -4.0 / 45.0);
        h = fma(u, h, -1.0 / 3.0);
        const double S = fma(u, h, 1.0);
        const float Td = fmaf(uf, (float)(7.0 * -25865068.0 / 1915538625.0), (float)(6.0 * -10719068.0 / 638512875.0));
        double g = fma(u, f2d_int(Td), 5.0 * -10196.0 / 467775.0);
        g = fma(u, g, 4.0 * -428.0 / 14175.0);
        g = fma(u, g, 3.0 * -44.0 / 945.0);
        g = fma(u, g, 2.0 * -4.0 / 45.0);
        const double dS = fma(u, g, -1.0 / 3.0);
        const double hS = 0.5 * S, w = 2.0 * t * dS * rs;
        L = s * hS;
        La = fma(w, b, hS);
        Lb = fma(-w, a, hS);
    } else {
        const double lr = log(a / b);
        L = d / lr;
        La = (1.0 - L / a) / lr;
        Lb = (L / b - 1.0) / lr;
    }
}
__device__ __forceinline__ void inv_ln_mean_grad_f64(double a, double b, float af, float bf, double &M, double &Ma,
                                                     double &Mb) {
    const double d = a - b, s = a + b;
    if (fabsf(af - bf) < 0.1f * (af + bf)) {
        const double rs = rcp_nr(s);
        const double t = d * rs, u = t * t;
        const float uf = d2f_int(u);
        const float T = fmaf(uf, fmaf(uf, fmaf(uf, (float)(1.0 / 17.0), (float)(1.0 / 15.0)), (float)(1.0 / 13.0)),
                             (float)(1.0 / 11.0));
        double h = fma(u, f2d_int(T), 1.0 / 9.0);
        h = fma(u, h, 1.0 / 7.0);
        h = fma(u, h, 1.0 / 5.0);
        h = fma(u, h, 1.0 / 3.0);
        const double P = fma(u, h, 1.0);
        const float Td = fmaf(uf, fmaf(uf, (float)(8.0 / 17.0), (float)(7.0 / 15.0)), (float)(6.0 / 13.0));
        double g = fma(u, f2d_int(Td), 5.0 / 11.0);
        g = fma(u, g, 4.0 / 9.0);
        g = fma(u, g, 3.0 / 7.0);
        g = fma(u, g, 2.0 / 5.0);
        const double dP = fma(u, g, 1.0 / 3.0);
        const double r2 = 2.0 * rs, c = r2 * rs, w = 4.0 * t * dP * rs;
        M = r2 * P;
        Ma = c * fma(w, b, -P);
        Mb = -c * fma(w, a, P);
    } else {
        const double lr = log(a / b), id = 1.0 / d;
        M = lr * id;
        Ma = (1.0 / a - M) * id;
        Mb = (M - 1.0 / b) * id;
    }
}

// Value and both partial derivatives of {a,b}_ln (FP64, for the adjoint).
// Band: L = (s/2) S(u), du/da = 4 t b / s^2, du/db = -4 t a / s^2, so
//   dL/da = S/2 + 2 t b S'(u) / s,  dL/db = S/2 - 2 t a S'(u) / s.
// Outside: dL/da = (1 - L/a) / ln(a/b),  dL/db = (L/b - 1) / ln(a/b).
__device__ __forceinline__ void ln_mean_grad(double a, double b, double &L, double &La, double &Lb) {
    const double d = a - b, s = a + b;
    if (d * d < kLnBand * (s * s)) {
        const double rs = 1.0 / s;
        const double t = d * rs, u = t * t;
        const double S = series_S(u), dS = series_dS(u);
        L = 0.5 * s * S;
        La = 0.5 * S + 2.0 * t * b * dS * rs;
        Lb = 0.5 * S - 2.0 * t * a * dS * rs;
    } else {
        const double lr = log(a / b);
        L = d / lr;
        La = (1.0 - L / a) / lr;
        Lb = (L / b - 1.0) / lr;
    }
}

// ---------------------------------------------------------------------------
// Compensated (Kahan) accumulation.  Every step is an explicitly rounded
// intrinsic so the compiler can neither contract nor reassociate it away:
//   y = q*f - c (one rounding, fused), t = s + y, c = (t - s) - y, s = t.
// The represented value is s - c.
// ---------------------------------------------------------------------------
struct KahanF {
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.0f; c = 0.0f; }
    __device__ __forceinline__ void add_prod(float q, float f) {
        const float y = __fmaf_rn(q, f, -c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ float value() const { return __fsub_rn(s, c); }
};

struct PlainD {
    double s;
    __device__ __forceinline__ void zero() { s = 0.0; }
    __device__ __forceinline__ void add_prod(double q, double f) { s = fma(q, f, s); }
    __device__ __forceinline__ double value() const { return s; }
};

template <class M> struct AccOf { using type = PlainD; };
template <> struct AccOf<ModeFP32K> { using type = KahanF; };
template <> struct AccOf<ModeMixed> { using type = KahanF; };

}  // namespace sfh
