/*
 * sfh_oracle.c -- plain FP64 CPU oracle for the sum-factorized Hadamard-product
 * volume term of entropy-conserving flux differencing
 * (Cicchino & Nadarajah, "Scalable evaluation of Hadamard products with tensor
 * product basis for entropy-stable high-order methods", arXiv 2306.11665).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library: it computes its own nodes,
 * its own derivative matrix, its own fluxes and its own metric terms.
 *
 * Everything here is written for readability, not speed: each function
 * follows one definition and loops over indices the way the definition reads.
 *
 * Conventions (Section 2, the three-dimensional listing):
 *   n = p + 1 nodes per direction; element node i <-> (a_0, .., a_{d-1}) with
 *   a_0 (x) running fastest: i = a_0 + n a_1 + n^2 a_2.
 *   u  [e][var][i]       conservative state (Burgers: 1 var; Euler: d + 2 vars)
 *   Ja [e][m][k][i]      J dxi_m/dx_k at node i
 *   r  [e][var][i]       r_i = sum_m sum_j (Q_m o F_m)_ij
 *   Q_m = (tensor product over axes k of A_k), A_m = W D, A_k = W for k != m
 *         (Eq. 5; the factor position names the direction, x runs fastest)
 *   F_m(u_i, u_j) = sum_k fsharp_k(u_i, u_j) (Ja^m_k(i) + Ja^m_k(j))
 *
 * Readings where the paper is silent (the paper gives no flux formulas):
 *   - Burgers: fsharp_k(a, b) = (a^2 + a b + b^2) / 6 in every direction k.
 *   - Euler: Ranocha's entropy-conserving, kinetic-energy-preserving flux with
 *     gamma = 1.4, logarithmic means with the near-equal series of Ranocha,
 *     Schlottke-Lakemper, Winters, Faulhaber, Chan, Gassner (2021) (threshold
 *     1e-4 on ((a-b)/(a+b))^2).
 *   - Euler, second flux: Chandrashekar's entropy-conserving, kinetic-energy-
 *     preserving flux (Commun. Comput. Phys. 2013), the flux the paper names
 *     for its TGV runs (Section 3; the pressure fix it cites is not stated in
 *     the paper and is not applied here).  With beta = rho/p:
 *     f_rho = {rho}_ln {v.n}, f_m = f_rho {v} + ({rho}/{beta}) n,
 *     f_E = f_rho (1/((g-1){beta}_ln) - {|v|^2}/2) + {v}.f_m.
 *     It differs from Ranocha's flux only in the pressure terms; the adjoint
 *     (orc_ec_flux_jac1) covers both.
 *
 * Return codes: 0 = ok, 1 = bad argument, 2 = non-positive density or
 * pressure met (the output is still filled).
 *
 * Parity status: every exported function is pinned by the CPU tests
 * (dense brute force, textbook nodes, SBP identities, Burgers closed form,
 * free stream, entropy identity, conservation, pressure equilibrium, finite
 * differences; for the modal path numpy's Legendre series, quadrature closed
 * forms, sum-factorized transforms and the entropy gradient).  No function
 * here is "parity unpinned".
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_GAMMA 1.4
#define ORC_FLUX_BURGERS 0
#define ORC_FLUX_EULER 1
#define ORC_FLUX_CHANDRASHEKAR 2
#define ORC_NODES_GLL 0
#define ORC_NODES_GAUSS 1

/* ------------------------------------------------------------------------ */
/* 1D collocated Lagrange basis on Gauss-Lobatto or Gauss-Legendre nodes.     */
/* Eq. 4-5 need the collocated nodal basis; these are the node sets the     */
/* paper's results use (Gauss-Legendre in Section 3).                       */
/* ------------------------------------------------------------------------ */

/* Legendre P_k(x), P_k'(x), P_k''(x) for k = q by the three-term recurrence
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}, and its derivative forms
 * P'_{k+1} = P'_{k-1} + (2k+1) P_k,  P''_{k+1} = P''_{k-1} + (2k+1) P'_k. */
static void legendre_eval(int q, long double x, long double *P, long double *dP,
                          long double *d2P)
{
    long double p0 = 1.0L, p1 = x;       /* P_0, P_1 */
    long double dp0 = 0.0L, dp1 = 1.0L;  /* P_0', P_1' */
    long double ddp0 = 0.0L, ddp1 = 0.0L;
    if (q == 0) { *P = 1.0L; *dP = 0.0L; *d2P = 0.0L; return; }
    for (int k = 1; k < q; ++k) {
        long double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
        long double dp2 = dp0 + (2 * k + 1) * p1;
        long double ddp2 = ddp0 + (2 * k + 1) * dp1;
        p0 = p1; p1 = p2; dp0 = dp1; dp1 = dp2; ddp0 = ddp1; ddp1 = ddp2;
    }
    *P = p1; *dP = dp1; *d2P = ddp1;
}

/* Nodes xi[0..p] (ascending) and weights w[0..p] on [-1, 1].
 *   Gauss-Lobatto (kind 0): xi = -1, roots of P_p', +1; w = 2 / (p (p+1) P_p(xi)^2).
 *   Gauss-Legendre (kind 1): roots of P_{p+1}; w = 2 / ((1 - xi^2) P'_{p+1}(xi)^2).
 * Newton iteration in long double from Chebyshev-like first guesses. */
int orc_nodes(int p, int kind, double *xi, double *w)
{
    int n = p + 1;
    if (p < 1 || p > 30 || (kind != ORC_NODES_GLL && kind != ORC_NODES_GAUSS)) return 1;
    if (kind == ORC_NODES_GAUSS) {
        for (int j = 0; j < n; ++j) {
            long double x = -cosl(3.14159265358979323846264338327950288L * (j + 0.75L) / (n + 0.5L));
            for (int it = 0; it < 100; ++it) {
                long double P, dP, d2P;
                legendre_eval(n, x, &P, &dP, &d2P);
                long double dx = P / dP;
                x -= dx;
                if (fabsl(dx) < 1e-19L) break;
            }
            long double P, dP, d2P;
            legendre_eval(n, x, &P, &dP, &d2P);
            xi[j] = (double)x;
            w[j] = (double)(2.0L / ((1.0L - x * x) * dP * dP));
        }
    } else {
        xi[0] = -1.0; xi[p] = 1.0;
        for (int j = 1; j < p; ++j) {
            long double x = -cosl(3.14159265358979323846264338327950288L * j / p);
            for (int it = 0; it < 100; ++it) {
                long double P, dP, d2P;
                legendre_eval(p, x, &P, &dP, &d2P);
                long double dx = dP / d2P;
                x -= dx;
                if (fabsl(dx) < 1e-19L) break;
            }
            xi[j] = (double)x;
        }
        for (int j = 0; j < n; ++j) {
            long double P, dP, d2P;
            legendre_eval(p, (long double)xi[j], &P, &dP, &d2P);
            w[j] = (double)(2.0L / ((long double)p * (p + 1) * P * P));
        }
    }
    return 0;
}

/* Collocation derivative D[i*n + j] = l_j'(xi_i) by the barycentric formula
 * (Berrut & Trefethen 2004): lambda_j = 1 / prod_{k != j} (xi_j - xi_k),
 * D_ij = (lambda_j / lambda_i) / (xi_i - xi_j) for i != j,
 * D_ii = -sum_{j != i} D_ij (negative-sum trick: rows sum to zero). */
void orc_dmat(int n, const double *xi, double *D)
{
    long double lam[64];
    for (int j = 0; j < n; ++j) {
        long double prod = 1.0L;
        for (int k = 0; k < n; ++k)
            if (k != j) prod *= ((long double)xi[j] - xi[k]);
        lam[j] = 1.0L / prod;
    }
    for (int i = 0; i < n; ++i) {
        long double diag = 0.0L;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            long double dij = (lam[j] / lam[i]) / ((long double)xi[i] - xi[j]);
            D[i * n + j] = (double)dij;
            diag -= dij;
        }
        D[i * n + i] = (double)diag;
    }
}

/* The 1D operators one direction of Eq. 5 needs: nodes, weights, D and the
 * weighted derivative Q1 = diag(w) D (the "stiffness" factor). */
int orc_op1d(int p, int kind, double *xi, double *w, double *D, double *Q1)
{
    int n = p + 1;
    if (orc_nodes(p, kind, xi, w)) return 1;
    orc_dmat(n, xi, D);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
            Q1[a * n + b] = w[a] * D[a * n + b];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Tensor-product index helpers (x fastest).                                  */
/* ------------------------------------------------------------------------ */
static int ipow(int b, int e) { int r = 1; while (e-- > 0) r *= b; return r; }

static void node_to_multi(int i, int n, int d, int *a)
{
    for (int k = 0; k < d; ++k) { a[k] = i % n; i /= n; }
}

static int multi_to_node(const int *a, int n, int d)
{
    int i = 0;
    for (int k = d - 1; k >= 0; --k) i = i * n + a[k];
    return i;
}

/* Dense Q_m (n^d x n^d, row-major) by the Kronecker-product definition:
 * Q_m[i][j] = prod_k A_k[a_k(i)][a_k(j)], A_m = Q1, A_k = diag(w) (k != m).
 * This is the full operator of Eq. 5 whose Hadamard product Eq. 1 evaluates. */
int orc_qmat_dense(int d, int p, int kind, int m, double *Q)
{
    int n = p + 1, nn = ipow(n, d);
    double xi[64], w[64], D[64 * 64], Q1[64 * 64];
    if (d < 1 || d > 3 || m < 0 || m >= d) return 1;
    if (orc_op1d(p, kind, xi, w, D, Q1)) return 1;
    for (int i = 0; i < nn; ++i) {
        int ai[3]; node_to_multi(i, n, d, ai);
        for (int j = 0; j < nn; ++j) {
            int aj[3]; node_to_multi(j, n, d, aj);
            double v = 1.0;
            for (int k = 0; k < d; ++k) {
                if (k == m) v *= Q1[ai[k] * n + aj[k]];
                else v *= (ai[k] == aj[k]) ? w[ai[k]] : 0.0;
            }
            Q[(long)i * nn + j] = v;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Logarithmic mean {a, b}_ln = (a - b) / (ln a - ln b), {a, a}_ln = a.       */
/* Near a = b: series in u = ((a - b)/(a + b))^2,                           */
/* {a,b}_ln = (a + b) / (2 + 2u/3 + 2u^2/5 + 2u^3/7)  (Ranocha et al. 2021). */
/* ------------------------------------------------------------------------ */
double orc_logmean(double a, double b)
{
    double d = a - b, s = a + b;
    double u = (d * d) / (s * s);
    if (u < 1e-4)
        return s / (2.0 + u * (2.0 / 3.0 + u * (2.0 / 5.0 + u * (2.0 / 7.0))));
    return d / log(a / b);
}

/* Partial derivatives of {a, b}_ln.
 * Away from a = b: d/da = (1 - L/a) / ln(a/b).
 * Near a = b: L = s / P(u), P(u) = 2 sum_k u^k / (2k+1) (seven terms here),
 * u = t^2, t = (a-b)/(a+b); du/da = 4 t b / s^2, du/db = -4 t a / s^2, so
 * dL/da = 1/P - s P'(u) du/da / P^2. */
void orc_logmean_grad(double a, double b, double *dLda, double *dLdb)
{
    double d = a - b, s = a + b;
    double u = (d * d) / (s * s);
    if (u < 1e-4) {
        double t = d / s, P = 0.0, dP = 0.0;
        for (int k = 6; k >= 0; --k) P = P * u + 2.0 / (2 * k + 1);
        for (int k = 6; k >= 1; --k) dP = dP * u + 2.0 * k / (2 * k + 1);
        double dudA = 4.0 * t * b / (s * s);
        double dudB = -4.0 * t * a / (s * s);
        *dLda = 1.0 / P - s * dP * dudA / (P * P);
        *dLdb = 1.0 / P - s * dP * dudB / (P * P);
    } else {
        double lr = log(a / b);
        double L = d / lr;
        *dLda = (1.0 - L / a) / lr;
        *dLdb = (L / b - 1.0) / lr;
    }
}

/* ------------------------------------------------------------------------ */
/* Two-point fluxes contracted with a metric vector nv (d components):       */
/* F(u_i, u_j; nv) = sum_k fsharp_k(u_i, u_j) nv_k.  The residual passes     */
/* nv = Ja^m(i) + Ja^m(j) (= 2 avg(J dxi_m/dx)).                            */
/* ------------------------------------------------------------------------ */

/* Euler primitives from conservative variables; returns 0 if rho, p > 0. */
static int euler_prim(int d, const double *u, double *rho, double *v, double *p)
{
    double ke = 0.0;
    *rho = u[0];
    for (int k = 0; k < d; ++k) { v[k] = u[1 + k] / u[0]; ke += u[1 + k] * v[k]; }
    *p = (ORC_GAMMA - 1.0) * (u[d + 1] - 0.5 * ke);
    return (*rho > 0.0 && *p > 0.0) ? 0 : 2;
}

int orc_ec_flux(int d, int flux, const double *ui, const double *uj, const double *nv, double *F)
{
    if (flux == ORC_FLUX_BURGERS) {
        double a = ui[0], b = uj[0], S = 0.0;
        for (int k = 0; k < d; ++k) S += nv[k];
        F[0] = (a * a + a * b + b * b) / 6.0 * S;
        return 0;
    }
    double ri, vi[3], pi, rj, vj[3], pj;
    int st = euler_prim(d, ui, &ri, vi, &pi) | euler_prim(d, uj, &rj, vj, &pj);
    double rho_ln = orc_logmean(ri, rj);
    double beta_ln = orc_logmean(ri / pi, rj / pj);
    if (flux == ORC_FLUX_CHANDRASHEKAR) {
        double vn = 0.0, v2 = 0.0, p_t = (ri + rj) / (ri / pi + rj / pj);   /* {rho} / {beta} */
        for (int k = 0; k < d; ++k) {
            vn += 0.5 * (vi[k] + vj[k]) * nv[k];
            v2 += 0.5 * (vi[k] * vi[k] + vj[k] * vj[k]);
        }
        double f_rho = rho_ln * vn, fe = 0.0;
        F[0] = f_rho;
        for (int l = 0; l < d; ++l) {
            F[1 + l] = f_rho * 0.5 * (vi[l] + vj[l]) + p_t * nv[l];
            fe += 0.5 * (vi[l] + vj[l]) * F[1 + l];
        }
        F[d + 1] = f_rho * (1.0 / ((ORC_GAMMA - 1.0) * beta_ln) - 0.5 * v2) + fe;
        return st;
    }
    double vni = 0.0, vnj = 0.0, vivj = 0.0;
    for (int k = 0; k < d; ++k) { vni += vi[k] * nv[k]; vnj += vj[k] * nv[k]; vivj += vi[k] * vj[k]; }
    double f_rho = rho_ln * 0.5 * (vni + vnj);
    double p_avg = 0.5 * (pi + pj);
    F[0] = f_rho;
    for (int l = 0; l < d; ++l) F[1 + l] = f_rho * 0.5 * (vi[l] + vj[l]) + p_avg * nv[l];
    F[d + 1] = f_rho * (0.5 * vivj + 1.0 / ((ORC_GAMMA - 1.0) * beta_ln)) + 0.5 * (pi * vnj + pj * vni);
    return st;
}

/* Jacobian of the contracted two-point flux with respect to the conservative
 * state of its FIRST argument: J[a*nvar + b] = dF_a / du_i,b.
 * Chain rule: conservative -> (rho, v, p) -> flux, with the log-mean
 * derivatives above (beta = rho / p). */
int orc_ec_flux_jac1(int d, int flux, const double *ui, const double *uj, const double *nv, double *J)
{
    if (flux == ORC_FLUX_BURGERS) {
        double a = ui[0], b = uj[0], S = 0.0;
        for (int k = 0; k < d; ++k) S += nv[k];
        J[0] = (2.0 * a + b) / 6.0 * S;
        return 0;
    }
    int nvar = d + 2;
    double ri, vi[3], pi, rj, vj[3], pj;
    int st = euler_prim(d, ui, &ri, vi, &pi) | euler_prim(d, uj, &rj, vj, &pj);
    double bi = ri / pi, bj = rj / pj;
    double Lr = orc_logmean(ri, rj), Lb = orc_logmean(bi, bj);
    double dLr, dLr_unused, dLb, dLb_unused;
    orc_logmean_grad(ri, rj, &dLr, &dLr_unused);
    orc_logmean_grad(bi, bj, &dLb, &dLb_unused);
    double vni = 0.0, vnj = 0.0, vivj = 0.0;
    for (int k = 0; k < d; ++k) { vni += vi[k] * nv[k]; vnj += vj[k] * nv[k]; vivj += vi[k] * vj[k]; }
    double f_rho = Lr * 0.5 * (vni + vnj);
    double K = 0.5 * vivj + 1.0 / ((ORC_GAMMA - 1.0) * Lb);
    double dK_dLb = -1.0 / ((ORC_GAMMA - 1.0) * Lb * Lb);

    /* dF/dw with w = (rho_i, v_i[0..d-1], p_i); dFw[a][c], c in 0..d+1 */
    double dFw[5][5];
    memset(dFw, 0, sizeof dFw);
    double dfrho_drho = dLr * 0.5 * (vni + vnj);
    double dfrho_dv[3];
    for (int k = 0; k < d; ++k) dfrho_dv[k] = Lr * 0.5 * nv[k];
    double dK_drho = dK_dLb * dLb * (1.0 / pi);
    double dK_dp = dK_dLb * dLb * (-ri / (pi * pi));
    /* Chandrashekar's pressure average pt = (rho_i + rho_j) / (beta_i + beta_j)
     * and its derivatives (through rho_i directly and through beta_i) */
    int ch = flux == ORC_FLUX_CHANDRASHEKAR;
    double sb = bi + bj, pt = (ri + rj) / sb;
    double dpt_drho = 1.0 / sb - pt / sb * (1.0 / pi);
    double dpt_dp = pt / sb * (ri / (pi * pi));
    /* mass */
    dFw[0][0] = dfrho_drho;
    for (int k = 0; k < d; ++k) dFw[0][1 + k] = dfrho_dv[k];
    /* momentum */
    for (int l = 0; l < d; ++l) {
        double vavg = 0.5 * (vi[l] + vj[l]);
        dFw[1 + l][0] = dfrho_drho * vavg;
        for (int k = 0; k < d; ++k)
            dFw[1 + l][1 + k] = dfrho_dv[k] * vavg + (k == l ? 0.5 * f_rho : 0.0);
        if (ch) {
            dFw[1 + l][0] += dpt_drho * nv[l];
            dFw[1 + l][d + 1] = dpt_dp * nv[l];
        } else {
            dFw[1 + l][d + 1] = 0.5 * nv[l];
        }
    }
    /* energy: pressure work 1/2 (p_i v_j + p_j v_i).n (Ranocha) or
     * pt {v}.n (Chandrashekar) */
    double vnavg = 0.5 * (vni + vnj);
    dFw[d + 1][0] = dfrho_drho * K + f_rho * dK_drho + (ch ? dpt_drho * vnavg : 0.0);
    for (int k = 0; k < d; ++k)
        dFw[d + 1][1 + k] = dfrho_dv[k] * K + f_rho * 0.5 * vj[k] + 0.5 * (ch ? pt : pj) * nv[k];
    dFw[d + 1][d + 1] = f_rho * dK_dp + (ch ? dpt_dp * vnavg : 0.5 * vnj);

    /* dw/du: rho = u0; v_k = u_{1+k}/u0; p = (g-1)(E - |m|^2/(2 rho)) */
    double dwu[5][5];
    memset(dwu, 0, sizeof dwu);
    double v2 = 0.0;
    for (int k = 0; k < d; ++k) v2 += vi[k] * vi[k];
    dwu[0][0] = 1.0;
    for (int k = 0; k < d; ++k) { dwu[1 + k][0] = -vi[k] / ri; dwu[1 + k][1 + k] = 1.0 / ri; }
    dwu[d + 1][0] = (ORC_GAMMA - 1.0) * 0.5 * v2;
    for (int k = 0; k < d; ++k) dwu[d + 1][1 + k] = -(ORC_GAMMA - 1.0) * vi[k];
    dwu[d + 1][d + 1] = ORC_GAMMA - 1.0;

    for (int a = 0; a < nvar; ++a)
        for (int b = 0; b < nvar; ++b) {
            double s = 0.0;
            for (int c = 0; c < nvar; ++c) s += dFw[a][c] * dwu[c][b];
            J[a * nvar + b] = s;
        }
    (void)dLr_unused; (void)dLb_unused;
    return st;
}

static int check_args(int d, int p, int kind, int nvar, int flux)
{
    if (d < 2 || d > 3 || p < 1 || p > 8) return 1;
    if (kind != ORC_NODES_GLL && kind != ORC_NODES_GAUSS) return 1;
    if (flux == ORC_FLUX_BURGERS && nvar != 1) return 1;
    if ((flux == ORC_FLUX_EULER || flux == ORC_FLUX_CHANDRASHEKAR) && nvar != d + 2) return 1;
    if (flux != ORC_FLUX_BURGERS && flux != ORC_FLUX_EULER && flux != ORC_FLUX_CHANDRASHEKAR) return 1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Volume residual, sum-factorized (Eq. 3 with Eq. 5): for every direction m */
/* and node i only the n partners j on the m-line through i contribute,     */
/*   r_i += omega_m(i) Q1[a_m(i)][a_m(j)] F_m(u_i, u_j),                      */
/*   omega_m(i) = prod_{k != m} w[a_k(i)],                                  */
/* which is d n^{d+1} flux evaluations per element (Theorem 2.1).           */
/* ------------------------------------------------------------------------ */
int orc_volume_sf(int d, int p, int kind, int nvar, int flux, long n_elem,
                  const double *u, const double *Ja, double *r)
{
    if (check_args(d, p, kind, nvar, flux) || n_elem < 0) return 1;
    int n = p + 1, nn = ipow(n, d), st = 0;
    double xi[16], w[16], D[256], Q1[256];
    orc_op1d(p, kind, xi, w, D, Q1);
    for (long e = 0; e < n_elem; ++e) {
        const double *ue = u + e * nvar * nn;
        const double *Je = Ja + e * d * d * nn;
        double *re = r + e * nvar * nn;
        for (int q = 0; q < nvar * nn; ++q) re[q] = 0.0;
        for (int m = 0; m < d; ++m) {
            for (int i = 0; i < nn; ++i) {
                int ai[3]; node_to_multi(i, n, d, ai);
                double omega = 1.0;
                for (int k = 0; k < d; ++k) if (k != m) omega *= w[ai[k]];
                double ui[5];
                for (int v = 0; v < nvar; ++v) ui[v] = ue[v * nn + i];
                for (int b = 0; b < n; ++b) {
                    int aj[3]; memcpy(aj, ai, sizeof aj); aj[m] = b;
                    int j = multi_to_node(aj, n, d);
                    double uj[5], nv[3], F[5];
                    for (int v = 0; v < nvar; ++v) uj[v] = ue[v * nn + j];
                    for (int k = 0; k < d; ++k) nv[k] = Je[(m * d + k) * nn + i] + Je[(m * d + k) * nn + j];
                    st |= orc_ec_flux(d, flux, ui, uj, nv, F);
                    for (int v = 0; v < nvar; ++v) re[v * nn + i] += omega * Q1[ai[m] * n + b] * F[v];
                }
            }
        }
    }
    return st;
}

/* Sum of the absolute terms of the sum-factorized residual (Eq. 3 with     */
/* Eq. 5), S_i = sum_m sum_j |omega_m(i) Q1[a_m(i)][a_m(j)] F_m(u_i, u_j)|    */
/* per variable: the magnitude the residual cancels from.  Test             */
/* infrastructure: rounding errors of a floating-point evaluation of r_i    */
/* scale with S_i, not with |r_i|.                                          */
int orc_volume_absterms(int d, int p, int kind, int nvar, int flux, long n_elem,
                        const double *u, const double *Ja, double *S)
{
    if (check_args(d, p, kind, nvar, flux) || n_elem < 0) return 1;
    int n = p + 1, nn = ipow(n, d), st = 0;
    double xi[16], w[16], D[256], Q1[256];
    orc_op1d(p, kind, xi, w, D, Q1);
    for (long e = 0; e < n_elem; ++e) {
        const double *ue = u + e * nvar * nn;
        const double *Je = Ja + e * d * d * nn;
        double *se = S + e * nvar * nn;
        for (int q = 0; q < nvar * nn; ++q) se[q] = 0.0;
        for (int m = 0; m < d; ++m) {
            for (int i = 0; i < nn; ++i) {
                int ai[3]; node_to_multi(i, n, d, ai);
                double omega = 1.0;
                for (int k = 0; k < d; ++k) if (k != m) omega *= w[ai[k]];
                double ui[5];
                for (int v = 0; v < nvar; ++v) ui[v] = ue[v * nn + i];
                for (int b = 0; b < n; ++b) {
                    int aj[3]; memcpy(aj, ai, sizeof aj); aj[m] = b;
                    int j = multi_to_node(aj, n, d);
                    double uj[5], nv[3], F[5];
                    for (int v = 0; v < nvar; ++v) uj[v] = ue[v * nn + j];
                    for (int k = 0; k < d; ++k) nv[k] = Je[(m * d + k) * nn + i] + Je[(m * d + k) * nn + j];
                    st |= orc_ec_flux(d, flux, ui, uj, nv, F);
                    for (int v = 0; v < nvar; ++v) se[v * nn + i] += fabs(omega * Q1[ai[m] * n + b] * F[v]);
                }
            }
        }
    }
    return st;
}

/* Volume residual, dense (Eq. 1): the full n^d x n^d operators Q_m and the
 * two-point flux over ALL node pairs (i, j), r_i = sum_m sum_j Q_m[i][j] F_m(u_i, u_j).
 * O(n^{2d}) per element: the brute-force form the sum-factorized one replaces. */
int orc_volume_dense(int d, int p, int kind, int nvar, int flux, long n_elem,
                     const double *u, const double *Ja, double *r)
{
    if (check_args(d, p, kind, nvar, flux) || n_elem < 0) return 1;
    int n = p + 1, nn = ipow(n, d), st = 0;
    double *Q = (double *)malloc(sizeof(double) * (size_t)d * nn * nn);
    if (!Q) return 1;
    for (int m = 0; m < d; ++m) orc_qmat_dense(d, p, kind, m, Q + (size_t)m * nn * nn);
    for (long e = 0; e < n_elem; ++e) {
        const double *ue = u + e * nvar * nn;
        const double *Je = Ja + e * d * d * nn;
        double *re = r + e * nvar * nn;
        for (int q = 0; q < nvar * nn; ++q) re[q] = 0.0;
        for (int m = 0; m < d; ++m) {
            const double *Qm = Q + (size_t)m * nn * nn;
            for (int i = 0; i < nn; ++i) {
                double ui[5];
                for (int v = 0; v < nvar; ++v) ui[v] = ue[v * nn + i];
                for (int j = 0; j < nn; ++j) {
                    double uj[5], nv[3], F[5];
                    for (int v = 0; v < nvar; ++v) uj[v] = ue[v * nn + j];
                    for (int k = 0; k < d; ++k) nv[k] = Je[(m * d + k) * nn + i] + Je[(m * d + k) * nn + j];
                    st |= orc_ec_flux(d, flux, ui, uj, nv, F);
                    for (int v = 0; v < nvar; ++v) re[v * nn + i] += Qm[(size_t)i * nn + j] * F[v];
                }
            }
        }
    }
    free(Q);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Vector-Jacobian product g = (dr/du)^T lambda (Ja is held fixed).           */
/* From r_i = sum_m sum_j Q_m,ij F_m(u_i, u_j) and F_m symmetric in its two   */
/* states (nv is symmetric in i, j):                                        */
/*   g_l = sum_m sum_{j on the m-line of l} (Q_m,lj lambda_l + Q_m,jl lambda_j)^T d1F_m(u_l, u_j). */
/* ------------------------------------------------------------------------ */
int orc_vjp_sf(int d, int p, int kind, int nvar, int flux, long n_elem,
               const double *u, const double *Ja, const double *lam, double *g)
{
    if (check_args(d, p, kind, nvar, flux) || n_elem < 0) return 1;
    int n = p + 1, nn = ipow(n, d), st = 0;
    double xi[16], w[16], D[256], Q1[256];
    orc_op1d(p, kind, xi, w, D, Q1);
    for (long e = 0; e < n_elem; ++e) {
        const double *ue = u + e * nvar * nn;
        const double *le = lam + e * nvar * nn;
        const double *Je = Ja + e * d * d * nn;
        double *ge = g + e * nvar * nn;
        for (int q = 0; q < nvar * nn; ++q) ge[q] = 0.0;
        for (int m = 0; m < d; ++m) {
            for (int l = 0; l < nn; ++l) {
                int al[3]; node_to_multi(l, n, d, al);
                double omega = 1.0;   /* omega_m is the same for l and j */
                for (int k = 0; k < d; ++k) if (k != m) omega *= w[al[k]];
                double ul[5];
                for (int v = 0; v < nvar; ++v) ul[v] = ue[v * nn + l];
                for (int b = 0; b < n; ++b) {
                    int aj[3]; memcpy(aj, al, sizeof aj); aj[m] = b;
                    int j = multi_to_node(aj, n, d);
                    double uj[5], nv[3], J1[25], c[5];
                    for (int v = 0; v < nvar; ++v) uj[v] = ue[v * nn + j];
                    for (int k = 0; k < d; ++k) nv[k] = Je[(m * d + k) * nn + l] + Je[(m * d + k) * nn + j];
                    st |= orc_ec_flux_jac1(d, flux, ul, uj, nv, J1);
                    double Qlj = omega * Q1[al[m] * n + b], Qjl = omega * Q1[b * n + al[m]];
                    for (int v = 0; v < nvar; ++v) c[v] = Qlj * le[v * nn + l] + Qjl * le[v * nn + j];
                    for (int bb = 0; bb < nvar; ++bb) {
                        double s = 0.0;
                        for (int a = 0; a < nvar; ++a) s += c[a] * J1[a * nvar + bb];
                        ge[bb * nn + l] += s;
                    }
                }
            }
        }
    }
    return st;
}

/* Dense-form VJP: assemble the element Jacobian dr/du (nvar nn x nvar nn)
 * from the dense Eq. 1 form, dr_i/du_l = sum_m sum_j Q_m[i][j]
 * (delta_il d1F(u_i,u_j) + delta_jl d2F(u_i,u_j)), d2F(u_i,u_j) = d1F(u_j,u_i),
 * then g = (dr/du)^T lambda. */
int orc_vjp_dense(int d, int p, int kind, int nvar, int flux, long n_elem,
                  const double *u, const double *Ja, const double *lam, double *g)
{
    if (check_args(d, p, kind, nvar, flux) || n_elem < 0) return 1;
    int n = p + 1, nn = ipow(n, d), st = 0, N = nvar * nn;
    double *Q = (double *)malloc(sizeof(double) * (size_t)d * nn * nn);
    double *Jac = (double *)malloc(sizeof(double) * (size_t)N * N);
    if (!Q || !Jac) { free(Q); free(Jac); return 1; }
    for (int m = 0; m < d; ++m) orc_qmat_dense(d, p, kind, m, Q + (size_t)m * nn * nn);
    for (long e = 0; e < n_elem; ++e) {
        const double *ue = u + e * nvar * nn;
        const double *le = lam + e * nvar * nn;
        const double *Je = Ja + e * d * d * nn;
        double *ge = g + e * nvar * nn;
        memset(Jac, 0, sizeof(double) * (size_t)N * N);
        for (int m = 0; m < d; ++m) {
            const double *Qm = Q + (size_t)m * nn * nn;
            for (int i = 0; i < nn; ++i)
                for (int j = 0; j < nn; ++j) {
                    double qij = Qm[(size_t)i * nn + j];
                    if (qij == 0.0) continue;     /* exact zeros of the Kronecker product */
                    double ui[5], uj[5], nv[3], J1[25], J2[25];
                    for (int v = 0; v < nvar; ++v) { ui[v] = ue[v * nn + i]; uj[v] = ue[v * nn + j]; }
                    for (int k = 0; k < d; ++k) nv[k] = Je[(m * d + k) * nn + i] + Je[(m * d + k) * nn + j];
                    st |= orc_ec_flux_jac1(d, flux, ui, uj, nv, J1);
                    st |= orc_ec_flux_jac1(d, flux, uj, ui, nv, J2);
                    for (int a = 0; a < nvar; ++a)
                        for (int b = 0; b < nvar; ++b) {
                            /* row (a, i); columns (b, i) and (b, j) */
                            Jac[(size_t)(a * nn + i) * N + (b * nn + i)] += qij * J1[a * nvar + b];
                            Jac[(size_t)(a * nn + i) * N + (b * nn + j)] += qij * J2[a * nvar + b];
                        }
                }
        }
        for (int col = 0; col < N; ++col) {
            double s = 0.0;
            for (int row = 0; row < N; ++row) s += Jac[(size_t)row * N + col] * le[row];
            ge[col] = s;
        }
    }
    free(Q); free(Jac);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Mesh and metric terms for the free-stream and pressure-equilibrium checks. */
/* Elements of [0,1]^d, N per direction (element e = ex + N ey + N^2 ez),    */
/* nodes x_k = (e_k + (xi + 1)/2) / N, then every axis is shifted by the same */
/* scalar amp * prod_l sin(pi x_l).  Metrics from the degree-p interpolant: */
/*   2D: Ja^0 = (y_eta, -x_eta), Ja^1 = (-y_xi, x_xi);                       */
/*   3D: conservative curl form (Kopriva 2006),                              */
/*       Ja^i_n = -[curl_xi (X_l grad_xi X_m)]_i,  (n, m, l) cyclic,         */
/* which satisfy sum_m D_m Ja^m_k = 0 to round-off.                          */
/* x [e][k][i], Ja [e][m][k][i].                                             */
/* ------------------------------------------------------------------------ */
static void deriv_dir(int d, int n, const double *D, int dir, const double *f, double *out)
{
    int nn = ipow(n, d);
    for (int i = 0; i < nn; ++i) {
        int a[3]; node_to_multi(i, n, d, a);
        double s = 0.0;
        for (int b = 0; b < n; ++b) {
            int aj[3]; memcpy(aj, a, sizeof aj); aj[dir] = b;
            s += D[a[dir] * n + b] * f[multi_to_node(aj, n, d)];
        }
        out[i] = s;
    }
}

int orc_mesh(int d, int p, int kind, int N, double amp, double *x, double *Ja)
{
    if (d < 2 || d > 3 || N < 1) return 1;
    int n = p + 1, nn = ipow(n, d);
    double xi[16], w[16], D[256], Q1[256];
    if (orc_op1d(p, kind, xi, w, D, Q1)) return 1;
    const double pi = 3.14159265358979323846;
    long n_elem = 1; for (int k = 0; k < d; ++k) n_elem *= N;
    double *dX = (double *)malloc(sizeof(double) * 9 * nn);   /* dX[(k*3 + j)*nn + i] = d x_k / d xi_j */
    double *V = (double *)malloc(sizeof(double) * 3 * nn);
    double *cV = (double *)malloc(sizeof(double) * nn);
    double *tmp = (double *)malloc(sizeof(double) * nn);
    for (long e = 0; e < n_elem; ++e) {
        int ee[3]; long t = e;
        for (int k = 0; k < d; ++k) { ee[k] = (int)(t % N); t /= N; }
        double *xe = x + e * d * nn;
        double *Je = Ja + e * d * d * nn;
        for (int i = 0; i < nn; ++i) {
            int a[3]; node_to_multi(i, n, d, a);
            double x0[3], s = amp;
            for (int k = 0; k < d; ++k) { x0[k] = (ee[k] + 0.5 * (xi[a[k]] + 1.0)) / N; s *= sin(pi * x0[k]); }
            for (int k = 0; k < d; ++k) xe[k * nn + i] = x0[k] + s;
        }
        for (int k = 0; k < d; ++k)
            for (int j = 0; j < d; ++j) deriv_dir(d, n, D, j, xe + k * nn, dX + (k * 3 + j) * nn);
        if (d == 2) {
            for (int i = 0; i < nn; ++i) {
                Je[(0 * 2 + 0) * nn + i] = dX[(1 * 3 + 1) * nn + i];    /*  y_eta */
                Je[(0 * 2 + 1) * nn + i] = -dX[(0 * 3 + 1) * nn + i];   /* -x_eta */
                Je[(1 * 2 + 0) * nn + i] = -dX[(1 * 3 + 0) * nn + i];   /* -y_xi  */
                Je[(1 * 2 + 1) * nn + i] = dX[(0 * 3 + 0) * nn + i];    /*  x_xi  */
            }
        } else {
            for (int nc = 0; nc < 3; ++nc) {
                int mc = (nc + 1) % 3, lc = (nc + 2) % 3;
                /* V_j = X_l * d X_m / d xi_j */
                for (int j = 0; j < 3; ++j)
                    for (int i = 0; i < nn; ++i)
                        V[j * nn + i] = xe[lc * nn + i] * dX[(mc * 3 + j) * nn + i];
                for (int ic = 0; ic < 3; ++ic) {
                    int jc = (ic + 1) % 3, kc = (ic + 2) % 3;
                    /* (curl V)_i = D_j V_k - D_k V_j */
                    deriv_dir(3, n, D, jc, V + kc * nn, cV);
                    deriv_dir(3, n, D, kc, V + jc * nn, tmp);
                    for (int i = 0; i < nn; ++i) Je[(ic * 3 + nc) * nn + i] = -(cV[i] - tmp[i]);
                }
            }
        }
    }
    free(dX); free(V); free(cV); free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The generic Hadamard workload of the paper's Section 3 timing experiment: */
/* y = (sum_j dl/dxi_j o C) 1 with C = c c^T in 3D, D_j = I x .. x D x .. x I */
/* (unweighted).  Dense: loop over all n^6 entries of each D_j.  Sum-        */
/* factorized (Eq. 3): only the n^4 entries on grid lines.                   */
/* ------------------------------------------------------------------------ */
static void fig1_ops(int p, double *D)
{
    double xi[64], w[64];
    orc_nodes(p, ORC_NODES_GLL, xi, w);
    orc_dmat(p + 1, xi, D);
}

int orc_fig1_dense(int p, const double *c, double *y)
{
    int n = p + 1, nn = n * n * n;
    double D[64 * 64];
    if (p < 1 || p > 30) return 1;
    fig1_ops(p, D);
    for (int i = 0; i < nn; ++i) y[i] = 0.0;
    for (int m = 0; m < 3; ++m)
        for (int i = 0; i < nn; ++i) {
            int ai[3]; node_to_multi(i, n, 3, ai);
            double s = 0.0;
            for (int j = 0; j < nn; ++j) {
                int aj[3]; node_to_multi(j, n, 3, aj);
                double q = 1.0;
                for (int k = 0; k < 3; ++k)
                    q *= (k == m) ? D[ai[k] * n + aj[k]] : (ai[k] == aj[k] ? 1.0 : 0.0);
                s += q * (c[i] * c[j]);
            }
            y[i] += s;
        }
    return 0;
}

int orc_fig1_sf(int p, const double *c, double *y)
{
    int n = p + 1, nn = n * n * n;
    double D[64 * 64];
    if (p < 1 || p > 30) return 1;
    fig1_ops(p, D);
    for (int i = 0; i < nn; ++i) y[i] = 0.0;
    for (int m = 0; m < 3; ++m)
        for (int i = 0; i < nn; ++i) {
            int ai[3]; node_to_multi(i, n, 3, ai);
            double s = 0.0;
            for (int b = 0; b < n; ++b) {
                int aj[3]; memcpy(aj, ai, sizeof aj); aj[m] = b;
                int j = multi_to_node(aj, n, 3);
                s += D[ai[m] * n + b] * (c[i] * c[j]);
            }
            y[i] += s;
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Modal / uncollocated path (Section 2, Eq. 4 and the theorem after it).    */
/* The solution lives in a tensor-product basis chi (n = p + 1 functions per */
/* direction) and is integrated on the volume cubature nodes xi of `kind`.   */
/* With V = chi(xi) (n^d x n^d, V[i][j] = prod_m V1[a_m(i)][b_m(j)]):         */
/*   u_v  = V u_hat                     (nodal values on the cubature)       */
/*   w_v  = w(u_v)                      (entropy variables)                  */
/*   w~   = V Pi w_v,  Pi = M^{-1} V^T W,  M = V^T W V   (entropy projection) */
/*   u~   = u(w~)                       (projected conservative state)       */
/*   r_v  = sum_m (Q_m o F_m(u~)) 1     (the collocated volume term, Eq. 3)  */
/*   r_hat = V^T r_v                    (tested against chi)                 */
/* Dense matrices throughout: the basis transform is written as the full     */
/* Kronecker product, not sum-factorized.                                    */
/* ------------------------------------------------------------------------ */
#define ORC_BASIS_LEGENDRE 0        /* orthonormal Legendre, sqrt((2k+1)/2) P_k */
#define ORC_BASIS_LAGRANGE_GLL 1    /* Lagrange on the p+1 Gauss-Lobatto nodes   */
#define ORC_BASIS_LAGRANGE_GAUSS 2  /* Lagrange on the p+1 Gauss-Legendre nodes  */

/* 1D basis on the cubature nodes of `kind`: V1[a*n + k] = chi_k(xi_a). */
int orc_basis_1d(int p, int kind, int basis, double *V1)
{
    int n = p + 1;
    double xi[16], w[16];
    if (p < 1 || p > 15 || orc_nodes(p, kind, xi, w)) return 1;
    if (basis == ORC_BASIS_LEGENDRE) {
        for (int a = 0; a < n; ++a)
            for (int k = 0; k < n; ++k) {
                long double P, dP, d2P;
                legendre_eval(k, (long double)xi[a], &P, &dP, &d2P);
                V1[a * n + k] = (double)(sqrtl((2.0L * k + 1.0L) / 2.0L) * P);
            }
        return 0;
    }
    if (basis != ORC_BASIS_LAGRANGE_GLL && basis != ORC_BASIS_LAGRANGE_GAUSS) return 1;
    double s[16], sw[16];
    orc_nodes(p, basis == ORC_BASIS_LAGRANGE_GLL ? ORC_NODES_GLL : ORC_NODES_GAUSS, s, sw);
    for (int a = 0; a < n; ++a)
        for (int k = 0; k < n; ++k) {
            long double l = 1.0L;
            for (int j = 0; j < n; ++j)
                if (j != k) l *= ((long double)xi[a] - s[j]) / ((long double)s[k] - s[j]);
            V1[a * n + k] = (double)l;
        }
    return 0;
}

/* Entropy variables w(u) of the flux's entropy: Burgers U = u^2/2 (w = u);
 * Euler U = -rho s/(g-1), s = ln p - g ln rho:
 *   w = ((g - s)/(g-1) - rho|v|^2/(2p), rho v/p, -rho/p). */
static int entropy_w(int d, int flux, const double *u, double *w)
{
    if (flux == ORC_FLUX_BURGERS) { w[0] = u[0]; return 0; }
    double rho, v[3], p;
    int st = euler_prim(d, u, &rho, v, &p);
    double v2 = 0.0;
    for (int k = 0; k < d; ++k) v2 += v[k] * v[k];
    double s = log(p) - ORC_GAMMA * log(rho);
    w[0] = (ORC_GAMMA - s) / (ORC_GAMMA - 1.0) - rho * v2 / (2.0 * p);
    for (int k = 0; k < d; ++k) w[1 + k] = rho * v[k] / p;
    w[d + 1] = -rho / p;
    return st;
}

/* Inverse map u(w): beta = -w_E = rho/p, v = w_m/beta,
 * s = g - (g-1)(w_0 + beta|v|^2/2), and from s = (1-g) ln rho - ln beta:
 * rho = exp(-(s + ln beta)/(g-1)), p = rho/beta. */
static int entropy_u(int d, int flux, const double *w, double *u)
{
    if (flux == ORC_FLUX_BURGERS) { u[0] = w[0]; return 0; }
    double beta = -w[d + 1];
    if (!(beta > 0.0)) return 2;
    double v[3], v2 = 0.0;
    for (int k = 0; k < d; ++k) { v[k] = w[1 + k] / beta; v2 += v[k] * v[k]; }
    double s = ORC_GAMMA - (ORC_GAMMA - 1.0) * (w[0] + 0.5 * beta * v2);
    double rho = exp(-(s + log(beta)) / (ORC_GAMMA - 1.0));
    double p = rho / beta;
    u[0] = rho;
    for (int k = 0; k < d; ++k) u[1 + k] = rho * v[k];
    u[d + 1] = p / (ORC_GAMMA - 1.0) + 0.5 * rho * v2;
    return 0;
}

/* Solve A x = b (A: m x m row-major, overwritten) by Gaussian elimination
 * with partial pivoting; nrhs right-hand sides stored as columns of B
 * (m x nrhs, row-major, overwritten by the solutions). */
static int dense_solve(int m, double *A, int nrhs, double *B)
{
    for (int c = 0; c < m; ++c) {
        int piv = c;
        for (int r = c + 1; r < m; ++r)
            if (fabs(A[(size_t)r * m + c]) > fabs(A[(size_t)piv * m + c])) piv = r;
        if (A[(size_t)piv * m + c] == 0.0) return 1;
        if (piv != c) {
            for (int k = 0; k < m; ++k) { double t = A[(size_t)c * m + k]; A[(size_t)c * m + k] = A[(size_t)piv * m + k]; A[(size_t)piv * m + k] = t; }
            for (int k = 0; k < nrhs; ++k) { double t = B[(size_t)c * nrhs + k]; B[(size_t)c * nrhs + k] = B[(size_t)piv * nrhs + k]; B[(size_t)piv * nrhs + k] = t; }
        }
        for (int r = c + 1; r < m; ++r) {
            double f = A[(size_t)r * m + c] / A[(size_t)c * m + c];
            if (f == 0.0) continue;
            for (int k = c; k < m; ++k) A[(size_t)r * m + k] -= f * A[(size_t)c * m + k];
            for (int k = 0; k < nrhs; ++k) B[(size_t)r * nrhs + k] -= f * B[(size_t)c * nrhs + k];
        }
    }
    for (int c = m - 1; c >= 0; --c)
        for (int k = 0; k < nrhs; ++k) {
            double s = B[(size_t)c * nrhs + k];
            for (int j = c + 1; j < m; ++j) s -= A[(size_t)c * m + j] * B[(size_t)j * nrhs + k];
            B[(size_t)c * nrhs + k] = s / A[(size_t)c * m + c];
        }
    return 0;
}

/* The n^d x n^d Kronecker matrix V[i][j] = prod_m V1[a_m(i)][b_m(j)] and the
 * cubature weights W_d[i] = prod_m w[a_m(i)]. */
static void modal_dense(int d, int p, int kind, const double *V1, double *V, double *Wd)
{
    int n = p + 1, nn = ipow(n, d);
    double xi[16], w[16];
    orc_nodes(p, kind, xi, w);
    for (int i = 0; i < nn; ++i) {
        int ai[3]; node_to_multi(i, n, d, ai);
        Wd[i] = 1.0;
        for (int m = 0; m < d; ++m) Wd[i] *= w[ai[m]];
        for (int j = 0; j < nn; ++j) {
            int bj[3]; node_to_multi(j, n, d, bj);
            double q = 1.0;
            for (int m = 0; m < d; ++m) q *= V1[ai[m] * n + bj[m]];
            V[(size_t)i * nn + j] = q;
        }
    }
}

/* Nodal states of the modal path: u_v = V u_hat and the entropy-projected
 * u~ = u(V Pi w(u_v)), both [e][var][i]. */
int orc_modal_states(int d, int p, int kind, int basis, int nvar, int flux, long n_elem,
                     const double *uhat, double *u_nodes, double *u_proj)
{
    if (check_args(d, p, kind, nvar, flux) || n_elem < 0) return 1;
    int n = p + 1, nn = ipow(n, d), st = 0;
    double V1[256];
    if (orc_basis_1d(p, kind, basis, V1)) return 1;
    double *V = (double *)malloc(sizeof(double) * (size_t)nn * nn);
    double *M = (double *)malloc(sizeof(double) * (size_t)nn * nn);
    double *Wd = (double *)malloc(sizeof(double) * nn);
    double *rhs = (double *)malloc(sizeof(double) * (size_t)nn * nvar);
    double *wv = (double *)malloc(sizeof(double) * (size_t)nn * nvar);
    if (!V || !M || !Wd || !rhs || !wv) { free(V); free(M); free(Wd); free(rhs); free(wv); return 1; }
    modal_dense(d, p, kind, V1, V, Wd);
    for (long e = 0; e < n_elem; ++e) {
        const double *ue = uhat + e * nvar * nn;
        double *uv = u_nodes + e * nvar * nn, *up = u_proj + e * nvar * nn;
        /* u_v = V u_hat */
        for (int v = 0; v < nvar; ++v)
            for (int i = 0; i < nn; ++i) {
                double s = 0.0;
                for (int j = 0; j < nn; ++j) s += V[(size_t)i * nn + j] * ue[v * nn + j];
                uv[v * nn + i] = s;
            }
        /* w_v = w(u_v) per node, stored [i][var] */
        for (int i = 0; i < nn; ++i) {
            double ui[5], wi[5];
            for (int v = 0; v < nvar; ++v) ui[v] = uv[v * nn + i];
            st |= entropy_w(d, flux, ui, wi);
            for (int v = 0; v < nvar; ++v) wv[(size_t)i * nvar + v] = wi[v];
        }
        /* M = V^T W V, rhs = V^T W w_v; solve M w_hat = rhs */
        for (int k = 0; k < nn; ++k) {
            for (int l = 0; l < nn; ++l) {
                double s = 0.0;
                for (int i = 0; i < nn; ++i) s += V[(size_t)i * nn + k] * Wd[i] * V[(size_t)i * nn + l];
                M[(size_t)k * nn + l] = s;
            }
            for (int v = 0; v < nvar; ++v) {
                double s = 0.0;
                for (int i = 0; i < nn; ++i) s += V[(size_t)i * nn + k] * Wd[i] * wv[(size_t)i * nvar + v];
                rhs[(size_t)k * nvar + v] = s;
            }
        }
        if (dense_solve(nn, M, nvar, rhs)) st |= 1;
        /* w~ = V w_hat, u~ = u(w~) */
        for (int i = 0; i < nn; ++i) {
            double wi[5], ui[5];
            for (int v = 0; v < nvar; ++v) {
                double s = 0.0;
                for (int k = 0; k < nn; ++k) s += V[(size_t)i * nn + k] * rhs[(size_t)k * nvar + v];
                wi[v] = s;
            }
            st |= entropy_u(d, flux, wi, ui);
            for (int v = 0; v < nvar; ++v) up[v * nn + i] = ui[v];
        }
    }
    free(V); free(M); free(Wd); free(rhs); free(wv);
    return st;
}

/* The modal volume residual r_hat = V^T r_v(u~) of the path above; with
 * project == 0 the flux takes u_v itself (the projection is the identity in
 * exact arithmetic whenever V is square, which the tests pin; skipping it
 * removes its round-off, about 1e-14 relative in u~, from the reference). */
int orc_volume_modal(int d, int p, int kind, int basis, int nvar, int flux, int project, long n_elem,
                     const double *uhat, const double *Ja, double *rhat)
{
    if (check_args(d, p, kind, nvar, flux) || n_elem < 0) return 1;
    int n = p + 1, nn = ipow(n, d), st;
    size_t tot = (size_t)n_elem * nvar * nn;
    double *uv = (double *)malloc(sizeof(double) * (tot ? tot : 1));
    double *up = (double *)malloc(sizeof(double) * (tot ? tot : 1));
    double *rv = (double *)malloc(sizeof(double) * (tot ? tot : 1));
    double *V = (double *)malloc(sizeof(double) * (size_t)nn * nn);
    double *Wd = (double *)malloc(sizeof(double) * nn);
    double V1[256];
    if (!uv || !up || !rv || !V || !Wd || orc_basis_1d(p, kind, basis, V1)) {
        free(uv); free(up); free(rv); free(V); free(Wd); return 1;
    }
    st = orc_modal_states(d, p, kind, basis, nvar, flux, n_elem, uhat, uv, up);
    st |= orc_volume_sf(d, p, kind, nvar, flux, n_elem, project ? up : uv, Ja, rv);
    modal_dense(d, p, kind, V1, V, Wd);
    for (long e = 0; e < n_elem; ++e)
        for (int v = 0; v < nvar; ++v)
            for (int k = 0; k < nn; ++k) {
                double s = 0.0;
                for (int i = 0; i < nn; ++i) s += V[(size_t)i * nn + k] * rv[(e * nvar + v) * nn + i];
                rhat[(e * nvar + v) * nn + k] = s;
            }
    free(uv); free(up); free(rv); free(V); free(Wd);
    return st;
}

/* Exported for the tests: entropy variables of one state and the inverse. */
int orc_entropy_vars(int d, int flux, const double *u, double *w) { return entropy_w(d, flux, u, w); }
int orc_entropy_state(int d, int flux, const double *w, double *u) { return entropy_u(d, flux, w, u); }

/* VJP of the modal residual (Ja fixed): from r_hat = V^T r_v(V u_hat) (the
 * projection being the identity map for square V, its derivative is the
 * identity too), g_hat = V^T J_v^T V lambda_hat with J_v = dr_v/du_v at
 * u_v = V u_hat: lambda_v = V lambda_hat, the nodal VJP, then V^T.  Dense
 * Kronecker transforms. */
int orc_vjp_modal(int d, int p, int kind, int basis, int nvar, int flux, long n_elem,
                  const double *uhat, const double *Ja, const double *lamhat, double *ghat)
{
    if (check_args(d, p, kind, nvar, flux) || n_elem < 0) return 1;
    int n = p + 1, nn = ipow(n, d), st = 0;
    size_t tot = (size_t)n_elem * nvar * nn;
    double V1[256];
    double *V = (double *)malloc(sizeof(double) * (size_t)nn * nn);
    double *Wd = (double *)malloc(sizeof(double) * nn);
    double *uv = (double *)malloc(sizeof(double) * (tot ? tot : 1));
    double *lv = (double *)malloc(sizeof(double) * (tot ? tot : 1));
    double *gv = (double *)malloc(sizeof(double) * (tot ? tot : 1));
    if (!V || !Wd || !uv || !lv || !gv || orc_basis_1d(p, kind, basis, V1)) {
        free(V); free(Wd); free(uv); free(lv); free(gv); return 1;
    }
    modal_dense(d, p, kind, V1, V, Wd);
    for (long e = 0; e < n_elem; ++e)
        for (int v = 0; v < nvar; ++v)
            for (int i = 0; i < nn; ++i) {
                double su = 0.0, sl = 0.0;
                for (int k = 0; k < nn; ++k) {
                    su += V[(size_t)i * nn + k] * uhat[(e * nvar + v) * nn + k];
                    sl += V[(size_t)i * nn + k] * lamhat[(e * nvar + v) * nn + k];
                }
                uv[(e * nvar + v) * nn + i] = su;
                lv[(e * nvar + v) * nn + i] = sl;
            }
    st = orc_vjp_sf(d, p, kind, nvar, flux, n_elem, uv, Ja, lv, gv);
    for (long e = 0; e < n_elem; ++e)
        for (int v = 0; v < nvar; ++v)
            for (int k = 0; k < nn; ++k) {
                double s = 0.0;
                for (int i = 0; i < nn; ++i) s += V[(size_t)i * nn + k] * gv[(e * nvar + v) * nn + i];
                ghat[(e * nvar + v) * nn + k] = s;
            }
    free(V); free(Wd); free(uv); free(lv); free(gv);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Surface Hadamard product of one element (Remark 1; the theorem's operator */
/* with alpha = 0 on the facet cubature; the surface coupling of Chan's     */
/* hybridised SBP form).  Face (m, side), side 0 at xi_m = -1, side 1 at    */
/* +1; facet cubature = the tensor product of the 1D nodes in the other    */
/* directions (lower axis fastest), n^{d-1} nodes f with weights           */
/* w_f = prod_{k != m} w[b_k(f)].  With the interpolation E = e (x) I (x) I */
/* (e in position m, e[b] = l_b(-1 or +1)) and a face state u~_f and face  */
/* normal nJ_f supplied by the caller, the dense Hadamard product          */
/*   H[f][j] = w_f E[f][j] fsharp(u~_f, u_j) . nJ_f                       */
/* gives the volume vector r_vol[j] = sum_{faces} sum_f H[f][j] and the    */
/* face vector r_face[f] = sum_j H[f][j].  Dense: every (f, j) pair, E from */
/* its Kronecker definition.                                                */
/* Layouts: u[e][var][i]; u_face[e][face][var][f]; nJ[e][face][k][f];       */
/* r_vol like u; r_face like u_face; face = 2 m + side.                    */
/* ------------------------------------------------------------------------ */
int orc_surface_dense(int d, int p, int kind, int nvar, int flux, long n_elem, const double *u,
                      const double *u_face, const double *nJ, double *r_vol, double *r_face)
{
    if (check_args(d, p, kind, nvar, flux) || n_elem < 0) return 1;
    int n = p + 1, nn = ipow(n, d), nf = ipow(n, d - 1), st = 0;
    double xi[16], w[16], e[2][16];
    orc_nodes(p, kind, xi, w);
    for (int side = 0; side < 2; ++side) {
        double x = side ? 1.0 : -1.0;
        for (int b = 0; b < n; ++b) {
            long double l = 1.0L;
            for (int j = 0; j < n; ++j)
                if (j != b) l *= ((long double)x - xi[j]) / ((long double)xi[b] - xi[j]);
            e[side][b] = (double)l;
        }
    }
    for (long el = 0; el < n_elem; ++el) {
        const double *ue = u + el * nvar * nn;
        double *rv = r_vol + el * nvar * nn;
        for (int q = 0; q < nvar * nn; ++q) rv[q] = 0.0;
        for (int m = 0; m < d; ++m)
            for (int side = 0; side < 2; ++side) {
                int face = 2 * m + side;
                const double *uf = u_face + (el * 2 * d + face) * nvar * nf;
                const double *nf_ = nJ + (el * 2 * d + face) * d * nf;
                double *rf = r_face + (el * 2 * d + face) * nvar * nf;
                for (int q = 0; q < nvar * nf; ++q) rf[q] = 0.0;
                for (int f = 0; f < nf; ++f) {
                    int bf[3]; node_to_multi(f, n, d - 1, bf);   /* the other directions, lower first */
                    double wf = 1.0;
                    for (int k = 0; k < d - 1; ++k) wf *= w[bf[k]];
                    double ufv[5], nv[3];
                    for (int v = 0; v < nvar; ++v) ufv[v] = uf[v * nf + f];
                    for (int k = 0; k < d; ++k) nv[k] = nf_[k * nf + f];
                    for (int j = 0; j < nn; ++j) {
                        int aj[3]; node_to_multi(j, n, d, aj);
                        /* E[f][j] = e[a_m(j)] * prod over the other axes of delta */
                        double E = e[side][aj[m]];
                        for (int k = 0, t = 0; k < d; ++k) {
                            if (k == m) continue;
                            if (aj[k] != bf[t]) E = 0.0;
                            ++t;
                        }
                        double uj[5], F[5];
                        for (int v = 0; v < nvar; ++v) uj[v] = ue[v * nn + j];
                        st |= orc_ec_flux(d, flux, ufv, uj, nv, F);
                        for (int v = 0; v < nvar; ++v) {
                            double h = wf * E * F[v];
                            rv[v * nn + j] += h;
                            rf[v * nf + f] += h;
                        }
                    }
                }
            }
    }
    return st;
}

/* ------------------------------------------------------------------------ */
/* Reverse mode of the surface Hadamard product above (derived from Remark  */
/* 1's operator; no paper counterpart).  For cotangents lam_vol (like       */
/* r_vol) and lam_face (like r_face), the scalar                            */
/*   L = sum lam_vol . r_vol + sum lam_face . r_face                         */
/*     = sum_{faces} sum_f sum_j w_f E[f][j] sum_v c_v(f, j) F_v(u~_f, u_j),  */
/* with c_v(f, j) = lam_vol[v][j] + lam_face[v][f], has the gradients        */
/*   g_u[b][j]    += w_f E[f][j] sum_v c_v dF_v/du_j[b]                        */
/*   g_face[b][f] += w_f E[f][j] sum_v c_v dF_v/du~_f[b]                       */
/* over every (face, f, j).  dF/du~_f is the flux Jacobian in its first      */
/* argument (orc_ec_flux_jac1); f# is symmetric, so dF/du_j(u~_f, u_j) is    */
/* the first-argument Jacobian at (u_j, u~_f).  The normals nJ are geometry  */
/* and get no gradient.  Dense: every (f, j) pair, E from its Kronecker      */
/* definition, as in orc_surface_dense.  Layouts: g_u like u, g_face like    */
/* u_face.                                                                   */
/* ------------------------------------------------------------------------ */
int orc_surface_vjp_dense(int d, int p, int kind, int nvar, int flux, long n_elem, const double *u,
                          const double *u_face, const double *nJ, const double *lam_vol,
                          const double *lam_face, double *g_u, double *g_face)
{
    if (check_args(d, p, kind, nvar, flux) || n_elem < 0) return 1;
    int n = p + 1, nn = ipow(n, d), nf = ipow(n, d - 1), st = 0;
    double xi[16], w[16], e[2][16];
    orc_nodes(p, kind, xi, w);
    for (int side = 0; side < 2; ++side) {
        double x = side ? 1.0 : -1.0;
        for (int b = 0; b < n; ++b) {
            long double l = 1.0L;
            for (int j = 0; j < n; ++j)
                if (j != b) l *= ((long double)x - xi[j]) / ((long double)xi[b] - xi[j]);
            e[side][b] = (double)l;
        }
    }
    for (long el = 0; el < n_elem; ++el) {
        const double *ue = u + el * nvar * nn;
        const double *lv = lam_vol + el * nvar * nn;
        double *gu = g_u + el * nvar * nn;
        for (int q = 0; q < nvar * nn; ++q) gu[q] = 0.0;
        for (int m = 0; m < d; ++m)
            for (int side = 0; side < 2; ++side) {
                int face = 2 * m + side;
                const double *uf = u_face + (el * 2 * d + face) * nvar * nf;
                const double *nf_ = nJ + (el * 2 * d + face) * d * nf;
                const double *lf = lam_face + (el * 2 * d + face) * nvar * nf;
                double *gf = g_face + (el * 2 * d + face) * nvar * nf;
                for (int q = 0; q < nvar * nf; ++q) gf[q] = 0.0;
                for (int f = 0; f < nf; ++f) {
                    int bf[3]; node_to_multi(f, n, d - 1, bf);
                    double wf = 1.0;
                    for (int k = 0; k < d - 1; ++k) wf *= w[bf[k]];
                    double ufv[5], nv[3];
                    for (int v = 0; v < nvar; ++v) ufv[v] = uf[v * nf + f];
                    for (int k = 0; k < d; ++k) nv[k] = nf_[k * nf + f];
                    for (int j = 0; j < nn; ++j) {
                        int aj[3]; node_to_multi(j, n, d, aj);
                        double E = e[side][aj[m]];
                        for (int k = 0, t = 0; k < d; ++k) {
                            if (k == m) continue;
                            if (aj[k] != bf[t]) E = 0.0;
                            ++t;
                        }
                        double uj[5], c[5], Jf[25], Jj[25];
                        for (int v = 0; v < nvar; ++v) {
                            uj[v] = ue[v * nn + j];
                            c[v] = wf * E * (lv[v * nn + j] + lf[v * nf + f]);
                        }
                        st |= orc_ec_flux_jac1(d, flux, ufv, uj, nv, Jf);   /* d F / d u~_f */
                        st |= orc_ec_flux_jac1(d, flux, uj, ufv, nv, Jj);   /* d F / d u_j  */
                        for (int b = 0; b < nvar; ++b) {
                            double sj = 0.0, sf = 0.0;
                            for (int a = 0; a < nvar; ++a) {
                                sj += c[a] * Jj[a * nvar + b];
                                sf += c[a] * Jf[a * nvar + b];
                            }
                            gu[b * nn + j] += sj;
                            gf[b * nf + f] += sf;
                        }
                    }
                }
            }
    }
    return st;
}
