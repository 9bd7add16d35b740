"""Pins of the oracle's volume residual r = sum_m (Q_m o F_m) 1.

  P1  sum-factorized (Eq. 3) == dense brute force (Eq. 1) on whole small meshes;
  P4  Burgers on an affine mesh == the split-form closed form built from plain
      numpy.kron matrix-vector products (no flux loop involved);
  P5  free stream: a constant state on the warped mesh gives r = 0 (discrete
      metric identities);
  P6  entropy identity for a general SBP Q (Q 1 = 0) and an entropy-
      conservative symmetric F, with entropy variables written out here;
  P7  conservation: 1^T r = 1/2 sum_ij (Q_m + Q_m^T)_ij F_m,ij;
  P8  pressure equilibrium of the Ranocha flux: constant v and p give
      r_mom = v r_rho and r_E = |v|^2/2 r_rho.
"""

import numpy as np
import pytest

import oracle as O
from paper_2306_11665_gb300 import inputs as I

GLL, GAUSS = O.NODES_GLL, O.NODES_GAUSS
G = O.GAMMA


def _kron_q(d, p, kind, m):
    _, w, _, Q1 = O.op1d(p, kind)
    W = np.diag(w)
    fac = [Q1 if k == m else W for k in range(d)]
    out = fac[d - 1]
    for k in range(d - 2, -1, -1):
        out = np.kron(out, fac[k])
    return out


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# ------------------------------------------------------------------- P1
def test_p1_burgers_2d_full_config():
    """The whole 2D Burgers configuration: p=3 Gauss-Lobatto, 8x8 affine."""
    u, Ja = I.workload(2, 3, GLL, 8, flux="burgers", amp=0.0)
    r_sf = O.volume_sf(2, 3, GLL, O.FLUX_BURGERS, u, Ja)
    r_de = O.volume_dense(2, 3, GLL, O.FLUX_BURGERS, u, Ja)
    assert _rel(r_sf, r_de) < 1e-14


@pytest.mark.parametrize("kind", [GLL, GAUSS])
@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 7])
def test_p1_euler_3d(kind, p):
    N = 2 if p <= 3 else 1
    u, Ja = I.workload(3, p, kind, N)
    r_sf = O.volume_sf(3, p, kind, O.FLUX_EULER, u, Ja)
    r_de = O.volume_dense(3, p, kind, O.FLUX_EULER, u, Ja)
    for v in range(5):
        assert _rel(r_sf[:, v], r_de[:, v]) < 1e-13


@pytest.mark.parametrize("d, flux", [(2, O.FLUX_EULER), (3, O.FLUX_BURGERS), (2, O.FLUX_BURGERS)])
@pytest.mark.parametrize("kind", [GLL, GAUSS])
def test_p1_other_shapes(d, flux, kind):
    u, Ja = I.workload(d, 3, kind, 2, flux="burgers" if flux == O.FLUX_BURGERS else "euler")
    r_sf = O.volume_sf(d, 3, kind, flux, u, Ja)
    r_de = O.volume_dense(d, 3, kind, flux, u, Ja)
    assert _rel(r_sf, r_de) < 1e-13


# ------------------------------------------------------------------- P4
@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("kind", [GLL, GAUSS])
@pytest.mark.parametrize("p", [1, 3, 5])
def test_p4_burgers_split_form_closed_form(d, kind, p):
    N = 3 if d == 2 else 2
    u, Ja = I.workload(d, p, kind, N, flux="burgers", amp=0.0)
    h = 1.0 / N
    c = (h / 2) ** (d - 1)
    # the generated affine metrics are c * identity up to round-off; the closed
    # form is checked with the exact metric
    eye = np.eye(d)[None, :, :, None]
    assert np.abs(Ja - c * eye).max() < 1e-12 * c
    Ja = np.ascontiguousarray(np.broadcast_to(c * eye, Ja.shape))
    r = O.volume_sf(d, p, kind, O.FLUX_BURGERS, u, Ja)
    Qs = [_kron_q(d, p, kind, m) for m in range(d)]
    for e in range(u.shape[0]):
        ue = u[e, 0]
        ref = sum(c / 3.0 * (ue * (Q @ ue) + Q @ (ue * ue)) for Q in Qs)
        assert np.abs(r[e, 0] - ref).max() < 1e-14 * max(1.0, np.abs(ref).max())


# --------------------------------------------------------- P5 / P8 (warped)
def _pair_scale(d, p, kind, flux, u, Ja):
    """max_i sum_{m,j} |Q_m,ij| |F_m,ij|: the size of the terms r_i sums."""
    nn = (p + 1) ** d
    scale = 0.0
    for e in range(u.shape[0]):
        for m in range(d):
            Q = _kron_q(d, p, kind, m)
            for i in range(nn):
                s = 0.0
                for j in np.nonzero(Q[i])[0]:
                    nv = Ja[e, m, :, i] + Ja[e, m, :, j]
                    s += abs(Q[i, j]) * np.abs(O.ec_flux(d, flux, u[e, :, i], u[e, :, j], nv)).max()
                scale = max(scale, s)
    return scale


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("kind", [GLL, GAUSS])
@pytest.mark.parametrize("p", [2, 4, 7])
def test_p5_free_stream(d, kind, p):
    N = 2
    _, Ja = O.mesh(d, p, kind, N, 0.1)      # the oracle's own metrics
    nn = (p + 1) ** d
    u = I.constant_state(N ** d, d, nn)
    r = O.volume_sf(d, p, kind, O.FLUX_EULER, u, Ja)
    scale = _pair_scale(d, p, kind, O.FLUX_EULER, u[:1], Ja[:1])
    assert np.abs(r).max() <= 1e-12 * scale
    # the warp is real: the metrics are far from affine
    assert np.abs(Ja - Ja[:, :, :, :1]).max() > 1e-3


@pytest.mark.parametrize("kind", [GLL, GAUSS])
@pytest.mark.parametrize("p", [3, 4])
def test_p8_pressure_equilibrium(kind, p):
    d, N = 3, 2
    x, Ja = O.mesh(d, p, kind, N, 0.1)
    rho = 1.0 + 0.2 * I.random_fourier(x, 11)
    v = np.array([0.3, -0.2, 0.1])
    u = I.conservative(rho, [np.full_like(rho, vk) for vk in v], np.full_like(rho, 1.0))
    r = O.volume_sf(d, p, kind, O.FLUX_EULER, u, Ja)
    scale = _pair_scale(d, p, kind, O.FLUX_EULER, u[:1], Ja[:1])
    for k in range(3):
        assert np.abs(r[:, 1 + k] - v[k] * r[:, 0]).max() <= 1e-12 * scale
    assert np.abs(r[:, 4] - 0.5 * (v @ v) * r[:, 0]).max() <= 1e-12 * scale
    assert np.abs(r[:, 0]).max() > 1e-6 * scale     # not trivially zero


# ------------------------------------------------------------- P6 / P7
def _entropy(u, d, flux):
    """Entropy variables w[var][i] and potentials psi[k][i] (U = u^2/2 for
    Burgers; U = -rho s/(gamma-1), s = ln p - gamma ln rho for Euler)."""
    if flux == O.FLUX_BURGERS:
        return u.copy(), np.repeat(u[0:1] ** 3 / 6.0, d, axis=0)
    rho = u[0]
    v = u[1:1 + d] / rho
    p = (G - 1) * (u[d + 1] - 0.5 * rho * (v * v).sum(0))
    s = np.log(p) - G * np.log(rho)
    w = np.concatenate([[(G - s) / (G - 1) - 0.5 * rho * (v * v).sum(0) / p], rho * v / p, [-rho / p]])
    return w, rho * v


@pytest.mark.parametrize("d, flux", [(3, O.FLUX_EULER), (2, O.FLUX_EULER), (2, O.FLUX_BURGERS), (3, O.FLUX_BURGERS)])
@pytest.mark.parametrize("kind", [GLL, GAUSS])
@pytest.mark.parametrize("p", [2, 4])
def test_p6_entropy_identity_and_p7_conservation(d, flux, kind, p):
    N = 2
    u, Ja = I.workload(d, p, kind, N, flux="burgers" if flux == O.FLUX_BURGERS else "euler")
    r = O.volume_sf(d, p, kind, flux, u, Ja)
    nn = (p + 1) ** d
    ones = np.ones(nn)
    for e in range(u.shape[0]):
        w, psi = _entropy(u[e], d, flux)
        lhs = np.sum(w * r[e])
        rhs = 0.0
        scale = 0.0
        cons_rhs = np.zeros(u.shape[1])
        for m in range(d):
            Q = _kron_q(d, p, kind, m)
            E = Q + Q.T
            J = Ja[e, m]                                   # [k][i]
            t1 = 0.0
            for i in range(nn):
                for j in np.nonzero(E[i] + np.abs(Q[i]))[0]:
                    F = O.ec_flux(d, flux, u[e, :, i], u[e, :, j], J[:, i] + J[:, j])
                    if E[i, j] != 0.0:
                        t1 += E[i, j] * (w[:, i] @ F)
                        cons_rhs += 0.5 * E[i, j] * F
                    scale += abs(Q[i, j]) * np.abs(w[:, i] * F).sum()
            psiJ = (psi * J).sum(0)                        # psi_i . Ja^m(i)
            rhs += 0.5 * t1 - 0.5 * ((E @ ones) * psiJ).sum() \
                - 0.5 * np.einsum("ki,ij,kj->", psi, E, J) + np.einsum("ki,ij,kj->", psi, Q, J)
        assert abs(lhs - rhs) <= 1e-13 * scale, (lhs, rhs, scale)
        # conservation
        cons_lhs = r[e].sum(axis=1)
        assert np.abs(cons_lhs - cons_rhs).max() <= 1e-13 * max(scale, 1.0)


def test_p6_lgl_boundary_entropy_flux_form():
    """Gauss-Lobatto: E_m = B_m is diagonal, so the identity becomes
    w^T r = sum_m sum_i (B_m)_ii (w_i . f(u_i; Ja^m(i)) - psi_i . Ja^m(i))
            + sum_m psi^T Q_m Ja^m,
    and the last sum vanishes when the metrics satisfy the discrete identities
    sum_m D_m Ja^m_k = 0: the stated form w^T (2 Q o F) 1 = 1^T B F_entropy."""
    d, p, kind = 3, 4, GLL
    u, Ja = I.workload(d, p, kind, 2)
    r = O.volume_sf(d, p, kind, O.FLUX_EULER, u, Ja)
    for e in range(u.shape[0]):
        w, psi = _entropy(u[e], d, O.FLUX_EULER)
        lhs = np.sum(w * r[e])
        bnd, gcl, scale = 0.0, 0.0, 0.0
        for m in range(d):
            Q = _kron_q(d, p, kind, m)
            B = np.diag(Q + Q.T)
            assert np.abs(Q + Q.T - np.diag(B)).max() < 1e-14
            J = Ja[e, m]
            for i in np.nonzero(B)[0]:
                rho = u[e, 0, i]
                v = u[e, 1:4, i] / rho
                pr = (G - 1) * (u[e, 4, i] - 0.5 * rho * v @ v)
                vn = v @ J[:, i]
                f = np.concatenate(([rho * vn], rho * v * vn + pr * J[:, i], [(u[e, 4, i] + pr) * vn]))
                bnd += B[i] * (w[:, i] @ f - psi[:, i] @ J[:, i])
                scale += abs(B[i]) * np.abs(w[:, i] * f).sum()
            gcl += np.einsum("ki,ij,kj->", psi, Q, J)
        assert abs(lhs - bnd - gcl) <= 1e-13 * scale
        assert abs(gcl) <= 1e-12 * scale


# ----------------------------------------------- absolute terms (error scale)
@pytest.mark.parametrize("d, flux, kind, p", [(3, O.FLUX_EULER, GLL, 2), (3, O.FLUX_EULER, GAUSS, 3),
                                              (2, O.FLUX_BURGERS, GLL, 3), (2, O.FLUX_EULER, GAUSS, 2)])
def test_absterms_against_dense_brute_force(d, flux, kind, p):
    """S_i = sum_m sum_j |Q_m,ij F_m,ij| from the full Kronecker matrices and
    a flux evaluation of every (i, j) pair (a path that shares no loop with
    the sum-factorized routine), and S >= |r| by the triangle inequality."""
    u, Ja = I.workload(d, p, kind, 2, flux="burgers" if flux == O.FLUX_BURGERS else "euler")
    u, Ja = u[:2], Ja[:2]
    S = O.volume_absterms(d, p, kind, flux, u, Ja)
    nn = u.shape[2]
    ref = np.zeros_like(u)
    for e in range(u.shape[0]):
        for m in range(d):
            Q = _kron_q(d, p, kind, m)
            for i in range(nn):
                for j in range(nn):
                    if Q[i, j] == 0.0:
                        continue
                    F = O.ec_flux(d, flux, u[e, :, i], u[e, :, j], Ja[e, m, :, i] + Ja[e, m, :, j])
                    ref[e, :, i] += np.abs(Q[i, j] * F)
    assert _rel(S, ref) <= 1e-14
    r = O.volume_sf(d, p, kind, flux, u, Ja)
    assert np.all(S >= np.abs(r) * (1 - 1e-14))
