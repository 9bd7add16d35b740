"""Pins of the oracle's surface Hadamard product (Remark 1: the operator of
the theorem with alpha = 0 on the facet cubature, m x n interpolation
factors): r_vol = sum_faces ((B E)^T o C^T) 1 and r_face = ((B E) o C) 1 with
(B E)[f][j] = w_f E[f][j], C[f][j] = fsharp(u~_f, u_j) . nJ_f.

  * a constant state (face state equal to it): r_face = w_f f(u) . nJ_f by
    consistency and the partition of unity of the interpolation;
  * Gauss-Lobatto: E picks the boundary node, r_face[f] = w_f F(u~_f, u_b(f)) . nJ_f;
  * Burgers with u~ = 0 and a state linear in each coordinate: r_face is
    w_f (sum nJ_f) / 6 times the square of the state at the face point (the
    interpolation of a quadratic is exact for p >= 2);
  * both contractions add up the same entries: sum_j r_vol = sum_f r_face;
  * Tadmor's condition gives the surface entropy identity
    w^T r_vol - sum_faces w~^T r_face = sum_faces sum_f w_f sum_j E[f][j] (psi_j - psi~_f) . nJ_f.
"""
import numpy as np
import pytest

import oracle as O
from paper_2306_11665_gb300 import inputs as I

G = O.GAMMA


def nodes(p, kind):
    xi, w = np.zeros(p + 1), np.zeros(p + 1)
    O._check(O._load().orc_nodes(p, kind, O._p(xi), O._p(w)))
    return xi, w


def face_rows(p, kind):
    """e[side][b] = l_b(-1) / l_b(+1) by numpy's polynomial fit through the nodes."""
    xi, _ = nodes(p, kind)
    n = p + 1
    e = np.zeros((2, n))
    for b in range(n):
        y = np.zeros(n)
        y[b] = 1.0
        c = np.polynomial.polynomial.polyfit(xi, y, p)
        e[0, b] = np.polynomial.polynomial.polyval(-1.0, c)
        e[1, b] = np.polynomial.polynomial.polyval(1.0, c)
    return e


def face_geometry(d, p, kind):
    """For each face (m, side) and face node f: the volume nodes of its normal
    line in order of a_m, and w_f."""
    n = p + 1
    _, w = nodes(p, kind)
    out = {}
    for m in range(d):
        others = [k for k in range(d) if k != m]
        lines, wf = [], []
        for f in range(n ** (d - 1)):
            bf = [(f // n ** t) % n for t in range(d - 1)]
            a = [0] * d
            for t, k in enumerate(others):
                a[k] = bf[t]
            line = []
            for am in range(n):
                a[m] = am
                line.append(sum(a[k] * n ** k for k in range(d)))
            lines.append(line)
            wf.append(np.prod([w[b] for b in bf]))
        out[m] = (lines, np.array(wf))
    return out


def psi(d, flux, u):
    if flux == O.FLUX_BURGERS:
        return np.full(d, u[0] ** 3 / 6.0)
    return u[1:1 + d].copy()


@pytest.mark.parametrize("d, kind", [(2, 0), (2, 1), (3, 0), (3, 1)])
def test_constant_state(d, kind):
    p = 3
    u, uf, nJ = I.surface_workload(d, p, kind, 2)
    c = np.array([1.1, 0.3, -0.2, 0.1, 2.7])[: d + 2]
    if d == 2:
        c = np.array([1.1, 0.3, -0.2, 2.7])
    u[:] = c[None, :, None]
    uf[:] = c[None, None, :, None]
    rv, rf = O.surface_dense(d, p, kind, O.FLUX_EULER, u, uf, nJ)
    geo = face_geometry(d, p, kind)
    for e in range(u.shape[0]):
        for m in range(d):
            _, wf = geo[m]
            for side in range(2):
                face = 2 * m + side
                for f in range(len(wf)):
                    want = wf[f] * O.ec_flux(d, O.FLUX_EULER, c, c, nJ[e, face, :, f])
                    assert np.abs(rf[e, face, :, f] - want).max() <= 1e-14 * (1 + np.abs(want).max())


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("flux", [O.FLUX_EULER, O.FLUX_CHANDRASHEKAR])
def test_gauss_lobatto_picks_the_boundary_node(d, flux):
    p = 4
    u, uf, nJ = I.surface_workload(d, p, 0, 2)
    rv, rf = O.surface_dense(d, p, 0, flux, u, uf, nJ)
    geo = face_geometry(d, p, 0)
    for e in range(u.shape[0]):
        for m in range(d):
            lines, wf = geo[m]
            for side in range(2):
                face = 2 * m + side
                for f, line in enumerate(lines):
                    j = line[-1] if side else line[0]
                    want = wf[f] * O.ec_flux(d, flux, uf[e, face, :, f], u[e, :, j], nJ[e, face, :, f])
                    assert np.abs(rf[e, face, :, f] - want).max() <= 1e-14 * (1 + np.abs(want).max())


@pytest.mark.parametrize("d, kind", [(2, 1), (3, 1), (3, 0)])
@pytest.mark.parametrize("p", [2, 5])
def test_burgers_interpolation_of_a_quadratic(d, kind, p):
    n = p + 1
    xi, _ = nodes(p, kind)
    u, uf, nJ = I.surface_workload(d, p, kind, 2, flux="burgers")
    coef = np.array([0.3, 0.2, 0.1])[:d]
    i = np.arange(n ** d)
    lin = 1.0 + sum(coef[k] * xi[(i // n ** k) % n] for k in range(d))
    u[:] = lin[None, None, :]
    uf[:] = 0.0
    rv, rf = O.surface_dense(d, p, kind, O.FLUX_BURGERS, u, uf, nJ)
    geo = face_geometry(d, p, kind)
    for m in range(d):
        lines, wf = geo[m]
        others = [k for k in range(d) if k != m]
        for side in range(2):
            face = 2 * m + side
            for f in range(len(wf)):
                bf = [(f // n ** t) % n for t in range(d - 1)]
                val = 1.0 + coef[m] * (1.0 if side else -1.0) + sum(coef[k] * xi[bf[t]] for t, k in enumerate(others))
                want = wf[f] * nJ[:, face, :, f].sum(axis=1) / 6.0 * val ** 2
                assert np.abs(rf[:, face, 0, f] - want).max() <= 1e-13 * (1 + np.abs(want).max())


@pytest.mark.parametrize("d, kind, flux", [(3, 1, O.FLUX_EULER), (3, 0, O.FLUX_CHANDRASHEKAR),
                                           (2, 1, O.FLUX_EULER), (2, 0, O.FLUX_BURGERS),
                                           (3, 1, O.FLUX_BURGERS)])
def test_sums_and_surface_entropy_identity(d, kind, flux):
    p = 3
    fl = "burgers" if flux == O.FLUX_BURGERS else "euler"
    u, uf, nJ = I.surface_workload(d, p, kind, 2, flux=fl)
    rv, rf = O.surface_dense(d, p, kind, flux, u, uf, nJ)
    # both contractions of the same entries
    assert np.abs(rv.sum(axis=2) - rf.sum(axis=(1, 3))).max() <= 1e-13 * np.abs(rv).sum()
    e_rows = face_rows(p, kind)
    geo = face_geometry(d, p, kind)
    for e in range(u.shape[0]):
        w_vol = np.stack([O.entropy_vars(d, flux, u[e, :, i]) for i in range(u.shape[2])], axis=1)
        lhs = np.sum(w_vol * rv[e])
        rhs, scale = 0.0, 0.0
        for m in range(d):
            lines, wf = geo[m]
            for side in range(2):
                face = 2 * m + side
                for f, line in enumerate(lines):
                    wt = O.entropy_vars(d, flux, uf[e, face, :, f])
                    lhs -= wt @ rf[e, face, :, f]
                    pf = psi(d, flux, uf[e, face, :, f])
                    for b, j in enumerate(line):
                        t = wf[f] * e_rows[side, b] * ((psi(d, flux, u[e, :, j]) - pf) @ nJ[e, face, :, f])
                        rhs += t
                        scale += abs(t)
                    scale += abs(wt @ rf[e, face, :, f])
        assert abs(lhs - rhs) <= 1e-12 * max(scale, 1.0), (lhs, rhs, scale)
