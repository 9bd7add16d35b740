"""Pins of the oracle's reverse mode of the surface Hadamard product
(orc_surface_vjp_dense: the gradients of lam_vol . r_vol + lam_face . r_face
with respect to the volume state u and the face state u~, Remark 1's operator):

  * every entry of both gradients against central differences of the forward
    oracle (orc_surface_dense) on a tiny element;
  * random directional derivatives against central differences, for every
    flux and both node sets, in 2D and 3D;
  * Burgers with u~ = 0, a closed form: dF/du_j = u_j S / 3 and dF/du~ =
    u_j S / 6 (S the sum of the normal's components), with the interpolation
    rows fitted by numpy -- a swap of the two Jacobians, of the cotangents or
    of the face weights fails it.
"""
import numpy as np
import pytest

import oracle as O
from paper_2306_11665_gb300 import inputs as I
from tests.test_oracle_surface import face_geometry, face_rows

FLUXES = [O.FLUX_EULER, O.FLUX_CHANDRASHEKAR, O.FLUX_BURGERS]


def _name(flux):
    return "burgers" if flux == O.FLUX_BURGERS else "euler"


def _loss(d, p, kind, flux, u, uf, nJ, lv, lf):
    rv, rf = O.surface_dense(d, p, kind, flux, u, uf, nJ)
    return float(np.sum(lv * rv) + np.sum(lf * rf))


def _cotangents(u, uf, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(u.shape), rng.standard_normal(uf.shape)


def test_every_entry_against_central_differences():
    d, p, kind, flux = 2, 2, 1, O.FLUX_EULER
    u, uf, nJ = I.surface_workload(d, p, kind, 1)
    lv, lf = _cotangents(u, uf, 3)
    gu, gf = O.surface_vjp_dense(d, p, kind, flux, u, uf, nJ, lv, lf)
    h = 1e-6
    for arr, g in ((u, gu), (uf, gf)):
        for idx in np.ndindex(arr.shape):
            x0 = arr[idx]
            arr[idx] = x0 + h
            lp = _loss(d, p, kind, flux, u, uf, nJ, lv, lf)
            arr[idx] = x0 - h
            lm = _loss(d, p, kind, flux, u, uf, nJ, lv, lf)
            arr[idx] = x0
            fd = (lp - lm) / (2 * h)
            assert abs(g[idx] - fd) <= 2e-7 * max(1.0, abs(fd)), (idx, g[idx], fd)


@pytest.mark.parametrize("flux", FLUXES)
@pytest.mark.parametrize("d, kind, p", [(2, 0, 3), (2, 1, 2), (3, 0, 2), (3, 1, 3)])
def test_directional_derivative(d, kind, p, flux):
    u, uf, nJ = I.surface_workload(d, p, kind, 2, flux=_name(flux))
    lv, lf = _cotangents(u, uf, 11 + p)
    gu, gf = O.surface_vjp_dense(d, p, kind, flux, u, uf, nJ, lv, lf)
    rng = np.random.default_rng(5 + d)
    du, duf = rng.standard_normal(u.shape), rng.standard_normal(uf.shape)
    h = 1e-6
    lp = _loss(d, p, kind, flux, u + h * du, uf + h * duf, nJ, lv, lf)
    lm = _loss(d, p, kind, flux, u - h * du, uf - h * duf, nJ, lv, lf)
    fd = (lp - lm) / (2 * h)
    ad = float(np.sum(gu * du) + np.sum(gf * duf))
    scale = float(np.sum(np.abs(gu * du)) + np.sum(np.abs(gf * duf)))
    assert abs(ad - fd) <= 1e-7 * max(scale, 1.0), (ad, fd, scale)


@pytest.mark.parametrize("d, kind", [(2, 0), (2, 1), (3, 1)])
def test_burgers_closed_form(d, kind):
    p = 3
    u, uf, nJ = I.surface_workload(d, p, kind, 2, flux="burgers")
    uf = np.zeros_like(uf)
    lv, lf = _cotangents(u, uf, 21)
    gu, gf = O.surface_vjp_dense(d, p, kind, O.FLUX_BURGERS, u, uf, nJ, lv, lf)
    e_rows = face_rows(p, kind)
    geo = face_geometry(d, p, kind)
    gu_ref, gf_ref = np.zeros_like(gu), np.zeros_like(gf)
    for e in range(u.shape[0]):
        for m in range(d):
            lines, wf = geo[m]
            for side in range(2):
                face = 2 * m + side
                for f, line in enumerate(lines):
                    S = nJ[e, face, :, f].sum()
                    for b, j in enumerate(line):
                        c = wf[f] * e_rows[side, b] * (lv[e, 0, j] + lf[e, face, 0, f])
                        gu_ref[e, 0, j] += c * u[e, 0, j] * S / 3.0
                        gf_ref[e, face, 0, f] += c * u[e, 0, j] * S / 6.0
    assert np.abs(gu - gu_ref).max() <= 1e-13 * max(np.abs(gu_ref).max(), 1.0)
    assert np.abs(gf - gf_ref).max() <= 1e-13 * max(np.abs(gf_ref).max(), 1.0)
