"""Pins of the oracle's vector-Jacobian product g = (dr/du)^T lambda.

  * central finite differences of the oracle's residual, per component on a
    sample of components (2^3 elements) and directionally at 8^3 elements
    (step 1e-6 max(1, |u|), the adjoint configuration p = 5 Gauss-Lobatto);
  * the dense-form VJP, i.e. the transpose of the assembled element Jacobian
    of the Eq. 1 form, on 2^3 elements.
"""
import numpy as np
import pytest

import oracle as O
from paper_2306_11665_gb300 import inputs as I

GLL, GAUSS = O.NODES_GLL, O.NODES_GAUSS


@pytest.mark.parametrize("kind", [GLL, GAUSS])
def test_vjp_vs_dense_form(kind):
    d, p = 3, 5
    u, Ja = I.workload(d, p, kind, 2)
    lam = I.cotangent(u.shape)
    g_sf = O.vjp_sf(d, p, kind, O.FLUX_EULER, u, Ja, lam)
    g_de = O.vjp_dense(d, p, kind, O.FLUX_EULER, u, Ja, lam)
    assert np.abs(g_sf - g_de).max() <= 1e-13 * np.abs(g_de).max()


@pytest.mark.parametrize("d, flux", [(2, O.FLUX_BURGERS), (2, O.FLUX_EULER), (3, O.FLUX_BURGERS)])
def test_vjp_vs_dense_other_shapes(d, flux):
    p, kind = 3, GAUSS
    u, Ja = I.workload(d, p, kind, 2, flux="burgers" if flux == O.FLUX_BURGERS else "euler")
    lam = I.cotangent(u.shape)
    g_sf = O.vjp_sf(d, p, kind, flux, u, Ja, lam)
    g_de = O.vjp_dense(d, p, kind, flux, u, Ja, lam)
    assert np.abs(g_sf - g_de).max() <= 1e-13 * np.abs(g_de).max()


def test_vjp_fd_per_component():
    d, p, kind = 3, 5, GLL
    u, Ja = I.workload(d, p, kind, 2)
    lam = I.cotangent(u.shape)
    g = O.vjp_sf(d, p, kind, O.FLUX_EULER, u, Ja, lam)
    rng = np.random.default_rng(5)
    flat = rng.choice(u.size, size=60, replace=False)
    for idx in flat:
        e, v, i = np.unravel_index(idx, u.shape)
        h = 1e-6 * max(1.0, abs(u[e, v, i]))
        up, um = u.copy(), u.copy()
        up[e, v, i] += h
        um[e, v, i] -= h
        # only element e changes: difference that element's residual
        rp = O.volume_sf(d, p, kind, O.FLUX_EULER, up[e:e + 1], Ja[e:e + 1])
        rm = O.volume_sf(d, p, kind, O.FLUX_EULER, um[e:e + 1], Ja[e:e + 1])
        fd = np.sum(lam[e:e + 1] * (rp - rm)) / (2 * h)
        assert abs(g[e, v, i] - fd) <= 1e-6 * max(abs(fd), np.abs(g).max() * 1e-3), (e, v, i, g[e, v, i], fd)


def test_vjp_fd_directional_8cubed():
    d, p, kind = 3, 5, GLL
    u, Ja = I.workload(d, p, kind, 8)
    lam = I.cotangent(u.shape)
    g = O.vjp_sf(d, p, kind, O.FLUX_EULER, u, Ja, lam)
    delta = np.random.default_rng(6).standard_normal(u.shape) * np.maximum(1.0, np.abs(u))
    h = 1e-6
    rp = O.volume_sf(d, p, kind, O.FLUX_EULER, u + h * delta, Ja)
    rm = O.volume_sf(d, p, kind, O.FLUX_EULER, u - h * delta, Ja)
    fd = np.sum(lam * (rp - rm)) / (2 * h)
    an = np.sum(g * delta)
    assert abs(an - fd) <= 1e-6 * abs(fd)
