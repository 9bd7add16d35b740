"""Pins of the oracle's second Euler flux, Chandrashekar's entropy-conserving
kinetic-energy-preserving flux (the flux the paper names for its TGV runs,
Section 3): consistency with the physical flux, symmetry, Tadmor's
entropy-conservation condition, the residual-level identities (dense =
sum-factorized, free stream, the SBP entropy identity, pressure
equilibrium), and how it differs from Ranocha's flux: only in the pressure
terms ({rho}/{beta} against {p} in the momentum flux, ({rho}/{beta}) {v}.n
against (p_i v_j + p_j v_i).n / 2 in the energy flux)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2306_11665_gb300 import inputs as I
from tests._entropy import identity_residual

G = O.GAMMA
CH, RA = O.FLUX_CHANDRASHEKAR, O.FLUX_EULER


def _prim(u, d):
    rho = u[0]
    v = u[1:1 + d] / rho
    p = (G - 1) * (u[d + 1] - 0.5 * rho * v @ v)
    return rho, v, p


def _state(rng, d, spread):
    rho = 1.0 + spread * rng.uniform(-1, 1)
    v = 0.5 * rng.uniform(-1, 1, size=d)
    p = 1.0 + spread * rng.uniform(-1, 1)
    return np.concatenate(([rho], rho * v, [p / (G - 1) + 0.5 * rho * v @ v]))


def _w(u, d):
    rho, v, p = _prim(u, d)
    s = math.log(p) - G * math.log(rho)
    return np.concatenate(([(G - s) / (G - 1) - 0.5 * rho * (v @ v) / p], rho * v / p, [-rho / p]))


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("spread", [1e-9, 1e-3, 0.3, 0.9])
def test_flux_consistent_symmetric_entropy_conservative(d, spread):
    rng = np.random.default_rng(5)
    for _ in range(50):
        ui, uj = _state(rng, d, spread), _state(rng, d, spread)
        nv = rng.uniform(-1, 1, size=d)
        F = O.ec_flux(d, CH, ui, uj, nv)
        sc = np.abs(F).max() + 1.0
        np.testing.assert_allclose(O.ec_flux(d, CH, uj, ui, nv), F, rtol=0, atol=1e-14 * sc)
        rho, v, p = _prim(ui, d)
        vn = v @ nv
        phys = np.concatenate(([rho * vn], rho * v * vn + p * nv, [(ui[d + 1] + p) * vn]))
        np.testing.assert_allclose(O.ec_flux(d, CH, ui, ui, nv), phys, rtol=0, atol=1e-14 * sc)
        dw = _w(uj, d) - _w(ui, d)
        lhs = dw @ F
        rhs = (_prim(uj, d)[0] * _prim(uj, d)[1] - rho * v) @ nv
        assert abs(lhs - rhs) <= 1e-12 * (np.abs(dw) @ np.abs(F) + 1e-300)


@pytest.mark.parametrize("d", [2, 3])
def test_fluxes_differ_only_in_the_pressure_terms(d):
    rng = np.random.default_rng(6)
    for _ in range(30):
        ui, uj = _state(rng, d, 0.5), _state(rng, d, 0.5)
        nv = rng.uniform(-1, 1, size=d)
        Fc, Fr = O.ec_flux(d, CH, ui, uj, nv), O.ec_flux(d, RA, ui, uj, nv)
        ri, vi, pi = _prim(ui, d)
        rj, vj, pj = _prim(uj, d)
        p_t = (ri + rj) / (ri / pi + rj / pj)
        vavg = 0.5 * (vi + vj)
        sc = np.abs(Fr).max() + 1.0
        assert abs(Fr[0] - Fc[0]) <= 1e-14 * sc                                   # same mass flux
        np.testing.assert_allclose(Fr[1:1 + d] - Fc[1:1 + d], (0.5 * (pi + pj) - p_t) * nv, rtol=0, atol=1e-13 * sc)
        dE = 0.5 * (pi * (vj @ nv) + pj * (vi @ nv)) - p_t * (vavg @ nv)
        assert abs((Fr[d + 1] - Fc[d + 1]) - dE) <= 1e-13 * sc


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("p", [2, 4])
def test_residual_dense_free_stream_entropy(kind, p):
    d = 3
    u, Ja = I.workload(d, p, kind, 2)
    r_sf = O.volume_sf(d, p, kind, CH, u, Ja)
    r_de = O.volume_dense(d, p, kind, CH, u, Ja)
    assert np.abs(r_sf - r_de).max() <= 1e-13 * np.abs(r_de).max()
    for e in (0, u.shape[0] - 1):
        assert identity_residual(d, p, kind, CH, u[e], Ja[e], r_sf[e]) <= 1e-13
    _, Jw = O.mesh(d, p, kind, 2, 0.1)
    uc = I.constant_state(8, d, (p + 1) ** d)
    rc = O.volume_sf(d, p, kind, CH, uc, Jw)
    assert np.abs(rc).max() <= 1e-12 * np.abs(r_sf).max()


@pytest.mark.parametrize("kind", [0, 1])
def test_pressure_equilibrium_both_fluxes(kind):
    """Constant velocity and pressure, varying density: with p constant,
    {rho}/{beta} = p and {beta}_ln = {rho}_ln / p, so both fluxes keep
    r_m = v r_rho and r_E = |v|^2/2 r_rho (no pressure oscillation is
    generated) -- while the two residuals differ once p varies."""
    d, p, N = 3, 3, 2
    x, Ja = O.mesh(d, p, kind, N, 0.1)
    rho = 1.0 + 0.2 * I.random_fourier(x, 11)
    v = np.array([0.3, -0.2, 0.1])
    u = I.conservative(rho, [np.full_like(rho, vk) for vk in v], np.full_like(rho, 1.0))
    for fl in (RA, CH):
        r = O.volume_sf(d, p, kind, fl, u, Ja)
        dm = max(np.abs(r[:, 1 + k] - v[k] * r[:, 0]).max() for k in range(3))
        dE = np.abs(r[:, 4] - 0.5 * (v @ v) * r[:, 0]).max()
        assert max(dm, dE) <= 1e-12 * np.abs(r).max(), fl
    u2, J2 = I.workload(d, p, kind, N)
    r_ra, r_ch = O.volume_sf(d, p, kind, RA, u2, J2), O.volume_sf(d, p, kind, CH, u2, J2)
    assert np.abs(r_ra - r_ch).max() >= 1e-6 * np.abs(r_ra).max()


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("spread", [1e-6, 0.01, 0.5])
def test_flux_jacobian_vs_fd(d, spread):
    """The adjoint's flux Jacobian (first state) against central differences of
    the flux itself."""
    rng = np.random.default_rng(7)
    for _ in range(10):
        ui, uj = _state(rng, d, spread), _state(rng, d, spread)
        nv = rng.uniform(-1, 1, size=d)
        J = O.ec_flux_jac1(d, CH, ui, uj, nv)
        for b in range(d + 2):
            h = 1e-6 * max(1.0, abs(ui[b]))
            e = np.zeros(d + 2)
            e[b] = h
            fd = (O.ec_flux(d, CH, ui + e, uj, nv) - O.ec_flux(d, CH, ui - e, uj, nv)) / (2 * h)
            np.testing.assert_allclose(J[:, b], fd, rtol=0, atol=2e-8 * (np.abs(fd).max() + 1))


@pytest.mark.parametrize("d, kind", [(3, 0), (3, 1), (2, 1)])
def test_vjp_dense_form_and_fd(d, kind):
    """Sum-factorized VJP = transpose of the assembled element Jacobian, and
    directional central differences of the residual."""
    p = 3
    u, Ja = I.workload(d, p, kind, 2)
    lam = I.cotangent(u.shape)
    g = O.vjp_sf(d, p, kind, CH, u, Ja, lam)
    g_de = O.vjp_dense(d, p, kind, CH, u, Ja, lam)
    assert np.abs(g - g_de).max() <= 1e-13 * np.abs(g_de).max()
    delta = np.random.default_rng(8).standard_normal(u.shape) * np.maximum(1.0, np.abs(u))
    h = 1e-6
    fd = np.sum(lam * (O.volume_sf(d, p, kind, CH, u + h * delta, Ja)
                       - O.volume_sf(d, p, kind, CH, u - h * delta, Ja))) / (2 * h)
    assert abs(np.sum(g * delta) - fd) <= 1e-6 * abs(fd)
    # the adjoints of the two fluxes differ (the pressure terms enter them)
    g_ra = O.vjp_sf(d, p, kind, RA, u, Ja, lam)
    assert np.abs(g - g_ra).max() >= 1e-6 * np.abs(g_ra).max()
