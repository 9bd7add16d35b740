"""Pins of the oracle's logarithmic mean and two-point fluxes.

The references here are independent of the oracle's formulas:
  * the logarithmic mean against a 50-digit evaluation of its definition;
  * consistency f#(u, u) = f(u) with the physical flux written out here;
  * Tadmor's entropy-conservation condition (w_j - w_i) . f# = psi_j - psi_i
    with entropy variables and potentials written out here (the property the
    method needs from its two-point flux);
  * symmetry, and the Jacobian against central finite differences.
"""
import math

import numpy as np
import pytest

import oracle as O

EPS = np.finfo(np.float64).eps
G = O.GAMMA


def _lm_exact(a, b):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    a, b = mp.mpf(a), mp.mpf(b)
    if a == b:
        return float(a)
    return float((a - b) / (mp.log(a) - mp.log(b)))


def _lm_bound(a, b):
    """Rounding bound of the two branches: a few ulp, plus eps / |ln(a/b)| for
    the direct branch, whose log of a rounded ratio carries the ratio's half
    ulp divided by |ln(a/b)|."""
    u = ((a - b) / (a + b)) ** 2
    if u < 1e-4:
        return 8 * EPS
    return 8 * EPS + 2 * EPS / abs(math.log(a / b))


@pytest.mark.parametrize("a, b", [
    (1.0, 1.0), (1.0, 1.0 + 1e-12), (1.0, 1.0 + 1e-6), (1.0, 1.015), (1.0, 1.0205),
    (1.0, 1.03), (0.8, 1.2), (1e-3, 2.0), (3.0, 1e5), (0.5, 0.5000001), (7.25, 7.0),
])
def test_logmean_vs_definition(a, b):
    for x, y in ((a, b), (b, a)):
        got = O.logmean(x, y)
        ref = _lm_exact(x, y)
        assert abs(got - ref) <= _lm_bound(x, y) * abs(ref), (x, y, got, ref)


def test_logmean_invariants():
    rng = np.random.default_rng(0)
    for _ in range(200):
        a, b = np.exp(rng.uniform(-3, 3, size=2))
        L = O.logmean(a, b)
        assert min(a, b) <= L <= max(a, b)
        assert abs(O.logmean(b, a) - L) <= 4 * EPS * L + _lm_bound(a, b) * L
        t = 2.0 ** rng.integers(-4, 5)   # exact scaling: homogeneity without rounding
        assert abs(O.logmean(t * a, t * b) - t * L) <= 2 * _lm_bound(a, b) * t * L
        # between the geometric and arithmetic means
        assert math.sqrt(a * b) * (1 - 1e-15) <= L <= 0.5 * (a + b) * (1 + 1e-15)
    for a in (1e-8, 0.3, 1.0, 17.0):
        assert O.logmean(a, a) == a


@pytest.mark.parametrize("a, b", [(1.0, 1.0), (1.0, 1.004), (1.0, 1.03), (0.7, 1.9), (2.0, 0.01)])
def test_logmean_grad(a, b):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50

    def L(x, y):
        x, y = mp.mpf(x), mp.mpf(y)
        return x if x == y else (x - y) / (mp.log(x) - mp.log(y))
    if a == b:
        ra = rb = 0.5
    else:
        ra = float(mp.diff(lambda t: L(t, b), a))
        rb = float(mp.diff(lambda t: L(a, t), b))
    ga, gb = O.logmean_grad(a, b)
    assert abs(ga - ra) < 1e-13 and abs(gb - rb) < 1e-13


# ---------------------------------------------------------------- Euler helpers
def _prim(u, d):
    rho = u[0]
    v = u[1:1 + d] / rho
    p = (G - 1) * (u[d + 1] - 0.5 * rho * v @ v)
    return rho, v, p


def _phys_flux(u, d, nv):
    rho, v, p = _prim(u, d)
    vn = v @ nv
    return np.concatenate(([rho * vn], rho * v * vn + p * nv, [(u[d + 1] + p) * vn]))


def _entropy_vars(u, d):
    rho, v, p = _prim(u, d)
    s = math.log(p) - G * math.log(rho)
    return np.concatenate(([(G - s) / (G - 1) - 0.5 * rho * (v @ v) / p], rho * v / p, [-rho / p]))


def _psi(u, d):
    rho, v, p = _prim(u, d)
    return rho * v


def _rand_state(rng, d, spread=0.3):
    rho = 1.0 + spread * rng.uniform(-1, 1)
    v = 0.5 * rng.uniform(-1, 1, size=d)
    p = 1.0 + spread * rng.uniform(-1, 1)
    return np.concatenate(([rho], rho * v, [p / (G - 1) + 0.5 * rho * v @ v]))


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("spread", [1e-9, 1e-3, 0.3, 0.9])
def test_euler_flux_ec_consistent_symmetric(d, spread):
    rng = np.random.default_rng(1)
    for _ in range(50):
        ui, uj = _rand_state(rng, d, spread), _rand_state(rng, d, spread)
        nv = rng.uniform(-1, 1, size=d)
        F = O.ec_flux(d, O.FLUX_EULER, ui, uj, nv)
        scale = np.abs(F).max() + 1.0
        # symmetry
        np.testing.assert_allclose(O.ec_flux(d, O.FLUX_EULER, uj, ui, nv), F, rtol=0, atol=1e-14 * scale)
        # consistency with the physical flux
        np.testing.assert_allclose(O.ec_flux(d, O.FLUX_EULER, ui, ui, nv), _phys_flux(ui, d, nv),
                                   rtol=0, atol=1e-14 * scale)
        # Tadmor: (w_j - w_i) . F = (psi_j - psi_i) . n
        lhs = (_entropy_vars(uj, d) - _entropy_vars(ui, d)) @ F
        rhs = (_psi(uj, d) - _psi(ui, d)) @ nv
        wsc = np.abs(_entropy_vars(uj, d) - _entropy_vars(ui, d)) @ np.abs(F) + 1e-300
        assert abs(lhs - rhs) <= 1e-12 * wsc, (lhs, rhs)


def test_burgers_flux():
    rng = np.random.default_rng(2)
    for d in (2, 3):
        for _ in range(50):
            a, b = rng.normal(size=2)
            nv = rng.uniform(-1, 1, size=d)
            F = O.ec_flux(d, O.FLUX_BURGERS, [a], [b], nv)[0]
            assert abs(O.ec_flux(d, O.FLUX_BURGERS, [a], [a], nv)[0] - 0.5 * a * a * nv.sum()) < 1e-15
            # entropy u^2/2: w = u, psi = u^3/6 per direction
            assert abs((b - a) * F - (b ** 3 - a ** 3) / 6 * nv.sum()) < 1e-14


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("flux", [O.FLUX_BURGERS, O.FLUX_EULER])
@pytest.mark.parametrize("spread", [1e-6, 0.01, 0.5])
def test_flux_jacobian_vs_fd(d, flux, spread):
    rng = np.random.default_rng(3)
    for _ in range(10):
        if flux == O.FLUX_EULER:
            ui, uj = _rand_state(rng, d, spread), _rand_state(rng, d, spread)
        else:
            ui, uj = rng.normal(size=1), rng.normal(size=1)
        nv = rng.uniform(-1, 1, size=d)
        J = O.ec_flux_jac1(d, flux, ui, uj, nv)
        nvar = ui.size
        for b in range(nvar):
            h = 1e-6 * max(1.0, abs(ui[b]))
            e = np.zeros(nvar); e[b] = h
            fd = (O.ec_flux(d, flux, ui + e, uj, nv) - O.ec_flux(d, flux, ui - e, uj, nv)) / (2 * h)
            np.testing.assert_allclose(J[:, b], fd, rtol=0, atol=2e-8 * (np.abs(fd).max() + 1))
