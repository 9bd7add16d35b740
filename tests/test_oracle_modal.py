"""Pins of the oracle's modal / uncollocated path (Section 2, Eq. 4 and the
theorem after it): u_v = V u_hat, entropy projection u~ = u(V Pi w(u_v)),
r_hat = V^T r_v(u~).

  * the 1D basis against numpy's Legendre series and closed forms
    (orthonormality under Gauss quadrature; the Gauss-Lobatto defect of the
    top mode, (2p+1)/p; Lagrange bases: identity on their own nodes, partition
    of unity, exact reproduction of degree-p polynomials);
  * the entropy variables against central differences of the entropy
    U = -rho s/(g-1), and their inverse map by a round trip;
  * the entropy projection: with as many cubature nodes as basis functions
    Pi = V^{-1}, so u~ = u_v to round-off;
  * the dense Kronecker transforms against sum-factorized einsum transforms,
    mode 0 of r_hat against the element sum of r_v (the transpose, not V);
  * a Lagrange basis on the cubature nodes gives the nodal residual; a
    constant state gives r_hat = 0 on the warped mesh; the modal residual
    satisfies the entropy identity with the projected entropy variables.
"""
import numpy as np
import pytest

import oracle as O
from paper_2306_11665_gb300 import inputs as I
from tests._entropy import identity_residual

LEG, LGLL, LGAUSS = O.BASIS_LEGENDRE, O.BASIS_LAGRANGE_GLL, O.BASIS_LAGRANGE_GAUSS
G = O.GAMMA


def nodes(p, kind):
    xi, w = np.zeros(p + 1), np.zeros(p + 1)
    O._check(O._load().orc_nodes(p, kind, O._p(xi), O._p(w)))
    return xi, w


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("p", [1, 2, 4, 7, 8, 12])
def test_legendre_basis(kind, p):
    V = O.basis_1d(p, kind, LEG)
    xi, w = nodes(p, kind)
    n = p + 1
    for k in range(n):
        c = np.zeros(n)
        c[k] = np.sqrt((2 * k + 1) / 2)
        np.testing.assert_allclose(V[:, k], np.polynomial.legendre.legval(xi, c), rtol=0, atol=1e-13)
    M = V.T @ np.diag(w) @ V
    want = np.eye(n)
    if kind == 0:
        want[p, p] = (2 * p + 1) / p   # GLL quadrature integrates P_p^2 to 2/p instead of 2/(2p+1)
    np.testing.assert_allclose(M, want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("basis", [LGLL, LGAUSS])
@pytest.mark.parametrize("p", [1, 3, 6, 8])
def test_lagrange_bases(kind, basis, p):
    V = O.basis_1d(p, kind, basis)
    sol_kind = 0 if basis == LGLL else 1
    if sol_kind == kind:
        assert np.array_equal(V, np.eye(p + 1))
    s, _ = nodes(p, sol_kind)
    xi, _ = nodes(p, kind)
    for k in range(p + 1):
        np.testing.assert_allclose(V @ s ** k, xi ** k, rtol=0, atol=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_entropy_variables_are_the_gradient_of_the_entropy(d):
    rng = np.random.default_rng(3)

    def U(u):
        rho = u[0]
        v = u[1:1 + d] / rho
        p = (G - 1) * (u[d + 1] - 0.5 * rho * v @ v)
        return -rho * (np.log(p) - G * np.log(rho)) / (G - 1)

    for _ in range(10):
        rho, p = 1 + 0.5 * rng.uniform(-1, 1), 1 + 0.5 * rng.uniform(-1, 1)
        v = rng.uniform(-0.5, 0.5, size=d)
        u = np.concatenate(([rho], rho * v, [p / (G - 1) + 0.5 * rho * v @ v]))
        w = O.entropy_vars(d, O.FLUX_EULER, u)
        for k in range(d + 2):
            h = 1e-6 * max(1.0, abs(u[k]))
            e = np.zeros(d + 2)
            e[k] = h
            assert abs((U(u + e) - U(u - e)) / (2 * h) - w[k]) <= 1e-8 * max(1.0, abs(w[k]))
        np.testing.assert_allclose(O.entropy_state(d, O.FLUX_EULER, w), u, rtol=1e-13, atol=1e-14)
    assert O.entropy_vars(d, O.FLUX_BURGERS, [0.7])[0] == 0.7


@pytest.mark.parametrize("d, kind, basis", [(3, 1, LEG), (3, 0, LEG), (2, 1, LGLL), (3, 1, LGLL), (2, 0, LGAUSS)])
@pytest.mark.parametrize("p", [2, 4])
def test_projection_is_the_identity_for_square_bases(d, kind, basis, p):
    uhat, _ = I.modal_workload(d, p, kind, basis, 2)
    uv, up = O.modal_states(d, p, kind, basis, O.FLUX_EULER, uhat)
    assert np.abs(up - uv).max() <= 1e-13 * np.abs(uv).max()


def _sf_apply(V1, x, d, transpose=False):
    """Apply V1 (or V1^T) along every axis of x[..., n^d] (x fastest)."""
    n = V1.shape[0]
    A = V1.T if transpose else V1
    lead = x.shape[:-1]
    t = x.reshape(lead + (n,) * d)   # C order: last axis is x (fastest)
    for ax in range(d):
        t = np.moveaxis(np.tensordot(t, A, axes=([t.ndim - 1 - ax], [1])), -1, t.ndim - 1 - ax)
    return t.reshape(lead + (n ** d,))


@pytest.mark.parametrize("d, kind, basis, flux", [(3, 1, LEG, O.FLUX_EULER), (3, 0, LGLL, O.FLUX_EULER),
                                                  (2, 1, LEG, O.FLUX_EULER), (2, 0, LEG, O.FLUX_BURGERS),
                                                  (3, 1, LGLL, O.FLUX_CHANDRASHEKAR)])
def test_dense_transforms_vs_sum_factorized(d, kind, basis, flux):
    p = 3
    fl = "burgers" if flux == O.FLUX_BURGERS else "euler"
    uhat, Ja = I.modal_workload(d, p, kind, basis, 2, flux=fl)
    V1 = O.basis_1d(p, kind, basis)
    uv, up = O.modal_states(d, p, kind, basis, flux, uhat)
    np.testing.assert_allclose(uv, _sf_apply(V1, uhat, d), rtol=0, atol=1e-13 * np.abs(uv).max())
    rv = O.volume_sf(d, p, kind, flux, up, Ja)
    rhat = O.volume_modal(d, p, kind, basis, flux, uhat, Ja)
    np.testing.assert_allclose(rhat, _sf_apply(V1, rv, d, transpose=True), rtol=0, atol=1e-13 * np.abs(rhat).max())
    if basis == LEG:
        # chi_0 = 2^(-d/2) at every node: mode 0 of r_hat is the element sum of r_v
        np.testing.assert_allclose(rhat[:, :, 0], 2.0 ** (-d / 2) * rv.sum(axis=2), rtol=0,
                                   atol=1e-13 * np.abs(rhat).max())


@pytest.mark.parametrize("d, kind", [(3, 0), (3, 1), (2, 1)])
def test_collocated_lagrange_basis_gives_the_nodal_residual(d, kind):
    p = 4
    basis = LGLL if kind == 0 else LGAUSS
    uhat, Ja = I.modal_workload(d, p, kind, basis, 2)
    r = O.volume_modal(d, p, kind, basis, O.FLUX_EULER, uhat, Ja)
    ref = O.volume_sf(d, p, kind, O.FLUX_EULER, uhat, Ja)
    assert np.abs(r - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("d, kind", [(3, 0), (3, 1), (2, 1)])
def test_constant_state_free_stream(d, kind):
    p = 4
    uhat, Ja = I.modal_workload(d, p, kind, LEG, 2)
    uhat[:, :, 1:] = 0.0                  # mode 0 only: a constant state
    r = O.volume_modal(d, p, kind, LEG, O.FLUX_EULER, uhat, Ja)
    uv, up = O.modal_states(d, p, kind, LEG, O.FLUX_EULER, uhat)
    scale = np.abs(O.ec_flux(d, O.FLUX_EULER, uv[0, :, 0], uv[0, :, 0], 2 * Ja[0, 0, :, 0])).max()
    assert np.abs(r).max() <= 1e-12 * scale


@pytest.mark.parametrize("d, kind, basis", [(3, 1, LEG), (3, 0, LEG), (2, 1, LGLL)])
def test_modal_entropy_identity(d, kind, basis):
    """w_hat . r_hat = w~ . r_v (the transform is V^T), and r_v at u~ satisfies
    the SBP entropy identity; w_hat = Pi w(u_v) = V^{-1} w(u_v) here."""
    p = 3
    uhat, Ja = I.modal_workload(d, p, kind, basis, 2)
    V1 = O.basis_1d(p, kind, basis)
    uv, up = O.modal_states(d, p, kind, basis, O.FLUX_EULER, uhat)
    rv = O.volume_sf(d, p, kind, O.FLUX_EULER, up, Ja)
    rhat = O.volume_modal(d, p, kind, basis, O.FLUX_EULER, uhat, Ja)
    Vinv = np.linalg.inv(V1)
    for e in range(uhat.shape[0]):
        w = np.stack([O.entropy_vars(d, O.FLUX_EULER, up[e, :, i]) for i in range(up.shape[2])], axis=1)
        what = _sf_apply(Vinv, w, d)
        lhs, rhs = np.sum(what * rhat[e]), np.sum(w * rv[e])
        assert abs(lhs - rhs) <= 1e-11 * np.sum(np.abs(w * rv[e]))
        assert identity_residual(d, p, kind, O.FLUX_EULER, up[e], Ja[e], rv[e]) <= 1e-12


@pytest.mark.parametrize("d, kind, basis", [(3, 1, LEG), (3, 0, LGLL), (2, 1, LEG)])
def test_projection_round_off_in_the_residual(d, kind, basis):
    """Skipping the projection changes r_hat only by its round-off amplified by
    the residual's cancellation: within 1e-11 relative per variable, while
    an actual change of the state (1e-8 relative) moves it by far more."""
    p = 4
    uhat, Ja = I.modal_workload(d, p, kind, basis, 2)
    a = O.volume_modal(d, p, kind, basis, O.FLUX_EULER, uhat, Ja)
    b = O.volume_modal(d, p, kind, basis, O.FLUX_EULER, uhat, Ja, project=False)
    den = np.abs(a).max(axis=(0, 2))
    assert np.all(np.abs(a - b).max(axis=(0, 2)) <= 1e-11 * den)
    c = O.volume_modal(d, p, kind, basis, O.FLUX_EULER, uhat * (1 + 1e-8 * np.cos(np.arange(uhat.size)).reshape(uhat.shape)), Ja)
    assert np.abs(a - c).max() >= 1e-9 * np.abs(a).max()


@pytest.mark.parametrize("d, kind, basis, flux", [(3, 1, LEG, O.FLUX_EULER), (3, 0, LGAUSS, O.FLUX_EULER),
                                                  (2, 1, LEG, O.FLUX_CHANDRASHEKAR), (2, 0, LEG, O.FLUX_BURGERS)])
def test_modal_vjp_against_finite_differences(d, kind, basis, flux):
    """g_hat . delta = d/dh lambda_hat . r_hat(u_hat + h delta) by central
    differences of the modal residual (unprojected and projected alike)."""
    p = 3
    fl = "burgers" if flux == O.FLUX_BURGERS else "euler"
    uhat, Ja = I.modal_workload(d, p, kind, basis, 2, flux=fl)
    lam = I.cotangent(uhat.shape)
    g = O.vjp_modal(d, p, kind, basis, flux, uhat, Ja, lam)
    delta = np.random.default_rng(9).standard_normal(uhat.shape) * np.maximum(0.1, np.abs(uhat))
    h = 1e-6
    for project in (False, True):
        rp = O.volume_modal(d, p, kind, basis, flux, uhat + h * delta, Ja, project=project)
        rm = O.volume_modal(d, p, kind, basis, flux, uhat - h * delta, Ja, project=project)
        fd = np.sum(lam * (rp - rm)) / (2 * h)
        assert abs(np.sum(g * delta) - fd) <= 1e-6 * abs(fd), project
    # per component on a sample
    rng = np.random.default_rng(10)
    for idx in rng.choice(uhat.size, size=12, replace=False):
        e, v, k = np.unravel_index(idx, uhat.shape)
        hh = 1e-6 * max(1.0, abs(uhat[e, v, k]))
        up, um = uhat.copy(), uhat.copy()
        up[e, v, k] += hh
        um[e, v, k] -= hh
        fd = np.sum(lam[e] * (O.volume_modal(d, p, kind, basis, flux, up[e:e + 1], Ja[e:e + 1], project=False)
                              - O.volume_modal(d, p, kind, basis, flux, um[e:e + 1], Ja[e:e + 1], project=False))) / (2 * hh)
        assert abs(g[e, v, k] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max())
