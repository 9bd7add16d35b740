"""Pins of the oracle's 1D operators and of its tensor-product assembly.

What is checked against what (none of it re-runs the oracle's own formula):
  * textbook node/weight values (closed forms) and numpy's Gauss rule;
  * SBP identities of Q1 = W D that hold for exact collocation derivatives;
  * polynomial exactness of D;
  * dense Q_m against numpy.kron in the x-fastest order (Eq. 5, Section 2);
  * the index maps of the paper's sparsity-pattern and basis-assembly
    algorithms (Algorithms 1-2) against the nonzeros of the same Q_m.
"""
import math

import numpy as np
import pytest

import oracle as O

GLL, GAUSS = O.NODES_GLL, O.NODES_GAUSS


@pytest.mark.parametrize("p, xi_ref, w_ref", [
    (1, [-1, 1], [1, 1]),
    (2, [-1, 0, 1], [1 / 3, 4 / 3, 1 / 3]),
    (3, [-1, -1 / math.sqrt(5), 1 / math.sqrt(5), 1], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    (4, [-1, -math.sqrt(3 / 7), 0, math.sqrt(3 / 7), 1], [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
])
def test_gll_textbook(p, xi_ref, w_ref):
    xi, w, _, _ = O.op1d(p, GLL)
    np.testing.assert_allclose(xi, xi_ref, rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, w_ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("p", range(0 + 1, 9))
def test_gauss_vs_numpy(p):
    xi, w, _, _ = O.op1d(p, GAUSS)
    xr, wr = np.polynomial.legendre.leggauss(p + 1)
    np.testing.assert_allclose(xi, xr, rtol=0, atol=2e-15)
    np.testing.assert_allclose(w, wr, rtol=0, atol=2e-15)


def test_gauss_textbook_two_point():
    xi, w, _, _ = O.op1d(1, GAUSS)
    np.testing.assert_allclose(xi, [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=1e-16)
    np.testing.assert_allclose(w, [1, 1], atol=1e-16)


def _lagrange_at(xi, x):
    """Values of the Lagrange basis on nodes xi at the point x (product form)."""
    n = xi.size
    out = np.ones(n)
    for j in range(n):
        for k in range(n):
            if k != j:
                out[j] *= (x - xi[k]) / (xi[j] - xi[k])
    return out


@pytest.mark.parametrize("kind", [GLL, GAUSS])
@pytest.mark.parametrize("p", range(1, 9))
def test_sbp_properties(kind, p):
    xi, w, D, Q1 = O.op1d(p, kind)
    n = p + 1
    # Q1 annihilates constants
    assert np.abs(Q1 @ np.ones(n)).max() < 1e-14
    # Q1 + Q1^T = t_R t_R^T - t_L t_L^T (diag(-1, 0, .., 0, 1) for Gauss-Lobatto)
    tR, tL = _lagrange_at(xi, 1.0), _lagrange_at(xi, -1.0)
    E = np.outer(tR, tR) - np.outer(tL, tL)
    np.testing.assert_allclose(Q1 + Q1.T, E, rtol=0, atol=2e-14)
    if kind == GLL:
        B = np.zeros((n, n)); B[0, 0] = -1; B[-1, -1] = 1
        np.testing.assert_allclose(Q1 + Q1.T, B, rtol=0, atol=2e-14)
    # D differentiates polynomials of degree <= p exactly
    for k in range(0, p + 1):
        exact = k * xi ** (k - 1) if k > 0 else np.zeros(n)
        np.testing.assert_allclose(D @ xi ** k, exact, rtol=0, atol=1e-13 * max(1, k * k))
    # the weights integrate degree 2p-1 (Lobatto) / 2p+1 (Gauss) exactly
    top = 2 * p - 1 if kind == GLL else 2 * p + 1
    for k in range(top + 1):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(w @ xi ** k - exact) < 1e-14


def _kron_q(d, Q1, w, m):
    """Q_m by numpy.kron with x fastest: the factor for axis k sits at
    Kronecker position d-1-k (standard Kronecker order runs slowest first)."""
    W = np.diag(w)
    factors = [Q1 if k == m else W for k in range(d)]
    out = factors[d - 1]
    for k in range(d - 2, -1, -1):
        out = np.kron(out, factors[k])
    return out


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("kind", [GLL, GAUSS])
@pytest.mark.parametrize("p", [1, 2, 4])
def test_dense_q_is_kronecker(d, kind, p):
    _, w, _, Q1 = O.op1d(p, kind)
    for m in range(d):
        Qd, Qk = O.qmat_dense(d, p, kind, m), _kron_q(d, Q1, w, m)
        # same entries up to the rounding order of the d-fold products
        np.testing.assert_allclose(Qd, Qk, rtol=4e-16, atol=0)
        np.testing.assert_array_equal(Qd == 0.0, Qk == 0.0)


def _paper_patterns(n):
    """Sparsity pattern of Algorithm 1 (3D), restated: for every (i, j, k, l)
    with l the position along the active direction, the row is the node
    (i, j, k) in z, y, x order and the x/y/z columns replace k/j/i by l."""
    i, j, k, l = np.meshgrid(*([np.arange(n)] * 4), indexing="ij")
    i, j, k, l = (t.ravel() for t in (i, j, k, l))
    row = i * n * n + j * n + k
    cols = [i * n * n + j * n + l, i * n * n + l * n + k, l * n * n + j * n + k]
    return row, cols


@pytest.mark.parametrize("kind", [GLL, GAUSS])
@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_algorithms_1_2_index_maps(kind, p):
    """Algorithm 2's entries, built from Algorithm 1's pattern, are exactly the
    nonzeros of the dense Q_m (Eq. 5 with 'basis' read as Q1 = W D, whose
    row weight supplies the W of the active direction)."""
    n = p + 1
    _, w, _, Q1 = O.op1d(p, kind)
    row, cols = _paper_patterns(n)
    counter = np.tile(np.arange(n), n ** 3)
    for m in range(3):
        Qd = O.qmat_dense(3, p, kind, m)
        col = cols[m]
        # 1D indices recovered from the flat indices with % and // (Algorithm 2)
        xr, yr, zr = row % n, (row // n) % n, row // (n * n)
        xc, yc, zc = col % n, (col // n) % n, col // (n * n)
        act_r, act_c = [(xr, xc), (yr, yc), (zr, zc)][m]
        others = [t for q, t in enumerate((xr, yr, zr)) if q != m]
        sparse = np.zeros((n ** 3, n))
        sparse[row, counter] = Q1[act_r, act_c] * w[others[0]] * w[others[1]]
        # same entries as the dense operator at (row, col) ...
        np.testing.assert_allclose(sparse[row, counter], Qd[row, col], rtol=1e-15, atol=0)
        # ... and nothing of the dense operator lies outside the pattern
        mask = np.zeros_like(Qd, dtype=bool)
        mask[row, col] = True
        assert np.all(Qd[~mask] == 0.0)
        # n^{d+1} stored entries instead of n^{2d} (Theorem 2.1)
        assert sparse.size == n ** 4
