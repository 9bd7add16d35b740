"""Seeded synthetic inputs: warped meshes, metric terms, states, cotangents.

This module only manufactures inputs.  It holds none of the volume-term
arithmetic (no two-point flux, no Hadamard product, no operator table used by
the kernels); it serves the tests, the smoke check and the benchmark alike.
Mesh geometry needs a node set and a collocation derivative to build discrete
metric terms; these are taken from numpy's Legendre routines and a plain
barycentric formula here, independently of both the CUDA library's tables and
the oracle's.

Recipe (the paper runs its timing on a warped periodic cube, Section 3):
  * Elements of [0,1]^d, N per direction, element e = ex + N ey + N^2 ez.
  * Nodes x_k = (e_k + (xi_{a_k} + 1)/2) / N, x fastest inside an element.
  * Warp: every axis is shifted by the same scalar amp * prod_l sin(pi x_l)
    (amp = 0.1); the shift vanishes on the faces of the cube, so states
    built from integer wavenumbers stay periodic.
  * Metric terms Ja[e][m][k][i] = J dxi_m/dx_k from the degree-p interpolant:
    2D (y_eta, -x_eta), (-y_xi, x_xi); 3D Kopriva's conservative curl form.
  * Euler states: rho = 1 + 0.2 g_rho, v_k = 0.3 g_vk, p = 1 + 0.2 g_p with
    g(x) = 1/4 sum_{q=1..4} sin(2 pi kappa_q . x + phi_q),
    kappa_q uniform in {-2..2}^d minus 0, phi_q ~ U[0, 2 pi), each field its
    own PCG64 stream (seeds 2, 3.., 3+d); then conservative variables.
  * Burgers states: u = sin(2 pi x) sin(2 pi y) + 0.1 N(0,1), seed 1.
  * Cotangents: N(0,1), seed 8.
  * Surface inputs: on each face (m, side) of an element the facet
    cubature points (xi_m = -1 or +1, the 1D nodes in the other directions,
    lower axis fastest) are mapped by the same warped map; the face state is
    the same state recipe at those points, the face normal the adjugate of
    the map's exact Jacobian there, row m, times -1 (side 0) or +1 (side 1).
  * Modal inputs (solution in a basis chi, integrated on the cubature nodes of
    `kind`): for a Lagrange basis on Gauss-Lobatto or Gauss nodes the
    coefficients are the state above at those solution nodes; for the
    orthonormal Legendre basis, mode 0 carries the mean state (rho = 1,
    v = (0.3, -0.2, 0.1), p = 1; Burgers 0.5) times 2^(d/2) (the constant
    mode's value is 2^(-d/2)) and every mode k of every variable adds
    0.04 N(0,1) / (1 + |k|_1)^2 (PCG64 seed 12); Ja is the mesh's metric on
    the cubature nodes.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 1.4
NODES_GLL = 0
NODES_GAUSS = 1


def nodes_1d(p: int, kind: int):
    """Nodes (ascending) and weights on [-1, 1] for n = p + 1 points."""
    n = p + 1
    L = np.polynomial.legendre
    if kind == NODES_GAUSS:
        xi, w = L.leggauss(n)
        return np.asarray(xi, dtype=np.float64), np.asarray(w, dtype=np.float64)
    if p < 1:
        raise ValueError("Gauss-Lobatto needs p >= 1")
    cp = np.zeros(p + 1)
    cp[p] = 1.0
    dcp = L.legder(cp)
    inner = np.sort(np.real(L.legroots(dcp))) if p > 1 else np.zeros(0)
    d2cp = L.legder(dcp)
    for _ in range(3):  # Newton polish of the library roots
        if inner.size:
            inner = inner - L.legval(inner, dcp) / L.legval(inner, d2cp)
    xi = np.concatenate(([-1.0], inner, [1.0]))
    w = 2.0 / (p * (p + 1) * L.legval(xi, cp) ** 2)
    return xi, w


def dmat_1d(xi: np.ndarray) -> np.ndarray:
    """Collocation derivative on the nodes xi (barycentric form)."""
    n = xi.size
    diff = xi[:, None] - xi[None, :]
    np.fill_diagonal(diff, 1.0)
    lam = 1.0 / np.prod(diff, axis=1)
    D = (lam[None, :] / lam[:, None]) / diff
    np.fill_diagonal(D, 0.0)
    np.fill_diagonal(D, -D.sum(axis=1))
    return D


def _deriv(f: np.ndarray, D: np.ndarray, d: int, n: int, j: int) -> np.ndarray:
    """Derivative along reference direction j of nodal fields f[E, n^d]."""
    E = f.shape[0]
    g = f.reshape((E,) + (n,) * d)   # axes: e, a_{d-1}, ..., a_0
    ax = d - j
    out = np.tensordot(g, D, axes=([ax], [1]))   # new axis appended last
    out = np.moveaxis(out, -1, ax)
    return out.reshape(E, n ** d)


def mesh(d: int, p: int, kind: int, N: int, amp: float = 0.1, n_elem: int | None = None):
    """Warped mesh of N^d elements (or its first n_elem elements).

    Returns x[e][k][i] and Ja[e][m][k][i] (float64, C-contiguous)."""
    n = p + 1
    nn = n ** d
    total = N ** d
    E = total if n_elem is None else int(n_elem)
    if E > total:
        raise ValueError("n_elem exceeds N^d")
    xi, _ = nodes_1d(p, kind)
    D = dmat_1d(xi)
    s = 0.5 * (xi + 1.0)
    e = np.arange(E)
    ek = [(e // N ** k) % N for k in range(d)]
    i = np.arange(nn)
    ak = [(i // n ** k) % n for k in range(d)]
    x0 = [(ek[k][:, None] + s[ak[k]][None, :]) / N for k in range(d)]
    shift = amp * np.ones((E, nn))
    for k in range(d):
        shift = shift * np.sin(math.pi * x0[k])
    x = np.stack([x0[k] + shift for k in range(d)], axis=1)
    del x0, shift
    dX = [[_deriv(x[:, k], D, d, n, j) for j in range(d)] for k in range(d)]  # dX[k][j] = dx_k/dxi_j
    Ja = np.empty((E, d, d, nn))
    if d == 2:
        Ja[:, 0, 0] = dX[1][1]
        Ja[:, 0, 1] = -dX[0][1]
        Ja[:, 1, 0] = -dX[1][0]
        Ja[:, 1, 1] = dX[0][0]
    else:
        for nc in range(3):
            mc, lc = (nc + 1) % 3, (nc + 2) % 3
            V = [x[:, lc] * dX[mc][j] for j in range(3)]
            for ic in range(3):
                jc, kc = (ic + 1) % 3, (ic + 2) % 3
                Ja[:, ic, nc] = -(_deriv(V[kc], D, 3, n, jc) - _deriv(V[jc], D, 3, n, kc))
    return np.ascontiguousarray(x), Ja


def random_fourier(x: np.ndarray, seed: int, modes: int = 4) -> np.ndarray:
    """g(x) = 1/4 sum_q sin(2 pi kappa_q . x + phi_q) on nodes x[e][k][i]."""
    rng = np.random.default_rng(seed)
    d = x.shape[1]
    g = np.zeros(x.shape[0:1] + x.shape[2:])
    for _ in range(modes):
        while True:
            kappa = rng.integers(-2, 3, size=d)
            if np.any(kappa != 0):
                break
        phi = rng.uniform(0.0, 2.0 * math.pi)
        arg = phi + sum(2.0 * math.pi * float(kappa[k]) * x[:, k] for k in range(d))
        g += np.sin(arg)
    return 0.25 * g


def euler_primitives(x: np.ndarray, seed0: int = 2):
    d = x.shape[1]
    rho = 1.0 + 0.2 * random_fourier(x, seed0)
    v = [0.3 * random_fourier(x, seed0 + 1 + k) for k in range(d)]
    p = 1.0 + 0.2 * random_fourier(x, seed0 + 1 + d)
    return rho, v, p


def conservative(rho, v, p) -> np.ndarray:
    d = len(v)
    ke = sum(vk * vk for vk in v)
    u = np.empty((rho.shape[0], d + 2) + rho.shape[1:])
    u[:, 0] = rho
    for k in range(d):
        u[:, 1 + k] = rho * v[k]
    u[:, d + 1] = p / (GAMMA - 1.0) + 0.5 * rho * ke
    return u


def euler_state(x: np.ndarray, seed0: int = 2) -> np.ndarray:
    """Conservative Euler state u[e][var][i] from the random-Fourier recipe."""
    return conservative(*euler_primitives(x, seed0))


def burgers_state(x: np.ndarray, seed: int = 1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    base = np.sin(2 * math.pi * x[:, 0]) * np.sin(2 * math.pi * x[:, 1])
    return (base + 0.1 * rng.standard_normal(base.shape))[:, None, :]


def constant_state(E: int, d: int, nn: int, rho=1.0, v=(0.3, -0.2, 0.1), p=1.0) -> np.ndarray:
    vv = [np.full((E, nn), v[k]) for k in range(d)]
    return conservative(np.full((E, nn), rho), vv, np.full((E, nn), p))


def cotangent(shape, seed: int = 8) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape)


def to_fp32(u: np.ndarray) -> np.ndarray:
    """Round to nearest FP32 (the FP32 precision modes' input)."""
    return np.ascontiguousarray(u, dtype=np.float32)


def workload(d: int, p: int, kind: int, N: int, flux: str = "euler", amp: float = 0.1,
             n_elem: int | None = None, seed0: int | None = None):
    """(u, Ja) of a named workload shape: warped mesh + state."""
    x, Ja = mesh(d, p, kind, N, amp, n_elem)
    if flux == "burgers":
        u = burgers_state(x, 1 if seed0 is None else seed0)
    else:
        u = euler_state(x, 2 if seed0 is None else seed0)
    return np.ascontiguousarray(u), Ja


BASIS_LEGENDRE, BASIS_LAGRANGE_GLL, BASIS_LAGRANGE_GAUSS = 0, 1, 2


def modal_workload(d: int, p: int, kind: int, basis: int, N: int, flux: str = "euler", amp: float = 0.1,
                   n_elem: int | None = None, seed: int = 12):
    """(u_hat, Ja) of a modal workload: coefficients in the basis, metrics on
    the cubature nodes of ``kind`` (recipe in the module docstring)."""
    _, Ja = mesh(d, p, kind, N, amp, n_elem)
    if basis in (BASIS_LAGRANGE_GLL, BASIS_LAGRANGE_GAUSS):
        sol = NODES_GLL if basis == BASIS_LAGRANGE_GLL else NODES_GAUSS
        uhat, _ = workload(d, p, sol, N, flux, amp, n_elem)
        return uhat, Ja
    if basis != BASIS_LEGENDRE:
        raise ValueError(f"unknown basis {basis}")
    return legendre_coefficients(d, p, Ja.shape[0], flux, seed), Ja


def legendre_coefficients(d: int, p: int, E: int, flux: str = "euler", seed: int = 12) -> np.ndarray:
    """u_hat[e][var][k] of the orthonormal Legendre recipe (module docstring)."""
    n = p + 1
    nn = n ** d
    if flux == "burgers":
        mean = np.array([0.5])
    else:
        v = np.array([0.3, -0.2, 0.1][:d])
        mean = np.concatenate(([1.0], v, [1.0 / (GAMMA - 1.0) + 0.5 * (v @ v)]))
    kk = np.zeros(nn)
    for i in range(nn):
        a, r = 0, i
        for _ in range(d):
            a += r % n
            r //= n
        kk[i] = a
    rng = np.random.Generator(np.random.PCG64(seed))
    uhat = 0.04 * rng.standard_normal((E, mean.size, nn)) / (1.0 + kk) ** 2
    uhat[:, :, 0] += mean * 2.0 ** (d / 2.0)
    return np.ascontiguousarray(uhat)


def surface_workload(d: int, p: int, kind: int, N: int, flux: str = "euler", amp: float = 0.1,
                     n_elem: int | None = None):
    """(u, u_face, nJ): the volume state of ``workload``, face states
    u_face[e][face][var][f] and face normals nJ[e][face][k][f], face = 2 m + side
    (recipe in the module docstring)."""
    u, _ = workload(d, p, kind, N, flux, amp, n_elem)
    n = p + 1
    nf = n ** (d - 1)
    E = u.shape[0]
    xi, _ = nodes_1d(p, kind)
    e = np.arange(E)
    ek = [(e // N ** k) % N for k in range(d)]
    f = np.arange(nf)
    bf = [(f // n ** k) % n for k in range(d - 1)]
    X = np.empty((E, 2 * d, d, nf))     # affine coordinates of the face points
    for m in range(d):
        others = [k for k in range(d) if k != m]
        for side in range(2):
            for k in range(d):
                xk = np.full(nf, 1.0 if side else -1.0) if k == m else xi[bf[others.index(k)]]
                X[:, 2 * m + side, k] = (ek[k][:, None] + 0.5 * (xk[None, :] + 1.0)) / N
    S = np.sin(math.pi * X)
    C = np.cos(math.pi * X)
    shift = amp * np.prod(S, axis=2)                      # [E][face][f]
    x = X + shift[:, :, None, :]
    # dx_k/dxi_j = (delta_kj + amp pi cos(pi X_j) prod_{l != j} sin(pi X_l)) / (2N)
    A = np.empty((E, 2 * d, d, d, nf))
    for j in range(d):
        dj = amp * math.pi * C[:, :, j] * np.prod(np.delete(S, j, axis=2), axis=2)
        for k in range(d):
            A[:, :, k, j] = ((1.0 if k == j else 0.0) + dj) / (2.0 * N)
    adj = np.empty_like(A)                                   # adj[m][k] = J dxi_m/dx_k
    if d == 2:
        adj[:, :, 0, 0] = A[:, :, 1, 1]
        adj[:, :, 0, 1] = -A[:, :, 0, 1]
        adj[:, :, 1, 0] = -A[:, :, 1, 0]
        adj[:, :, 1, 1] = A[:, :, 0, 0]
    else:
        for m in range(3):
            for k in range(3):
                r = [q for q in range(3) if q != k]
                c = [q for q in range(3) if q != m]
                minor = A[:, :, r[0], c[0]] * A[:, :, r[1], c[1]] - A[:, :, r[0], c[1]] * A[:, :, r[1], c[0]]
                adj[:, :, m, k] = (-1.0) ** (m + k) * minor
    nJ = np.empty((E, 2 * d, d, nf))
    for m in range(d):
        for side in range(2):
            nJ[:, 2 * m + side] = (1.0 if side else -1.0) * adj[:, 2 * m + side, m]
    xf = x.reshape(E * 2 * d, d, nf)
    if flux == "burgers":
        uf = burgers_state(xf, 13)
    else:
        uf = euler_state(xf, 2)
    u_face = np.ascontiguousarray(uf.reshape(E, 2 * d, -1, nf))
    return u, u_face, np.ascontiguousarray(nJ)
