"""Entropy identity of the volume term, evaluated in FP64 with the oracle's flux.

For r = sum_m (Q_m o F_m) 1 with Q_m 1 = 0 and an entropy-conservative,
symmetric F (Tadmor's condition (w_i - w_j).F_ij = (psi_i - psi_j).(J_i + J_j)):
  w^T r = sum_m [ 1/2 sum_ij E_ij w_i.F_ij - 1/2 sum_i (E 1)_i psi_i.J_i
                 - 1/2 psi^T E J + psi^T Q J ],   E = Q_m + Q_m^T, J = Ja^m.
Returns (lhs - rhs) / scale with scale = sum_m sum_ij |Q_ij| |w_i . F_ij|.
"""
import numpy as np

import oracle as O

G = O.GAMMA


def kron_q(d, p, kind, m):
    _, w, _, Q1 = O.op1d(p, kind)
    W = np.diag(w)
    fac = [Q1 if k == m else W for k in range(d)]
    out = fac[d - 1]
    for k in range(d - 2, -1, -1):
        out = np.kron(out, fac[k])
    return out


def entropy_vars(ue, d, flux):
    if flux == O.FLUX_BURGERS:
        return ue.copy(), np.repeat(ue[0:1] ** 3 / 6.0, d, axis=0)
    rho = ue[0]
    v = ue[1:1 + d] / rho
    p = (G - 1) * (ue[d + 1] - 0.5 * rho * (v * v).sum(0))
    s = np.log(p) - G * np.log(rho)
    w = np.concatenate([[(G - s) / (G - 1) - 0.5 * rho * (v * v).sum(0) / p], rho * v / p, [-rho / p]])
    return w, rho * v


def identity_residual(d, p, kind, flux, ue, Je, re):
    """Relative defect of the entropy identity for one element (u FP64 state,
    r the residual under test)."""
    nn = (p + 1) ** d
    w, psi = entropy_vars(ue, d, flux)
    lhs = float(np.sum(w * re))
    ones = np.ones(nn)
    rhs, scale = 0.0, 0.0
    for m in range(d):
        Q = kron_q(d, p, kind, m)
        E = Q + Q.T
        J = Je[m]
        t1 = 0.0
        rows, cols = np.nonzero(Q)
        for i, j in zip(rows, cols):
            F = O.ec_flux(d, flux, ue[:, i], ue[:, j], J[:, i] + J[:, j])
            wf = w[:, i] @ F
            if E[i, j] != 0.0:
                t1 += E[i, j] * wf
            scale += abs(Q[i, j]) * np.abs(w[:, i] * F).sum()
        psiJ = (psi * J).sum(0)
        rhs += 0.5 * t1 - 0.5 * ((E @ ones) * psiJ).sum() \
            - 0.5 * np.einsum("ki,ij,kj->", psi, E, J) + np.einsum("ki,ij,kj->", psi, Q, J)
    return abs(lhs - rhs) / scale
