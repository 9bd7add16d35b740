"""FP64 CPU oracle for the sum-factorized Hadamard-product volume term.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product library never does, and the two share no code: the oracle computes
its own nodes, derivative matrix, fluxes and metric terms (``sfh_oracle.c``).

The C source is compiled with gcc (no fast-math) into ``oracle/_build`` on
first use; ``build()`` forces it.  Arrays are numpy float64, C-contiguous,
with the layouts documented in ``sfh_oracle.c``:
``u[e][var][i]``, ``Ja[e][m][k][i]``, ``x[e][k][i]``, nodes x fastest.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfh_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libsfh_oracle.so")

NODES_GLL = 0
NODES_GAUSS = 1
FLUX_BURGERS = 0
FLUX_EULER = 1
FLUX_CHANDRASHEKAR = 2
GAMMA = 1.4

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libsfh_oracle.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        i, L = ctypes.c_int, ctypes.c_long
        lib.orc_nodes.argtypes = [i, i, dp, dp]
        lib.orc_dmat.argtypes = [i, dp, dp]
        lib.orc_dmat.restype = None
        lib.orc_op1d.argtypes = [i, i, dp, dp, dp, dp]
        lib.orc_qmat_dense.argtypes = [i, i, i, i, dp]
        lib.orc_logmean.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.orc_logmean.restype = ctypes.c_double
        lib.orc_logmean_grad.argtypes = [ctypes.c_double, ctypes.c_double, dp, dp]
        lib.orc_logmean_grad.restype = None
        lib.orc_ec_flux.argtypes = [i, i, dp, dp, dp, dp]
        lib.orc_ec_flux_jac1.argtypes = [i, i, dp, dp, dp, dp]
        for name in ("orc_volume_sf", "orc_volume_dense", "orc_volume_absterms"):
            getattr(lib, name).argtypes = [i, i, i, i, i, L, dp, dp, dp]
        for name in ("orc_vjp_sf", "orc_vjp_dense"):
            getattr(lib, name).argtypes = [i, i, i, i, i, L, dp, dp, dp, dp]
        lib.orc_mesh.argtypes = [i, i, i, i, ctypes.c_double, dp, dp]
        lib.orc_fig1_dense.argtypes = [i, dp, dp]
        lib.orc_fig1_sf.argtypes = [i, dp, dp]
        lib.orc_basis_1d.argtypes = [i, i, i, dp]
        lib.orc_modal_states.argtypes = [i, i, i, i, i, i, L, dp, dp, dp]
        lib.orc_volume_modal.argtypes = [i, i, i, i, i, i, i, L, dp, dp, dp]
        lib.orc_vjp_modal.argtypes = [i, i, i, i, i, i, L, dp, dp, dp, dp]
        lib.orc_surface_dense.argtypes = [i, i, i, i, i, L, dp, dp, dp, dp, dp]
        lib.orc_surface_vjp_dense.argtypes = [i, i, i, i, i, L, dp, dp, dp, dp, dp, dp, dp]
        lib.orc_entropy_vars.argtypes = [i, i, dp, dp]
        lib.orc_entropy_state.argtypes = [i, i, dp, dp]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleDomainError(ValueError):
    """Raised when a state has non-positive density or pressure."""


def _check(rc: int, allow_domain: bool = False):
    if rc == 1:
        raise ValueError("oracle: bad argument")
    if rc == 2 and not allow_domain:
        raise OracleDomainError("oracle: non-positive density or pressure")


def nvar_of(d: int, flux: int) -> int:
    return 1 if flux == FLUX_BURGERS else d + 2


def op1d(p: int, kind: int):
    """(xi, w, D, Q1) of the collocated 1D basis on n = p+1 nodes."""
    n = p + 1
    xi, w = np.zeros(n), np.zeros(n)
    D, Q1 = np.zeros((n, n)), np.zeros((n, n))
    _check(_load().orc_op1d(p, kind, _p(xi), _p(w), _p(D), _p(Q1)))
    return xi, w, D, Q1


def qmat_dense(d: int, p: int, kind: int, m: int) -> np.ndarray:
    nn = (p + 1) ** d
    Q = np.zeros((nn, nn))
    _check(_load().orc_qmat_dense(d, p, kind, m, _p(Q)))
    return Q


def logmean(a: float, b: float) -> float:
    return _load().orc_logmean(float(a), float(b))


def logmean_grad(a: float, b: float):
    da, db = ctypes.c_double(), ctypes.c_double()
    _load().orc_logmean_grad(float(a), float(b), ctypes.byref(da), ctypes.byref(db))
    return da.value, db.value


def ec_flux(d: int, flux: int, ui, uj, nv) -> np.ndarray:
    ui, uj, nv = _f64(ui), _f64(uj), _f64(nv)
    F = np.zeros(nvar_of(d, flux))
    _check(_load().orc_ec_flux(d, flux, _p(ui), _p(uj), _p(nv), _p(F)))
    return F


def ec_flux_jac1(d: int, flux: int, ui, uj, nv) -> np.ndarray:
    ui, uj, nv = _f64(ui), _f64(uj), _f64(nv)
    nvar = nvar_of(d, flux)
    J = np.zeros((nvar, nvar))
    _check(_load().orc_ec_flux_jac1(d, flux, _p(ui), _p(uj), _p(nv), _p(J)))
    return J


def _volume(fn, d, p, kind, flux, u, Ja, allow_domain=False):
    u, Ja = _f64(u), _f64(Ja)
    n_elem = u.shape[0]
    nvar = nvar_of(d, flux)
    nn = (p + 1) ** d
    assert u.shape == (n_elem, nvar, nn), u.shape
    assert Ja.shape == (n_elem, d, d, nn), Ja.shape
    r = np.zeros_like(u)
    _check(fn(d, p, kind, nvar, flux, n_elem, _p(u), _p(Ja), _p(r)), allow_domain)
    return r


def volume_sf(d, p, kind, flux, u, Ja, allow_domain=False) -> np.ndarray:
    """Sum-factorized residual r[e][var][i] (Eq. 3 with the Eq. 5 operators)."""
    return _volume(_load().orc_volume_sf, d, p, kind, flux, u, Ja, allow_domain)


def volume_absterms(d, p, kind, flux, u, Ja) -> np.ndarray:
    """S[e][var][i] = sum_m sum_j |Q_m,ij F_m,ij,var| (the terms of Eq. 3 with
    the Eq. 5 operators in absolute value): the magnitude each residual entry
    cancels from, the scale of its rounding errors in floating point."""
    return _volume(_load().orc_volume_absterms, d, p, kind, flux, u, Ja)


def volume_dense(d, p, kind, flux, u, Ja) -> np.ndarray:
    """Dense O(n^{2d}) residual (Eq. 1 with the full Kronecker operators)."""
    return _volume(_load().orc_volume_dense, d, p, kind, flux, u, Ja)


def _vjp(fn, d, p, kind, flux, u, Ja, lam):
    u, Ja, lam = _f64(u), _f64(Ja), _f64(lam)
    assert lam.shape == u.shape
    g = np.zeros_like(u)
    _check(fn(d, p, kind, nvar_of(d, flux), flux, u.shape[0], _p(u), _p(Ja), _p(lam), _p(g)))
    return g


def vjp_sf(d, p, kind, flux, u, Ja, lam) -> np.ndarray:
    """g = (dr/du)^T lambda, line by line with the analytic flux Jacobian."""
    return _vjp(_load().orc_vjp_sf, d, p, kind, flux, u, Ja, lam)


def vjp_dense(d, p, kind, flux, u, Ja, lam) -> np.ndarray:
    """g from the assembled dense element Jacobian of the Eq. 1 form."""
    return _vjp(_load().orc_vjp_dense, d, p, kind, flux, u, Ja, lam)


def mesh(d: int, p: int, kind: int, N: int, amp: float):
    """Warped mesh on [0,1]^d: node coordinates x[e][k][i] and metrics Ja[e][m][k][i]."""
    nn = (p + 1) ** d
    n_elem = N ** d
    x = np.zeros((n_elem, d, nn))
    Ja = np.zeros((n_elem, d, d, nn))
    _check(_load().orc_mesh(d, p, kind, N, float(amp), _p(x), _p(Ja)))
    return x, Ja


def fig1_dense(p: int, c) -> np.ndarray:
    c = _f64(c)
    y = np.zeros_like(c)
    _check(_load().orc_fig1_dense(p, _p(c), _p(y)))
    return y


def fig1_sf(p: int, c) -> np.ndarray:
    c = _f64(c)
    y = np.zeros_like(c)
    _check(_load().orc_fig1_sf(p, _p(c), _p(y)))
    return y


BASIS_LEGENDRE, BASIS_LAGRANGE_GLL, BASIS_LAGRANGE_GAUSS = 0, 1, 2


def basis_1d(p: int, kind: int, basis: int) -> np.ndarray:
    """V1[a, k] = chi_k(xi_a) on the cubature nodes of ``kind``."""
    n = p + 1
    V = np.zeros((n, n))
    _check(_load().orc_basis_1d(p, kind, basis, _p(V)))
    return V


def modal_states(d, p, kind, basis, flux, uhat, allow_domain=False):
    """(u_v, u~): nodal values V u_hat and the entropy-projected state."""
    uhat = _f64(uhat)
    nvar = nvar_of(d, flux)
    assert uhat.shape[1:] == (nvar, (p + 1) ** d), uhat.shape
    uv, up = np.zeros_like(uhat), np.zeros_like(uhat)
    _check(_load().orc_modal_states(d, p, kind, basis, nvar, flux, uhat.shape[0], _p(uhat), _p(uv), _p(up)),
           allow_domain)
    return uv, up


def volume_modal(d, p, kind, basis, flux, uhat, Ja, allow_domain=False, project=True) -> np.ndarray:
    """Modal volume residual r_hat = V^T r_v(u~) (dense transforms, literal
    entropy projection; project=False evaluates the flux at u_v = V u_hat)."""
    uhat, Ja = _f64(uhat), _f64(Ja)
    nvar = nvar_of(d, flux)
    assert uhat.shape[1:] == (nvar, (p + 1) ** d) and Ja.shape[0] == uhat.shape[0]
    r = np.zeros_like(uhat)
    _check(_load().orc_volume_modal(d, p, kind, basis, nvar, flux, int(bool(project)), uhat.shape[0], _p(uhat),
                                    _p(Ja), _p(r)), allow_domain)
    return r


def entropy_vars(d: int, flux: int, u) -> np.ndarray:
    """Entropy variables w(u) of one state (Burgers: u)."""
    u = _f64(u)
    w = np.zeros_like(u)
    _check(_load().orc_entropy_vars(d, flux, _p(u), _p(w)))
    return w


def entropy_state(d: int, flux: int, w) -> np.ndarray:
    """Conservative state u(w) of one vector of entropy variables."""
    w = _f64(w)
    u = np.zeros_like(w)
    _check(_load().orc_entropy_state(d, flux, _p(w), _p(u)))
    return u


def vjp_modal(d, p, kind, basis, flux, uhat, Ja, lamhat) -> np.ndarray:
    """g_hat = V^T (dr_v/du_v)^T V lambda_hat, the VJP of the modal residual."""
    uhat, Ja, lamhat = _f64(uhat), _f64(Ja), _f64(lamhat)
    assert lamhat.shape == uhat.shape
    g = np.zeros_like(uhat)
    _check(_load().orc_vjp_modal(d, p, kind, basis, nvar_of(d, flux), flux, uhat.shape[0], _p(uhat), _p(Ja),
                                 _p(lamhat), _p(g)))
    return g


def surface_dense(d, p, kind, flux, u, u_face, nJ):
    """(r_vol, r_face) of the dense surface Hadamard product (B E) o C of each
    element's 2d faces; u_face [E][2d][nvar][n^(d-1)], nJ [E][2d][d][n^(d-1)]."""
    u, u_face, nJ = _f64(u), _f64(u_face), _f64(nJ)
    nvar = nvar_of(d, flux)
    E, nf = u.shape[0], (p + 1) ** (d - 1)
    assert u.shape == (E, nvar, (p + 1) ** d) and u_face.shape == (E, 2 * d, nvar, nf) and nJ.shape == (E, 2 * d, d, nf)
    rv, rf = np.zeros_like(u), np.zeros_like(u_face)
    _check(_load().orc_surface_dense(d, p, kind, nvar, flux, E, _p(u), _p(u_face), _p(nJ), _p(rv), _p(rf)))
    return rv, rf


def surface_vjp_dense(d, p, kind, flux, u, u_face, nJ, lam_vol, lam_face):
    """(g_u, g_face): the gradients of lam_vol . r_vol + lam_face . r_face of
    surface_dense with respect to u and u_face (reverse mode of Remark 1's
    surface operator, every (f, j) pair with the flux Jacobian)."""
    u, u_face, nJ, lam_vol, lam_face = _f64(u), _f64(u_face), _f64(nJ), _f64(lam_vol), _f64(lam_face)
    nvar = nvar_of(d, flux)
    E, nf = u.shape[0], (p + 1) ** (d - 1)
    assert u.shape == (E, nvar, (p + 1) ** d) and u_face.shape == (E, 2 * d, nvar, nf) and nJ.shape == (E, 2 * d, d, nf)
    assert lam_vol.shape == u.shape and lam_face.shape == u_face.shape
    gu, gf = np.zeros_like(u), np.zeros_like(u_face)
    _check(_load().orc_surface_vjp_dense(d, p, kind, nvar, flux, E, _p(u), _p(u_face), _p(nJ), _p(lam_vol),
                                         _p(lam_face), _p(gu), _p(gf)))
    return gu, gf
