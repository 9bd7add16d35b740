"""Shared helpers for the tests (no arithmetic of the method lives here)."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sfhad.h")


def header_functions():
    """Names of every function the public header declares."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sfh_[a-z0-9_]+)\s*\(", src)))


def rel_err_per_var(got, ref):
    """max_{e,i} |got - ref| / max_{e,i} |ref| for every variable; returns the worst
    variable's value (the error norm of the parity bars)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    worst = 0.0
    for v in range(ref.shape[1]):
        den = np.abs(ref[:, v]).max()
        num = np.abs(got[:, v] - ref[:, v]).max()
        worst = max(worst, num / den if den > 0 else num)
    return worst


def rel_err_global(got, ref):
    """max |got - ref| / max |ref| over the whole residual vector (all
    variables): the relative max norm of the FP32 bar."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(got - ref).max() / np.abs(ref).max()


def rel_err_vars(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.array([np.abs(got[:, v] - ref[:, v]).max() / max(np.abs(ref[:, v]).max(), 1e-300)
                     for v in range(ref.shape[1])])


# The FP32 kernels' own arithmetic error, node by node: |r_gpu - r_w| <=
# C_ARITH * 2^-24 * S with r_w the oracle on the FP32-rounded state and S the
# sum of the absolute terms (oracle volume_absterms).  Each term carries a few
# FP32 roundings (primitives, two logarithmic means, the flux products, the
# compensated row sum), hence a small multiple of the unit roundoff of the
# terms' magnitude; 32 leaves room for the terms whose own parts cancel.
C_ARITH = 32.0


def fp32_check(got, ref, ref_w, kappa_fn=None, global_bar=2e-5, terms=None, c_arith=C_ARITH, arith_per_node=True):
    """The FP32 bars.  (1) 2e-5 (global_bar) in the relative max norm of the
    residual vector (callers with a derived global bar check it themselves).  (2) Per variable, the largest of
      2e-5;
      6 x that variable's input-rounding floor (ref_w = oracle on the
        FP32-rounded state): FP32 arithmetic moves each node's primitives and
        each pair's flux by at most ~3 ulp, six times the half-ulp rounding;
      2.5 u32 kappa_v, u32 = 2^-24, kappa_v = max_i sum_{m,j} |Q_m,ij F_m,ij,v|
        / max_i |r_i,v| (the sum the residual cancels over its size), the
        worst-case rounding bound of the sums (from `terms` when given, else
        kappa_fn() when the first two bounds are not met).
    (3) With `terms` (S, the oracle's absolute terms of the same entries): the
    arithmetic error alone, |got - ref_w| <= c_arith u32 S node by node (or,
    arith_per_node=False, per variable in the max norm: max|got - ref_w|_v <=
    c_arith u32 kappa_v max|ref_v|).
    Returns the measured errors, kappa_v and the bars used."""
    u32 = 2.0 ** -24
    g = rel_err_global(got, ref)
    pv = rel_err_vars(got, ref)
    floor = rel_err_vars(ref_w, ref)
    bar = np.maximum(2e-5, 6.0 * floor)
    kap = None
    if terms is not None:
        S = np.asarray(terms, dtype=np.float64)
        ref64 = np.asarray(ref, dtype=np.float64)
        kap = np.array([S[:, v].max() / max(np.abs(ref64[:, v]).max(), 1e-300) for v in range(ref64.shape[1])])
    elif np.any(pv > bar) and kappa_fn is not None:
        kap = np.asarray(kappa_fn())
    if kap is not None and np.any(pv > bar):
        bar = np.maximum(bar, 2.5 * u32 * kap)
    out = {"global": float(g), "per_variable": pv.tolist(), "input_floor": floor.tolist(), "bar": bar.tolist(),
           "kappa": None if kap is None else kap.tolist()}
    if terms is not None:
        dev = np.abs(np.asarray(got, dtype=np.float64) - np.asarray(ref_w, dtype=np.float64))
        if arith_per_node:
            ratio = dev / (u32 * np.maximum(S, 1e-300))
            out["arith_ratio_per_variable"] = [float(ratio[:, v].max()) for v in range(ratio.shape[1])]
        else:
            out["arith_ratio_per_variable"] = [float(dev[:, v].max() / (u32 * kap[v] * np.abs(ref64[:, v]).max()))
                                               for v in range(dev.shape[1])]
        out["arith_ratio_max"] = max(out["arith_ratio_per_variable"])
        out["arith_norm"] = "node" if arith_per_node else "variable"
        out["arith_bar"] = c_arith
        assert out["arith_ratio_max"] <= c_arith, ("arithmetic", out["arith_ratio_per_variable"])
    assert g <= global_bar, ("global", g)
    assert np.all(pv <= bar), ("per-variable", pv, bar)
    return out


def have_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
