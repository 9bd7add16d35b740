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


def fp32_check(got, ref, ref_w, kappa_fn=None, global_bar=2e-5):
    """The FP32 bars.  (1) 2e-5 (global_bar) in the relative max norm of the
    residual vector (callers with a derived global bar check it themselves).  (2) Per variable, the largest of
      2e-5;
      6 x that variable's input-rounding floor (ref_w = oracle on the
        FP32-rounded state): FP32 arithmetic moves each node's primitives and
        each pair's flux by at most ~3 ulp, six times the half-ulp rounding;
      2.5 u32 kappa_v, u32 = 2^-24, kappa_v = max_i sum_{m,j} |Q_m,ij F_m,ij,v|
        / max_i |r_i,v| (the sum the residual cancels over its size), the
        worst-case rounding bound of the sums (kappa_fn() computes it, only
        when the first two bounds are not met).
    Returns the measured errors and the bars used."""
    g = rel_err_global(got, ref)
    pv = rel_err_vars(got, ref)
    floor = rel_err_vars(ref_w, ref)
    bar = np.maximum(2e-5, 6.0 * floor)
    if np.any(pv > bar) and kappa_fn is not None:
        bar = np.maximum(bar, 2.5 * 2.0 ** -24 * np.asarray(kappa_fn()))
    assert g <= global_bar, ("global", g)
    assert np.all(pv <= bar), ("per-variable", pv, bar)
    return {"global": float(g), "per_variable": pv.tolist(), "input_floor": floor.tolist(), "bar": bar.tolist()}


def have_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
