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


def have_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
