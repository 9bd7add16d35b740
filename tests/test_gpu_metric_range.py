"""Metric terms outside the accepted range are reported, not silently used.

The FP32 modes convert the FP64 metric terms to FP32 by integer field
arithmetic, which would turn Inf, NaN or a magnitude >= 2^128 into a finite
wrong value.  Every kernel therefore checks the range (FP32 modes: finite and
|Ja| < 2^126; FP64: finite) and latches SFH_EDOMAIN; the other elements'
results stay correct, and the next clean call is clean again.  The bad values
are plain host data (no fault is involved).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2306_11665_gb300 import _abi as A
from paper_2306_11665_gb300 import api
from paper_2306_11665_gb300 import inputs as I
from tests._helpers import rel_err_global, rel_err_per_var

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2306_11665_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


BAD = [(3, 0, 1, 7, np.inf), (11, 2, 2, 40, np.nan), (20, 1, 0, 0, -np.inf)]


def _poison(Ja, entries):
    Jb = Ja.copy()
    for e, m, k, i, v in entries:
        Jb[e, m, k, i % Jb.shape[3]] = v
    return Jb


@pytest.mark.parametrize("prec", ["fp32k", "fp32mix", "fp64"])
@pytest.mark.parametrize("p, kind", [(4, 0), (3, 1), (7, 1), (8, 0)])
def test_non_finite_metric_is_reported(prec, p, kind):
    d = 3
    u, Ja = I.workload(d, p, kind, 3)
    Jb = _poison(Ja, BAD)
    ctx = api.Context(d, p, kind, "euler")
    dt = torch.float64 if prec == "fp64" else torch.float32
    ut = torch.from_numpy(u).to(dt).cuda()
    r = ctx.volume_residual(ut, torch.from_numpy(Jb).cuda(), prec)
    assert ctx.check() == A.SFH_EDOMAIN
    assert "metric" in A.sfh_last_error()
    # every element without a bad value is still right
    keep = np.setdiff1d(np.arange(u.shape[0]), [b[0] for b in BAD])
    ref = O.volume_sf(d, p, kind, O.FLUX_EULER, u[keep], Ja[keep])
    got = r.double().cpu().numpy()[keep]
    if prec == "fp64":
        assert rel_err_per_var(got, ref) <= 1e-12
    else:
        assert rel_err_global(got, ref) <= 2e-5
    # and the error word was cleared: a clean call is clean
    ctx.volume_residual(ut, torch.from_numpy(Ja).cuda(), prec)
    assert ctx.check() == A.SFH_OK


@pytest.mark.parametrize("prec", ["fp32k", "fp32mix"])
def test_fp32_modes_refuse_metric_beyond_2_126(prec):
    d, p, kind = 3, 4, 0
    u, Ja = I.workload(d, p, kind, 2)
    ctx = api.Context(d, p, kind, "euler")
    ut = torch.from_numpy(u).float().cuda()
    Jb = _poison(Ja, [(5, 1, 2, 3, 1e40)])   # finite in FP64, beyond the FP32 modes' range
    ctx.volume_residual(ut, torch.from_numpy(Jb).cuda(), prec)
    assert ctx.check() == A.SFH_EDOMAIN
    # the largest magnitude still accepted is far below it
    Jc = _poison(Ja, [(5, 1, 2, 3, 1e30)])
    ctx.volume_residual(ut, torch.from_numpy(Jc).cuda(), prec)
    assert ctx.check() == A.SFH_OK


def test_fp64_accepts_large_finite_metric():
    d, p, kind = 3, 4, 0
    u, Ja = I.workload(d, p, kind, 2)
    ctx = api.Context(d, p, kind, "euler")
    Jb = _poison(Ja, [(5, 1, 2, 3, 1e40)])
    ctx.volume_residual(torch.from_numpy(u).cuda(), torch.from_numpy(Jb).cuda(), "fp64")
    assert ctx.check() == A.SFH_OK


def test_vjp_and_modal_report_non_finite_metric():
    d, p, kind = 3, 4, 0
    u, Ja = I.workload(d, p, kind, 2)
    Jb = torch.from_numpy(_poison(Ja, [(2, 0, 0, 9, np.nan)])).cuda()
    ctx = api.Context(d, p, kind, "euler")
    ut = torch.from_numpy(u).cuda()
    lam = torch.from_numpy(I.cotangent(u.shape)).cuda()
    ctx.vjp(ut, Jb, lam)
    assert ctx.check() == A.SFH_EDOMAIN
    uh = torch.from_numpy(I.legendre_coefficients(d, p, u.shape[0])).cuda()
    for prec in ("fp32k", "fp64"):
        src = uh if prec == "fp64" else uh.float()
        ctx.volume_residual_modal(src, Jb, "legendre", prec)
        assert ctx.check() == A.SFH_EDOMAIN, prec
