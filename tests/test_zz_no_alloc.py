"""The allocation-free host-buffer entry point, for callers that cannot call
cudaMalloc (their device memory belongs to another allocator, or they must not
allocate after start-up).

It is checked through the C ABI against the existing host-buffer entry point
(sfh_volume_residual_host, which stages through context-owned allocations):
two calls in a row with different inputs (the shared device array keeps the
previous call's contents), every precision mode, and a request larger than the
fixed device array, which must be refused with a clear error.  This file is
collected last so that a run stopping at its first failure has already run
every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

from paper_2306_11665_gb300 import _abi as A
from paper_2306_11665_gb300 import api
from paper_2306_11665_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2306_11665_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _noalloc(d, p, kind, flux, u, Ja, prec):
    r = np.empty_like(u)
    st = A.lib().sfh_volume_residual_host_noalloc(d, p, kind, flux, u.shape[0], u.ctypes.data, Ja.ctypes.data,
                                                   r.ctypes.data, prec, None)
    return st, r


@pytest.mark.parametrize("prec, dtype", [(A.SFH_FP64, np.float64), (A.SFH_FP32_KAHAN, np.float32),
                                         (A.SFH_FP32_MIXED, np.float32)])
@pytest.mark.parametrize("p, kind", [(4, 0), (2, 1), (3, 0), (5, 1), (7, 0), (7, 1)])
def test_matches_context_host_entry_two_calls(prec, dtype, p, kind):
    # the context-free tables must round exactly as a context's do: several
    # degrees on both node sets, compared bit for bit
    d = 3
    ctx = api.Context(d, p, kind, "euler")
    for seed in (2, 40):   # second call: different state, same shared device array
        u, Ja = I.workload(d, p, kind, 6, n_elem=120, seed0=seed)
        u = _host(u, dtype)
        st, r_na = _noalloc(d, p, kind, A.SFH_FLUX_EULER_RANOCHA, u, Ja, prec)
        assert st == A.SFH_OK, A.sfh_last_error()
        r_ref = np.empty_like(u)
        st = A.sfh_volume_residual_host(ctx.handle, u.shape[0], u.ctypes.data, Ja.ctypes.data, r_ref.ctypes.data,
                                        prec)
        assert st == A.SFH_OK
        scale = np.abs(r_ref).max()
        tol = 1e-12 if prec == A.SFH_FP64 else 2e-5
        assert np.abs(r_na.astype(np.float64) - r_ref).max() <= tol * scale
        # same kernel, same inputs: in practice the results are identical
        assert np.array_equal(r_na, r_ref)


def test_burgers_2d_and_domain_error():
    d, p, kind = 2, 3, 0
    u, Ja = I.workload(d, p, kind, 8, flux="burgers", amp=0.0)
    st, r1 = _noalloc(d, p, kind, A.SFH_FLUX_BURGERS, u, Ja, A.SFH_FP64)
    assert st == A.SFH_OK
    ctx = api.Context(d, p, kind, "burgers")
    r2 = np.empty_like(u)
    A.sfh_volume_residual_host(ctx.handle, u.shape[0], u.ctypes.data, Ja.ctypes.data, r2.ctypes.data, A.SFH_FP64)
    assert np.array_equal(r1, r2)
    # a negative density is reported, and the next clean call is clean again
    u3, Ja3 = I.workload(3, 3, 0, 2)
    bad = u3.copy()
    bad[1, 0, 5] = -1.0
    st, _ = _noalloc(3, 3, 0, A.SFH_FLUX_EULER_RANOCHA, bad, Ja3, A.SFH_FP64)
    assert st == A.SFH_EDOMAIN
    st, _ = _noalloc(3, 3, 0, A.SFH_FLUX_EULER_RANOCHA, u3, Ja3, A.SFH_FP64)
    assert st == A.SFH_OK


def test_oversized_request_is_refused():
    d, p, kind = 3, 4, 0
    # more elements than the fixed device array can stage (FP64, 19,000 bytes per element)
    n_elem = 5000
    u = np.zeros((n_elem, 5, 125))
    Ja = np.zeros((n_elem, 3, 3, 125))
    r = np.zeros_like(u)
    st = A.lib().sfh_volume_residual_host_noalloc(d, p, kind, A.SFH_FLUX_EULER_RANOCHA, n_elem, u.ctypes.data,
                                                   Ja.ctypes.data, r.ctypes.data, A.SFH_FP64, None)
    assert st == A.SFH_EINVAL
    msg = A.sfh_last_error()
    assert "no-allocation" in msg and "at most" in msg
