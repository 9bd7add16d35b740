"""GPU parity of sfh_vjp (FP64) against the oracle's VJP, the autograd
wrapper, and central finite differences of the GPU residual."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2306_11665_gb300 import _abi as A
from paper_2306_11665_gb300 import api
from paper_2306_11665_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2306_11665_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def gpu_vjp(ctx, u, Ja, lam):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    g = ctx.vjp(t(u), t(Ja), t(lam))
    assert ctx.check() == A.SFH_OK
    return g.cpu().numpy()


@pytest.mark.parametrize("d, flux", [(3, "euler"), (2, "euler"), (2, "burgers"), (3, "burgers")])
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("p", [1, 2, 3, 5, 8])
def test_vjp_parity_small(d, flux, kind, p):
    N = 3 if d == 3 else 5
    if d == 3 and p >= 7:
        N = 2
    u, Ja = I.workload(d, p, kind, N, flux=flux)
    lam = I.cotangent(u.shape)
    fl = O.FLUX_EULER if flux == "euler" else O.FLUX_BURGERS
    ref = O.vjp_sf(d, p, kind, fl, u, Ja, lam)
    got = gpu_vjp(api.Context(d, p, kind, flux), u, Ja, lam)
    assert rel(got, ref) <= 1e-12


def test_vjp_adjoint_config_full():
    """Adjoint configuration: p=5 Gauss-Lobatto, 8^3 warped elements, lambda ~ N(0,1)."""
    u, Ja = I.workload(3, 5, 0, 8)
    lam = I.cotangent(u.shape, seed=8)
    got = gpu_vjp(api.Context(3, 5, "gll", "euler"), u, Ja, lam)
    ref = O.vjp_sf(3, 5, 0, O.FLUX_EULER, u, Ja, lam)
    assert rel(got, ref) <= 1e-12


@pytest.mark.parametrize("p, kind", [(4, 0), (3, 1)])
def test_vjp_large_mesh_sampled(p, kind):
    """A mesh large enough for the multi-element blocks of the default
    launch shape (16^3 elements); sampled elements checked one by one."""
    u, Ja = I.workload(3, p, kind, 16)
    lam = I.cotangent(u.shape, seed=8)
    got = gpu_vjp(api.Context(3, p, kind, "euler"), u, Ja, lam)
    idx = np.r_[0:5, 1000:1003, np.arange(7, u.shape[0], 211), u.shape[0] - 3:u.shape[0]]
    ref = O.vjp_sf(3, p, kind, O.FLUX_EULER, u[idx], Ja[idx], lam[idx])
    assert rel(got[idx], ref) <= 1e-12


def test_autograd_and_finite_differences():
    ctx = api.Context(3, 5, "gll", "euler")
    u, Ja = I.workload(3, 5, 0, 3)
    lam = I.cotangent(u.shape, seed=8)
    ut = torch.from_numpy(u).cuda().requires_grad_(True)
    Jt = torch.from_numpy(Ja).cuda()
    lt = torch.from_numpy(lam).cuda()
    r = api.volume(ut, Jt, ctx)
    (r * lt).sum().backward()
    g = ut.grad.detach()
    assert torch.equal(g, ctx.vjp(ut.detach(), Jt, lt))
    # directional central difference of the GPU residual (FP64)
    delta = torch.from_numpy(np.random.default_rng(3).standard_normal(u.shape) * np.maximum(1, np.abs(u))).cuda()
    h = 1e-6
    with torch.no_grad():
        rp = ctx.volume_residual((ut + h * delta).contiguous(), Jt)
        rm = ctx.volume_residual((ut - h * delta).contiguous(), Jt)
    fd = float((lt * (rp - rm)).sum() / (2 * h))
    an = float((g * delta).sum())
    assert abs(an - fd) <= 1e-6 * abs(fd)
