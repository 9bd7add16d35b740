"""GPU parity of Chandrashekar's flux (SFH_FLUX_EULER_CHANDRASHEKAR, the flux
named for the TGV runs of Section 3) against the oracle's flux id 2, with
the bars of the Ranocha-flux tests: FP64 1e-12 per variable, the FP32 bars of
fp32_check, VJP 1e-12, the entropy identity 1e-10 / 1e-4.  Small cases span
several CTAs and a ragged tail; the full-size 3D p = 4 Gauss-Lobatto 32^3
workload is checked on sampled elements; rough states exercise the logarithm
branch of every mode."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2306_11665_gb300 import _abi as A
from paper_2306_11665_gb300 import api
from paper_2306_11665_gb300 import inputs as I
from tests._entropy import identity_residual
from tests._helpers import fp32_check, rel_err_per_var

pytestmark = pytest.mark.gpu

CH = O.FLUX_CHANDRASHEKAR
NAME = "euler_chandrashekar"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2306_11665_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def run_gpu(ctx, u, Ja, prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    ut = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float64)).to(dt).cuda()
    r = ctx.volume_residual(ut, torch.from_numpy(Ja).cuda(), prec)
    return r.double().cpu().numpy(), ctx.check()


def small_case(d, p, kind):
    N = 2 if (d == 3 and p >= 7) else (3 if d == 3 else 5)
    return I.workload(d, p, kind, N)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("p", range(1, 9))
def test_parity_small_all_modes(d, kind, p):
    u, Ja = small_case(d, p, kind)
    ref = O.volume_sf(d, p, kind, CH, u, Ja)
    ctx = api.Context(d, p, kind, NAME)
    got, st = run_gpu(ctx, u, Ja, "fp64")
    assert st == A.SFH_OK
    assert rel_err_per_var(got, ref) <= 1e-12
    u32 = I.to_fp32(u)
    ref_w = O.volume_sf(d, p, kind, CH, u32.astype(np.float64), Ja)
    S = O.volume_absterms(d, p, kind, CH, u32.astype(np.float64), Ja)
    for prec in ("fp32k", "fp32mix"):
        got, st = run_gpu(ctx, u32, Ja, prec)
        assert st == A.SFH_OK
        fp32_check(got, ref, ref_w, terms=S)


def test_differs_from_ranocha_on_the_gpu():
    """The context's flux reaches the kernels: the two Euler fluxes give
    residuals that differ by far more than round-off, in every mode."""
    u, Ja = I.workload(3, 4, 0, 3)
    for prec in ("fp64", "fp32k", "fp32mix"):
        src = u if prec == "fp64" else I.to_fp32(u)
        a, _ = run_gpu(api.Context(3, 4, 0, "euler"), src, Ja, prec)
        b, _ = run_gpu(api.Context(3, 4, 0, NAME), src, Ja, prec)
        assert np.abs(a - b).max() >= 1e-4 * np.abs(a).max(), prec


def test_full_size_p4_32cubed_sampled():
    """3D p = 4 Gauss-Lobatto on 32^3 warped elements (the launch shape of the
    FP32 benchmark), sampled elements recomputed by the oracle."""
    d, p, kind = 3, 4, 0
    u, Ja = I.workload(d, p, kind, 32)
    E = u.shape[0]
    rng = np.random.default_rng(41)
    idx = np.unique(np.concatenate([[0, E - 1], rng.choice(E, size=64, replace=False)]))
    ref = O.volume_sf(d, p, kind, CH, u[idx], Ja[idx])
    ref_w = O.volume_sf(d, p, kind, CH, I.to_fp32(u[idx]).astype(np.float64), Ja[idx])
    S = O.volume_absterms(d, p, kind, CH, I.to_fp32(u[idx]).astype(np.float64), Ja[idx])
    ctx = api.Context(d, p, kind, NAME)
    for prec in ("fp64", "fp32k", "fp32mix"):
        got, st = run_gpu(ctx, u if prec == "fp64" else I.to_fp32(u), Ja, prec)
        assert st == A.SFH_OK
        if prec == "fp64":
            assert rel_err_per_var(got[idx], ref) <= 1e-12
        else:
            fp32_check(got[idx], ref, ref_w, terms=S)


@pytest.mark.parametrize("d, p, kind", [(3, 4, 0), (3, 7, 1), (3, 8, 0), (2, 5, 0)])
def test_rough_states_take_the_logarithm_path(d, p, kind):
    rng = np.random.default_rng(43)
    x, Ja = I.mesh(d, p, kind, 2, 0.1)
    E, nn = x.shape[0], x.shape[2]
    rho = 1.0 + 0.8 * rng.uniform(-1, 1, size=(E, nn))
    pr = 1.0 + 0.8 * rng.uniform(-1, 1, size=(E, nn))
    v = [0.3 * rng.uniform(-1, 1, size=(E, nn)) for _ in range(d)]
    u = np.ascontiguousarray(I.conservative(rho, v, pr))
    ref = O.volume_sf(d, p, kind, CH, u, Ja)
    ctx = api.Context(d, p, kind, NAME)
    got, st = run_gpu(ctx, u, Ja, "fp64")
    assert st == A.SFH_OK
    assert rel_err_per_var(got, ref) <= 1e-12
    u32 = I.to_fp32(u)
    ref_w = O.volume_sf(d, p, kind, CH, u32.astype(np.float64), Ja)
    S = O.volume_absterms(d, p, kind, CH, u32.astype(np.float64), Ja)
    for prec in ("fp32k", "fp32mix"):
        got, st = run_gpu(ctx, u32, Ja, prec)
        assert st == A.SFH_OK
        fp32_check(got, ref, ref_w, terms=S)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("p", [1, 3, 5, 8])
def test_vjp_parity(d, kind, p):
    u, Ja = small_case(d, p, kind)
    lam = I.cotangent(u.shape)
    ref = O.vjp_sf(d, p, kind, CH, u, Ja, lam)
    ctx = api.Context(d, p, kind, NAME)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    got = ctx.vjp(t(u), t(Ja), t(lam)).cpu().numpy()
    assert ctx.check() == A.SFH_OK
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("d, p, kind", [(3, 4, 0), (3, 7, 1), (2, 5, 1)])
def test_entropy_identity(d, p, kind):
    """Chandrashekar's flux conserves the same entropy: the GPU's identity
    defect of GPU residuals is at round-off and matches the host evaluation."""
    N = 2 if (d == 3 and p >= 7) else 3
    u, Ja = I.workload(d, p, kind, N)
    ctx = api.Context(d, p, kind, NAME)
    ut, Jt = torch.from_numpy(u).cuda(), torch.from_numpy(Ja).cuda()
    for prec, bar in (("fp64", 1e-10), ("fp32k", 1e-4), ("fp32mix", 1e-4)):
        src = u if prec == "fp64" else I.to_fp32(u)
        r = ctx.volume_residual(torch.from_numpy(np.ascontiguousarray(src)).cuda(), Jt, prec)
        dev = ctx.entropy_residual(ut, Jt, r).cpu().numpy()
        assert ctx.check() == A.SFH_OK
        assert np.all(dev <= bar), (prec, dev.max())
        rh = r.double().cpu().numpy()
        for e in (0, u.shape[0] - 1):
            host = identity_residual(d, p, kind, CH, u[e], Ja[e], rh[e])
            assert abs(dev[e] - host) <= 1e-15 + 1e-6 * host, (prec, e, dev[e], host)


@pytest.mark.parametrize("prec", ["fp64", "fp32k", "fp32mix"])
def test_host_entry_points(prec):
    """The host-buffer entry point and the allocation-free one give the device
    path's result bit for bit."""
    ctx = api.Context(3, 4, "gll", NAME)
    u, Ja = I.workload(3, 4, 0, 5)
    src = u if prec == "fp64" else I.to_fp32(u)
    dev, _ = run_gpu(ctx, src, Ja, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    uh = torch.from_numpy(np.ascontiguousarray(src)).to(dt).pin_memory()
    host = ctx.volume_residual_host(uh, torch.from_numpy(Ja).pin_memory(), prec).double().numpy()
    assert np.array_equal(host, dev)
    un = np.ascontiguousarray(src)
    rn = np.empty_like(un)
    st = A.lib().sfh_volume_residual_host_noalloc(3, 4, 0, A.SFH_FLUX_EULER_CHANDRASHEKAR, u.shape[0],
                                                   un.ctypes.data, Ja.ctypes.data, rn.ctypes.data,
                                                   api.PREC[prec], None)
    assert st == A.SFH_OK
    assert np.array_equal(rn.astype(np.float64), dev)
