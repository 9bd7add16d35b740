"""GPU parity of sfh_volume_residual against the FP64 oracle.

Bars (relative, max norm, per variable, worst variable):
  FP64 1e-12; FP32 modes 2e-5 against the oracle on the FP64 state;
  entropy identity 1e-10 (FP64) and 1e-4 (FP32).
Small cases span several CTAs and a ragged tail; the full-size workloads
(3D Euler p=4 Gauss-Lobatto 32^3, p=7 Gauss 16^3) are checked on sampled
elements the oracle recomputes one by one, in the launch configuration the
benchmark times.
"""
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

FLUXES = {"burgers": O.FLUX_BURGERS, "euler": O.FLUX_EULER}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2306_11665_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def run_gpu(ctx, u, Ja, prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    ut = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float64)).to(dt).cuda()
    Jt = torch.from_numpy(Ja).cuda()
    r = ctx.volume_residual(ut, Jt, prec)
    st = ctx.check()
    return r.double().cpu().numpy(), st


def small_case(d, p, kind, flux):
    N = 3 if d == 3 else 5
    if d == 3 and p >= 7:
        N = 2
    amp = 0.0 if (flux == "burgers" and d == 2) else 0.1
    return I.workload(d, p, kind, N, flux=flux, amp=amp)


CASES = [(3, "euler"), (2, "burgers"), (2, "euler"), (3, "burgers")]


@pytest.mark.parametrize("d, flux", CASES)
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("p", range(1, 9))
def test_fp64_parity_small(d, flux, kind, p):
    u, Ja = small_case(d, p, kind, flux)
    ref = O.volume_sf(d, p, kind, FLUXES[flux], u, Ja)
    ctx = api.Context(d, p, kind, flux)
    got, st = run_gpu(ctx, u, Ja, "fp64")
    assert st == A.SFH_OK
    assert rel_err_per_var(got, ref) <= 1e-12


@pytest.mark.parametrize("d, flux", CASES)
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("p", range(1, 9))
@pytest.mark.parametrize("prec", ["fp32k", "fp32mix"])
def test_fp32_parity_small(d, flux, kind, p, prec):
    u, Ja = small_case(d, p, kind, flux)
    ref = O.volume_sf(d, p, kind, FLUXES[flux], u, Ja)
    u32 = I.to_fp32(u)
    ref_w = O.volume_sf(d, p, kind, FLUXES[flux], u32.astype(np.float64), Ja)
    ctx = api.Context(d, p, kind, flux)
    got, st = run_gpu(ctx, u32, Ja, prec)
    assert st == A.SFH_OK
    S = O.volume_absterms(d, p, kind, FLUXES[flux], u32.astype(np.float64), Ja)
    fp32_check(got, ref, ref_w, terms=S)


def test_burgers_2d_full_config_fp64():
    """2D Burgers, p=3 Gauss-Lobatto, 8x8 affine: all elements, against the
    sum-factorized and the dense oracle."""
    u, Ja = I.workload(2, 3, 0, 8, flux="burgers", amp=0.0)
    ctx = api.Context(2, 3, "gll", "burgers")
    got, st = run_gpu(ctx, u, Ja, "fp64")
    assert st == A.SFH_OK
    assert rel_err_per_var(got, O.volume_sf(2, 3, 0, O.FLUX_BURGERS, u, Ja)) <= 1e-12
    assert rel_err_per_var(got, O.volume_dense(2, 3, 0, O.FLUX_BURGERS, u, Ja)) <= 1e-12


def _sampled(d, p, kind, N, precs, n_sample, seed):
    """Full-size run on the GPU, the oracle on sampled elements; FP64 is held
    to 1e-12 per variable, the FP32 modes to the FP32 bars (fp32_check)."""
    u, Ja = I.workload(d, p, kind, N)
    E = u.shape[0]
    rng = np.random.default_rng(seed)
    idx = np.unique(np.concatenate([[0, E - 1], rng.choice(E, size=n_sample, replace=False)]))
    ref = O.volume_sf(d, p, kind, O.FLUX_EULER, u[idx], Ja[idx])
    ref_w = O.volume_sf(d, p, kind, O.FLUX_EULER, I.to_fp32(u[idx]).astype(np.float64), Ja[idx])
    S = O.volume_absterms(d, p, kind, O.FLUX_EULER, I.to_fp32(u[idx]).astype(np.float64), Ja[idx])
    ctx = api.Context(d, p, kind, "euler")
    out = {}
    for prec in precs:
        src = u if prec == "fp64" else I.to_fp32(u)
        got, st = run_gpu(ctx, src, Ja, prec)
        assert st == A.SFH_OK
        if prec == "fp64":
            out[prec] = {"per_variable_worst": float(rel_err_per_var(got[idx], ref))}
            assert out[prec]["per_variable_worst"] <= 1e-12
        else:
            out[prec] = fp32_check(got[idx], ref, ref_w, terms=S)
    return out, u, Ja, idx, ctx


def _report(name, data):
    import json
    import os
    d = os.environ.get("SFH_REPORT_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, f"{name}.json"), "w") as f:
            json.dump(data, f, indent=1)


def test_euler_p4_32cubed_sampled():
    errs, *_ = _sampled(3, 4, 0, 32, ["fp64", "fp32k", "fp32mix"], 96, 21)
    _report("parity_euler_p4_gll_32cubed", errs)


def test_euler_p7_gauss_16cubed_sampled():
    errs, *_ = _sampled(3, 7, 1, 16, ["fp64", "fp32k", "fp32mix"], 24, 22)
    _report("parity_euler_p7_gauss_16cubed", errs)


@pytest.mark.parametrize("p, kind", [(6, 0), (6, 1)])
def test_euler_p6_two_element_blocks_sampled(p, kind):
    """At n = 7 the warp-specialized kernel takes two elements per block, one
    residual buffer and two service warps; 21^3 = 9,261 elements (an odd
    count: a one-element tail block) checked on sampled elements, and the
    same elements as a small mesh (other block boundaries) meet the same bars."""
    errs, u, Ja, idx, ctx = _sampled(3, p, kind, 21, ["fp32k", "fp32mix"], 16, 31)
    u32 = I.to_fp32(u[idx]).astype(np.float64)
    ref = O.volume_sf(3, p, kind, O.FLUX_EULER, u[idx], Ja[idx])
    ref_w = O.volume_sf(3, p, kind, O.FLUX_EULER, u32, Ja[idx])
    S = O.volume_absterms(3, p, kind, O.FLUX_EULER, u32, Ja[idx])
    for prec in ("fp32k", "fp32mix"):
        small, st = run_gpu(ctx, I.to_fp32(u[idx]), Ja[idx], prec)
        assert st == A.SFH_OK
        fp32_check(small, ref, ref_w, terms=S)


@pytest.mark.parametrize("p, kind, N", [(4, 0, 8), (7, 1, 4)])
def test_entropy_identity_on_gpu_results(p, kind, N):
    d = 3
    u, Ja = I.workload(d, p, kind, N)
    ctx = api.Context(d, p, kind, "euler")
    r64, _ = run_gpu(ctx, u, Ja, "fp64")
    r32, _ = run_gpu(ctx, I.to_fp32(u), Ja, "fp32k")
    rmx, _ = run_gpu(ctx, I.to_fp32(u), Ja, "fp32mix")
    worst = {"fp64": 0.0, "fp32k": 0.0, "fp32mix": 0.0}
    for e in (0, u.shape[0] // 2, u.shape[0] - 1):
        for prec, r in (("fp64", r64), ("fp32k", r32), ("fp32mix", rmx)):
            worst[prec] = max(worst[prec], identity_residual(d, p, kind, O.FLUX_EULER, u[e], Ja[e], r[e]))
    assert worst["fp64"] <= 1e-10
    assert worst["fp32k"] <= 1e-4 and worst["fp32mix"] <= 1e-4
    _report(f"entropy_identity_euler_p{p}_{'gll' if kind == 0 else 'gauss'}_{N}cubed", worst)


@pytest.mark.parametrize("prec", ["fp32k", "fp64"])
def test_large_mesh_64bit_offsets(prec):
    """2^21 elements of 3D Euler p = 4 (the 32^3 state tiled 64 times on the
    device): Ja alone spans 18.9 GB, so element offsets pass 2^31 floats and
    2^32 bytes; sampled elements, the last ones included, match the oracle."""
    u, Ja = I.workload(3, 4, 0, 32)
    E0, rep = u.shape[0], 64
    dt = torch.float64 if prec == "fp64" else torch.float32
    src = u if prec == "fp64" else I.to_fp32(u)
    ut = torch.from_numpy(np.ascontiguousarray(src)).to(dt).cuda().repeat(rep, 1, 1)
    Jt = torch.from_numpy(Ja).cuda().repeat(rep, 1, 1, 1)
    ctx = api.Context(3, 4, "gll", "euler")
    r = ctx.volume_residual(ut, Jt, prec)
    assert ctx.check() == A.SFH_OK
    E = E0 * rep
    idx = np.array([0, 1, E0 - 1, E0, E // 2 + 7, E - E0, E - 2, E - 1])
    got = r[torch.from_numpy(idx).cuda()].double().cpu().numpy()
    del ut, Jt, r
    torch.cuda.empty_cache()
    base = idx % E0
    ref = O.volume_sf(3, 4, 0, O.FLUX_EULER, u[base], Ja[base])
    if prec == "fp64":
        assert rel_err_per_var(got, ref) <= 1e-12
    else:
        u32 = I.to_fp32(u[base]).astype(np.float64)
        ref_w = O.volume_sf(3, 4, 0, O.FLUX_EULER, u32, Ja[base])
        fp32_check(got, ref, ref_w, terms=O.volume_absterms(3, 4, 0, O.FLUX_EULER, u32, Ja[base]))


@pytest.mark.parametrize("d, p, kind, flux", [(3, 4, 0, "euler"), (3, 7, 1, "euler"), (3, 3, 1, "euler"),
                                             (2, 5, 1, "euler"), (2, 4, 0, "burgers"), (3, 2, 1, "burgers")])
def test_entropy_residual_kernel_matches_host(d, p, kind, flux):
    """The GPU's FP64 entropy-identity defect against the host evaluation of
    the same identity (tests/_entropy.py), for FP64 and FP32 residuals; and the
    whole mesh under the bars."""
    N = 2 if (d == 3 and p >= 7) else 3
    u, Ja = I.workload(d, p, kind, N, flux=flux)
    ctx = api.Context(d, p, kind, flux)
    ut, Jt = torch.from_numpy(u).cuda(), torch.from_numpy(Ja).cuda()
    for prec, bar in (("fp64", 1e-10), ("fp32k", 1e-4)):
        src = u if prec == "fp64" else I.to_fp32(u)
        r = ctx.volume_residual(torch.from_numpy(np.ascontiguousarray(src)).cuda(), Jt, prec)
        dev = ctx.entropy_residual(ut, Jt, r).cpu().numpy()
        assert ctx.check() == A.SFH_OK
        assert dev.shape == (u.shape[0],) and np.all(dev <= bar), (prec, dev.max())
        rh = r.double().cpu().numpy()
        fl = FLUXES[flux]
        for e in (0, u.shape[0] - 1):
            host = identity_residual(d, p, kind, fl, u[e], Ja[e], rh[e])
            assert abs(dev[e] - host) <= 1e-15 + 1e-6 * host, (prec, e, dev[e], host)


def test_entropy_residual_detects_a_wrong_residual():
    u, Ja = I.workload(3, 4, 0, 2)
    ctx = api.Context(3, 4, "gll", "euler")
    ut, Jt = torch.from_numpy(u).cuda(), torch.from_numpy(Ja).cuda()
    r = ctx.volume_residual(ut, Jt, "fp64")
    r[3, 4, 17] += 1e-3 * r[3].abs().max()   # one energy component off by 0.1 % of the element's scale
    dev = ctx.entropy_residual(ut, Jt, r).cpu().numpy()
    assert dev[3] > 1e-8 and np.delete(dev, 3).max() <= 1e-10
    # an output that overlaps an input is refused before any launch
    with pytest.raises(A.SfhError) as e:
        A.sfh_entropy_residual(ctx.handle, u.shape[0], ut.data_ptr(), Jt.data_ptr(), r.data_ptr(), A.SFH_FP64,
                               ut.data_ptr() + 8)
    assert e.value.status == A.SFH_EINVAL


def test_edge_cases():
    ctx = api.Context(3, 4, "gll", "euler")
    # n_elem = 0 is a no-op
    A.sfh_volume_residual(ctx.handle, 0, 0, 0, 0, A.SFH_FP64, 0)
    # one element
    u, Ja = I.workload(3, 4, 0, 2, n_elem=1)
    got, st = run_gpu(ctx, u, Ja, "fp64")
    assert st == A.SFH_OK
    assert rel_err_per_var(got, O.volume_sf(3, 4, 0, O.FLUX_EULER, u, Ja)) <= 1e-12
    # every element count 1..12 (ragged tails of the 5-element CTAs)
    u, Ja = I.workload(3, 4, 0, 3)
    for E in range(1, 13):
        got, _ = run_gpu(ctx, u[:E], Ja[:E], "fp64")
        assert rel_err_per_var(got, O.volume_sf(3, 4, 0, O.FLUX_EULER, u[:E], Ja[:E])) <= 1e-12
    # misaligned / overlapping arguments are rejected before any launch
    ut = torch.from_numpy(u).cuda()
    Jt = torch.from_numpy(Ja).cuda()
    with pytest.raises(A.SfhError) as e:
        A.sfh_volume_residual(ctx.handle, 2, ut.data_ptr(), Jt.data_ptr(), ut.data_ptr(), A.SFH_FP64, 0)
    assert e.value.status == A.SFH_EINVAL
    with pytest.raises(A.SfhError) as e:
        r2 = torch.empty_like(ut)
        A.sfh_volume_residual(ctx.handle, 2, ut.data_ptr() + 4, Jt.data_ptr(), r2.data_ptr(), A.SFH_FP64, 0)
    assert e.value.status == A.SFH_EINVAL


def test_domain_error_is_reported_and_cleared():
    ctx = api.Context(3, 3, "gll", "euler")
    u, Ja = I.workload(3, 3, 0, 2)
    bad = u.copy()
    bad[3, 0, 7] = -1.0         # negative density in element 3
    got, st = run_gpu(ctx, bad, Ja, "fp64")
    assert st == A.SFH_EDOMAIN
    assert ctx.check() == A.SFH_OK    # cleared by the check
    # elements without the bad node are unaffected
    ref = O.volume_sf(3, 3, 0, O.FLUX_EULER, u, Ja)
    keep = [e for e in range(u.shape[0]) if e != 3]
    assert rel_err_per_var(got[keep], ref[keep]) <= 1e-12
    # the FP32 path reports it too
    _, st = run_gpu(ctx, I.to_fp32(bad), Ja, "fp32k")
    assert st == A.SFH_EDOMAIN


def test_deterministic_and_stream():
    ctx = api.Context(3, 5, "gauss", "euler")
    u, Ja = I.workload(3, 5, 1, 3)
    a, _ = run_gpu(ctx, u, Ja, "fp64")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b, _ = run_gpu(ctx, u, Ja, "fp64")
    assert np.array_equal(a, b)
    c, _ = run_gpu(ctx, I.to_fp32(u), Ja, "fp32k")
    d_, _ = run_gpu(ctx, I.to_fp32(u), Ja, "fp32k")
    assert np.array_equal(c, d_)


@pytest.mark.parametrize("prec", ["fp64", "fp32k"])
def test_host_entry_point_matches_device(prec):
    ctx = api.Context(3, 4, "gll", "euler")
    u, Ja = I.workload(3, 4, 0, 6)
    src = u if prec == "fp64" else I.to_fp32(u)
    dev, _ = run_gpu(ctx, src, Ja, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    uh = torch.from_numpy(np.ascontiguousarray(src)).to(dt).pin_memory()
    Jh = torch.from_numpy(Ja).pin_memory()
    host = ctx.volume_residual_host(uh, Jh, prec).double().numpy()
    assert np.array_equal(host, dev)


@pytest.mark.parametrize("prec", ["fp32k", "fp32mix", "fp64"])
def test_bound_metric_host_entry_point(prec):
    """sfh_volume_residual_host_bound on a metric bound once equals the
    host-buffer entry point that copies Ja every call, on two calls in a row;
    a smaller element count uses the first elements of the bound metric, and
    more elements than are bound are refused."""
    ctx = api.Context(3, 4, "gll", "euler")
    u, Ja = I.workload(3, 4, 0, 14)       # 2,744 elements: several 4 MB chunks and a ragged tail
    src = u if prec == "fp64" else I.to_fp32(u)
    dt = torch.float64 if prec == "fp64" else torch.float32
    uh = torch.from_numpy(np.ascontiguousarray(src)).to(dt).pin_memory()
    Jh = torch.from_numpy(Ja).pin_memory()
    want = ctx.volume_residual_host(uh, Jh, prec).double().numpy()
    E = u.shape[0]
    A.sfh_bind_metric(ctx.handle, E, Jh.data_ptr())
    mode = {"fp64": A.SFH_FP64, "fp32k": A.SFH_FP32_KAHAN, "fp32mix": A.SFH_FP32_MIXED}[prec]
    for _ in range(2):
        rh = torch.full_like(uh, float("nan")).pin_memory()
        assert A.sfh_volume_residual_host_bound(ctx.handle, E, uh.data_ptr(), rh.data_ptr(), mode) == A.SFH_OK
        got = rh.double().numpy()
        if prec == "fp64":   # another chunking may pick another FP64 kernel: equal to round-off
            assert rel_err_per_var(got, want) <= 1e-13
        else:
            assert np.array_equal(got, want)
    part = 1000
    rh = torch.full_like(uh, float("nan")).pin_memory()
    A.sfh_volume_residual_host_bound(ctx.handle, part, uh.data_ptr(), rh.data_ptr(), mode)
    assert rel_err_per_var(rh[:part].double().numpy(), want[:part]) <= (1e-13 if prec == "fp64" else 0.0)
    assert np.isnan(rh[part:].numpy()).all()
    with pytest.raises(A.SfhError) as e:
        A.sfh_volume_residual_host_bound(ctx.handle, E + 1, uh.data_ptr(), rh.data_ptr(), mode)
    assert e.value.status == A.SFH_EINVAL
    A.sfh_bind_metric(ctx.handle, 0, 0)   # unbind
    with pytest.raises(A.SfhError) as e:
        A.sfh_volume_residual_host_bound(ctx.handle, 1, uh.data_ptr(), rh.data_ptr(), mode)
    assert e.value.status == A.SFH_EINVAL


@pytest.mark.parametrize("d, p, kind", [(3, 4, 0), (3, 2, 1), (2, 5, 0), (3, 7, 1), (3, 6, 0), (3, 8, 0)])
def test_rough_states_take_the_logarithm_path(d, p, kind):
    """States with large jumps between neighbouring nodes put many pairs
    outside the series band of the logarithmic mean (|a-b| >= 0.1 (a+b)),
    exercising the logarithm branch of every precision mode."""
    rng = np.random.default_rng(31)
    x, Ja = I.mesh(d, p, kind, 2, 0.1)
    E, nn = x.shape[0], x.shape[2]
    rho = 1.0 + 0.8 * rng.uniform(-1, 1, size=(E, nn))
    pr = 1.0 + 0.8 * rng.uniform(-1, 1, size=(E, nn))
    v = [0.3 * rng.uniform(-1, 1, size=(E, nn)) for _ in range(d)]
    u = np.ascontiguousarray(I.conservative(rho, v, pr))
    ref = O.volume_sf(d, p, kind, O.FLUX_EULER, u, Ja)
    ctx = api.Context(d, p, kind, "euler")
    got, st = run_gpu(ctx, u, Ja, "fp64")
    assert st == A.SFH_OK
    assert rel_err_per_var(got, ref) <= 1e-12
    u32 = I.to_fp32(u)
    ref_w = O.volume_sf(d, p, kind, O.FLUX_EULER, u32.astype(np.float64), Ja)
    S = O.volume_absterms(d, p, kind, O.FLUX_EULER, u32.astype(np.float64), Ja)
    for prec in ("fp32k", "fp32mix"):
        got, st = run_gpu(ctx, u32, Ja, prec)
        assert st == A.SFH_OK
        fp32_check(got, ref, ref_w, terms=S)
