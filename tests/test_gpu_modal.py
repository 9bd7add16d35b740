"""GPU parity of the modal / uncollocated entry point
(sfh_volume_residual_modal: r_hat = V^T r_v(V u_hat), transforms fused into
the residual kernels) against the oracle's modal path (dense Kronecker
transforms).  The kernels apply the theorem that the entropy projection is
the identity for square V; the parity cases compare with the oracle's
unprojected path, and one case with its literal projection, whose round-off
(about 1e-14 relative in the state) the residual's cancellation amplifies:
there the FP64 bar is max(1e-12, 16 u64 kappa_v).

Bars: FP64 1e-12 per variable; FP32 modes, per variable, max(2e-5, 6 x the
input-rounding floor, 2.5 u32 kappa_v) with kappa_v the cancellation ratio of
the modal residual, max_k sum_i |V_ik| S_v,i / max_k |r_hat_k,v|,
S_v,i = sum_{m,j} |Q_m,ij F_m,ij,v| (the sums the residual and its transform
cancel), and in the global relative max norm max(2e-5, 2.5 u32 kappa) with
kappa the same ratio over all variables at once: the FP32 forward transform
rounds the nodal state (a few ulp, like the nodal path's input rounding) and
the residual's cancellation amplifies it."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2306_11665_gb300 import _abi as A
from paper_2306_11665_gb300 import api
from paper_2306_11665_gb300 import inputs as I
from tests._entropy import kron_q
from tests._helpers import fp32_check, rel_err_global, rel_err_per_var

pytestmark = pytest.mark.gpu

LEG, LGLL, LGAUSS = I.BASIS_LEGENDRE, I.BASIS_LAGRANGE_GLL, I.BASIS_LAGRANGE_GAUSS
FLUX = {"euler": O.FLUX_EULER, "euler_chandrashekar": O.FLUX_CHANDRASHEKAR, "burgers": O.FLUX_BURGERS}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2306_11665_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def run_modal(ctx, uhat, Ja, basis, prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    ut = torch.from_numpy(np.ascontiguousarray(uhat, dtype=np.float64)).to(dt).cuda()
    r = ctx.volume_residual_modal(ut, torch.from_numpy(Ja).cuda(), basis, prec)
    return r.double().cpu().numpy(), ctx.check()


def modal_terms(d, p, kind, basis, flux, uhat, Ja):
    """T[e, v, k] = sum_i |V_ik| S_v,i: the absolute terms of the nodal
    residual (oracle volume_absterms at the nodal states V u_hat) carried
    through |V^T|, the magnitude the modal residual cancels from."""
    _, up = O.modal_states(d, p, kind, basis, flux, uhat)
    V1 = O.basis_1d(p, kind, basis)
    V = V1
    for _ in range(d - 1):
        V = np.kron(V1, V)
    S = O.volume_absterms(d, p, kind, flux, up, Ja)
    return np.einsum("ik,evi->evk", np.abs(V), S)


def kappa_modal(d, p, kind, basis, flux, uhat, Ja, rhat):
    """Per-variable cancellation ratios of the modal residual."""
    T = modal_terms(d, p, kind, basis, flux, uhat, Ja)
    return [T[:, v].max() / np.abs(rhat[:, v]).max() for v in range(rhat.shape[1])]


def fp32_check_modal(got, ref, ref_w, T):
    """The FP32 bars of the modal path: the global relative max norm within
    max(2e-5, 2.5 u32 kappa) (kappa over all variables: the FP32 forward
    transform rounds the nodal state by a few ulp, and the residual amplifies
    that by its cancellation ratio), the per-variable bars of fp32_check, and
    the arithmetic error against the oracle on the FP32-rounded coefficients
    per variable at C_ARITH u32 kappa_v."""
    g = rel_err_global(got, ref)
    kap = T.max() / np.abs(ref).max()
    assert g <= max(2e-5, 2.5 * 2.0 ** -24 * kap), ("global", g, kap)
    out = fp32_check(got, ref, ref_w, global_bar=np.inf, terms=T, arith_per_node=False)
    out["kappa_global"] = float(kap)
    return out


def check(d, p, kind, basis, flux_name, N=None, precs=("fp64", "fp32k", "fp32mix")):
    fl = FLUX[flux_name]
    N = N or (2 if (d == 3 and p >= 6) else 3)
    uhat, Ja = I.modal_workload(d, p, kind, basis, N, flux="burgers" if fl == O.FLUX_BURGERS else "euler")
    ref = O.volume_modal(d, p, kind, basis, fl, uhat, Ja, project=False)
    ctx = api.Context(d, p, kind, flux_name)
    out = {}
    for prec in precs:
        if prec == "fp64":
            got, st = run_modal(ctx, uhat, Ja, basis, prec)
            assert st == A.SFH_OK
            out[prec] = rel_err_per_var(got, ref)
            assert out[prec] <= 1e-12, (prec, out[prec])
        else:
            u32 = I.to_fp32(uhat)
            ref_w = O.volume_modal(d, p, kind, basis, fl, u32.astype(np.float64), Ja, project=False)
            got, st = run_modal(ctx, u32, Ja, basis, prec)
            assert st == A.SFH_OK
            out[prec] = fp32_check_modal(got, ref, ref_w, modal_terms(d, p, kind, basis, fl, I.to_fp32(uhat).astype(np.float64), Ja))
    return out


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8])
def test_legendre_euler_all_modes(d, kind, p):
    check(d, p, kind, LEG, "euler")


@pytest.mark.parametrize("d, kind, p", [(3, 1, 4), (3, 0, 7), (2, 1, 5)])
def test_fp64_against_the_literal_entropy_projection(d, kind, p):
    N = 2 if (d == 3 and p >= 6) else 3
    uhat, Ja = I.modal_workload(d, p, kind, LEG, N)
    ref = O.volume_modal(d, p, kind, LEG, O.FLUX_EULER, uhat, Ja, project=True)
    got, st = run_modal(api.Context(d, p, kind, "euler"), uhat, Ja, LEG, "fp64")
    assert st == A.SFH_OK
    kap = np.asarray(kappa_modal(d, p, kind, LEG, O.FLUX_EULER, uhat, Ja, ref))
    err = np.array([np.abs(got[:, v] - ref[:, v]).max() / np.abs(ref[:, v]).max() for v in range(ref.shape[1])])
    assert np.all(err <= np.maximum(1e-12, 16 * 2.0 ** -53 * kap)), (err, kap)


@pytest.mark.parametrize("d, kind, basis, p", [(3, 1, LGLL, 4), (3, 0, LGAUSS, 3), (2, 1, LGLL, 6),
                                               (3, 1, LGLL, 7), (2, 0, LGAUSS, 8)])
def test_uncollocated_lagrange_bases(d, kind, basis, p):
    check(d, p, kind, basis, "euler")


@pytest.mark.parametrize("d, kind, p", [(3, 0, 4), (3, 1, 7), (2, 1, 3)])
def test_chandrashekar_and_burgers(d, kind, p):
    check(d, p, kind, LEG, "euler_chandrashekar")
    check(d, p, kind, LEG, "burgers")


@pytest.mark.parametrize("prec", ["fp64", "fp32k"])
@pytest.mark.parametrize("d, kind, p", [(3, 0, 4), (3, 1, 2), (2, 1, 5)])
def test_collocated_basis_matches_the_nodal_entry_point(prec, d, kind, p):
    """With the Lagrange basis of the cubature nodes V = I: the modal entry
    point gives the nodal residual (FP32: bit for bit, same kernel and sums)."""
    basis = LGLL if kind == 0 else LGAUSS
    u, Ja = I.workload(d, p, kind, 3)
    ctx = api.Context(d, p, kind, "euler")
    src = u if prec == "fp64" else I.to_fp32(u)
    dt = torch.float64 if prec == "fp64" else torch.float32
    ut = torch.from_numpy(np.ascontiguousarray(src)).to(dt).cuda()
    Jt = torch.from_numpy(Ja).cuda()
    rn = ctx.volume_residual(ut, Jt, prec).double().cpu().numpy()
    rm = ctx.volume_residual_modal(ut, Jt, basis, prec).double().cpu().numpy()
    if prec == "fp32k":
        assert np.array_equal(rn, rm)
    else:
        assert rel_err_per_var(rm, rn) <= 1e-12


def test_full_size_p4_32cubed_sampled():
    """3D Euler p = 4, Legendre coefficients on 32^3 warped elements with
    Gauss-Lobatto cubature (the benchmark's shape), sampled elements
    recomputed by the oracle."""
    d, p, kind = 3, 4, 0
    uhat, Ja = I.modal_workload(d, p, kind, LEG, 32)
    E = uhat.shape[0]
    rng = np.random.default_rng(51)
    idx = np.unique(np.concatenate([[0, E - 1], rng.choice(E, size=48, replace=False)]))
    ref = O.volume_modal(d, p, kind, LEG, O.FLUX_EULER, uhat[idx], Ja[idx], project=False)
    ref_w = O.volume_modal(d, p, kind, LEG, O.FLUX_EULER, I.to_fp32(uhat[idx]).astype(np.float64), Ja[idx],
                           project=False)
    ctx = api.Context(d, p, kind, "euler")
    errs = {}
    for prec in ("fp64", "fp32k", "fp32mix"):
        got, st = run_modal(ctx, uhat if prec == "fp64" else I.to_fp32(uhat), Ja, LEG, prec)
        assert st == A.SFH_OK
        if prec == "fp64":
            assert rel_err_per_var(got[idx], ref) <= 1e-12
        else:
            errs[prec] = fp32_check_modal(got[idx], ref, ref_w,
                                          modal_terms(d, p, kind, LEG, O.FLUX_EULER,
                                                      I.to_fp32(uhat[idx]).astype(np.float64), Ja[idx]))
    from tests.test_gpu_volume import _report
    _report("parity_modal_legendre_euler_p4_gll_32cubed", errs)


def test_errors_and_domain():
    uhat, Ja = I.modal_workload(3, 3, 1, LEG, 2)
    ctx = api.Context(3, 3, 1, "euler")
    ut, Jt = torch.from_numpy(uhat).cuda(), torch.from_numpy(Ja).cuda()
    r = torch.empty_like(ut)
    with pytest.raises(A.SfhError) as e:
        A.sfh_volume_residual_modal(ctx.handle, 3, ut.shape[0], ut.data_ptr(), Jt.data_ptr(), r.data_ptr(), A.SFH_FP64)
    assert e.value.status == A.SFH_EINVAL
    with pytest.raises(A.SfhError) as e:
        A.sfh_volume_residual_modal(ctx.handle, 0, ut.shape[0], ut.data_ptr(), Jt.data_ptr(), ut.data_ptr(), A.SFH_FP64)
    assert e.value.status == A.SFH_EINVAL
    bad = uhat.copy()
    bad[1, 0, 0] = -bad[1, 0, 0]          # negative mean density in element 1
    for prec in ("fp64", "fp32k", "fp32mix"):
        _, st = run_modal(ctx, bad if prec == "fp64" else I.to_fp32(bad), Ja, LEG, prec)
        assert st == A.SFH_EDOMAIN, prec
        assert ctx.check() == A.SFH_OK     # the error word is cleared by the read
    # empty input is a no-op
    A.sfh_volume_residual_modal(ctx.handle, 0, 0, ut.data_ptr(), Jt.data_ptr(), r.data_ptr(), A.SFH_FP64)



@pytest.mark.parametrize("d, kind, basis, flux_name, p", [(3, 1, LEG, "euler", 4), (3, 0, LGAUSS, "euler", 3),
                                                          (2, 1, LEG, "euler_chandrashekar", 5),
                                                          (3, 1, LEG, "burgers", 2), (3, 0, LEG, "euler", 7),
                                                          (2, 0, LGLL, "euler", 8)])
def test_modal_vjp_parity(d, kind, basis, flux_name, p):
    fl = FLUX[flux_name]
    N = 2 if (d == 3 and p >= 6) else 3
    uhat, Ja = I.modal_workload(d, p, kind, basis, N, flux="burgers" if fl == O.FLUX_BURGERS else "euler")
    lam = I.cotangent(uhat.shape)
    ref = O.vjp_modal(d, p, kind, basis, fl, uhat, Ja, lam)
    ctx = api.Context(d, p, kind, flux_name)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    got = ctx.vjp_modal(t(uhat), t(Ja), t(lam), basis).cpu().numpy()
    assert ctx.check() == A.SFH_OK
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_modal_autograd():
    """torch.autograd through the modal residual: backward calls the modal
    adjoint; its result against the oracle and a directional difference of
    the GPU residual."""
    d, p, kind = 3, 4, 1
    uhat, Ja = I.modal_workload(d, p, kind, LEG, 2)
    lam = I.cotangent(uhat.shape, seed=11)
    ctx = api.Context(d, p, kind, "euler")
    ut = torch.from_numpy(uhat).cuda().requires_grad_()
    Jt, lt = torch.from_numpy(Ja).cuda(), torch.from_numpy(lam).cuda()
    r = api.volume_modal(ut, Jt, ctx, "legendre")
    (r * lt).sum().backward()
    g = ut.grad.cpu().numpy()
    ref = O.vjp_modal(d, p, kind, LEG, O.FLUX_EULER, uhat, Ja, lam)
    assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()
    delta = torch.from_numpy(np.random.default_rng(12).standard_normal(uhat.shape)).cuda()
    h = 1e-6
    with torch.no_grad():
        rp = ctx.volume_residual_modal(ut.detach() + h * delta, Jt, "legendre", "fp64")
        rm = ctx.volume_residual_modal(ut.detach() - h * delta, Jt, "legendre", "fp64")
    fd = float(((rp - rm) * lt).sum() / (2 * h))
    assert abs(float((ut.grad * delta).sum()) - fd) <= 1e-6 * abs(fd)


@pytest.mark.parametrize("modal", [False, True])
@pytest.mark.parametrize("d, p, kind", [(3, 4, 0), (3, 3, 1), (2, 6, 1)])
def test_fp32_unaligned_bases_take_the_plain_load_path(modal, d, p, kind):
    """u and r 4 bytes past a 16-byte boundary: the persistent FP32 kernel
    stages with plain loads instead of bulk copies; the result is the same
    bit for bit (nodal and modal)."""
    if modal:
        src, Ja = I.modal_workload(d, p, kind, LEG, 3)
    else:
        src, Ja = I.workload(d, p, kind, 3)
    ctx = api.Context(d, p, kind, "euler")
    u32 = torch.from_numpy(I.to_fp32(src)).cuda()
    Jt = torch.from_numpy(Ja).cuda()
    n = u32.numel()
    ub = torch.empty(n + 1, dtype=torch.float32, device="cuda")
    rb = torch.empty(n + 1, dtype=torch.float32, device="cuda")
    uo, ro = ub[1:].view(u32.shape), rb[1:].view(u32.shape)
    uo.copy_(u32)
    assert uo.data_ptr() % 16 != 0 and ro.data_ptr() % 16 != 0
    if modal:
        ref = ctx.volume_residual_modal(u32, Jt, "legendre", "fp32k")
        ctx.volume_residual_modal(uo, Jt, "legendre", "fp32k", out=ro)
    else:
        ref = ctx.volume_residual(u32, Jt, "fp32k")
        ctx.volume_residual(uo, Jt, "fp32k", out=ro)
    assert ctx.check() == A.SFH_OK
    assert torch.equal(ref, ro)
