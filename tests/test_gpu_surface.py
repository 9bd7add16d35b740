"""GPU parity of the surface Hadamard product (sfh_surface_hadamard, FP64)
against the oracle's dense definition: both outputs (the volume sums and the
face sums) within 1e-12 relative per variable, for Burgers, Ranocha's and
Chandrashekar's flux, Gauss-Lobatto (selector interpolation) and Gauss
(dense interpolation rows) nodes, d = 2, 3, p = 1..8; a full-size mesh on
sampled elements; argument errors."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2306_11665_gb300 import _abi as A
from paper_2306_11665_gb300 import api
from paper_2306_11665_gb300 import inputs as I
from tests._helpers import rel_err_per_var

pytestmark = pytest.mark.gpu

FLUX = {"euler": O.FLUX_EULER, "euler_chandrashekar": O.FLUX_CHANDRASHEKAR, "burgers": O.FLUX_BURGERS}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2306_11665_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def run(ctx, u, uf, nJ):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    rv, rf = ctx.surface_hadamard(t(u), t(uf), t(nJ))
    return rv.cpu().numpy(), rf.cpu().numpy(), ctx.check()


def rel_face(got, ref):
    E, F, V, nf = ref.shape
    return rel_err_per_var(got.transpose(0, 1, 3, 2).reshape(E * F * nf, V, 1),
                           ref.transpose(0, 1, 3, 2).reshape(E * F * nf, V, 1))


@pytest.mark.parametrize("flux", ["euler", "euler_chandrashekar", "burgers"])
@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("p", [1, 2, 4, 7, 8])
def test_parity_small(flux, d, kind, p):
    N = 2 if (d == 3 and p >= 6) else 3
    fl = "burgers" if flux == "burgers" else "euler"
    u, uf, nJ = I.surface_workload(d, p, kind, N, flux=fl)
    ref_v, ref_f = O.surface_dense(d, p, kind, FLUX[flux], u, uf, nJ)
    rv, rf, st = run(api.Context(d, p, kind, flux), u, uf, nJ)
    assert st == A.SFH_OK
    assert rel_err_per_var(rv, ref_v) <= 1e-12
    assert rel_face(rf, ref_f) <= 1e-12


def test_full_size_p4_32cubed_sampled():
    d, p, kind = 3, 4, 1
    u, uf, nJ = I.surface_workload(d, p, kind, 32)
    E = u.shape[0]
    rv, rf, st = run(api.Context(d, p, kind, "euler"), u, uf, nJ)
    assert st == A.SFH_OK
    idx = np.unique(np.concatenate([[0, E - 1], np.random.default_rng(61).choice(E, size=40, replace=False)]))
    ref_v, ref_f = O.surface_dense(d, p, kind, O.FLUX_EULER, u[idx], uf[idx], nJ[idx])
    assert rel_err_per_var(rv[idx], ref_v) <= 1e-12
    assert rel_face(rf[idx], ref_f) <= 1e-12


def test_errors_and_domain():
    d, p, kind = 3, 3, 1
    u, uf, nJ = I.surface_workload(d, p, kind, 2)
    ctx = api.Context(d, p, kind, "euler")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    ut, ft, jt = t(u), t(uf), t(nJ)
    rv, rf = torch.empty_like(ut), torch.empty_like(ft)
    with pytest.raises(A.SfhError) as e:       # output overlapping an input
        A.sfh_surface_hadamard(ctx.handle, u.shape[0], ut.data_ptr(), ft.data_ptr(), jt.data_ptr(), ut.data_ptr(),
                               rf.data_ptr())
    assert e.value.status == A.SFH_EINVAL
    with pytest.raises(A.SfhError) as e:       # misaligned
        A.sfh_surface_hadamard(ctx.handle, u.shape[0], ut.data_ptr() + 4, ft.data_ptr(), jt.data_ptr(), rv.data_ptr(),
                               rf.data_ptr())
    assert e.value.status == A.SFH_EINVAL
    A.sfh_surface_hadamard(ctx.handle, 0, 0, 0, 0, 0, 0)   # empty: no-op
    bad = uf.copy()
    bad[1, 2, 0, 3] = -1.0                     # negative density in a face state
    _, _, st = run(ctx, u, bad, nJ)
    assert st == A.SFH_EDOMAIN
    assert ctx.check() == A.SFH_OK
