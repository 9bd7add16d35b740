"""Failure detection on the GPU without a fault: a bounded wait that runs
out (a barrier phase nothing completes) returns SFH_ETIMEOUT to the host,
and the context stays usable afterwards."""
import pytest
import torch

import oracle as O
from paper_2306_11665_gb300 import _abi as A
from paper_2306_11665_gb300 import api
from paper_2306_11665_gb300 import inputs as I
from tests._helpers import rel_err_per_var

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2306_11665_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def test_bounded_wait_gives_up_and_reports_timeout():
    st, el = A.sfh_selftest_bounded_wait(50_000, torch.cuda.current_stream().cuda_stream)
    assert st == A.SFH_ETIMEOUT
    assert 45_000 <= el <= 5_000_000, el
    # the device and a context work normally afterwards
    ctx = api.Context(3, 3, "gll", "euler")
    u, Ja = I.workload(3, 3, 0, 2)
    r = ctx.volume_residual(torch.from_numpy(u).cuda(), torch.from_numpy(Ja).cuda(), "fp64")
    assert ctx.check() == A.SFH_OK
    assert rel_err_per_var(r.cpu().numpy(), O.volume_sf(3, 3, 0, O.FLUX_EULER, u, Ja)) <= 1e-12


def test_bounded_wait_rejects_bad_limits():
    for bad in (0, -5, 10_000_001):
        with pytest.raises(A.SfhError) as e:
            A.sfh_selftest_bounded_wait(bad)
        assert e.value.status == A.SFH_EINVAL
