"""GPU form of the paper's timing experiment (Section 3, Fig. 1): the
generic Hadamard product y = sum_m (D_m o c c^T) 1 on Gauss-Lobatto nodes,
sum-factorized and dense, against the oracle's two evaluations."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2306_11665_gb300 import _abi as A

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2306_11665_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _run(p, c, dense):
    ct = torch.from_numpy(c).cuda()
    y = torch.empty_like(ct)
    A.sfh_fig1_hadamard(p, c.shape[0], ct.data_ptr(), y.data_ptr(), dense, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("p", [1, 3, 6, 9, 12, 15])
def test_fig1_matches_oracle(p):
    n3 = (p + 1) ** 3
    rng = np.random.default_rng(100 + p)
    c = rng.uniform(1e-8, 30.0, size=(3, n3))
    sf = _run(p, c, False)
    dn = _run(p, c, True)
    for e in range(3):
        ref_sf, ref_dn = O.fig1_sf(p, c[e]), O.fig1_dense(p, c[e])
        scale = np.abs(ref_dn).max()
        assert np.abs(sf[e] - ref_sf).max() <= 1e-12 * scale
        assert np.abs(dn[e] - ref_dn).max() <= 1e-12 * scale
    assert np.abs(sf - dn).max() <= 1e-12 * np.abs(dn).max()


def test_fig1_argument_errors():
    c = torch.ones(2, 64, dtype=torch.float64, device="cuda")
    y = torch.empty_like(c)
    for bad_p in (0, 16):
        with pytest.raises(A.SfhError) as e:
            A.sfh_fig1_hadamard(bad_p, 2, c.data_ptr(), y.data_ptr(), False)
        assert e.value.status == A.SFH_EINVAL
    with pytest.raises(A.SfhError) as e:
        A.sfh_fig1_hadamard(3, 2, c.data_ptr(), c.data_ptr() + 8, False)
    assert e.value.status == A.SFH_EINVAL
    A.sfh_fig1_hadamard(3, 0, 0, 0, True)   # no elements: no-op
