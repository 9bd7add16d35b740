"""The benchmark's work accounting (pairs per element, algorithmic bytes and
flops) checked against the operators themselves: every off-diagonal nonzero
of Q_m = Q1 (x) W (x) W couples an unordered pair of nodes on one line, each
pair appearing twice (Q1[a][b] and Q1[b][a] are both nonzero)."""
import numpy as np
import pytest

import bench
from tests._entropy import kron_q


@pytest.mark.parametrize("d, p, kind", [(3, 2, 0), (3, 4, 0), (3, 3, 1), (2, 5, 1), (2, 6, 0)])
def test_pairs_per_element_matches_q_nonzeros(d, p, kind):
    off = 0
    diag = 0
    for m in range(d):
        Q = kron_q(d, p, kind, m)
        # the oracle's negative-sum diagonal leaves round-off where the exact
        # entry is zero (interior Gauss-Lobatto nodes, the middle Gauss node)
        nz = np.abs(Q) > 1e-12 * np.abs(Q).max()
        off += int(nz.sum() - np.trace(nz))
        diag += int(np.trace(nz))
    assert off % 2 == 0
    assert bench.pairs_per_element(d, p) == off // 2
    # diagonal terms: Gauss-Lobatto only at the two endpoints of each line
    n = p + 1
    lines = d * n ** (d - 1)
    if kind == 0:
        assert diag == 2 * lines
    else:
        assert diag == lines * sum(1 for a in range(n) if not (n % 2 == 1 and a == n // 2))


def test_bytes_per_node():
    assert bench.bytes_per_node("fp32k", 3) == 112
    assert bench.bytes_per_node("fp64", 3) == 152
    assert bench.bytes_per_node("fp32k", 2) == 2 * 4 * 4 + 4 * 8


def test_flops_per_element_composition():
    d, p = 3, 4
    n = p + 1
    lines = d * n ** (d - 1)
    expected = bench.pairs_per_element(d, p) * bench.PAIR_FLOPS + lines * 2 * bench.GAMMA_DIAG \
        + n ** d * (bench.NODE_FLOPS + 10 * d)
    assert bench.flops_per_element(d, p, 0) == expected
    # Gauss: a diagonal term at every node of every line
    assert bench.flops_per_element(d, p, 1) - bench.flops_per_element(d, p, 0) == lines * (n - 2) * bench.GAMMA_DIAG


@pytest.mark.parametrize("d, p, kind", [(3, 4, 0), (3, 4, 1), (2, 3, 1), (3, 7, 1), (2, 6, 0)])
def test_surface_fluxes_match_interpolation_nonzeros(d, p, kind):
    """The surface product's flux count against the nonzeros of the face
    interpolation rows l_b(-1), l_b(+1) (numpy polynomial fit through the
    nodes; Gauss-Lobatto rows are selectors, Gauss rows dense)."""
    import oracle as O
    n = p + 1
    xi, w = np.zeros(n), np.zeros(n)
    O._check(O._load().orc_nodes(p, kind, O._p(xi), O._p(w)))
    nnz = 0
    for b in range(n):
        y = np.zeros(n)
        y[b] = 1.0
        c = np.polynomial.polynomial.polyfit(xi, y, p)
        for x in (-1.0, 1.0):
            nnz += abs(np.polynomial.polynomial.polyval(x, c)) > 1e-10
    assert bench.surface_fluxes_per_element(d, p, kind) == d * n ** (d - 1) * nnz


@pytest.mark.parametrize("p, kind", [(4, 0), (4, 1), (7, 1), (2, 0)])
def test_fp32_pipe_count_and_binding_roofline(p, kind):
    """The FP32-pipe count: pairs x 85 + nonzero diagonal terms x 49 + nodes
    x 45 (3D Euler), diagonal terms counted from the nonzeros of diag(Q1);
    the binding roofline takes the larger of the two floors."""
    import oracle as O
    _, _, _, Q1 = O.op1d(p, kind)
    n = p + 1
    ndiag = int(np.count_nonzero(np.abs(np.diag(Q1)) > 1e-12))
    want = bench.pairs_per_element(3, p) * 85 + 3 * n * n * ndiag * 49 + n ** 3 * 45
    assert bench.fp32_pipe_ops_per_element(3, p, kind) == want
    r = bench.fp32_roofline(3, p, kind, 1000, 1.0, 6800.0)
    assert r["frac"] == pytest.approx(max(r["hbm_frac"], r["fp32_pipe_frac"]))
    assert r["bound"] == ("hbm" if r["t_hbm_ms"] >= r["t_fp32_pipe_ms"] else "alu")


def test_mixed_fp64_work_per_kernel():
    """The mixed mode's FP64 count follows the kernel: 9 instructions and 11
    flops per pair plus 3 / 5 per node on the warp-specialized kernel (3D,
    n = 3..8), 35 flops per pair on the thread-per-line kernel (2D, n = 9)."""
    fl, ins = bench.mix_fp64_work(3, 4, 0)
    assert (fl, ins) == (750 * 11 + 125 * 5, 750 * 9 + 125 * 3)
    assert bench.mix_fp64_work(3, 7, 1)[0] == bench.pairs_per_element(3, 7) * 11 + 8 ** 3 * 5
    assert bench.mix_fp64_work(3, 8, 1)[0] == bench.pairs_per_element(3, 8) * 35
    assert bench.mix_fp64_work(2, 4, 0)[0] == bench.pairs_per_element(2, 4) * 35
