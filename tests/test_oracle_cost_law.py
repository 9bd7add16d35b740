"""The paper's timing experiment (Section 3, Fig. 1) on the oracle: the
generic Hadamard product (sum_j D_j o C) 1 with C = c c^T, c ~ U[1e-8, 30],
evaluated densely costs O(n^{2d}) and sum-factorized O(n^{d+1}) in 3D; the
fitted log-log slopes are 6 and 4.  The two forms agree to round-off."""
import time

import numpy as np
import pytest

import oracle as O


def _best_time(fn, *args, reps=3, min_time=0.02):
    best = float("inf")
    for _ in range(reps):
        k, t0 = 0, time.perf_counter()
        while True:
            fn(*args)
            k += 1
            el = time.perf_counter() - t0
            if el >= min_time:
                break
        best = min(best, el / k)
    return best


@pytest.mark.parametrize("p", [3, 6, 9])
def test_fig1_forms_agree(p):
    c = np.random.default_rng(p).uniform(1e-8, 30.0, size=(p + 1) ** 3)
    yd, ys = O.fig1_dense(p, c), O.fig1_sf(p, c)
    assert np.abs(yd - ys).max() <= 1e-13 * np.abs(yd).max()


def test_fig1_slopes():
    # Each call also builds the nodes and D (O(n^2) work with a large
    # constant), which flattens the sum-factorized curve at small n: its slope
    # is fitted where the n^4 term dominates (p = 14 .. 30); the dense form's
    # n^6 dominates from p = 8 on.
    def slope(fn, ps, **kw):
        t = []
        for p in ps:
            c = np.random.default_rng(p).uniform(1e-8, 30.0, size=(p + 1) ** 3)
            t.append(_best_time(fn, p, c, **kw))
        return np.polyfit(np.log(np.array(ps) + 1.0), np.log(t), 1)[0]
    sd = slope(O.fig1_dense, [8, 10, 12, 14], reps=2, min_time=0.0)
    ss = slope(O.fig1_sf, [14, 18, 24, 30], reps=3, min_time=0.05)
    assert 5.0 < sd < 7.0, sd
    assert 3.0 < ss < 5.0, ss
