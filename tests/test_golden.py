"""Fixtures under tests/golden: the paper's printed values (cited there) and
the oracle's regression values (written by make_oracle_golden.py)."""
import json
import os

import numpy as np

import oracle as O
from paper_2306_11665_gb300 import inputs as I

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_paper_values_present_and_consistent():
    pv = json.load(open(os.path.join(HERE, "paper_values.json")))
    d = 3
    # the paper's slopes are the exponents of the two cost laws in 3D
    assert pv["fig1_slope_dense_3d"]["value"] == 2 * d
    assert pv["fig1_slope_sum_factorized_3d"]["value"] == d + 1


def test_oracle_regression():
    g = json.load(open(os.path.join(HERE, "oracle_regression.json")))
    u, Ja = I.workload(2, 3, O.NODES_GLL, 8, flux="burgers", amp=0.0)
    r = O.volume_sf(2, 3, O.NODES_GLL, O.FLUX_BURGERS, u, Ja).ravel()
    ent = g["burgers2d_p3_8x8"]
    np.testing.assert_allclose(r[ent["flat_index"]], ent["r"], rtol=1e-13, atol=1e-16)
    u, Ja = I.workload(3, 4, O.NODES_GLL, 4, n_elem=3)
    r = O.volume_sf(3, 4, O.NODES_GLL, O.FLUX_EULER, u, Ja).ravel()
    ent = g["euler3d_p4_gll_warped_4cubed_e0_3"]
    np.testing.assert_allclose(r[ent["flat_index"]], ent["r"], rtol=1e-13, atol=1e-16)
