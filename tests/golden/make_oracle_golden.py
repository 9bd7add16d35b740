"""Writes tests/golden/oracle_regression.json from the oracle alone.

The stored values are a regression fixture: any later change to the oracle's
arithmetic that moves them must say, in its commit message, which passage of
the paper (or which reading of it) justifies the change.
Run:  python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2306_11665_gb300 import inputs as I  # noqa: E402


def main():
    out = {}
    # 2D Burgers, p=3 Gauss-Lobatto, 8x8 affine elements on [0,1]^2
    u, Ja = I.workload(2, 3, O.NODES_GLL, 8, flux="burgers", amp=0.0)
    r = O.volume_sf(2, 3, O.NODES_GLL, O.FLUX_BURGERS, u, Ja)
    idx = list(range(0, r.size, 37))
    out["burgers2d_p3_8x8"] = {"flat_index": idx, "r": [float(r.ravel()[i]) for i in idx]}
    # 3D Euler, p=4 Gauss-Lobatto, first 3 elements of the warped 4^3 mesh
    u, Ja = I.workload(3, 4, O.NODES_GLL, 4, n_elem=3)
    r = O.volume_sf(3, 4, O.NODES_GLL, O.FLUX_EULER, u, Ja)
    idx = list(range(0, r.size, 53))
    out["euler3d_p4_gll_warped_4cubed_e0_3"] = {"flat_index": idx, "r": [float(r.ravel()[i]) for i in idx]}
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
