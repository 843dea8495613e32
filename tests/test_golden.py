"""Fixtures under tests/golden: the numbers the paper prints that the implementation adopts, and
a regression record of the oracle written by tests/golden/make_oracle_golden.py."""
import json
import os

import numpy as np

import oracle
from synthetic import bumpy_plane

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def test_paper_values_are_the_defaults():
    g = load("paper_values.json")
    p = oracle.OracleParams(nx=10, ny=10, n_yaw=8, res=0.1, length=0.6, width=0.4)
    assert p.phi_x_max == g["phi_x_max_rad"]["value"] and p.phi_y_max == g["phi_y_max_rad"]["value"]
    from paper_2503_02412_gb300.maps import SebParams

    q = SebParams(nx=10, ny=10, n_yaw=8, res=0.1, length=0.6, width=0.4)
    assert abs(q.phi_x_max - 0.52) < 1e-7 and abs(q.phi_y_max - 0.52) < 1e-7


def test_cycle_configuration_is_the_papers_densest():
    import bench

    g = load("paper_values.json")
    assert bench.CYCLE_SIDE ** 2 * bench.CYCLE_YAWS == g["densest_se2_grids"]["value"]
    assert abs(bench.CYCLE_SIDE * bench.CYCLE_RES - g["map_side_m_max"]["value"]) < 1e-9
    assert bench.CYCLE_RES == g["map_res_m"]["value"]
    lo, hi = g["so2_bins_range"]["value"]
    assert lo <= bench.CYCLE_YAWS <= hi


def test_oracle_regression_record():
    g = load("oracle_bumpy_c1.json")
    p = oracle.OracleParams(nx=100, ny=100, n_yaw=36, res=0.1, length=0.6, width=0.4)
    out, flags, _ = oracle.assess_cells(p, bumpy_plane(0).astype(np.float64), np.array(g["cells"], np.int32))
    assert np.array_equal(flags, np.array(g["flags"], np.uint8))
    ref = np.array(g["out"])
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(out), fin) and np.allclose(out[fin], ref[fin], rtol=0, atol=1e-12)
