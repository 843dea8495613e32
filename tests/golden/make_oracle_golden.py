"""Writes oracle_bumpy_c1.json: FP64 oracle outputs at fixed cells of a seeded 100x100x36 map, a
regression record of the oracle itself (calls only oracle/ and synthetic/).  Run from the repo
root: python tests/golden/make_oracle_golden.py"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from synthetic import bumpy_plane  # noqa: E402

CELLS = [[c, r, k] for c, r, k in zip(range(5, 95, 9), range(90, 0, -8), range(0, 36, 3))]


def main():
    e = bumpy_plane(0).astype(np.float64)
    p = oracle.OracleParams(nx=100, ny=100, n_yaw=36, res=0.1, length=0.6, width=0.4)
    out, flags, gap = oracle.assess_cells(p, e, np.array(CELLS, np.int32))
    rec = {"_about": "oracle.assess_cells on synthetic.bumpy_plane(0), 100x100x36, 0.1 m, 0.6x0.4 m footprint",
           "cells": CELLS, "out": out.tolist(), "flags": flags.tolist()}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_bumpy_c1.json"), "w") as f:
        json.dump(rec, f, indent=1)


if __name__ == "__main__":
    main()
