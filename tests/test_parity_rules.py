"""The comparison rules of tests/parity.py on synthetic rows (no GPU): ill-conditioned cells are
checked against the gap-scaled bound, not skipped, and the other cells against the plain
tolerances."""
import numpy as np
import pytest

from .parity import C_GAP, U32, compare


def rows(n=6):
    ref = np.zeros((n, 5))
    ref[:, 0] = 1.0
    ref[:, 1] = 0.1
    ref[:, 2] = -0.05
    ref[:, 3] = 0.01
    ref[:, 4] = 0.2
    return ref, np.zeros(n, np.uint8)


def test_plain_cells_hold_the_plain_tolerance():
    ref, fl = rows()
    gap = np.full(len(ref), 0.3)
    gpu = ref.copy()
    gpu[2, 1] += 0.9e-4
    s = compare(gpu, fl, ref, fl, gap=gap)
    assert s["ill"] == 0 and s["max1"] == pytest.approx(0.9e-4)
    gpu[2, 1] += 0.2e-4
    with pytest.raises(AssertionError, match="channel 1"):
        compare(gpu, fl, ref, fl, gap=gap)


def test_ill_cells_are_checked_against_the_gap_bound():
    ref, fl = rows()
    gap = np.full(len(ref), 0.3)
    gap[3] = 1e-7  # bound C_GAP u / (1e-7 n_z)
    nz = np.sqrt(1 - np.sin(0.1) ** 2 - np.sin(-0.05) ** 2)
    bound = C_GAP * U32 / (1e-7 * nz)
    assert bound > 1e-4
    gpu = ref.copy()
    gpu[3, 1] += 0.9 * bound
    s = compare(gpu, fl, ref, fl, gap=gap)
    assert s["ill"] == 1 and 0.85 < s["ill_ratio"] < 0.95
    gpu[3, 1] += 0.2 * bound
    with pytest.raises(AssertionError, match="channel 1"):
        compare(gpu, fl, ref, fl, gap=gap)


def test_ill_cells_keep_the_plain_roughness_tolerance():
    ref, fl = rows()
    gap = np.full(len(ref), 0.3)
    gap[1] = 1e-9
    gpu = ref.copy()
    gpu[1, 3] += 4e-5  # an eigenvalue is not divided by the gap
    with pytest.raises(AssertionError, match="channel 3"):
        compare(gpu, fl, ref, fl, gap=gap)


def test_unknown_bits_must_match():
    ref, fl = rows()
    g = fl.copy()
    g[0] = 1
    with pytest.raises(AssertionError, match="UNKNOWN"):
        compare(ref, g, ref, fl)
