"""Host-side statistics of the bench: the two observations of Sec. 5.2.2 on
the enumerated best omega (share in [0.5, 2]; zigzag of its moves), checked
on sequences whose answers are known."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_alternating_sequence_is_a_perfect_zigzag():
    st = bench.best_omega_stats([np.array([0.5, 2.0] * 20)])
    assert st["in_0.5_2"] == 1.0
    assert st["turning_points"] == 1.0
    assert st["lag1_autocorr"] == pytest.approx(-1.0)


def test_monotone_sequence_has_no_turning_point():
    st = bench.best_omega_stats([np.arange(0.0, 9.5, 0.5)])
    assert st["turning_points"] == 0.0
    assert st["in_0.5_2"] == pytest.approx(4 / 19)


def test_independent_sequence_matches_its_expectations():
    rng = np.random.default_rng(0)
    st = bench.best_omega_stats([rng.random(200000)])
    assert st["turning_points"] == pytest.approx(2 / 3, abs=0.01)
    assert st["lag1_autocorr"] == pytest.approx(-0.5, abs=0.01)


def test_repeats_are_not_moves():
    # omega held for a while then changed: only the changes count
    st = bench.best_omega_stats([np.array([1.0, 1.0, 2.0, 2.0, 1.0, 1.0, 2.0])])
    assert st["turning_points"] == 1.0
