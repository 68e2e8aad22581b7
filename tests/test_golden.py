"""The oracle still reproduces its committed 8^3-cube summary (drift guard)."""
import json
import os

import pytest

from tests.golden.make_golden import summary

HERE = os.path.dirname(os.path.abspath(__file__))


def test_cube8_summary_unchanged():
    with open(os.path.join(HERE, "golden", "cube8_oracle.json")) as f:
        ref = json.load(f)
    got = summary()
    for key in ("nnz", "row_ptr_sum", "col_idx_sum"):
        assert got[key] == ref[key]
    for key in ("A_sum", "A_abs_sum"):
        assert got[key] == pytest.approx(ref[key], rel=1e-13, abs=1e-15)
    for key in ("G_abs_sum", "rhs_abs_sum"):
        assert got[key] == pytest.approx(ref[key], rel=1e-13)
    # signed sums cancel to ~0: compare on the scale of the absolute sums
    for key, scale in (("G_sum", "G_abs_sum"), ("rhs_sum", "rhs_abs_sum")):
        for g, r, s in zip(got[key], ref[key], ref[scale]):
            assert abs(g - r) <= 1e-13 * s
    for p, v in ref["A_at"].items():
        assert got["A_at"][p] == pytest.approx(v, rel=1e-13, abs=1e-18)
