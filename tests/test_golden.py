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


def test_cube8_stabilized_summary_unchanged():
    """The stabilised oracle's committed summary: component sums (the
    diagonal components sum to rho/dt times the cube's volume, 100, since
    every other term annihilates constants), absolute sums, five entries'
    blocks and one element's tau1, tau2."""
    from tests.golden.make_golden import stab_summary

    with open(os.path.join(HERE, "golden", "cube8_stab_oracle.json")) as f:
        ref = json.load(f)
    got = stab_summary()
    assert got["nnz"] == ref["nnz"]
    for c in range(9):
        assert abs(got["Auu_sum"][c] - ref["Auu_sum"][c]) <= 1e-13 * ref["Auu_abs_sum"][c]
        assert got["Auu_abs_sum"][c] == pytest.approx(ref["Auu_abs_sum"][c], rel=1e-13)
    for c in (0, 4, 8):
        assert ref["Auu_sum"][c] == pytest.approx(100.0, rel=1e-13)
    for p, v in ref["Auu_at"].items():
        assert got["Auu_at"][p] == pytest.approx(v, rel=1e-13, abs=1e-18)
    assert got["tau_element0"] == pytest.approx(ref["tau_element0"], rel=1e-14)
