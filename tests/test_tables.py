"""The accuracy-table harness: every row is consistent with the library's own outputs.

The chosen update's exact error equals the error of the returned P; the offline references
order as they must (the truncated SVD is optimal, so no rank-k ID beats it); estimates are
non-negative errors of the same magnitude as the exact ones; least squares on Algorithm 3's J is
no worse than any coefficient update on it; Algorithm 1 selects at most k columns."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_table_rows_are_consistent():
    from paper_2405_16076_gb300 import tables
    from workloads import config1_matrix
    A = config1_matrix(3, m=2048, n=120)
    for k in (8, 16):
        r = tables.table_row(A, k, block=4, seed=3)
        assert r["q_star"] in (4, 5, 6, 7)
        assert abs(r["chosen_exact"] - r["exact"][r["q_star"] - 4]) <= 1e-12
        assert r["svd"] <= r["cpqr"] + 1e-12
        assert r["svd"] <= min(r["exact"]) + 1e-12
        assert all(e >= 0.0 for e in r["estimated"])
        assert r["alg3_ls"] <= r["chosen_exact"] + 1e-12      # least squares is optimal for its J
        assert r["svd"] <= r["alg1_ls"] + 1e-12 and r["svd"] <= r["alg3_ls"] + 1e-12
        assert 0 < r["alg1_n"] <= k
        o = r["alg1_online"]
        assert o["q_star"] in (4, 5, 6, 7)
        assert abs(o["chosen_exact"] - o["exact"][o["q_star"] - 4]) <= 1e-12
        assert r["alg1_ls"] <= o["chosen_exact"] + 1e-12     # same subset: least squares is optimal
    md = tables.markdown([r], "check")
    assert md.count("|") > 10
