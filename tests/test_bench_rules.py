"""Measurement rules of bench.py checked against the paper's own printed
numbers (no GPU): the order-beta regression of Table 1."""
import os

import numpy as np

import bench

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_beta_regression_reproduces_table1():
    """Table 1 (Section 5.1): beta is the log-log slope of T against N divided
    by d = 2, per M row; pooled over the rows (one intercept each) it is the
    printed 1.03."""
    rows = np.loadtxt(os.path.join(GOLDEN, "paper_table1_complexity.txt"))
    Ns = [180, 360, 720, 1440, 2880]
    per_row, pooled = bench.fit_beta(Ns, [r[1:6] for r in rows])
    for b, r in zip(per_row, rows):
        assert abs(b - r[6]) <= 0.01, (b, r[6])
    assert abs(pooled - 1.03) <= 0.005
