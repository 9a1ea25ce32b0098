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


def test_workload_table_is_consistent():
    """Every benchmark workload has the GPU step count the reference arm
    scales by and a positive node damping; both arms report the same alpha."""
    for name, (fac, alpha, graphs, label, l2) in bench.WORKLOADS.items():
        assert name in bench.GPU_STEPS_PER_SOLVE and bench.GPU_STEPS_PER_SOLVE[name] > 0
        assert alpha > 0 and label and l2


def test_job_rate_and_clock_reasons():
    """Whole-job rate on one process, and the throttle reasons the clock
    sampler reports from nvidia-smi lines (median SM clock, max power)."""
    ms, rate = bench.job_rate(None, 1, 4, 2000.0)
    assert ms == 2000.0 and abs(rate - 2.0) < 1e-12

    class P:  # a finished nvidia-smi process
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs = bench.ClockSampler(0)
    cs.proc = P()
    cs.lines = ["2070, 2070, 600.5, 0x0, Not Active, Not Active, Not Active, Not Active",
                "2040, 2070, 640.0, 0x4, Not Active, Not Active, Not Active, Active",
                "2070, 2070, 610.0, 0x0, Not Active, Not Active, Not Active, Not Active",
                "garbage"]
    c = cs.stop()
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["power_w_max"] == 640.0 and c["reasons"] == ["sw_power_cap"]
