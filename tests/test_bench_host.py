"""Host arithmetic of bench.py's report (no GPU): the roofline object of the
ORAS apply and the whole-job value."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_roofline_of_the_oras_apply():
    """Algorithmic bytes: c64 factor entries (panels + one D^-1 per local row)
    once, plus x in and y out (n x m c64 each); the implementation's count is
    reported beside it."""
    res = {"kernel_calls": [10, 26, 26, 1], "kernel_ms": [5.0, 78.0, 17.0, 37.0],
           "factor": {"oras_bytes_per_call": 7.74e9, "factor_entries": 2.76e8, "nloc": 864937}}
    r = bench.roofline(res, ndof=458220, m=32)
    per_call = 78.0 / 26
    alg = (2.76e8 + 864937) * 8 + 2 * 458220 * 32 * 8
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] is None
    assert r["ms_per_call"] == pytest.approx(per_call)
    assert r["algorithmic_bytes_per_call"] == pytest.approx(alg)
    assert r["achieved"] == pytest.approx(alg / (per_call / 1e3) / 1e9, abs=0.05)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)
    assert r["impl_bytes_per_call"] == 7.74e9
    assert r["frac_impl_traffic"] == pytest.approx(7.74e9 / (per_call / 1e3) / 1e9 / r["peak"], rel=1e-3)
    t = bench.roofline(res, ndof=458220, m=32, traffic={"bytes_per_call": 2 * alg, "source": "x"})
    assert t["traffic"] == 2 * alg and t["traffic_over_algorithmic"] == pytest.approx(2.0)


def test_roofline_absent_without_calls():
    res = {"kernel_calls": [0, 0, 0, 0], "kernel_ms": [0.0] * 4, "factor": {"oras_bytes_per_call": 1.0}}
    assert bench.roofline(res, ndof=1, m=1) is None


def test_whole_job_value_counts_all_replicas():
    assert bench.whole_job_value(4, 64, 5, 1000.0) == pytest.approx(4 * 64 * 5 / 1.0)
