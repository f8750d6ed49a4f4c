"""CPU checks of bench.py's roofline arithmetic: the algorithmic work of a
V-cycle, the achieved rate and fraction, and the whole-job throughput."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _stats(nnz, n, vcycles):
    return {"n_levels": len(n), "nnz_blocks": list(nnz), "n_nodes": list(n), "vcycles": vcycles}


def test_vcycle_block_visits_per_level():
    """Per level m < M-1: 3.5 sweeps over the off-diagonal blocks (the first
    forward half needs only the earlier-colored half) plus one residual over
    all blocks; the coarsest level (PCG) is not counted."""
    nnz, n = [1000, 200, 30], [100, 20, 3]
    st = _stats(nnz, n, vcycles=3)
    visits = sum((7 * (a - b)) // 2 + a for a, b in zip(nnz[:-1], n[:-1])) * 3
    assert visits == ((3150 + 1000) + (630 + 200)) * 3
    flop, unit = bench.algorithmic_units("vcycle", [st], 0, precision=0)
    assert unit == "flop" and flop == 18 * visits
    byte, unit = bench.algorithmic_units("vcycle", [st, st], 0, precision=1)
    assert unit == "byte" and byte == 2 * 40 * visits


def test_hessian_flop_count():
    flop, unit = bench.algorithmic_units("hessian_cells", [{}, {}], 1000, 0)
    assert unit == "flop" and flop == 2 * (27 * 27 * 3 + 378 * 9 * 3) * 1000 * 2


def test_roofline_fraction_and_bound():
    st = _stats([1000, 30], [100, 3], vcycles=4)
    prof = {"vcycle": {"ms": 2.0, "launches": 4}}
    r = bench.roofline_entry("vcycle", prof, [st], 0, 1, {"hbm_gbs": 5000.0})
    byte = 40 * ((7 * 900) // 2 + 1000) * 4
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(byte / 2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 5000.0)
    assert r["avg_launch_ms"] == pytest.approx(0.5)
    r64 = bench.roofline_entry("vcycle", prof, [st], 0, 0, {"hbm_gbs": 5000.0})
    assert r64["bound"] == "alu" and r64["peak"] == pytest.approx(152 * 4 * 2.07e9 / 1e12, rel=1e-3)
    assert bench.roofline_entry("vcycle", {}, [st], 0, 0, {}) is None


def test_job_throughput_is_whole_job_over_slowest_rank():
    # 4 ranks, 1000 units each, 5 steps, slowest rank 250 ms
    assert bench.job_throughput(1000, 4, 5, 250.0) == pytest.approx(4 * 1000 * 5 / 0.25)
