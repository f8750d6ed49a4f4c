"""CPU checks of bench.py's roofline arithmetic: the algorithmic work of a
V-cycle, the achieved rate and fraction, and the whole-job throughput."""
import os
import sys

import numpy as np
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


def _st(status, iters=10, norm=1e-6, dt=1e-2):
    return {"status": status, "iters": iters, "final_norm": norm, "dt": dt, "n_particles": 100, "n_levels": 2,
            "nnz_blocks": [900, 60], "n_nodes": [40, 8], "ls_trials": iters, "vcycles": iters}


def test_only_converged_steps_earn_particle_steps():
    """A step that stopped at the iteration cap costs its time and earns
    nothing: 3 of 4 steps converged over 2 s -> 3 N / 2 s."""
    stats = [_st(0), _st(4, 500), _st(0), _st(0)]
    assert bench.credited_rate(1000, stats, 2000.0) == pytest.approx(1500.0)
    assert bench.credited_rate(1000, stats, 2000.0, ws=2) == pytest.approx(3000.0)
    rec = bench.step_record(stats, [1.0, 2.0, 3.0, 4.0])
    assert rec["converged"] == 3 and rec["steps"] == 4
    assert rec["status"] == [0, 4, 0, 0] and rec["iters"] == [10, 500, 10, 10] and rec["ms"][3] == 4.0


def test_mixed_error_metrics():
    c = np.arange(12).reshape(4, 3)
    v64 = np.ones((4, 3))
    v32 = v64.copy()
    v32[2, 1] += 1e-6
    xp = np.full((2, 3), 0.5)
    x64 = xp + 1e-3
    x32 = x64.copy()
    x32[1, 0] += 2e-9
    e = bench.mixed_error(c, v64, x64, c, v32, x32, xp, 0.01)
    assert e["grid_v_rel"] == pytest.approx(1e-6)
    assert e["x_rel"] == pytest.approx(2e-9 / 0.501)
    assert e["x_cells"] == pytest.approx(2e-7)
    assert e["x_rel_to_step_displacement"] == pytest.approx(2e-6)
    e2 = bench.mixed_error(c, v64, x64, c[::-1].copy(), v32, x32, xp, 0.01)
    assert e2["grid_v_rel"] is None
    # mass-weighted: a node of vanishing mass barely counts
    m = np.array([1.0, 1.0, 1e-12, 1.0])
    v32b = v64.copy()
    v32b[2] += 1.0
    e3 = bench.mixed_error(c, v64, x64, c, v32b, x32, xp, 0.01, m=m, vp64=v64[:2], vp32=v64[:2] * 1.5)
    assert e3["grid_v_rel"] == pytest.approx(1.0)
    assert e3["grid_v_rel_mass_weighted"] == pytest.approx(np.sqrt(3e-12 / (9.0 + 3e-12)))
    assert e3["particle_v_rel"] == pytest.approx(0.5)


def test_pair_summary_speedup_and_error_maxima():
    class Sc:
        n, name = 100, "s"
    stats64 = [_st(0), _st(0)]
    stats32 = [_st(0), _st(4, 500)]
    errs = [{"grid_v_rel": 1e-6, "x_rel": 1e-9, "x_cells": 1e-5, "x_rel_to_step_displacement": 1e-4},
            {"grid_v_rel": 3e-6, "x_rel": 2e-9, "x_cells": 3e-5, "x_rel_to_step_displacement": 2e-4}]
    r = {"stats": stats64, "step_ms": [10.0, 10.0], "total_ms": 20.0, "prof_stats": stats64,
         "partner": {"stats": stats32, "step_ms": [4.0, 6.0], "total_ms": 10.0, "errors": errs,
                     "prof_stats": stats32}}
    out = bench.summarize_pair(r, Sc(), {"hbm_gbs": 5000.0}, None)
    assert out["fp64"]["value"] == pytest.approx(200 / 0.02)
    assert out["mixed"]["value"] == pytest.approx(100 / 0.01)      # one converged step of two
    assert out["speedup_mixed_over_fp64"] == pytest.approx(1.0)
    assert out["error_vs_fp64"]["max"]["grid_v_rel"] == pytest.approx(3e-6)
    assert out["mixed"]["converged_steps"] == 1
    assert out["mixed"]["step_hbm"]["bytes_per_step"] == bench.step_traffic(stats32, 1, bench.REFRESH) / 2


def test_reference_arm_line(capsys):
    """bench.py --impl reference: the oracle on the CPU sample, one JSON line
    with the GPU arm's metric and credit rule (one oracle step, ~10 s)."""
    import argparse
    import json
    bench.run_reference(argparse.Namespace(gpus=1, steps=1, warmup=0))
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["converged_steps"] == 1 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_hessian_roofline_counts_every_build():
    """With the hierarchy refreshed, the fine Hessian is assembled several
    times per step: its flops are counted per launch, not per step."""
    st = _stats([1000, 30], [100, 3], vcycles=4)
    prof = {"hessian_cells": {"ms": 10.0, "launches": 5}}
    r = bench.roofline_entry("hessian_cells", prof, [st, st], 1000, 0, {})
    flop = 2 * (27 * 27 * 3 + 378 * 9 * 3) * 1000 * 5
    assert r["algorithmic_total"] == flop and r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(flop / 10e-3 / 1e12)


def test_kernel_traffic_is_pinned_to_its_source(tmp_path, monkeypatch):
    """The ncu DRAM figure is reported only while the kernel's source file
    hashes to the value recorded beside it; otherwise traffic is null."""
    import hashlib
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_1911_07913_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "elastic.cu").write_bytes(b"kernel source v1")
    sha = hashlib.sha256(b"kernel source v1").hexdigest()
    (tmp_path / "profiles" / "hessian_cells_dram.txt").write_text(
        f"# comment: not a value\nelastic_cu_sha256: {sha}\ntwo_bars_600k_fp64_bytes_per_launch: 1234\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("hessian_cells", "two_bars_600k_fp64_bytes_per_launch") == 1234.0
    assert bench.kernel_traffic("hessian_cells", "missing_key") is None
    assert bench.kernel_traffic("vcycle", "two_bars_600k_fp64_l5_bytes_per_vcycle") is None   # no summary file
    (csrc / "elastic.cu").write_bytes(b"kernel source v2")
    assert bench.kernel_traffic("hessian_cells", "two_bars_600k_fp64_bytes_per_launch") is None


def test_committed_traffic_summaries_parse():
    """Both committed summaries carry a source hash and the keys bench.py
    asks for."""
    for name, (summary, source) in bench.TRAFFIC_FILES.items():
        lines = open(os.path.join(ROOT, "profiles", summary)).read().splitlines()
        kv = dict(line.split(": ", 1) for line in lines if ": " in line and not line.startswith("#"))
        assert len(kv[source.replace(".", "_") + "_sha256"]) == 64
    kv = dict(line.split(": ", 1) for line in open(os.path.join(ROOT, "profiles", "vcycle_dram.txt")).read().splitlines()
              if ": " in line and not line.startswith("#"))
    assert float(kv["two_bars_600k_fp64_l5_bytes_per_vcycle"]) > 1e9
    assert float(kv[f"two_bars_2m_mixed_l{bench.LEVELS_2M}_bytes_per_vcycle"]) > 1e9


def test_step_traffic_counts_each_phase():
    """Whole-step algorithmic bytes: the transfers once, an energy per trial
    plus the one at dv = 0, a gradient per iteration plus the first, the
    two-loop per iteration, each V-cycle's block visits and one hierarchy
    build at the first iteration plus one every `refresh` iterations; a step
    that needs no iteration builds nothing."""
    st = {"n_particles": 1000, "n_levels": 3, "nnz_blocks": [5000, 800, 90], "n_nodes": [300, 50, 10],
          "iters": 11, "ls_trials": 13, "vcycles": 11}
    visits = ((7 * (5000 - 300)) // 2 + 5000) + ((7 * (800 - 50)) // 2 + 800)
    fixed = (128 + 288) * 1000 + (32 + 24) * 300
    energies = 14 * (112 * 1000 + 48 * 300)
    grads = 12 * (112 * 1000 + 72 * 300)
    twoloop = 11 * 66 * 24 * 300
    build64 = 2 * 45 * 8 * 1000 + 5000 * 72 + (5000 + 800) * 72 + (800 + 90) * 72
    # refresh 5: builds at the first iteration and after iterations 5 and 10
    assert bench.step_traffic([st], 0, 5) == fixed + energies + grads + twoloop + 11 * visits * 76 + 3 * build64
    build32 = 2 * 45 * 4 * 1000 + 5000 * 36 + (5000 + 800) * 36 + (800 + 90) * 36
    assert bench.step_traffic([st], 1, 0) == fixed + energies + grads + twoloop + 11 * visits * 40 + build32
    rest = {**st, "iters": 0, "ls_trials": 0, "vcycles": 0}
    assert bench.step_traffic([rest], 0, 5) == fixed + (112 * 1000 + 48 * 300) + (112 * 1000 + 72 * 300)
    e = bench.step_hbm_entry([st, st], 0, 5, 2.0, {"hbm_gbs": 5000.0})
    assert abs(e["achieved"] - 2 * bench.step_traffic([st], 0, 5) / 2e-3 / 1e9) < 1e-9
    assert abs(e["frac"] - e["achieved"] / 5000.0) < 1e-12 and e["bytes_per_step"] == bench.step_traffic([st], 0, 5)
