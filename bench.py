#!/usr/bin/env python
"""Throughput of the HOT implicit MPM step on GB300: particle-steps/s at a
fixed residual tolerance.

Default workload: two twisted bars, 601,600 particles on a sparse 256^3 grid
(dx = 1/256), Neo-Hookean E = 1e5 / 1e9 Pa, nu = 0.4, rho = 2000, ends
rotating at +-1 rad/s, dt at CFL 0.6 (24 FPS cap), 5-level multigrid, FP64,
characteristic-norm tolerance eps = 1e-7 (Sec. 5.2, Sec. 6.1).  A step is one
full implicit step (P2G, HOT solve, G2P) on device-resident particles.  Only
steps whose solve met the tolerance earn particle-steps; every step's status,
iteration count and final norm is printed.  Also reported: the same metric
end to end through the C ABI with host buffers, the mixed-precision form
against FP64 on the same scenes (600k and 2M particles) with its per-step
error, the dominant kernel against its roofline, p50/p99 step latency, batched
and served stepping, the paper's comparison solvers, and the FP64 oracle on
the host cores (one core and all cores).

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1911_07913_gb300 import scenes  # noqa: E402

METRIC = "particle-steps/s at fixed residual tol (HOT implicit MPM step)"
UNIT = "particle-steps/s"

# FP64 pipe of GB300: 2 FP64 FMA per SM per clock -> 152 SMs x 4 flop x 2.07
# GHz = 1.259 TFLOP/s (the nominal 1.25 TFLOP/s); bench.py also measures it
# live with the library's FMA probe and reports both.
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12

# Every timed configuration rebuilds the projected Hessian and its hierarchy
# at the current iterate every REFRESH iterations of an unconverged solve (an
# extension of Alg. 3, which builds it once per step): with the hierarchy of
# dv = 0 alone, L-BFGS stalls on steps whose Hessian changes strongly within
# the step (measured on these scenes; the comparison is in the design notes).
REFRESH = 5
# Multigrid levels of the 2M-particle scene: one more than the 600k scene's 5,
# so that the coarsest level has the same 105 nodes in both (measured: mixed
# V-cycle 3.50 -> 2.63 ms, the coarsest CG's ~80 iterations per V-cycle on
# 312 nodes gone; FP64 step time unchanged, mixed step 4% faster).
LEVELS_2M = 6


def workload_opts(precision: int, refresh: int = REFRESH, levels: int = 5) -> scenes.SolverOptions:
    return scenes.SolverOptions(eps=1e-7, cn_mode=0, lbfgs_m=8, levels=levels, precision=precision,
                                max_iters=500, refresh_every=refresh)


def workload_desc(sc, opts, extra=None):
    if sc.name.startswith("cube"):
        what = f"{sc.name}: FCR cube E=1e5 Pa, nu=0.3, random initial velocity, sticky floor, 32^3 grid"
    else:
        what = (f"{sc.name}: two twisted Neo-Hookean bars E=1e5/1e9 Pa, nu=0.4, rho=2000, "
                f"ends at +-1 rad/s, sparse {int(sc.grid_dims[0])}^3 grid")
    d = {"workload": what,
         "particles": sc.n, "dx": sc.dx, "levels": opts.levels, "lbfgs_window": opts.lbfgs_m,
         "tolerance": f"CN eps={opts.eps}" if opts.cn_mode == 0 else f"||g|| <= {opts.eps} ||g1||",
         "dt": "min(1/24, 0.6 dx / v_max)" if opts.dt <= 0 else opts.dt,
         "solver": ("HOT: L-BFGS (Alg. 3) preconditioned by the Galerkin V-cycle (Alg. 2)"
                    + (f", hierarchy rebuilt at the iterate every {opts.refresh_every} iterations"
                       if opts.refresh_every else "")),
         "max_iters": opts.max_iters,
         "precision": "fp64" if opts.precision == 0 else "mixed (fp32 Hessian/V-cycle, fp64 E/grad/L-BFGS/CN)",
         "l2": "inputs larger than L2 (particles + Hessian > 129 MB)"}
    if extra:
        d.update(extra)
    return d


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, ws: int, steps: int, t_max_ms: float) -> float:
    """Whole-job rate: the units every rank processed over the slowest rank's time."""
    return units_per_rank * ws * steps / (t_max_ms / 1e3)


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def algorithmic_units(name: str, stats_list, n_particles: int, precision: int, launches=None):
    """Algorithmic work of kernel `name` summed over the timed steps.

    vcycle (the captured V-cycle of Alg. 2): per level m < M-1 four
    Gauss-Seidel sweeps over the off-diagonal blocks, of which the first
    (forward, from u = 0) needs only the blocks of earlier-colored
    neighbours -- exactly half of the off-diagonal blocks, since every
    coupling joins two colors -- and one residual over all blocks.  FP64:
    9 FMA = 18 flop per block visit (the FP64 pipe bounds it).  FP32: 36 B of
    block values + 4 B column index per block visit (HBM bounds it).  The
    coarsest PCG (latency bound, shared-memory resident) is not counted.
    hessian_cells: 27*27*3 + 378*9*3 FMA = 24,786 flop per particle and
    launch (one launch per hierarchy build: several per step with the
    refresh; `launches` when known, else one per step)."""
    if name == "hessian_cells":
        n_launch = launches if launches is not None else len(stats_list)
        return 2 * (27 * 27 * 3 + 378 * 9 * 3) * n_particles * n_launch, "flop"
    visits = 0
    for st in stats_list:
        nl = st["n_levels"]
        for m in range(nl - 1):
            nnz, n = st["nnz_blocks"][m], st["n_nodes"][m]
            visits += ((7 * (nnz - n)) // 2 + nnz) * st["vcycles"]
    if precision == 0:
        return 18 * visits, "flop"
    return 40 * visits, "byte"


def step_traffic(stats_list, precision: int, refresh: int) -> int:
    """Algorithmic HBM bytes of whole steps, summed over stats_list:
    P2G 128 B per particle (x, v, C, m) + 32 B per node (m, m v written);
    G2P 288 B per particle (x, F read; x, v, C, F written) + 24 B per node;
    every energy evaluation (the one at dv = 0 and each line-search trial)
    112 B per particle + 48 B per node; every gradient (at dv = 0 and after
    each iteration) 112 B per particle + 72 B per node; the two-loop 66 vector
    passes of 24 B per node per iteration (window 8); each V-cycle its block
    visits (as in algorithmic_units) at 76 B (FP64: 72 B of values and a
    column index) or 40 B (FP32); each hierarchy build (at the first
    iteration, and again every `refresh` iterations) the per-particle
    stiffness (45 values) written and read, the fine matrix written, and
    every Galerkin level's finer matrix read and its own written."""
    vb = 76 if precision == 0 else 40
    bb = 72 if precision == 0 else 36
    sb = 8 if precision == 0 else 4
    total = 0
    for st in stats_list:
        npart, n0, its, trials = st["n_particles"], st["n_nodes"][0], st["iters"], st["ls_trials"]
        nnz, nodes, nl = st["nnz_blocks"], st["n_nodes"], st["n_levels"]
        total += 128 * npart + 32 * n0 + 288 * npart + 24 * n0
        total += (1 + trials) * (112 * npart + 48 * n0)
        total += (1 + its) * (112 * npart + 72 * n0)
        total += its * 66 * 24 * n0
        visits = sum((7 * (nnz[m] - nodes[m])) // 2 + nnz[m] for m in range(nl - 1))
        total += st["vcycles"] * visits * vb
        builds = 0 if its == 0 else 1 + ((its - 1) // refresh if refresh > 0 else 0)
        build = 2 * 45 * sb * npart + nnz[0] * bb + sum((nnz[m] + nnz[m + 1]) * bb for m in range(nl - 1))
        total += builds * build
    return total


def step_hbm_entry(stats_list, precision, refresh, total_ms, peaks):
    """Whole-step achieved bandwidth: step_traffic over the timed steps' time."""
    if not stats_list or total_ms <= 0:
        return None
    b = step_traffic(stats_list, precision, refresh)
    achieved = b / (total_ms / 1e3) / 1e9
    hbm = peaks.get("hbm_gbs", 6800.0)
    return {"bytes_per_step": b / len(stats_list), "achieved": achieved, "unit": "GB/s", "peak": hbm,
            "frac": achieved / hbm, "peak_source": "of measured" if "hbm_gbs" in peaks else "of fallback",
            "note": "algorithmic bytes of the whole step (P2G, energies, gradients, two-loop, V-cycles, hierarchy "
                    "builds, G2P) over the device time of the timed steps; the FP64 step is bound by the FP64 "
                    "pipe, not by these bytes"}


# committed ncu DRAM figures per roofline unit: summary file and the source file whose hash pins them
TRAFFIC_FILES = {"vcycle": ("vcycle_dram.txt", "multigrid.cu"),
                 "hessian_cells": ("hessian_cells_dram.txt", "elastic.cu")}


def kernel_traffic(name, key):
    """DRAM bytes per roofline unit (dram__bytes_read.sum + dram__bytes_write.sum:
    over the kernels of one V-cycle, or of one Hessian-assembly launch) from
    the committed ncu summary, or None when the kernel's source changed after
    that capture."""
    if name not in TRAFFIC_FILES:
        return None
    summary, source = TRAFFIC_FILES[name]
    try:
        lines = open(os.path.join(ROOT, "profiles", summary)).read().splitlines()
        src = open(os.path.join(ROOT, "paper_1911_07913_gb300", "csrc", source), "rb").read()
    except OSError:
        return None
    kv = dict(line.split(": ", 1) for line in lines if ": " in line and not line.startswith("#"))
    if kv.get(source.replace(".", "_") + "_sha256") != hashlib.sha256(src).hexdigest():
        return None
    v = kv.get(key)
    return float(v) if v else None


def roofline_entry(name, prof, stats_list, n_particles, precision, peaks, traffic_key=None, fp64_probe=None):
    """Dominant-kernel roofline from live CUDA-event times over the timed steps."""
    p = prof.get(name)
    if not p or p["launches"] == 0:
        return None
    units, kind = algorithmic_units(name, stats_list, n_particles, precision, launches=p["launches"])
    secs = p["ms"] / 1e3
    traffic = kernel_traffic(name, traffic_key) if traffic_key else None
    base = {"kernel": name, "traffic": traffic,
            "traffic_unit": "DRAM bytes per V-cycle (ncu)" if name == "vcycle" else "DRAM bytes per launch (ncu)",
            "launches": p["launches"],
            "avg_launch_ms": p["ms"] / p["launches"], "algorithmic_total": units, "algorithmic_unit": kind,
            "timed": f"CUDA events around every {name} launch, over a replay of the timed steps from their start state"}
    if kind == "flop":
        achieved = units / secs / 1e12
        out = {**base, "bound": "alu", "achieved": achieved, "peak": round(FP64_PEAK_TFLOPS, 3),
               "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
               "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2.07 GHz (nominal 1.25 TFLOP/s)"}
        if fp64_probe:
            out["fp64_probe_tflops"] = fp64_probe
            out["frac_of_probe"] = achieved / fp64_probe
        return out
    achieved = units / secs / 1e9
    hbm = peaks.get("hbm_gbs", 6800.0)
    return {**base, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "peak_source": "of measured" if "hbm_gbs" in peaks else "of fallback"}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# --------------------------------------------------------------------------- our arm
def step_record(stats, step_ms=None):
    """Per-step status of a run: iterations, mpm_status, final termination
    norm, dt (and device time); `converged` counts the steps whose solve met
    the tolerance (status 0)."""
    rec = {"iters": [int(s["iters"]) for s in stats], "status": [int(s["status"]) for s in stats],
           "cn_norm": [float("%.4g" % s["final_norm"]) for s in stats],
           "dt": [float("%.5g" % s["dt"]) for s in stats]}
    if step_ms is not None:
        rec["ms"] = [round(float(x), 3) for x in step_ms]
    rec["converged"] = sum(1 for s in stats if int(s["status"]) == 0)
    rec["steps"] = len(stats)
    return rec


def credited_rate(n_particles: int, stats, total_ms: float, ws: int = 1) -> float:
    """Particle-steps/s counting only the steps that met the tolerance, over
    the time of all steps: an unconverged step costs time and earns nothing."""
    conv = sum(1 for s in stats if int(s["status"]) == 0)
    return n_particles * ws * conv / (total_ms / 1e3)


def timed_steps(g, steps, stream):
    """K steps of scene g between CUDA events on its stream."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    stats = []
    torch.cuda.synchronize()
    ev[0].record(stream)
    for k in range(steps):
        stats.append(g.step(check=False))
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    return stats, [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)], ev[0].elapsed_time(ev[steps])


def grid_velocity(g):
    """Node coordinates, v^{n+1} = v^n + dv of the last solved step, node masses."""
    gr = g.grid()
    return gr["coords"], gr["v"] + gr["dv"], gr["m"]


def mixed_error(c64, v64, x64, c32, v32, x32, x_prev, dx, m=None, vp64=None, vp32=None):
    """Error of a mixed-precision step against the FP64 step from the same
    state: grid v^{n+1} (relative infinity norm over the nodes, and relative
    in the mass-weighted norm |M^1/2 v| -- nodes of vanishing mass carry
    velocities the step barely constrains), particle velocities, and particle
    positions (relative to |x|, in cells, and relative to the step's
    displacement)."""
    if c64.shape != c32.shape or not np.array_equal(c64, c32):
        return {"grid_v_rel": None, "x_rel": None, "note": "node sets differ"}
    dvx = np.abs(x32 - x64).max()
    disp = np.abs(x64 - x_prev).max()
    out = {"grid_v_rel": float(np.abs(v32 - v64).max() / max(np.abs(v64).max(), 1e-300)),
           "x_rel": float(dvx / np.abs(x64).max()), "x_cells": float(dvx / dx),
           "x_rel_to_step_displacement": float(dvx / max(disp, 1e-300))}
    if m is not None:
        w = m[:, None]
        out["grid_v_rel_mass_weighted"] = float(np.sqrt(np.sum(w * (v32 - v64) ** 2) /
                                                        max(np.sum(w * v64 ** 2), 1e-300)))
    if vp64 is not None:
        out["particle_v_rel"] = float(np.abs(vp32 - vp64).max() / max(np.abs(vp64).max(), 1e-300))
    return out


def run_gpu(sc, opts, steps, warmup, with_e2e, local, sample_clocks=True, profile_run=False,
            partner_opts=None, fp64_probe=None):
    """Warm-up, one profiled breakdown step, K timed steps (the L-BFGS loop on
    the device), the same K steps of the partner precision from the same start
    state (timed alike), then a replay of the K steps with CUDA events around
    every V-cycle and every fine-Hessian assembly for the rooflines, in which
    the partner also steps from each FP64 state so that its per-step error is
    measured, and the end-to-end pass through host buffers."""
    import torch
    from paper_1911_07913_gb300 import hot
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    g = hot.HotScene(sc, opts, stream=stream.cuda_stream)
    warm = [g.step(check=False) for _ in range(warmup)]
    breakdown = {}
    if warmup > 0 and not profile_run:
        g.profile(True)
        g.step(check=False)
        breakdown = g.profile_read()
        g.profile(False)
    start_state = g.get_state()
    clocks = ClockSampler(local)
    launches0 = hot.kernel_launch_count()
    if sample_clocks:
        clocks.start()
    stats, step_ms, total_ms = timed_steps(g, steps, stream)
    clk = clocks.stop() if sample_clocks else {"sm_mhz": None, "sm_max_mhz": None,
                                                 "reasons": ["not sampled (profiling run)"]}
    launches = hot.kernel_launch_count() - launches0
    out = {"total_ms": total_ms, "step_ms": step_ms, "stats": stats, "warm": warm, "breakdown": breakdown,
           "clocks": clk, "launches": launches, "device_loop": all(st.get("device_loop", 0) == 1 for st in stats)}
    g2 = None
    if partner_opts is not None:
        stream2 = torch.cuda.Stream()
        g2 = hot.HotScene(sc, partner_opts, stream=stream2.cuda_stream)
        replay_state(g2, sc, start_state)
        clocks2 = ClockSampler(local)
        clocks2.start()
        st2, ms2, tot2 = timed_steps(g2, steps, stream2)
        out["partner"] = {"stats": st2, "step_ms": ms2, "total_ms": tot2, "clocks": clocks2.stop()}
        g2.profile(True)
        g2.step(check=False)
        out["partner"]["breakdown"] = g2.profile_read()
        g2.profile(False)
    if not profile_run:
        replay_state(g, sc, start_state)
        g.profile(True, only="vcycle,hessian_cells")
        if g2 is not None:
            g2.profile(True, only="vcycle")
        prof_stats, errors, partner_stats = [], [], []
        for k in range(steps):
            s_k = g.get_state() if g2 is not None else None
            prof_stats.append(g.step(check=False))
            if g2 is not None:
                c64, v64, m64 = grid_velocity(g)
                s64 = g.get_state()
                replay_state(g2, sc, s_k)
                partner_stats.append(g2.step(check=False))
                c32, v32, _ = grid_velocity(g2)
                s32 = g2.get_state()
                errors.append(mixed_error(c64, v64, s64["x"], c32, v32, s32["x"], s_k["x"], sc.dx, m=m64,
                                          vp64=s64["v"], vp32=s32["v"]))
        torch.cuda.synchronize()
        out["prof"] = g.profile_read()
        out["prof_stats"] = prof_stats
        g.profile(False)
        if g2 is not None:
            out["partner"]["prof"] = g2.profile_read()
            out["partner"]["prof_stats"] = partner_stats
            out["partner"]["errors"] = errors
            g2.profile(False)
    else:
        out["prof"], out["prof_stats"] = {}, []
    if g2 is not None:
        g2.close()
    out["e2e"] = run_e2e(g, sc, steps, stream, start_state) if with_e2e else None
    g.close()
    return out


def replay_state(g, sc, st):
    n = sc.n
    g.set_state(st["x"], st["v"], st["F"].reshape(n, 9), st["C"].reshape(n, 9))


def run_e2e(g, sc, steps, stream, st):
    """The same steps, from the same starting state, through the C ABI with
    host buffers: each step copies the particle state in from pinned host
    memory and the result back out.  Only converged steps earn credit."""
    import torch
    n = sc.n
    pin = lambda *shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()  # noqa: E731
    x, v, F, Cm = pin(n, 3), pin(n, 3), pin(n, 9), pin(n, 9)
    x[:], v[:], F[:], Cm[:] = st["x"], st["v"], st["F"].reshape(n, 9), st["C"].reshape(n, 9)
    stream.synchronize()
    stats = []
    t0 = time.perf_counter()
    for _ in range(steps):
        g.set_state(x, v, F, Cm)
        stats.append(g.step(check=False))
        g.lib.mpm_get_state(g.h, x.ctypes.data, v.ctypes.data, F.ctypes.data, Cm.ctypes.data, 0)
    stream.synchronize()
    secs = time.perf_counter() - t0
    per = 8 * n * (3 + 3 + 9 + 9)
    rec = step_record(stats)
    return {"value": credited_rate(n, stats, 1e3 * secs), "unit": UNIT, "h2d_bytes_per_step": per,
            "d2h_bytes_per_step": per, "ms_per_step": 1e3 * secs / steps,
            "converged_steps": rec["converged"], "steps": steps, "iters": rec["iters"],
            "status": rec["status"]}


def run_batching(seed, steps, count=64):
    """64 independent scenes (particle counts log-uniform 5k-200k, grids
    64^3-128^3, E log-uniform 1e4-1e8, half von Mises, FP32 preconditioner)
    stepped together: each scene on its own stream, driven by its own host
    thread, so their kernels overlap on the GPU."""
    import torch
    from paper_1911_07913_gb300 import hot
    scs = scenes.batch_scenes(seed=seed, count=count)
    opts = scenes.SolverOptions(eps=1e-7, cn_mode=0, levels=3, precision=1, max_iters=500, refresh_every=REFRESH)
    gs = [hot.HotScene(sc, opts) for sc in scs]
    hot.step_batch(gs, check=False)       # warm-up: allocations, first hierarchy
    tuned = hot.batch_autotune(gs, 1)     # launch configuration: more (ordinary) steps
    f = tuned["flags"]
    tuned["launch"] = ("V-cycle graph, cooperative sweeps" if not f & 1 else
                       "eager V-cycle, one launch per color" if f & 4 else
                       "eager V-cycle, one launch per color on the finest level, cluster or cooperative sweeps on "
                       "the others" if f & 8 else "eager V-cycle, cooperative sweeps")
    if f & 12:
        tuned["sweep_rows_per_block"] = (8, 2, 4, 16)[(f >> 8) & 3]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    iters, conv = [], 0
    for _ in range(steps):
        st = hot.step_batch(gs, check=False)
        iters.append(sum(x["iters"] for x in st))
        conv += sum(1 for x in st if x["status"] == 0)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    n_total = sum(sc.n for sc in scs)
    # the same scenes one after another, for comparison
    t1 = time.perf_counter()
    for g in gs:
        g.step(check=False)
    torch.cuda.synchronize()
    seq = time.perf_counter() - t1
    for g in gs:
        g.close()
    return {"value": n_total * steps / secs, "unit": UNIT, "scenes": count, "particles": n_total,
            "ms_per_batch_step": 1e3 * secs / steps, "sequential_value": n_total / seq,
            "speedup_vs_sequential": (n_total * steps / secs) / (n_total / seq),
            "autotuned": tuned,
            "lbfgs_iters_per_batch_step": iters, "converged_scene_steps": conv, "scene_steps": steps * count,
            "config": "64 boxes, N_p log-uniform 5k-200k, grids 64^3/96^3/128^3, FCR E log-uniform 1e4-1e8, "
                      "half von Mises (yield 1e4 Pa), FP32 preconditioner, 3 levels, CN eps 1e-7, CFL dt"}


def run_solvers(seed, steps=4, warmup=2):
    """HOT against the paper's comparison solvers (Alg. 1: PN-PCG, PN-MGPCG)
    on the two-bar scene at dx = 1/128 (75,200 particles, FP64, CN eps 1e-7,
    4 levels): device time per step, the same steps from the same state for
    each solver.  HOT runs both as printed in Alg. 3 (hierarchy built once
    per step) and with the hierarchy refreshed every REFRESH iterations."""
    import torch
    from paper_1911_07913_gb300 import hot
    sc = scenes.two_bars_scene(seed=seed, res=128, width=10, length=47, gap=10)
    out = {"workload": f"two bars at dx=1/128, {sc.n} particles, FP64, CN eps 1e-7, 4 levels, {steps} steps "
                       f"after {warmup} warm-up step(s)"}
    runs = [("hot", 0, REFRESH), ("hot_alg3", 0, 0), ("pn_pcg", 1, 0), ("pn_mgpcg", 2, 0)]
    for name, solver, refresh in runs:
        opts = scenes.SolverOptions(eps=1e-7, cn_mode=0, levels=4, precision=0, max_iters=500, solver=solver,
                                    refresh_every=refresh)
        stream = torch.cuda.Stream()
        g = hot.HotScene(sc, opts, stream=stream.cuda_stream)
        for _ in range(warmup):
            g.step(check=False)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        stats, inner = [], []
        for _ in range(steps):
            stats.append(g.step(check=False))
            inner.append(int(sum(g.inner_iters())) if solver else 0)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / steps
        rec = step_record(stats)
        out[name] = {"ms_per_step": ms, "outer_iters": rec["iters"], "converged_steps": rec["converged"],
                     "cg_iters": inner if solver else None}
        g.close()
    out["hot_speedup_vs_pn_pcg"] = out["pn_pcg"]["ms_per_step"] / out["hot"]["ms_per_step"]
    out["hot_speedup_vs_pn_mgpcg"] = out["pn_mgpcg"]["ms_per_step"] / out["hot"]["ms_per_step"]
    return out


def _serve_phase(srv, gs, scs, rng, count, requests, load, cap_rate=None, rid0=0):
    """A saturating burst (capacity), or Poisson arrivals at `load` x the
    given capacity; returns (latencies in ms, wall s, particle-steps)."""
    pick = rng.integers(count, size=requests)
    lat = []
    t0 = time.perf_counter()
    if cap_rate is None:
        for r, i in enumerate(pick):
            srv.submit(gs[i], rid0 + r)
    else:
        gaps = rng.exponential(1.0 / (load * cap_rate), size=requests)
        t_next = t0
        for r, i in enumerate(pick):
            t_next += gaps[r]
            while True:
                now = time.perf_counter()
                if now >= t_next:
                    break
                out = srv.poll(wait=False)
                if out is not None:
                    lat.append(out["latency_s"])
                else:
                    time.sleep(min(5e-4, t_next - now))
            srv.submit(gs[i], rid0 + r)
    bad = 0
    while True:
        out = srv.poll(wait=True)
        if out is None:
            break
        lat.append(out["latency_s"])
        bad += out["code"] != 0
    wall = time.perf_counter() - t0
    return np.array(lat) * 1e3, wall, sum(scs[i].n for i in pick), bad


def run_stiffness_sweep(seed, steps=2, warmup=2, E_mids=(1e5, 1e6, 1e7, 1e8, 1e9, 1e10)):
    """The varying-stiffness experiment of Sec. 6.4: a bar of three segments
    twisted by its ends, the end segments at 1e5 Pa, the middle one swept up
    to 1e10 Pa (38,400 particles, dx = 1/128, FCR, FP64, CN eps 1e-7, 4
    levels): L-BFGS iterations and device time per step for HOT (with the
    benchmark's hierarchy refresh) and PN-MGPCG, the same steps for each."""
    import torch
    from paper_1911_07913_gb300 import hot
    out = {"workload": f"three-material bar 10x10x48 cells at dx=1/128, {steps} steps after {warmup} warm-up "
                       "steps per stiffness, FP64, CN eps 1e-7, 4 levels", "E_mid": list(E_mids)}
    for name, solver, refresh in (("hot", 0, REFRESH), ("pn_mgpcg", 2, 0)):
        rows = []
        for E in E_mids:
            sc = scenes.three_material_bar_scene(seed=seed, E_mid=E)
            opts = scenes.SolverOptions(eps=1e-7, cn_mode=0, levels=4, precision=0, max_iters=500, solver=solver,
                                        refresh_every=refresh)
            stream = torch.cuda.Stream()
            g = hot.HotScene(sc, opts, stream=stream.cuda_stream)
            for _ in range(warmup):
                g.step(check=False)
            stats, ms, tot = timed_steps(g, steps, stream)
            g.close()
            rec = step_record(stats)
            rows.append({"iters": rec["iters"], "converged": rec["converged"], "ms_per_step": round(tot / steps, 2)})
        out[name] = rows
    return out


def run_serving(seed, count=256, requests=512, workers=12, budget_gb=150.0, load=0.8, flags=0,
                bind_fraction=0.25):
    """Resident scenes behind the continuous-batching server.  For each budget
    -- the configured 150 GB, and one at `bind_fraction` of the scenes' summed
    peak footprint, where residency admission binds (idle scenes are parked to
    host memory, requests wait for memory) -- a saturating burst measures
    capacity, then a Poisson stream at `load` of that capacity measures
    request latency (arrival -> result).  `flags`: the launch configuration
    the batch autotuner chose for the same kind of workload."""
    import torch
    from paper_1911_07913_gb300 import hot
    scs = scenes.serving_scenes(seed=seed, count=count)
    opts = scenes.SolverOptions(eps=1e-7, cn_mode=0, levels=3, precision=1, max_iters=500, flags=flags,
                                refresh_every=REFRESH)
    gs = [hot.HotScene(sc, opts) for sc in scs]
    srv = hot.StepServer(budget_bytes=int(budget_gb * (1 << 30)), n_workers=workers)
    for i, g in enumerate(gs):           # first step of every scene: its footprint becomes known
        srv.submit(g, i)
    while srv.poll(wait=True) is not None:
        pass
    srv.close()
    peak_total = sum(g.residency()["peak_bytes"] for g in gs)
    out = {"unit": UNIT, "scenes": count, "resident_particles": sum(sc.n for sc in scs),
           "scenes_peak_footprint_gb": peak_total / 2 ** 30, "requests": requests, "workers": workers,
           "launch_flags": flags, "offered_load": load,
           "config": "scenes with N_p lognormal (median 50k, sigma 1, <= 1M), E log-uniform 1e4-1e9, FCR/NH, "
                     f"every third von Mises, FP32 preconditioner, 3 levels, CN eps 1e-7, refresh every {REFRESH}; "
                     "Poisson arrivals"}
    rng = np.random.default_rng(seed + 1)
    for tag, budget in (("configured", budget_gb * (1 << 30)), ("binding", bind_fraction * peak_total)):
        if tag == "binding":
            for g in gs:             # start from nothing resident: the server decides what comes back
                g.park()
        srv = hot.StepServer(budget_bytes=int(budget), n_workers=workers)
        lat_b, wall_b, ps_b, bad_b = _serve_phase(srv, gs, scs, rng, count, requests, load)
        cap_rate = requests / wall_b
        lat, wall, ps, bad = _serve_phase(srv, gs, scs, rng, count, requests, load, cap_rate, rid0=requests)
        info = srv.info()
        srv.close()
        out[tag] = {"budget_gb": budget / 2 ** 30, "value": ps / wall,
                    "capacity_requests_per_s": cap_rate, "capacity_particle_steps_per_s": ps_b / wall_b,
                    "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                    "mean_ms": float(lat.mean()), "failed_requests": int(bad + bad_b),
                    "peak_resident_gb": info["peak_resident_bytes"] / 2 ** 30,
                    "peak_in_flight_gb": info["peak_in_flight_bytes"] / 2 ** 30,
                    "parks": info["parks"], "unparks": info["unparks"], "deferred_requests": info["deferred"],
                    "admission_binds": bool(info["parks"] > 0 or info["deferred"] > 0)}
    out["value"] = out["configured"]["value"]
    out["p50_ms"], out["p99_ms"] = out["configured"]["p50_ms"], out["configured"]["p99_ms"]
    for g in gs:
        g.close()
    return out


# --------------------------------------------------------------------------- host oracle
# Bounded sample of the two-bar workload for the FP64 oracle: the same dx,
# materials, hold regions and solver settings, with 6 x 6 x 12-cell bars (6,912
# particles); the end rotation is scaled by the ratio of the free lengths
# (7 / 85 cells) so that the twist per unit length, and hence the shear rate,
# equals that of the 601,600-particle scene.
SAMPLE = dict(res=256, width=6, length=12, end_cells=2, gap=8, omega=7.0 / 85.0)


def sample_scene(seed: int = 0):
    return scenes.two_bars_scene(seed=seed, **SAMPLE)


def _oracle_sample_step(seed: int):
    """One oracle step of a seeded sample (runs in a spawned worker process)."""
    from oracle import hot_oracle as O
    sc = sample_scene(seed)
    t0 = time.perf_counter()
    _out, info = O.hot_step(sc, workload_opts(0))
    return sc.n, time.perf_counter() - t0, info["trace"].iters, info["trace"].status


def _noop(_x):
    return 0


def cpu_baseline_sample():
    """The oracle, as it stands, on bounded samples of the same workload: one
    step of the seed-0 sample on one core, then one step of an independent
    seeded sample per host core in as many spawned processes at once (each
    single-threaded, no shared state), timed by the wall clock."""
    import multiprocessing as mp
    n, secs, iters, status = _oracle_sample_step(0)
    single = n / secs
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_noop, range(cores))              # workers up and imports done before the clock
        t0 = time.perf_counter()
        res = pool.map(_oracle_sample_step, range(1, cores + 1))
        wall = time.perf_counter() - t0
    allcore = sum(r[0] for r in res) / wall
    conv = sum(1 for r in res if r[3] == "ok")
    return {"value": allcore, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"one step of the two-bar sample (6x6x12-cell bars, {n} particles, dx=1/256, end rotation "
                       f"scaled to the same twist per length, 5 levels, CN eps=1e-7, refresh every {REFRESH}), "
                       f"numpy/scipy FP64: one process per core on {cores} independently seeded samples "
                       f"({conv}/{cores} converged), wall {wall:.1f} s"),
            "single_core": {"value": single, "unit": UNIT, "cores": 1, "seconds": secs, "lbfgs_iters": iters,
                            "status": status},
            "nproc": cores}


def run_reference(args):
    """The oracle arm: W + K consecutive oracle steps of the seed-0 sample on
    the host (rank 0 only), the same metric and credit rule as the GPU arm."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from oracle import hot_oracle as O
    sc = sample_scene(0)
    opts = workload_opts(0)
    state = sc
    for _ in range(args.warmup):
        state, _info = O.hot_step(state, opts)
    t0 = time.perf_counter()
    iters, status = [], []
    for _ in range(args.steps):
        state, info = O.hot_step(state, opts)
        iters.append(info["trace"].iters)
        status.append(info["trace"].status)
    secs = time.perf_counter() - t0
    conv = sum(1 for x in status if x == "ok")
    value = sc.n * conv / secs
    sample = (f"two-bar sample, 6x6x12-cell bars ({sc.n} particles, dx=1/256, end rotation scaled to the same twist "
              f"per length, 5 levels, CN eps=1e-7, refresh every {REFRESH}), {args.steps} consecutive steps after "
              f"{args.warmup} warm-up steps, {conv}/{args.steps} converged, L-BFGS iterations {iters}, one core")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": workload_desc(scenes.two_bars_scene(), workload_opts(0), {"reference_sample": sample}),
            "converged_steps": conv,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def summarize_pair(r, sc, peaks, traffic_key_mixed, ws=1, refresh=REFRESH):
    """FP64 against mixed precision on one scene from the same start state:
    throughput (converged steps only), per-step status, and the mixed step's
    error against the FP64 step from the same state."""
    def arm(stats, step_ms, total_ms, precision):
        rec = step_record(stats, step_ms)
        sm = sorted(step_ms)
        return {"value": credited_rate(sc.n, stats, total_ms, ws), "unit": UNIT, "ms_per_step": total_ms / len(stats),
                "p50_ms": float(np.percentile(sm, 50)), "p99_ms": float(np.percentile(sm, 99)),
                "converged_steps": rec["converged"], "steps": rec["steps"], "per_step": rec,
                "step_hbm": step_hbm_entry(stats, precision, refresh, total_ms, peaks)}
    p = r["partner"]
    out = {"workload": sc.name, "particles": sc.n, "start": "the same state (after the FP64 warm-up steps)",
           "fp64": arm(r["stats"], r["step_ms"], r["total_ms"], 0),
           "mixed": arm(p["stats"], p["step_ms"], p["total_ms"], 1)}
    f, m = out["fp64"]["value"], out["mixed"]["value"]
    out["speedup_mixed_over_fp64"] = (m / f) if f > 0 else None
    errs = p.get("errors") or []
    keys = ("grid_v_rel", "grid_v_rel_mass_weighted", "particle_v_rel", "x_rel", "x_cells",
            "x_rel_to_step_displacement")
    out["error_vs_fp64"] = {
        "how": "each step k: the mixed scene steps from the FP64 state S_k; its grid v^{n+1} and particle x are "
               "compared with the FP64 step from S_k",
        "max": {k: max((e[k] for e in errs if e.get(k) is not None), default=None) for k in keys},
        "per_step": [{k: (float("%.3g" % e[k]) if e.get(k) is not None else None) for k in keys} for e in errs],
        "mixed_status_in_comparison": [int(s["status"]) for s in p.get("prof_stats", [])],
        "mixed_iters_in_comparison": [int(s["iters"]) for s in p.get("prof_stats", [])],
        "fp64_iters_in_comparison": [int(s["iters"]) for s in r.get("prof_stats", [])]}
    out["roofline_mixed_vcycle"] = roofline_entry("vcycle", p.get("prof", {}), p.get("prof_stats", []), sc.n, 1,
                                                  peaks, traffic_key=traffic_key_mixed)
    out["mixed_kernel_ms_one_step"] = {k: round(v["ms"], 3) for k, v in p.get("breakdown", {}).items()}
    out["mixed_clocks"] = p.get("clocks")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dominant", default="auto",
                    help="kernel of the roofline entry (auto: the top kernel of the launch list, the fine Hessian "
                         "assembly in FP64, the V-cycle in mixed precision)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision arms")
    ap.add_argument("--no-2m", action="store_true", help="skip the 2M-particle FP64 / mixed pair")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--small", action="store_true", help="8k-particle cube (for profiling runs)")
    ap.add_argument("--workload", default="two_bars_600k",
                    choices=["two_bars_600k", "two_bars_2m", "two_bars_75k", "cube8k"])
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1])
    ap.add_argument("--refresh", type=int, default=REFRESH, help="hierarchy refresh interval (0: Alg. 3 as printed)")
    ap.add_argument("--levels", type=int, default=0,
                    help="multigrid levels (0: the workload's own, 5 at 600k particles, 6 at 2M)")
    ap.add_argument("--levels-2m", type=int, default=LEVELS_2M, help="multigrid levels of the 2M pair run after the headline")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-solvers", action="store_true", help="skip the HOT / PN-PCG / PN-MGPCG comparison")
    ap.add_argument("--serve-scenes", type=int, default=256)
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--profile-run", action="store_true",
                    help="profiling run under ncu: warm-up and timed steps of one workload only (no breakdown, "
                         "no replay), warm-up allowed below 3")
    args = ap.parse_args()
    if args.small:
        args.workload = "cube8k"
    if args.profile_run:
        args.no_mixed = args.no_2m = args.no_e2e = args.no_cpu = args.no_batch = args.no_serve = True
        args.no_solvers = True
    elif args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    ws, rank, local = dist_env()
    import torch
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_1911_07913_gb300 import hot
    torch.cuda.set_device(local)
    if args.workload == "cube8k":
        sc = scenes.cube_scene(seed=rank)
        opts = scenes.SolverOptions(eps=1e-6, cn_mode=1, dt=2e-3, levels=3, precision=args.precision)
    elif args.workload == "two_bars_2m":
        sc = scenes.two_bars_2m_scene(seed=rank)
        opts = workload_opts(args.precision, args.refresh, args.levels or LEVELS_2M)
    elif args.workload == "two_bars_75k":     # small case of the same scene (profiling captures)
        sc = scenes.two_bars_scene(seed=rank, res=128, width=10, length=47, gap=10)
        opts = workload_opts(args.precision, args.refresh)
        opts.levels = 4
    else:
        sc = scenes.two_bars_scene(seed=rank)
        opts = workload_opts(args.precision, args.refresh, args.levels or 5)
    peaks = load_peaks()
    probe = None if args.profile_run else hot.probe_fp64_tflops()
    partner = None
    if not args.no_mixed and args.workload != "cube8k":
        partner = workload_opts(1 - args.precision, args.refresh, opts.levels)
    barrier(ws)
    r = run_gpu(sc, opts, args.steps, args.warmup, not args.no_e2e, local,
                sample_clocks=not args.profile_run, profile_run=args.profile_run, partner_opts=partner,
                fp64_probe=probe)
    barrier(ws)
    t_max = max_over_ranks(r["total_ms"], ws)
    value = credited_rate(sc.n, r["stats"], t_max, ws)
    prec_key = "fp64" if opts.precision == 0 else "mixed"
    roof_vc = roofline_entry("vcycle", r["prof"], r["prof_stats"], sc.n, opts.precision, peaks,
                             traffic_key=f"{args.workload}_{prec_key}_l{opts.levels}_bytes_per_vcycle",
                             fp64_probe=probe)
    roof_hess = roofline_entry("hessian_cells", r["prof"], r["prof_stats"], sc.n, opts.precision, peaks,
                               traffic_key=f"{args.workload}_{prec_key}_bytes_per_launch",
                               fp64_probe=probe) if opts.precision == 0 else None
    dominant = args.dominant if args.dominant != "auto" else ("hessian_cells" if opts.precision == 0 else "vcycle")
    roof = roof_hess if dominant == "hessian_cells" else roof_vc
    mixed = {}
    if partner is not None and "partner" in r and opts.precision == 0:
        mixed[args.workload] = summarize_pair(r, sc, peaks, f"{args.workload}_mixed_l{opts.levels}_bytes_per_vcycle", ws,
                                              args.refresh)
    if partner is not None and not args.no_2m and args.workload == "two_bars_600k" and opts.precision == 0:
        sc2 = scenes.two_bars_2m_scene(seed=rank)
        r2 = run_gpu(sc2, workload_opts(0, args.refresh, args.levels_2m), args.steps, args.warmup, False, local,
                     partner_opts=workload_opts(1, args.refresh, args.levels_2m), fp64_probe=probe)
        mixed["two_bars_2m"] = summarize_pair(r2, sc2, peaks, f"two_bars_2m_mixed_l{args.levels_2m}_bytes_per_vcycle", ws,
                                              args.refresh)
        mixed["two_bars_2m"]["roofline_fp64_vcycle"] = roofline_entry(
            "vcycle", r2["prof"], r2["prof_stats"], sc2.n, 0, peaks, fp64_probe=probe)
    batching = serving = solvers = None
    if args.workload == "two_bars_600k" and args.precision == 0:
        if not args.no_solvers:
            solvers = run_solvers(rank)
            solvers["stiffness_sweep"] = run_stiffness_sweep(rank)
        if not args.no_batch:
            batching = run_batching(rank, max(2, args.steps // 2))
        if not args.no_serve:
            tuned = batching["autotuned"] if batching else {"flags": 0, "workers": 12}
            serving = run_serving(rank, count=args.serve_scenes, requests=args.serve_requests,
                                  workers=tuned["workers"], flags=tuned["flags"])
    if rank != 0:
        return
    cpu = None if args.no_cpu else cpu_baseline_sample()
    rec = step_record(r["stats"], r["step_ms"])
    sm = sorted(r["step_ms"])
    e2e = r["e2e"]
    if e2e is not None:
        e2e["device_pass_iters"] = rec["iters"]
        e2e["same_iterations_as_device_pass"] = e2e["iters"] == rec["iters"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if opts.precision == 0 else "f64+f32",
            "data": "synthetic",
            "config": workload_desc(sc, opts, {"parallelism": f"replicas x{ws}",
                                               "credit": "particle-steps of steps whose solve met the tolerance, "
                                                         "over the time of all timed steps"}),
            "at_tolerance": rec["converged"] == args.steps, "converged_steps": rec["converged"],
            "per_step": rec, "warmup_status": [int(s["status"]) for s in r["warm"]],
            "p50_ms": float(np.percentile(sm, 50)), "p99_ms": float(np.percentile(sm, 99)),
            "e2e": e2e, "gpu_launches": int(r["launches"]), "roofline": roof,
            "roofline_vcycle": roof_vc, "roofline_hessian_assembly": roof_hess,
            "step_hbm": step_hbm_entry(r["stats"], opts.precision, args.refresh, t_max, peaks),
            "lbfgs_loop_on_device": r["device_loop"],
            "kernel_ms_one_step": {k: round(v["ms"], 3) for k, v in r["breakdown"].items()},
            "clocks": r["clocks"], "fp64_probe_tflops": probe, "mixed": mixed or None,
            "batching": batching, "serving": serving, "solvers": solvers, "cpu_baseline": cpu}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
