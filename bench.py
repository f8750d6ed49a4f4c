#!/usr/bin/env python
"""Throughput of the HOT implicit MPM step on GB300: particle-steps/s.

Default workload: two twisted bars, 601,600 particles on a sparse 256^3 grid
(dx = 1/256), Neo-Hookean E = 1e5 / 1e9 Pa, nu = 0.4, rho = 2000, ends
rotating at +-1 rad/s, dt at CFL 0.6 (24 FPS cap), 5-level multigrid, FP64,
characteristic-norm tolerance eps = 1e-7.  A step is one full implicit step
(P2G, HOT solve, G2P) on device-resident particles.  Also reported: the same
metric end to end through the C ABI with host buffers, the mixed-precision
form on the 2M-particle version of the scene, the dominant kernel against its
roofline, p50/p99 step latency, and the FP64 oracle on the host cores.

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

# measured FP64 FMA throughput unit count: 2 FP64 FMA per SM per clock on
# GB300 -> 152 SMs x 4 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12


def workload_opts(precision: int) -> scenes.SolverOptions:
    return scenes.SolverOptions(eps=1e-7, cn_mode=0, lbfgs_m=8, levels=5, precision=precision,
                                max_iters=500)


def workload_desc(sc, opts, extra=None):
    if sc.name.startswith("cube"):
        what = f"{sc.name}: FCR cube E=1e5 Pa, nu=0.3, random initial velocity, sticky floor, 32^3 grid"
    else:
        what = (f"{sc.name}: two twisted Neo-Hookean bars E=1e5/1e9 Pa, nu=0.4, rho=2000, "
                f"ends at +-1 rad/s, sparse {int(sc.grid_dims[0])}^3 grid")
    d = {"workload": what,
         "particles": sc.n, "dx": sc.dx, "levels": opts.levels, "lbfgs_window": opts.lbfgs_m,
         "tolerance": f"CN eps={opts.eps}", "dt": "min(1/24, 0.6 dx / v_max)",
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


def algorithmic_units(name: str, stats_list, n_particles: int, precision: int):
    """Algorithmic work of kernel `name` summed over the timed steps.

    vcycle (the captured V-cycle of Alg. 2): per level m < M-1 four
    Gauss-Seidel sweeps over the off-diagonal blocks, of which the first
    (forward, from u = 0) needs only the blocks of earlier-colored
    neighbours -- exactly half of the off-diagonal blocks, since every
    coupling joins two colors -- and one residual over all blocks.  FP64:
    9 FMA = 18 flop per block visit (the FP64 pipe bounds it).  FP32: 36 B of
    block values + 4 B column index per block visit (HBM bounds it).  The
    coarsest PCG (latency bound, shared-memory resident) is not counted.
    hessian_cells: 27*27*3 + 378*9*3 FMA = 24,786 flop per particle."""
    if name == "hessian_cells":
        return 2 * (27 * 27 * 3 + 378 * 9 * 3) * n_particles * len(stats_list), "flop"
    visits = 0
    for st in stats_list:
        nl = st["n_levels"]
        for m in range(nl - 1):
            nnz, n = st["nnz_blocks"][m], st["n_nodes"][m]
            visits += ((7 * (nnz - n)) // 2 + nnz) * st["vcycles"]
    if precision == 0:
        return 18 * visits, "flop"
    return 40 * visits, "byte"


def vcycle_traffic(key):
    """DRAM bytes per V-cycle (dram__bytes_read.sum + dram__bytes_write.sum
    over the kernels of one V-cycle) from the committed ncu summary, or None
    when the V-cycle's source changed after that capture."""
    try:
        lines = open(os.path.join(ROOT, "profiles", "vcycle_dram.txt")).read().splitlines()
        src = open(os.path.join(ROOT, "paper_1911_07913_gb300", "csrc", "multigrid.cu"), "rb").read()
    except OSError:
        return None
    kv = dict(line.split(": ", 1) for line in lines if ": " in line and not line.startswith("#"))
    if kv.get("multigrid_cu_sha256") != hashlib.sha256(src).hexdigest():
        return None
    v = kv.get(key)
    return float(v) if v else None


def roofline_entry(name, prof, stats_list, n_particles, precision, peaks, traffic_key=None):
    """Dominant-kernel roofline from live CUDA-event times over the timed steps."""
    p = prof.get(name)
    if not p or p["launches"] == 0:
        return None
    units, kind = algorithmic_units(name, stats_list, n_particles, precision)
    secs = p["ms"] / 1e3
    traffic = vcycle_traffic(traffic_key) if (traffic_key and name == "vcycle") else None
    base = {"kernel": name, "traffic": traffic, "traffic_unit": "DRAM bytes per V-cycle (ncu)", "launches": p["launches"],
            "avg_launch_ms": p["ms"] / p["launches"], "algorithmic_total": units, "algorithmic_unit": kind,
            "timed": "CUDA events around every V-cycle, over a replay of the timed steps from their start state"}
    if kind == "flop":
        achieved = units / secs / 1e12
        return {**base, "bound": "alu", "achieved": achieved, "peak": round(FP64_PEAK_TFLOPS, 3),
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2.07 GHz (probe: 1.20 TFLOP/s at 1995 MHz)"}
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
def run_gpu(sc, opts, steps, warmup, dominant, with_e2e, rank, local, sample_clocks=True, profile_run=False):
    """Warm-up, one profiled breakdown step, K timed steps (the L-BFGS loop as
    one device-driven CUDA graph, no profiling), then the same K steps replayed
    from the same state with CUDA events around every V-cycle (`dominant`) for
    the roofline, and the end-to-end pass through host buffers."""
    import torch
    from paper_1911_07913_gb300 import hot
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    g = hot.HotScene(sc, opts, stream=stream.cuda_stream)
    for _ in range(warmup):
        g.step(check=False)
    breakdown = {}
    if warmup > 0 and not profile_run:
        # full kernel breakdown on one extra untimed step
        g.profile(True)
        g.step()
        breakdown = g.profile_read()
        g.profile(False)
    start_state = g.get_state()
    stats = []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    launches0 = hot.kernel_launch_count()
    if sample_clocks:
        clocks.start()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for k in range(steps):
        stats.append(g.step(check=False))
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if sample_clocks else {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled (profiling run)"]}
    launches = hot.kernel_launch_count() - launches0
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    total_ms = ev[0].elapsed_time(ev[steps])
    # roofline: the same steps again, every V-cycle between CUDA events
    prof, prof_stats = {}, []
    if not profile_run:
        replay_state(g, sc, start_state)
        g.profile(True, only=dominant)
        prof_stats = [g.step(check=False) for _ in range(steps)]
        torch.cuda.synchronize()
        prof = g.profile_read()
        g.profile(False)
    e2e = None
    if with_e2e:
        e2e = run_e2e(g, sc, steps, stream, start_state)
    g.close()
    return {"total_ms": total_ms, "step_ms": step_ms, "stats": stats, "prof": prof, "prof_stats": prof_stats,
            "breakdown": breakdown, "clocks": clk, "launches": launches, "e2e": e2e,
            "device_loop": all(st.get("device_loop", 0) == 1 for st in stats)}


def replay_state(g, sc, st):
    n = sc.n
    g.set_state(st["x"], st["v"], st["F"].reshape(n, 9), st["C"].reshape(n, 9))


def run_e2e(g, sc, steps, stream, st):
    """The same steps, from the same starting state, through the C ABI with
    host buffers: each step copies the particle state in from pinned host
    memory and the result back out."""
    import torch
    n = sc.n
    pin = lambda *shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()  # noqa: E731
    x, v, F, Cm = pin(n, 3), pin(n, 3), pin(n, 9), pin(n, 9)
    x[:], v[:], F[:], Cm[:] = st["x"], st["v"], st["F"].reshape(n, 9), st["C"].reshape(n, 9)
    stream.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        g.set_state(x, v, F, Cm)
        g.step(check=False)
        g.lib.mpm_get_state(g.h, x.ctypes.data, v.ctypes.data, F.ctypes.data, Cm.ctypes.data, 0)
    stream.synchronize()
    secs = time.perf_counter() - t0
    per = 8 * n * (3 + 3 + 9 + 9)
    return {"value": n * steps / secs, "unit": UNIT, "h2d_bytes_per_step": per, "d2h_bytes_per_step": per,
            "ms_per_step": 1e3 * secs / steps}


def run_batching(seed, steps, count=64):
    """64 independent scenes (particle counts log-uniform 5k-200k, grids
    64^3-128^3, E log-uniform 1e4-1e8, half von Mises, FP32 preconditioner)
    stepped together: each scene on its own stream, driven by its own host
    thread, so their kernels overlap on the GPU."""
    import torch
    from paper_1911_07913_gb300 import hot
    scs = scenes.batch_scenes(seed=seed, count=count)
    opts = scenes.SolverOptions(eps=1e-7, cn_mode=0, levels=3, precision=1, max_iters=500)
    gs = [hot.HotScene(sc, opts) for sc in scs]
    hot.step_batch(gs, check=False)       # warm-up: allocations, first hierarchy
    tuned = hot.batch_autotune(gs, 1)     # launch configuration: 6 more (ordinary) steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    iters = []
    for _ in range(steps):
        st = hot.step_batch(gs, check=False)
        iters.append(sum(x["iters"] for x in st))
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
            "lbfgs_iters_per_batch_step": iters,
            "config": "64 boxes, N_p log-uniform 5k-200k, grids 64^3/96^3/128^3, FCR E log-uniform 1e4-1e8, "
                      "half von Mises (yield 1e4 Pa), FP32 preconditioner, 3 levels, CN eps 1e-7, CFL dt"}


def run_solvers(seed, steps=2, warmup=1):
    """HOT against the paper's comparison solvers (Alg. 1: PN-PCG, PN-MGPCG)
    on the two-bar scene at dx = 1/128 (75,200 particles, FP64, CN eps 1e-7,
    4 levels): wall time per step on the device, same steps from the same
    state for each solver."""
    import torch
    from paper_1911_07913_gb300 import hot
    sc = scenes.two_bars_scene(seed=seed, res=128, width=10, length=47, gap=4)
    out = {"workload": f"two bars at dx=1/128, {sc.n} particles, FP64, CN eps 1e-7, 4 levels, {steps} steps "
                       f"after {warmup} warm-up step(s)"}
    names = {0: "hot", 1: "pn_pcg", 2: "pn_mgpcg"}
    for solver in (0, 1, 2):
        opts = scenes.SolverOptions(eps=1e-7, cn_mode=0, levels=4, precision=0, max_iters=500, solver=solver)
        stream = torch.cuda.Stream()
        g = hot.HotScene(sc, opts, stream=stream.cuda_stream)
        for _ in range(warmup):
            g.step(check=False)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        its, inner = [], []
        for _ in range(steps):
            st = g.step(check=False)
            its.append(st["iters"])
            inner.append(int(sum(g.inner_iters())) if solver else 0)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / steps
        out[names[solver]] = {"ms_per_step": ms, "outer_iters": its, "cg_iters": inner if solver else None}
        g.close()
    out["hot_speedup_vs_pn_pcg"] = out["pn_pcg"]["ms_per_step"] / out["hot"]["ms_per_step"]
    out["hot_speedup_vs_pn_mgpcg"] = out["pn_mgpcg"]["ms_per_step"] / out["hot"]["ms_per_step"]
    return out


def run_serving(seed, count=256, requests=512, workers=12, budget_gb=150.0, load=0.8, flags=0):
    """Resident scenes behind the continuous-batching server: a saturating
    burst measures capacity, then a Poisson stream at `load` of that capacity
    measures request latency (arrival -> result).  `flags`: the launch
    configuration the batch autotuner chose for the same kind of workload."""
    import torch
    from paper_1911_07913_gb300 import hot
    scs = scenes.serving_scenes(seed=seed, count=count)
    opts = scenes.SolverOptions(eps=1e-7, cn_mode=0, levels=3, precision=1, max_iters=500, flags=flags)
    gs = [hot.HotScene(sc, opts) for sc in scs]
    srv = hot.StepServer(budget_bytes=int(budget_gb * (1 << 30)), n_workers=workers)
    for i, g in enumerate(gs):           # first step of every scene: buffers become resident
        srv.submit(g, i)
    while srv.poll(wait=True) is not None:
        pass
    footprint = sum(g.footprint() for g in gs)
    rng = np.random.default_rng(seed + 1)
    # capacity: a burst of requests
    pick = rng.integers(count, size=requests)
    t0 = time.perf_counter()
    for r, i in enumerate(pick):
        srv.submit(gs[i], r)
    done = 0
    while srv.poll(wait=True) is not None:
        done += 1
    cap_s = time.perf_counter() - t0
    cap_rate = requests / cap_s
    cap_particles = sum(scs[i].n for i in pick) / cap_s
    # Poisson arrivals at a fraction of capacity
    rate = load * cap_rate
    pick = rng.integers(count, size=requests)
    gaps = rng.exponential(1.0 / rate, size=requests)
    lat = []
    t0 = time.perf_counter()
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
        srv.submit(gs[i], requests + r)
    while True:
        out = srv.poll(wait=True)
        if out is None:
            break
        lat.append(out["latency_s"])
    wall = time.perf_counter() - t0
    info = srv.info()
    srv.close()
    for g in gs:
        g.close()
    lat = np.array(lat) * 1e3
    return {"value": sum(scs[i].n for i in pick) / wall, "unit": UNIT, "scenes": count,
            "resident_particles": sum(sc.n for sc in scs), "resident_footprint_gb": footprint / 2 ** 30,
            "requests": requests, "workers": workers, "launch_flags": flags, "budget_gb": budget_gb,
            "capacity_requests_per_s": cap_rate, "capacity_particle_steps_per_s": cap_particles,
            "offered_load": load, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "peak_in_flight_gb": info["peak_in_flight_bytes"] / 2 ** 30,
            "config": "resident scenes, N_p lognormal (median 50k, sigma 1, <= 1M), E log-uniform 1e4-1e9, FCR/NH, "
                      "every third von Mises, FP32 preconditioner, 3 levels, CN eps 1e-7; Poisson arrivals"}


def cpu_baseline_sample():
    """The oracle, as it stands, on a bounded sample of the same workload: the
    two-bar scene at the same dx, materials and boundary conditions, with bars
    of 12 x 12 x 8 cells (18,432 particles), one implicit step."""
    from oracle import hot_oracle as O
    sc = scenes.two_bars_scene(res=256, width=12, length=8, end_cells=2)
    opts = workload_opts(0)
    t0 = time.perf_counter()
    out, info = O.hot_step(sc, opts)
    secs = time.perf_counter() - t0
    return {"value": sc.n / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one step of the two-bar scene with 12x12x8-cell bars ({sc.n} particles, "
                      f"dx=1/256, 5 levels, CN eps=1e-7, {info['trace'].iters} L-BFGS iterations), "
                      f"numpy/scipy FP64, single thread, {secs:.1f} s"}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from oracle import hot_oracle as O
    sc = scenes.two_bars_scene(res=256, width=8, length=8, end_cells=2)
    opts = workload_opts(0)
    state = sc
    for _ in range(args.warmup):
        state, _info = O.hot_step(state, opts)
    t0 = time.perf_counter()
    iters = []
    for _ in range(args.steps):
        state, info = O.hot_step(state, opts)
        iters.append(info["trace"].iters)
    secs = time.perf_counter() - t0
    value = sc.n * args.steps / secs
    sample = (f"two-bar scene with 8x8x8-cell bars ({sc.n} particles, dx=1/256, 5 levels, CN eps=1e-7), "
              f"{args.steps} consecutive steps, L-BFGS iterations {iters}")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": workload_desc(scenes.two_bars_scene(), workload_opts(0),
                                    {"reference_sample": sample}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dominant", default="vcycle", help="kernel timed live for the roofline entry")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--small", action="store_true", help="8k-particle cube (for profiling runs)")
    ap.add_argument("--workload", default="two_bars_600k", choices=["two_bars_600k", "two_bars_2m", "cube8k"])
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1])
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-solvers", action="store_true", help="skip the HOT / PN-PCG / PN-MGPCG comparison")
    ap.add_argument("--serve-scenes", type=int, default=256)
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--profile-run", action="store_true",
                    help="profiling run under ncu: warm-up and timed steps of one workload only (no breakdown, "
                         "no roofline replay), warm-up allowed below 3")
    args = ap.parse_args()
    if args.small:
        args.workload = "cube8k"
    if args.profile_run:
        args.no_mixed = args.no_e2e = args.no_cpu = args.no_batch = args.no_serve = args.no_solvers = True
    elif args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    ws, rank, local = dist_env()
    import torch
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if args.workload == "cube8k":
        sc = scenes.cube_scene(seed=rank)
        opts = scenes.SolverOptions(eps=1e-6, cn_mode=1, dt=2e-3, levels=3, precision=args.precision)
    elif args.workload == "two_bars_2m":
        sc = scenes.two_bars_2m_scene(seed=rank)
        opts = workload_opts(args.precision)
    else:
        sc = scenes.two_bars_scene(seed=rank)
        opts = workload_opts(args.precision)
    peaks = load_peaks()
    barrier(ws)
    r = run_gpu(sc, opts, args.steps, args.warmup, args.dominant, not args.no_e2e, rank, local,
                sample_clocks=not args.profile_run, profile_run=args.profile_run)
    barrier(ws)
    t_max = max_over_ranks(r["total_ms"], ws)
    value = job_throughput(sc.n, ws, args.steps, t_max)
    roof = roofline_entry(args.dominant, r["prof"], r["prof_stats"], sc.n, opts.precision, peaks,
                          traffic_key=f"{args.workload}_{'fp64' if opts.precision == 0 else 'mixed'}_bytes_per_vcycle")
    mixed = None
    if not args.no_mixed and args.workload == "two_bars_600k" and args.precision == 0:
        sc2 = scenes.two_bars_2m_scene(seed=rank)
        o2 = workload_opts(1)
        r2 = run_gpu(sc2, o2, args.steps, args.warmup, "vcycle", False, rank, local)
        t2 = max_over_ranks(r2["total_ms"], ws)
        sm = sorted(r2["step_ms"])
        mixed = {"value": sc2.n * ws * args.steps / (t2 / 1e3), "unit": UNIT, "ms_per_step": t2 / args.steps,
                 "p50_ms": float(np.percentile(sm, 50)), "p99_ms": float(np.percentile(sm, 99)),
                 "config": workload_desc(sc2, o2), "iters": [s["iters"] for s in r2["stats"]],
                 "roofline": roofline_entry("vcycle", r2["prof"], r2["prof_stats"], sc2.n, 1, peaks,
                                            traffic_key="two_bars_2m_mixed_bytes_per_vcycle"),
                 "kernel_ms": {k: round(v["ms"], 3) for k, v in r2["breakdown"].items()},
                 "clocks": r2["clocks"]}
    batching = serving = solvers = None
    if args.workload == "two_bars_600k" and args.precision == 0:
        if not args.no_solvers:
            solvers = run_solvers(rank)
        if not args.no_batch:
            batching = run_batching(rank, max(2, args.steps // 2))
        if not args.no_serve:
            tuned = batching["autotuned"] if batching else {"flags": 0, "workers": 12}
            serving = run_serving(rank, count=args.serve_scenes, requests=args.serve_requests,
                                  workers=tuned["workers"], flags=tuned["flags"])
    if rank != 0:
        return
    cpu = None if args.no_cpu else cpu_baseline_sample()
    sm = sorted(r["step_ms"])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if opts.precision == 0 else "f64+f32",
            "data": "synthetic",
            "config": workload_desc(sc, opts, {"parallelism": f"replicas x{ws}"}),
            "p50_ms": float(np.percentile(sm, 50)), "p99_ms": float(np.percentile(sm, 99)),
            "iters": [s["iters"] for s in r["stats"]],
            "e2e": r["e2e"], "gpu_launches": int(r["launches"]), "roofline": roof,
            "lbfgs_loop_on_device": r["device_loop"],
            "kernel_ms_one_step": {k: round(v["ms"], 3) for k, v in r["breakdown"].items()},
            "clocks": r["clocks"], "mixed": mixed, "batching": batching, "serving": serving, "solvers": solvers,
            "cpu_baseline": cpu}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
