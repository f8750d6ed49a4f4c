"""Seeded synthetic MPM scenes (inputs only).

This module builds particle arrays, material tables and boundary-condition
lists for the workloads the HOT step is exercised on.  It contains no part of
the method's arithmetic: no kernel weights, no transfers, no energies.  Both
the CUDA path and the FP64 oracle receive the arrays it returns, so the two
sides always see bit-identical inputs.

Shapes follow the paper's benchmark set (Table 2: bar-twisting scene "Twist",
stiffness-contrast bars, soft boxes) at sizes chosen for one GPU; the paper's
meshes are not available, so boxes and bars of the stated cell counts stand in
for them.  Every scene is drawn from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

MODEL_FCR = 0   # fixed-corotated elasticity (Stomakhin et al. 2012), Sec. 6.1
MODEL_NH = 1    # compressible Neo-Hookean

BC_STICKY = 0   # nodes inside the box get v = 0
BC_ROTATE = 1   # nodes inside the box get v = omega * axis x (x_i - center)


@dataclasses.dataclass
class Material:
    E: float
    nu: float
    rho: float
    model: int = MODEL_FCR
    plasticity: int = 0
    yield_stress: float = 0.0


@dataclasses.dataclass
class BoundaryBox:
    type: int
    lo: tuple
    hi: tuple
    axis: tuple = (0.0, 0.0, 1.0)
    center: tuple = (0.0, 0.0, 0.0)
    omega: float = 0.0
    radius: float = 0.0   # > 0: only nodes within this distance of the axis line through center


@dataclasses.dataclass
class Scene:
    """Particle state plus grid description of one MPM scene.

    Arrays are C-contiguous float64 (int32 for ``mat``):
    x, v: (N, 3); F, C: (N, 3, 3) row-major; vol, mass: (N,); mat: (N,).
    ``grid_dims`` counts cells per axis; nodes run 0..grid_dims inclusive.
    """
    x: np.ndarray
    v: np.ndarray
    F: np.ndarray
    C: np.ndarray
    vol: np.ndarray
    mass: np.ndarray
    mat: np.ndarray
    materials: List[Material]
    dx: float
    origin: np.ndarray
    grid_dims: np.ndarray
    gravity: np.ndarray
    bcs: List[BoundaryBox]
    name: str = "scene"

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def copy(self) -> "Scene":
        return dataclasses.replace(
            self, x=self.x.copy(), v=self.v.copy(), F=self.F.copy(), C=self.C.copy(),
            vol=self.vol.copy(), mass=self.mass.copy(), mat=self.mat.copy(),
            materials=list(self.materials), origin=self.origin.copy(),
            grid_dims=self.grid_dims.copy(), gravity=self.gravity.copy(), bcs=list(self.bcs))

    def subset(self, idx: np.ndarray) -> "Scene":
        s = self.copy()
        for k in ("x", "v", "F", "C", "vol", "mass", "mat"):
            setattr(s, k, np.ascontiguousarray(getattr(self, k)[idx]))
        return s


@dataclasses.dataclass
class SolverOptions:
    """Solver settings; defaults are the paper's (Sec. 6.1: 3 levels, one SGS
    sweep, L-BFGS window 8, eps = 1e-7, CFL 0.6, 24 FPS)."""
    eps: float = 1e-7
    cn_mode: int = 0          # 0: characteristic norm (Sec. 5.2); 1: ||g|| <= eps ||g^1||
    lbfgs_m: int = 8
    levels: int = 3
    precision: int = 0        # 0: FP64 everywhere; 1: FP32 Hessian/V-cycle
    max_iters: int = 500
    max_ls: int = 50
    max_coarse_cg: int = 0    # 0: number of coarsest-level DOFs
    dt: float = 0.0           # > 0: fixed step; else CFL rule
    fps: float = 24.0
    cfl: float = 0.6
    flags: int = 0            # bit 0: V-cycle launched eagerly (no CUDA graph); 1: cooperative
                              # coarsest PCG; 2: one launch per SGS color; 3: the same, finest level;
                              # 4: host-driven L-BFGS loop; 5: device-side graph loop always;
                              # 6: no cluster-launched sweeps on levels with few rows per color;
                              # 7: half-matrix residual; 8-9: rows per block of per-color launches;
                              # 10: cluster sweeps with u in global instead of shared memory;
                              # 11: cluster barrier instead of per-CTA byte counts between colors
    solver: int = 0           # 0: HOT (Alg. 3); 1: PN-PCG; 2: PN-MGPCG (Alg. 1, comparison solvers)
    refresh_every: int = 0    # HOT extension: rebuild the hierarchy at the iterate every k iterations (0: off)
    fallback_after: int = 0   # HOT extension: finish an unconverged step with PN-MGPCG after k iterations


def _jittered_block(rng, cell_lo, cell_hi, dx, origin, ppc_axis=2):
    """Particles ``ppc_axis**3`` per cell, each uniform inside its sub-cell."""
    lo = np.asarray(cell_lo, np.int64)
    hi = np.asarray(cell_hi, np.int64)
    counts = (hi - lo) * ppc_axis
    gz, gy, gx = np.meshgrid(np.arange(counts[2]), np.arange(counts[1]),
                             np.arange(counts[0]), indexing="ij")
    sub = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1).astype(np.float64)
    jitter = rng.random(sub.shape)
    x = origin + (lo + (sub + jitter) / ppc_axis) * dx
    return np.ascontiguousarray(x)


def _assemble(x, v, mat, materials, dx, ppc, origin, dims, gravity, bcs, name, F=None):
    n = x.shape[0]
    vol = np.full(n, dx ** 3 / ppc)
    rho = np.array([materials[m].rho for m in mat])
    mass = rho * vol
    if F is None:
        F = np.tile(np.eye(3), (n, 1, 1))
    return Scene(x=np.ascontiguousarray(x, np.float64), v=np.ascontiguousarray(v, np.float64),
                 F=np.ascontiguousarray(F, np.float64), C=np.zeros((n, 3, 3)),
                 vol=vol, mass=mass, mat=np.ascontiguousarray(mat, np.int32),
                 materials=materials, dx=float(dx), origin=np.asarray(origin, np.float64),
                 grid_dims=np.asarray(dims, np.int32), gravity=np.asarray(gravity, np.float64),
                 bcs=bcs, name=name)


def cube_scene(seed: int = 0, res: int = 32, cube_lo=(11, 4, 11), side: int = 10,
               E: float = 1e5, nu: float = 0.3, rho: float = 1000.0,
               model: int = MODEL_FCR, vel_amp: float = 0.5, floor_nodes: float = 3.5,
               gravity=(0.0, -9.8, 0.0)) -> Scene:
    """Elastic cube with random initial velocity over a sticky floor.

    Default: 10^3 cells x 8 particles = 8000 particles on a 32^3 grid,
    dx = 1/32, FCR E = 1e5, nu = 0.3, rho = 1000, v ~ U[-0.5, 0.5]^3; the floor
    holds every node with y <= 3.5 dx, so the cube's lowest node layer is held.
    """
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    origin = np.zeros(3)
    lo = np.asarray(cube_lo)
    x = _jittered_block(rng, lo, lo + side, dx, origin)
    v = rng.uniform(-vel_amp, vel_amp, size=x.shape)
    mats = [Material(E, nu, rho, model)]
    big = 1e30
    bcs = [BoundaryBox(BC_STICKY, (-big, -big, -big), (big, floor_nodes * dx, big))]
    return _assemble(x, v, np.zeros(x.shape[0], np.int32), mats, dx, 8, origin,
                     (res, res, res), gravity, bcs, f"cube{side}_r{res}")


def two_bars_scene(seed: int = 0, res: int = 256, width: int = 20, length: int = 94,
                   gap: int = 14, E_a: float = 1e5, E_b: float = 1e9, nu: float = 0.4,
                   rho: float = 2000.0, model: int = MODEL_NH, omega: float = 1.0,
                   end_cells: int = 4, gravity=(0.0, -9.8, 0.0), hold: str = "cylinder") -> Scene:
    """Two parallel bars along z, twisted by prescribed end rotations.

    Stand-in for the paper's Twist scene (Fig. 1, Table 2: rho = 2000,
    nu = 0.4, stiffness contrast).  Default: res 256 (dx = 1/256), bars of
    20 x 20 x 94 cells, 8 particles per cell (601,600 particles), bar A
    E = 1e5, bar B E = 1e9, Neo-Hookean.  The ``end_cells`` end layers of
    each bar rotate about the bar axis at +omega (low-z end) and -omega
    (high-z end).

    hold = "cylinder": the held region of each end is a cylinder about the
    bar axis, 2 cells wider than the bar's half diagonal (capped half a cell
    short of the other bar's nearest stencil node), so the turning end stays
    inside it.  hold = "box": an axis-aligned box 3 cells wider than the bar,
    which the end's corners leave after about 0.4 rad of rotation.
    """
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    origin = np.zeros(3)
    c = res // 2
    half_gap = gap // 2
    y0, y1 = c - width // 2, c - width // 2 + width
    z0, z1 = c - length // 2, c - length // 2 + length
    xs = [(c - half_gap - width, c - half_gap), (c + half_gap, c + half_gap + width)]
    mats = [Material(E_a, nu, rho, model), Material(E_b, nu, rho, model)]
    parts, mids = [], []
    bcs = []
    for b, (x0, x1) in enumerate(xs):
        xb = _jittered_block(rng, (x0, y0, z0), (x1, y1, z1), dx, origin)
        parts.append(xb)
        mids.append(np.full(xb.shape[0], b, np.int32))
        center = (0.5 * (x0 + x1) * dx, 0.5 * (y0 + y1) * dx, 0.0)
        if hold == "cylinder":
            reach = gap + 0.5 * width - 1.0          # axis -> other bar's nearest stencil node, cells
            radius = min(np.sqrt(0.5) * width + 2.0, reach - 0.5)
            lo_x, hi_x = center[0] - radius * dx, center[0] + radius * dx
            lo_y, hi_y = center[1] - radius * dx, center[1] + radius * dx
            rad = radius * dx
        else:
            lo_x, hi_x = (x0 - 3) * dx, (x1 + 3) * dx
            lo_y, hi_y = (y0 - 3) * dx, (y1 + 3) * dx
            rad = 0.0
        bcs.append(BoundaryBox(BC_ROTATE, (lo_x, lo_y, (z0 - 3) * dx),
                               (hi_x, hi_y, (z0 + end_cells + 0.5) * dx),
                               (0.0, 0.0, 1.0), center, omega, rad))
        bcs.append(BoundaryBox(BC_ROTATE, (lo_x, lo_y, (z1 - end_cells - 0.5) * dx),
                               (hi_x, hi_y, (z1 + 3) * dx),
                               (0.0, 0.0, 1.0), center, -omega, rad))
    x = np.concatenate(parts)
    mat = np.concatenate(mids)
    v = np.zeros_like(x)
    return _assemble(x, v, mat, mats, dx, 8, origin, (res, res, res), gravity, bcs,
                     f"two_bars_w{width}_l{length}_r{res}")


def three_material_bar_scene(seed: int = 0, res: int = 128, width: int = 10, length: int = 48,
                             E_ends: float = 1e5, E_mid: float = 1e8, nu: float = 0.4, rho: float = 2000.0,
                             model: int = MODEL_FCR, omega: float = 1.0, end_cells: int = 3,
                             gravity=(0.0, -9.8, 0.0)) -> Scene:
    """A bar along z in three equal segments, twisted by its ends (the
    varying-stiffness experiment of Sec. 6.4): the two end segments keep
    E_ends, the middle one takes E_mid (the paper sweeps it from 1e5 to 1e10
    Pa).  FCR as in all of the paper's examples; the end layers are held in
    cylinders about the bar axis and rotate at +omega / -omega."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    origin = np.zeros(3)
    c = res // 2
    x0, y0, z0 = c - width // 2, c - width // 2, c - length // 2
    x1, y1, z1 = x0 + width, y0 + width, z0 + length
    xb = _jittered_block(rng, (x0, y0, z0), (x1, y1, z1), dx, origin)
    seg = (xb[:, 2] / dx - z0) * 3.0 / length
    mat = np.where((seg >= 1.0) & (seg < 2.0), 1, 0).astype(np.int32)
    mats = [Material(E_ends, nu, rho, model), Material(E_mid, nu, rho, model)]
    center = (0.5 * (x0 + x1) * dx, 0.5 * (y0 + y1) * dx, 0.0)
    radius = (np.sqrt(0.5) * width + 2.0) * dx
    lo_x, hi_x = center[0] - radius, center[0] + radius
    lo_y, hi_y = center[1] - radius, center[1] + radius
    bcs = [BoundaryBox(BC_ROTATE, (lo_x, lo_y, (z0 - 3) * dx), (hi_x, hi_y, (z0 + end_cells + 0.5) * dx),
                       (0.0, 0.0, 1.0), center, omega, radius),
           BoundaryBox(BC_ROTATE, (lo_x, lo_y, (z1 - end_cells - 0.5) * dx), (hi_x, hi_y, (z1 + 3) * dx),
                       (0.0, 0.0, 1.0), center, -omega, radius)]
    return _assemble(xb, np.zeros_like(xb), mat, mats, dx, 8, origin, (res, res, res), gravity, bcs,
                     f"three_material_bar_w{width}_l{length}_r{res}_Emid{E_mid:g}")


def two_bars_2m_scene(seed: int = 0) -> Scene:
    """The two-bar scene at 1.5x resolution: dx = 1/384, bars 30 x 30 x 141
    cells, 8 particles per cell (2,030,400 particles)."""
    return two_bars_scene(seed=seed, res=384, width=30, length=141, gap=18)


def tiny_scene(seed: int = 0, res: int = 8, cells=(2, 2, 2), lo=(3, 3, 3), ppc_axis: int = 1,
               E: float = 1e4, nu: float = 0.3, rho: float = 1000.0, model: int = MODEL_FCR,
               vel_amp: float = 0.3, F_jitter: float = 0.0, gravity=(0.0, -9.8, 0.0),
               bcs: Optional[list] = None) -> Scene:
    """A handful of particles for finite-difference and dense-solve checks."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    origin = np.zeros(3)
    lo = np.asarray(lo)
    x = _jittered_block(rng, lo, lo + np.asarray(cells), dx, origin, ppc_axis)
    n = x.shape[0]
    v = rng.uniform(-vel_amp, vel_amp, size=x.shape)
    F = np.tile(np.eye(3), (n, 1, 1)) + F_jitter * rng.uniform(-1, 1, size=(n, 3, 3))
    sc = _assemble(x, v, np.zeros(n, np.int32), [Material(E, nu, rho, model)], dx,
                   ppc_axis ** 3, origin, (res, res, res), gravity, bcs or [], "tiny", F=F)
    sc.C = rng.uniform(-vel_amp, vel_amp, size=(n, 3, 3)) * res * 0.1
    return sc


def stretched_box_scene(seed: int = 0, res: int = 32, side: int = 8, E: float = 1e4,
                        nu: float = 0.3, rho: float = 1000.0) -> Scene:
    """Soft box whose particles start with diag(F) ~ U[0.7, 1.3] (Sec. 6.3,
    'Visualization of Convergence'); no gravity, no boundary conditions."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    origin = np.zeros(3)
    lo = np.full(3, (res - side) // 2)
    x = _jittered_block(rng, lo, lo + side, dx, origin)
    n = x.shape[0]
    F = np.zeros((n, 3, 3))
    d = rng.uniform(0.7, 1.3, size=(n, 3))
    F[:, 0, 0], F[:, 1, 1], F[:, 2, 2] = d[:, 0], d[:, 1], d[:, 2]
    return _assemble(x, np.zeros_like(x), np.zeros(n, np.int32), [Material(E, nu, rho)], dx, 8,
                     origin, (res, res, res), (0.0, 0.0, 0.0), [], f"stretched{side}", F=F)


def batch_scenes(seed: int = 0, count: int = 64, n_min: int = 5000, n_max: int = 200_000,
                 E_range=(1e4, 1e8), yield_stress: float = 1e4) -> List[Scene]:
    """Independent boxes for batched stepping: particle counts log-uniform in
    [n_min, n_max] (8 per cell, aspect ratios in [1/2, 2]), a grid drawn from
    64^3, 96^3, 128^3 among those that fit the box with a 5-cell margin, FCR
    with E log-uniform in E_range, nu = 0.3, rho = 1000; every second scene
    von Mises with the given yield stress; random velocity, sticky floor."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        target = float(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        cells = max(8.0, target / 8.0)
        a = rng.uniform(0.5, 2.0, size=3)
        a /= np.cbrt(a.prod())
        side = np.maximum(2, np.round(a * np.cbrt(cells)).astype(int))
        fits = [r for r in (64, 96, 128) if side.max() + 10 <= r] or [128]
        res = int(fits[int(rng.integers(len(fits)))])
        side = np.minimum(side, res - 10)
        lo = np.array([(res - side[0]) // 2, 5, (res - side[2]) // 2])
        dx = 1.0 / res
        x = _jittered_block(rng, lo, lo + side, dx, np.zeros(3))
        v = rng.uniform(-0.3, 0.3, size=x.shape)
        E = float(np.exp(rng.uniform(np.log(E_range[0]), np.log(E_range[1]))))
        plastic = k % 2
        mats = [Material(E, 0.3, 1000.0, MODEL_FCR, plastic, yield_stress if plastic else 0.0)]
        big = 1e30
        bcs = [BoundaryBox(BC_STICKY, (-big, -big, -big), (big, 4.5 * dx, big))]
        out.append(_assemble(x, v, np.zeros(x.shape[0], np.int32), mats, dx, 8, np.zeros(3),
                             (res, res, res), (0.0, -9.8, 0.0), bcs, f"batch{k}_n{x.shape[0]}_r{res}"))
    return out


def serving_scenes(seed: int = 0, count: int = 256, median: float = 50_000, sigma: float = 1.0,
                   n_max: int = 1_000_000) -> List[Scene]:
    """Resident scenes for the step server: particle counts lognormal (median
    50k, sigma 1, clipped at 1M), boxes as in batch_scenes, materials mixed:
    E log-uniform in [1e4, 1e9], FCR or Neo-Hookean, every third scene von
    Mises (yield 1e4 Pa)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = float(min(n_max, max(1000.0, np.exp(rng.normal(np.log(median), sigma)))))
        sc = batch_scenes(seed=int(rng.integers(1 << 31)), count=1, n_min=n, n_max=n,
                          E_range=(1e4, 1e9))[0]
        m = sc.materials[0]
        plastic = 1 if k % 3 == 0 else 0
        model = int(rng.integers(2))
        sc.materials = [Material(m.E, m.nu, m.rho, model, plastic, 1e4 if plastic else 0.0)]
        sc.name = f"serve{k}_n{sc.n}"
        out.append(sc)
    return out


def scene_by_name(name: str, seed: int = 0) -> Scene:
    if name == "cube8k":
        return cube_scene(seed)
    if name == "two_bars_600k":
        return two_bars_scene(seed)
    if name == "two_bars_2m":
        return two_bars_2m_scene(seed)
    raise KeyError(name)
