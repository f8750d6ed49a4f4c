"""Python binding of the HOT CUDA library (include/hot_mpm.h).

Argument marshalling only: every step of the MPM time step runs in the
library's CUDA kernels.  PyTorch provides the device memory pool (its caching
allocator is installed as the library's allocator) and the CUDA stream.
Importing this module does not need a GPU; creating a scene does, and fails
loudly when the compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import scenes as _scenes

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhotmpm.so")

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "NOT_CONVERGED", 5: "LINESEARCH",
          6: "NUMERIC", 7: "ADMISSION", 8: "STATE", 9: "DOMAIN", 10: "TIMEOUT"}
OK, NOT_CONVERGED, LINESEARCH = 0, 4, 5

EXPORTED = ["mpm_set_allocator", "mpm_create_scene", "mpm_destroy_scene", "mpm_last_error",
            "mpm_set_options", "mpm_p2g", "mpm_build_hierarchy", "mpm_solve_step", "mpm_g2p",
            "mpm_step", "mpm_get_state", "mpm_set_state", "mpm_get_grid", "mpm_eval_energy",
            "mpm_eval_gradient", "mpm_get_hessian", "mpm_apply_vcycle", "mpm_get_trace", "mpm_get_inner_iters",
            "mpm_batch_autotune",
            "mpm_scene_footprint", "mpm_step_batch", "mpm_profile", "mpm_profile_read",
            "mpm_kernel_launch_count", "mpm_particle_energy_noalloc", "mpm_server_create",
            "mpm_server_submit", "mpm_server_poll", "mpm_server_info", "mpm_server_destroy",
            "mpm_probe_fp64_fma", "mpm_set_wait_limit", "mpm_scene_park", "mpm_scene_unpark",
            "mpm_scene_residency", "mpm_server_residency"]


class mpm_material(C.Structure):
    _fields_ = [("E", C.c_double), ("nu", C.c_double), ("rho", C.c_double),
                ("yield_stress", C.c_double), ("model", C.c_int32), ("plasticity", C.c_int32)]


class mpm_bc(C.Structure):
    _fields_ = [("type", C.c_int32), ("reserved", C.c_int32), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("axis", C.c_double * 3), ("center", C.c_double * 3),
                ("omega", C.c_double), ("radius", C.c_double)]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class mpm_scene_desc(C.Structure):
    _fields_ = [("n_particles", C.c_int64), ("x", _dp), ("v", _dp), ("F", _dp), ("C", _dp),
                ("vol", _dp), ("mass", _dp), ("material_id", _ip),
                ("materials", C.POINTER(mpm_material)), ("n_materials", C.c_int32),
                ("grid_dims", C.c_int32 * 3), ("dx", C.c_double), ("origin", C.c_double * 3),
                ("gravity", C.c_double * 3), ("bcs", C.POINTER(mpm_bc)), ("n_bcs", C.c_int32),
                ("inputs_on_device", C.c_int32), ("cuda_stream", C.c_void_p)]


class mpm_solver_opts(C.Structure):
    _fields_ = [("eps", C.c_double), ("cn_mode", C.c_int32), ("lbfgs_m", C.c_int32),
                ("levels", C.c_int32), ("precision", C.c_int32), ("max_iters", C.c_int32),
                ("max_ls", C.c_int32), ("max_coarse_cg", C.c_int32), ("record_trace", C.c_int32),
                ("dt", C.c_double), ("fps", C.c_double), ("cfl", C.c_double), ("flags", C.c_int32),
                ("solver", C.c_int32), ("refresh_every", C.c_int32), ("fallback_after", C.c_int32)]


class mpm_step_stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("ls_trials", C.c_int32), ("coarse_cg_iters", C.c_int32),
                ("vcycles", C.c_int32), ("final_norm", C.c_double), ("energy", C.c_double),
                ("dt_used", C.c_double), ("n_particles", C.c_int64), ("n_nodes", C.c_int64 * 8),
                ("nnz_blocks", C.c_int64 * 8), ("n_levels", C.c_int32), ("status", C.c_int32),
                ("graph_vcycles", C.c_int32), ("device_loop", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

_lib = None
_alloc_refs = None


class HotError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def library_path() -> str:
    return LIB_PATH


def load(install_torch_allocator: bool = True):
    """Load libhotmpm.so (built by paper_1911_07913_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"HOT CUDA library not built: {LIB_PATH} is missing "
                           "(run __graft_entry__.build())")
    lib = C.CDLL(LIB_PATH)
    for name in EXPORTED:
        getattr(lib, name).restype = C.c_int
    lib.mpm_last_error.restype = C.c_char_p
    lib.mpm_last_error.argtypes = [C.c_void_p]
    lib.mpm_create_scene.argtypes = [C.POINTER(mpm_scene_desc), C.POINTER(mpm_solver_opts),
                                     C.POINTER(C.c_void_p)]
    lib.mpm_destroy_scene.argtypes = [C.c_void_p]
    lib.mpm_set_options.argtypes = [C.c_void_p, C.POINTER(mpm_solver_opts)]
    for f in ("mpm_p2g", "mpm_build_hierarchy", "mpm_g2p"):
        getattr(lib, f).argtypes = [C.c_void_p]
    lib.mpm_solve_step.argtypes = [C.c_void_p, C.POINTER(mpm_step_stats)]
    lib.mpm_step.argtypes = [C.c_void_p, C.POINTER(mpm_step_stats)]
    lib.mpm_get_state.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
    lib.mpm_set_state.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
    lib.mpm_get_grid.argtypes = [C.c_void_p, C.POINTER(C.c_int64), C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p]
    lib.mpm_eval_energy.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]
    lib.mpm_eval_gradient.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    lib.mpm_get_hessian.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.mpm_apply_vcycle.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]
    lib.mpm_get_trace.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.POINTER(C.c_int32), C.c_void_p]
    lib.mpm_get_inner_iters.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.c_void_p]
    lib.mpm_scene_footprint.argtypes = [C.c_void_p, C.POINTER(C.c_int64)]
    lib.mpm_step_batch.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(mpm_step_stats)]
    lib.mpm_batch_autotune.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.c_int32, C.POINTER(C.c_int32),
                                       C.POINTER(C.c_int32), C.POINTER(C.c_double), C.POINTER(C.c_int32)]
    lib.mpm_set_allocator.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    lib.mpm_profile.argtypes = [C.c_void_p, C.c_int32, C.c_char_p]
    lib.mpm_profile_read.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.c_void_p, C.c_void_p,
                                     C.c_void_p]
    lib.mpm_kernel_launch_count.restype = C.c_int64
    lib.mpm_kernel_launch_count.argtypes = []
    lib.mpm_server_create.argtypes = [C.c_int64, C.c_int32, C.POINTER(C.c_void_p)]
    lib.mpm_server_submit.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
    lib.mpm_server_poll.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_int64), C.POINTER(mpm_step_stats),
                                    C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int32)]
    lib.mpm_server_info.argtypes = [C.c_void_p] + [C.POINTER(C.c_int64)] * 4
    lib.mpm_server_destroy.argtypes = [C.c_void_p]
    lib.mpm_particle_energy_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(mpm_material),
                                                C.c_int32, C.c_int64, C.c_void_p, C.c_int32, C.c_void_p]
    lib.mpm_set_wait_limit.argtypes = [C.c_void_p, C.c_int64]
    lib.mpm_scene_park.argtypes = [C.c_void_p]
    lib.mpm_scene_unpark.argtypes = [C.c_void_p]
    lib.mpm_scene_residency.argtypes = [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64)]
    lib.mpm_server_residency.argtypes = [C.c_void_p] + [C.POINTER(C.c_int64)] * 5
    lib.mpm_probe_fp64_fma.argtypes = [C.c_void_p, C.POINTER(C.c_double)]
    _lib = lib
    if install_torch_allocator:
        _install_torch_allocator(lib)
    return lib


def _install_torch_allocator(lib):
    """Route the library's device allocations through PyTorch's caching
    allocator on the current device."""
    global _alloc_refs
    try:
        import torch
    except ImportError:
        return
    if not torch.cuda.is_available():
        return

    def _alloc(nbytes, stream, ctx):
        try:
            dev = torch.cuda.current_device()
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0))
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    _alloc_refs = (a, f)
    lib.mpm_set_allocator(C.cast(a, C.c_void_p), C.cast(f, C.c_void_p), None)


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(C.c_void_p)


def opts_struct(o: _scenes.SolverOptions) -> mpm_solver_opts:
    return mpm_solver_opts(eps=o.eps, cn_mode=o.cn_mode, lbfgs_m=o.lbfgs_m, levels=o.levels,
                           precision=o.precision, max_iters=o.max_iters, max_ls=o.max_ls,
                           max_coarse_cg=o.max_coarse_cg, record_trace=1, dt=o.dt, fps=o.fps,
                           cfl=o.cfl, flags=getattr(o, "flags", 0), solver=getattr(o, "solver", 0),
                           refresh_every=getattr(o, "refresh_every", 0),
                           fallback_after=getattr(o, "fallback_after", 0))


def stats_dict(s: mpm_step_stats) -> dict:
    nl = s.n_levels
    return {"iters": s.iters, "ls_trials": s.ls_trials, "coarse_cg_iters": s.coarse_cg_iters,
            "vcycles": s.vcycles, "final_norm": s.final_norm, "energy": s.energy, "dt": s.dt_used,
            "n_particles": s.n_particles, "n_nodes": list(s.n_nodes[:nl]),
            "nnz_blocks": list(s.nnz_blocks[:nl]), "n_levels": nl, "status": s.status,
            "status_name": STATUS.get(s.status, str(s.status)), "graph_vcycles": s.graph_vcycles,
            "device_loop": s.device_loop}


class HotScene:
    """One MPM scene resident on the GPU."""

    def __init__(self, sc: _scenes.Scene, opts: _scenes.SolverOptions, stream=None):
        self.lib = load()
        self.n = sc.n
        self._keep = {}
        x = np.ascontiguousarray(sc.x, np.float64)
        v = np.ascontiguousarray(sc.v, np.float64)
        F = np.ascontiguousarray(sc.F.reshape(-1, 9), np.float64)
        Cm = np.ascontiguousarray(sc.C.reshape(-1, 9), np.float64)
        vol = np.ascontiguousarray(sc.vol, np.float64)
        mass = np.ascontiguousarray(sc.mass, np.float64)
        mat = np.ascontiguousarray(sc.mat, np.int32)
        mats = (mpm_material * len(sc.materials))(*[
            mpm_material(m.E, m.nu, m.rho, m.yield_stress, m.model, m.plasticity) for m in sc.materials])
        bcs = (mpm_bc * max(1, len(sc.bcs)))()
        for k, b in enumerate(sc.bcs):
            bcs[k] = mpm_bc(b.type, 0, (C.c_double * 3)(*b.lo), (C.c_double * 3)(*b.hi),
                            (C.c_double * 3)(*b.axis), (C.c_double * 3)(*b.center), b.omega,
                            getattr(b, "radius", 0.0))
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except ImportError:
                stream = 0
        d = mpm_scene_desc()
        d.n_particles = sc.n
        d.x, d.v, d.F, d.C = (a.ctypes.data_as(_dp) for a in (x, v, F, Cm))
        d.vol, d.mass = vol.ctypes.data_as(_dp), mass.ctypes.data_as(_dp)
        d.material_id = mat.ctypes.data_as(_ip)
        d.materials = mats
        d.n_materials = len(sc.materials)
        d.grid_dims = (C.c_int32 * 3)(*[int(k) for k in sc.grid_dims])
        d.dx = sc.dx
        d.origin = (C.c_double * 3)(*sc.origin)
        d.gravity = (C.c_double * 3)(*sc.gravity)
        d.bcs = bcs
        d.n_bcs = len(sc.bcs)
        d.inputs_on_device = 0
        d.cuda_stream = C.c_void_p(int(stream)) if stream else None
        self.opts = opts
        o = opts_struct(opts)
        h = C.c_void_p()
        self._check(self.lib.mpm_create_scene(C.byref(d), C.byref(o), C.byref(h)), None)
        self.h = h

    # ------------------------------------------------------------------
    def _check(self, code, h="self"):
        if code != OK:
            hh = self.h if h == "self" else h
            msg = self.lib.mpm_last_error(hh).decode()
            raise HotError(code, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.mpm_destroy_scene(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_wait_limit(self, polls: int):
        """Poll limit of the scene's device-side barrier waits (default 2^24)."""
        self._check(self.lib.mpm_set_wait_limit(self.h, C.c_int64(int(polls))))

    def set_options(self, opts):
        self.opts = opts
        o = opts_struct(opts)
        self._check(self.lib.mpm_set_options(self.h, C.byref(o)))

    def p2g(self):
        self._check(self.lib.mpm_p2g(self.h))

    def build_hierarchy(self):
        self._check(self.lib.mpm_build_hierarchy(self.h))

    def solve(self, check=True) -> dict:
        st = mpm_step_stats()
        code = self.lib.mpm_solve_step(self.h, C.byref(st))
        if check and code not in (OK,):
            self._check(code)
        return stats_dict(st)

    def g2p(self):
        self._check(self.lib.mpm_g2p(self.h))

    def step(self, check=True) -> dict:
        st = mpm_step_stats()
        code = self.lib.mpm_step(self.h, C.byref(st))
        if check and code != OK:
            self._check(code)
        out = stats_dict(st)
        out["code"] = code
        return out

    def get_state(self):
        n = self.n
        x = np.empty((n, 3))
        v = np.empty((n, 3))
        F = np.empty((n, 3, 3))
        Cm = np.empty((n, 3, 3))
        self._check(self.lib.mpm_get_state(self.h, _ptr(x), _ptr(v), _ptr(F), _ptr(Cm), 0))
        return {"x": x, "v": v, "F": F, "C": Cm}

    def get_state_device(self, x, v, F, Cm):
        """Copy the state into device buffers given as integer pointers."""
        self._check(self.lib.mpm_get_state(self.h, C.c_void_p(x), C.c_void_p(v), C.c_void_p(F),
                                           C.c_void_p(Cm), 1))

    def set_state(self, x=None, v=None, F=None, Cm=None):
        arrs = [None if a is None else np.ascontiguousarray(a, np.float64) for a in (x, v, F, Cm)]
        self._check(self.lib.mpm_set_state(self.h, *[_ptr(a) for a in arrs], 0))

    def grid(self) -> dict:
        n = C.c_int64()
        self._check(self.lib.mpm_get_grid(self.h, C.byref(n), None, None, None, None, None, None))
        nn = n.value
        ijk = np.empty((nn, 3), np.int32)
        m = np.empty(nn)
        v = np.empty((nn, 3))
        xi = np.empty(nn)
        fixed = np.empty(nn, np.int32)
        dv = np.empty((nn, 3))
        self._check(self.lib.mpm_get_grid(self.h, C.byref(n), _ptr(ijk), _ptr(m), _ptr(v), _ptr(xi),
                                          _ptr(fixed), _ptr(dv)))
        return {"coords": ijk, "m": m, "v": v, "xi": xi, "fixed": fixed.astype(bool), "dv": dv}

    def energy(self, dv) -> float:
        dv = np.ascontiguousarray(dv, np.float64)
        e = C.c_double()
        self._check(self.lib.mpm_eval_energy(self.h, _ptr(dv), C.byref(e)))
        return e.value

    def gradient(self, dv) -> np.ndarray:
        dv = np.ascontiguousarray(dv, np.float64)
        g = np.empty_like(dv)
        self._check(self.lib.mpm_eval_gradient(self.h, _ptr(dv), _ptr(g)))
        return g

    def hessian(self, level: int = 0) -> dict:
        nr, nb = C.c_int64(), C.c_int64()
        self._check(self.lib.mpm_get_hessian(self.h, level, C.byref(nr), C.byref(nb), None, None, None, None))
        rp = np.empty(nr.value + 1, np.int32)
        cols = np.empty(nb.value, np.int32)
        vals = np.empty((nb.value, 3, 3))
        coords = np.empty((nr.value, 3), np.int32)
        self._check(self.lib.mpm_get_hessian(self.h, level, C.byref(nr), C.byref(nb), _ptr(rp), _ptr(cols),
                                             _ptr(vals), _ptr(coords)))
        return {"row_ptr": rp, "cols": cols, "vals": vals, "coords": coords}

    def vcycle(self, b):
        b = np.ascontiguousarray(b, np.float64)
        u = np.empty_like(b)
        its = C.c_int32()
        self._check(self.lib.mpm_apply_vcycle(self.h, _ptr(b), _ptr(u), C.byref(its)))
        return u, its.value

    def trace(self, capacity: int = 100000) -> dict:
        ni, nv = C.c_int32(), C.c_int32()
        al = np.zeros(capacity)
        ls = np.zeros(capacity, np.int32)
        sk = np.zeros(capacity, np.int32)
        fb = np.zeros(capacity, np.int32)
        cg = np.zeros(capacity, np.int32)
        self._check(self.lib.mpm_get_trace(self.h, capacity, C.byref(ni), _ptr(al), _ptr(ls), _ptr(sk),
                                           _ptr(fb), C.byref(nv), _ptr(cg)))
        k = ni.value
        return {"iters": k, "alphas": al[:k].tolist(), "ls_trials": ls[:k].tolist(),
                "skipped": sk[:k].tolist(), "fallback": fb[:k].tolist(),
                "cg_counts": cg[:nv.value].tolist()}

    def inner_iters(self, capacity: int = 100000) -> list:
        """CG iterations of each Newton iteration (projected-Newton solvers)."""
        n = C.c_int32()
        out = np.zeros(capacity, np.int32)
        self._check(self.lib.mpm_get_inner_iters(self.h, capacity, C.byref(n), _ptr(out)))
        return out[:min(n.value, capacity)].tolist()

    def profile(self, enable: bool = True, only: Optional[str] = None):
        self._check(self.lib.mpm_profile(self.h, 1 if enable else 0, only.encode() if only else None))

    def profile_read(self) -> dict:
        cap = 64
        cnt = C.c_int32()
        names = C.create_string_buffer(32 * cap)
        ms = np.zeros(cap)
        nl = np.zeros(cap, np.int64)
        self._check(self.lib.mpm_profile_read(self.h, cap, C.byref(cnt), names, _ptr(ms), _ptr(nl)))
        out = {}
        for k in range(min(cnt.value, cap)):
            nm = names.raw[32 * k:32 * (k + 1)].split(b"\0", 1)[0].decode()
            out[nm] = {"ms": float(ms[k]), "launches": int(nl[k])}
        return out

    def park(self):
        """Particle state to host memory, every device buffer released."""
        self._check(self.lib.mpm_scene_park(self.h))

    def unpark(self):
        self._check(self.lib.mpm_scene_unpark(self.h))

    def residency(self) -> dict:
        p, b = C.c_int32(), C.c_int64()
        self._check(self.lib.mpm_scene_residency(self.h, C.byref(p), C.byref(b)))
        return {"parked": bool(p.value), "peak_bytes": b.value}

    def footprint(self) -> int:
        b = C.c_int64()
        self._check(self.lib.mpm_scene_footprint(self.h, C.byref(b)))
        return b.value


def particle_energy_noalloc(F_dev: int, vol_dev: int, mat_dev: int, materials, n: int,
                            out_dev: Optional[int] = None, stream: int = 0) -> Optional[float]:
    """Elastic energy of n particles from device arrays (F n x 9, vol n,
    material ids n) without any device allocation: for callers that cannot
    allocate (allocation-free loops, fixed device-memory budgets).  Returns
    the value (host result) or None when out_dev (a device double*) is given."""
    lib = load()
    mats = (mpm_material * len(materials))(*[
        mpm_material(m.E, m.nu, m.rho, m.yield_stress, m.model, m.plasticity) for m in materials])
    if out_dev is None:
        e = C.c_double()
        code = lib.mpm_particle_energy_noalloc(C.c_void_p(F_dev), C.c_void_p(vol_dev), C.c_void_p(mat_dev),
                                               mats, len(materials), n, C.cast(C.byref(e), C.c_void_p), 0,
                                               C.c_void_p(stream) if stream else None)
        if code != OK:
            raise HotError(code, lib.mpm_last_error(None).decode())
        return e.value
    code = lib.mpm_particle_energy_noalloc(C.c_void_p(F_dev), C.c_void_p(vol_dev), C.c_void_p(mat_dev), mats,
                                           len(materials), n, C.c_void_p(out_dev), 1,
                                           C.c_void_p(stream) if stream else None)
    if code != OK:
        raise HotError(code, lib.mpm_last_error(None).decode())
    return None


class StepServer:
    """Continuous-batching server of implicit steps for resident scenes
    (mpm_server_* in the C ABI)."""

    def __init__(self, budget_bytes: int, n_workers: int = 8):
        self.lib = load()
        h = C.c_void_p()
        code = self.lib.mpm_server_create(int(budget_bytes), int(n_workers), C.byref(h))
        if code != OK:
            raise HotError(code, "mpm_server_create")
        self.h = h

    def submit(self, scene: "HotScene", request_id: int):
        code = self.lib.mpm_server_submit(self.h, scene.h, int(request_id))
        if code != OK:
            raise HotError(code, f"request {request_id} not admitted")

    def poll(self, wait: bool = True):
        rid = C.c_int64()
        st = mpm_step_stats()
        lat, qd = C.c_double(), C.c_double()
        code = C.c_int32()
        self.lib.mpm_server_poll(self.h, 1 if wait else 0, C.byref(rid), C.byref(st), C.byref(lat), C.byref(qd),
                                 C.byref(code))
        if rid.value < 0:
            return None
        out = stats_dict(st)
        out.update({"request_id": rid.value, "latency_s": lat.value, "queue_s": qd.value, "code": code.value})
        return out

    def info(self) -> dict:
        v = [C.c_int64() for _ in range(4)]
        self.lib.mpm_server_info(self.h, *[C.byref(x) for x in v])
        out = dict(zip(("queued", "in_flight", "in_flight_bytes", "peak_in_flight_bytes"), [x.value for x in v]))
        w = [C.c_int64() for _ in range(5)]
        self.lib.mpm_server_residency(self.h, *[C.byref(x) for x in w])
        out.update(zip(("resident_bytes", "peak_resident_bytes", "parks", "unparks", "deferred"),
                       [x.value for x in w]))
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.mpm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe_fp64_tflops(stream: int = 0) -> float:
    """Measured FP64 FMA throughput of the current device (TFLOP/s)."""
    lib = load()
    t = C.c_double()
    code = lib.mpm_probe_fp64_fma(C.c_void_p(stream) if stream else None, C.byref(t))
    if code != OK:
        raise HotError(code, lib.mpm_last_error(None).decode())
    return t.value


def kernel_launch_count() -> int:
    return int(load().mpm_kernel_launch_count())


def batch_autotune(scene_list, steps: int = 1) -> dict:
    """Times real batched steps under each launch configuration and keeps the
    fastest (see mpm_batch_autotune); returns the choice."""
    lib = load()
    n = len(scene_list)
    hs = (C.c_void_p * n)(*[s.h for s in scene_list])
    fl, wk, rate, ran = C.c_int32(), C.c_int32(), C.c_double(), C.c_int32()
    code = lib.mpm_batch_autotune(hs, n, steps, C.byref(fl), C.byref(wk), C.byref(rate), C.byref(ran))
    if code != OK:
        raise HotError(code, lib.mpm_last_error(None).decode())
    return {"flags": fl.value, "workers": wk.value, "particle_steps_per_s": rate.value, "steps_run": ran.value}


def step_batch(scene_list, check=True):
    lib = load()
    n = len(scene_list)
    hs = (C.c_void_p * n)(*[s.h for s in scene_list])
    st = (mpm_step_stats * n)()
    code = lib.mpm_step_batch(hs, n, st)
    if check and code != OK:
        raise HotError(code, lib.mpm_last_error(None).decode())
    return [stats_dict(st[i]) for i in range(n)]
