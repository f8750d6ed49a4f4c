"""Error paths of the C ABI, driven from the host (no GPU fault, trap or
hang): a failing device allocator, a NaN in the particle input, and the
L-BFGS iteration cap.  Each call returns its status and leaves the library
usable."""
import ctypes as C

import numpy as np
import pytest

from paper_1911_07913_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hot():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1911_07913_gb300 import hot as H
    H.load()
    return H


def small_cube():
    sc = scenes.cube_scene(seed=5, res=16, cube_lo=(5, 4, 5), side=4)
    return sc, scenes.SolverOptions(eps=1e-6, cn_mode=1, dt=4e-3, levels=2)


def test_allocation_failure_is_reported_and_recoverable(hot):
    """An allocator that fails from its fourth request on: scene creation
    returns MPM_ERR_OOM and frees what it had taken; with the normal
    allocator back, a scene steps as usual."""
    import torch
    lib = hot.load()
    sc, opts = small_cube()
    calls = {"n": 0}
    live = set()   # pointers this allocator handed out and the library has not freed

    def _alloc(nbytes, stream, ctx):
        calls["n"] += 1
        if calls["n"] >= 4:
            return None
        ptr = int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0))
        live.add(ptr)
        return ptr

    def _free(ptr, stream, ctx):
        live.discard(int(ptr))
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = hot.ALLOC_FN(_alloc), hot.FREE_FN(_free)
    assert lib.mpm_set_allocator(C.cast(a, C.c_void_p), C.cast(f, C.c_void_p), None) == 0
    try:
        with pytest.raises(hot.HotError) as err:
            hot.HotScene(sc, opts)
        assert err.value.code == 2          # MPM_ERR_OOM
        assert calls["n"] == 4 and not live
    finally:
        hot._install_torch_allocator(lib)
    g = hot.HotScene(sc, opts)
    st = g.step()
    assert st["status"] == 0 and st["iters"] >= 1
    g.close()


def test_nan_input_reports_numeric(hot):
    """A NaN velocity reaches the gradient; the convergence test reports
    MPM_ERR_NUMERIC and G2P is not applied."""
    sc, opts = small_cube()
    sc.v[7, 1] = np.nan
    g = hot.HotScene(sc, opts)
    x0 = g.get_state()["x"].copy()
    st = g.step(check=False)
    assert st["code"] == 6                  # MPM_ERR_NUMERIC
    np.testing.assert_array_equal(g.get_state()["x"], x0)
    g.close()


def test_iteration_cap_reports_not_converged_and_advances(hot):
    """With max_iters = 2 and a tolerance no two iterations reach, the step
    returns MPM_ERR_NOT_CONVERGED after exactly two iterations and G2P
    applies the last accepted iterate."""
    sc, opts = small_cube()
    opts = scenes.SolverOptions(**{**opts.__dict__, "eps": 1e-13, "max_iters": 2})
    g = hot.HotScene(sc, opts)
    x0 = g.get_state()["x"].copy()
    st = g.step(check=False)
    assert st["code"] == 4                  # MPM_ERR_NOT_CONVERGED
    assert st["iters"] == 2
    x1 = g.get_state()["x"]
    assert np.all(np.isfinite(x1)) and not np.array_equal(x1, x0)
    g.close()


def test_device_wait_timeout_is_reported_and_scene_recovers(hot):
    """Every device-side barrier wait is bounded.  With the poll limit cut to
    one poll, the cooperative Gauss-Seidel sweeps and the cooperative coarsest
    PCG (flag bits 6 and 1: grid barriers on every level) give up waiting,
    record the timeout and return; mpm_apply_vcycle reports MPM_ERR_TIMEOUT.
    No index leaves its buffer, so the early exits race but cannot fault.
    With the default limit back, the same scene applies a V-cycle that the
    oracle reproduces and takes a step whose result the oracle replays."""
    from oracle import hot_oracle as O
    sc = scenes.two_bars_scene(seed=4, res=64, width=6, length=14, gap=8, E_a=1e5, E_b=1e8)
    opts = scenes.SolverOptions(eps=1e-7, cn_mode=0, levels=3, flags=64 | 2)
    g = hot.HotScene(sc, opts)
    g.p2g()
    g.build_hierarchy()
    og = O.p2g(sc)
    prob = O.Problem(sc, og, O.step_dt(sc, opts))
    b = np.random.default_rng(6).normal(size=(prob.n, 3))
    g.set_wait_limit(1)
    timed_out = False
    for _ in range(3):
        try:
            g.vcycle(b)
        except hot.HotError as e:
            assert e.code == 10 and "timed out" in str(e)     # MPM_ERR_TIMEOUT
            timed_out = True
            break
    assert timed_out
    with pytest.raises(hot.HotError):
        g.set_wait_limit(0)
    g.set_wait_limit(1 << 24)
    u, its = g.vcycle(b)
    L = O.build_hierarchy(og.coords, prob.hessian(), prob.hessian_pattern(), opts.levels)
    vc = O.VCycle(L, og.fixed, opts.eps, opts.max_coarse_cg)
    vc.forced = [its]
    uo = vc(b)
    assert np.abs(u - uo).max() <= 1e-9 * np.abs(uo).max()
    st = g.solve()
    assert st["status"] == 0
    tr = g.trace()
    dv = g.grid()["dv"]
    g.close()
    rep = O.Trace(iters=tr["iters"], alphas=tr["alphas"], ls_trials=tr["ls_trials"], cg_counts=tr["cg_counts"],
                  skipped=tr["skipped"], fallback=tr["fallback"])
    dvo, _ = O.hot_solve(O.Problem(sc, og, st["dt"]), opts, replay=rep)
    assert np.abs(dv - dvo).max() <= 1e-9 * np.abs(dvo).max()


def test_cluster_sweep_wait_past_limit_is_reported_and_completes(hot):
    """The cluster sweeps that keep u in shared memory wait on per-CTA byte
    counts; past the poll limit they record the timeout but keep waiting
    (the bytes of a color always arrive), so no CTA leaves while stores into
    its shared memory may be in flight.  With the limit cut to one poll and
    the default launches, the V-cycle reports MPM_ERR_TIMEOUT (or completes
    within one poll per wait); with the default limit back the scene applies
    the same V-cycle, bitwise, as before the limit was cut."""
    sc = scenes.two_bars_scene(seed=4, res=64, width=6, length=14, gap=8, E_a=1e5, E_b=1e8)
    opts = scenes.SolverOptions(eps=1e-7, cn_mode=0, levels=3, flags=1)   # eager: each launch on its own
    g = hot.HotScene(sc, opts)
    g.p2g()
    g.build_hierarchy()
    b = np.random.default_rng(7).normal(size=(len(g.grid()["m"]), 3))
    u_ref, its_ref = g.vcycle(b)
    g.set_wait_limit(1)
    try:
        g.vcycle(b)
    except hot.HotError as e:
        assert e.code == 10 and "timed out" in str(e)     # MPM_ERR_TIMEOUT
    g.set_wait_limit(1 << 24)
    u, its = g.vcycle(b)
    assert its == its_ref and np.array_equal(u, u_ref)
    g.close()
