"""GPU parity at the benchmark's full size: the 601,600-particle two-bar scene
(dx = 1/256, 5 levels, FP64, CN eps = 1e-7) in the launch configuration
bench.py times (a scene on its own CUDA stream, V-cycle as a CUDA graph).

The oracle runs in float64 on the host where that is affordable at this size
(P2G, energy, gradient, G2P, Galerkin products, one V-cycle), and on sampled
rows where it is not (the fine Hessian: only the particles whose stencils
contain the sampled nodes)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import hot_oracle as O
from paper_1911_07913_gb300 import scenes

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

OPTS = scenes.SolverOptions(eps=1e-7, cn_mode=0, lbfgs_m=8, levels=5, precision=0, max_iters=500)


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1911_07913_gb300 import hot
    sc = scenes.two_bars_scene(seed=0)
    stream = torch.cuda.Stream()
    g = hot.HotScene(sc, OPTS, stream=stream.cuda_stream)
    g.p2g()
    og = O.p2g(sc)
    prob = O.Problem(sc, og, O.step_dt(sc, OPTS))
    yield sc, g, og, prob
    g.close()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_fullsize_p2g_nodes_and_values(setup):
    sc, g, og, prob = setup
    gd = g.grid()
    assert sc.n == 601_600
    assert np.array_equal(gd["coords"], og.coords.astype(np.int32))
    assert np.array_equal(gd["fixed"], og.fixed)
    assert rel(gd["m"], og.m) < 1e-12
    assert rel(gd["v"], og.v) < 1e-12
    assert rel(gd["xi"], og.xi) < 1e-12


def test_fullsize_energy_and_gradient(setup):
    sc, g, og, prob = setup
    rng = np.random.default_rng(5)
    dv = 0.01 * rng.normal(size=(prob.n, 3))
    dv[og.fixed] = 0.0
    E_g, E_o = g.energy(dv), prob.energy(dv)
    assert abs(E_g - E_o) <= 1e-12 * abs(E_o)
    assert rel(g.gradient(dv), prob.gradient(dv)) < 1e-11


def test_fullsize_hessian_sampled_rows(setup):
    sc, g, og, prob = setup
    g.build_hierarchy()
    H = g.hessian(0)
    n = H["coords"].shape[0]
    rng = np.random.default_rng(6)
    rows = rng.choice(n, 12, replace=False)
    # particles whose stencil contains a sampled node
    touch = np.isin(og.pidx, rows).any(axis=1)
    sub = np.nonzero(touch)[0]
    F0 = prob.deformation(np.zeros((n, 3)))[sub]
    A = O.project_psd(O.dPdF(F0, prob.mu[sub], prob.lam[sub], prob.model[sub])).reshape(-1, 3, 3, 3, 3)
    d = np.einsum("pba,pkb->pka", sc.F[sub], og.gw[sub])
    blk = np.einsum("pagbd,pig,pld->pilab", A, d, d) * (prob.dt ** 2 * sc.vol[sub])[:, None, None, None, None]
    pidx = og.pidx[sub]
    fixed = og.fixed
    for r in rows:
        ref = {}
        for p in range(sub.size):
            hits = np.nonzero(pidx[p] == r)[0]
            for i in hits:
                for l in range(27):
                    c = pidx[p, l]
                    ref[c] = ref.get(c, 0.0) + blk[p, i, l]
        ref[r] = ref.get(r, 0.0) + og.m[r] * np.eye(3)
        for c in list(ref):
            if fixed[r] or fixed[c]:
                ref[c] = np.zeros((3, 3))
        if fixed[r]:
            ref[r] = (og.m[r] if og.m[r] > 0 else 1.0) * np.eye(3)
        a, b = H["row_ptr"][r], H["row_ptr"][r + 1]
        got = {int(c): H["vals"][k] for k, c in zip(range(a, b), H["cols"][a:b])}
        assert set(got) == set(ref)
        scale = max(np.abs(v).max() for v in ref.values())
        for c in ref:
            assert np.abs(got[c] - ref[c]).max() <= 1e-11 * scale


def gpu_level_matrix(h):
    n = h["coords"].shape[0]
    return sp.bsr_matrix((h["vals"], h["cols"], h["row_ptr"]), shape=(3 * n, 3 * n)).tocsr()


def test_fullsize_galerkin_levels(setup):
    """Each coarse level equals R H^m R^T of the GPU's own finer level (the
    oracle's restriction on the GPU's node sets)."""
    sc, g, og, prob = setup
    g.build_hierarchy()
    levels = [g.hessian(m) for m in range(OPTS.levels)]
    for m in range(OPTS.levels - 1):
        fc, cc = levels[m]["coords"].astype(np.int64), levels[m + 1]["coords"].astype(np.int64)
        ref_coarse = O.coarse_nodes(fc)
        assert np.array_equal(ref_coarse, cc)
        R3 = sp.kron(O.restriction(fc, cc), sp.eye(3)).tocsr()
        Hf, Hc = gpu_level_matrix(levels[m]), gpu_level_matrix(levels[m + 1])
        ref = (R3 @ Hf @ R3.T).tocsr()
        diff = abs(Hc - ref)
        assert diff.max() <= 1e-11 * abs(ref).max(), m


def test_fullsize_vcycle_against_oracle_on_gpu_hierarchy(setup):
    sc, g, og, prob = setup
    g.build_hierarchy()
    levels = []
    mats = [g.hessian(m) for m in range(OPTS.levels)]
    for m, h in enumerate(mats):
        coords = h["coords"].astype(np.int64)
        Hm = gpu_level_matrix(h)
        R = O.restriction(coords, mats[m + 1]["coords"].astype(np.int64)) if m + 1 < len(mats) else None
        pat = sp.csr_matrix((np.ones(h["cols"].size), h["cols"], h["row_ptr"]), shape=(coords.shape[0],) * 2)
        levels.append(O.Level(coords=coords, H=Hm, pattern=pat, R=R, colors=O.node_colors(coords),
                              Dblk=O.diag_blocks(Hm, coords.shape[0])))
    rng = np.random.default_rng(7)
    b = rng.normal(size=(prob.n, 3))
    u, its = g.vcycle(b)
    vc = O.VCycle(levels, og.fixed, OPTS.eps, OPTS.max_coarse_cg)
    vc.forced = [its]
    assert rel(u, vc(b)) < 1e-9


def test_fullsize_step_converges_and_g2p_matches(setup):
    sc, g, og, prob = setup
    g.p2g()
    st = g.solve()
    assert st["status"] == 0 and st["iters"] >= 1
    gd = g.grid()
    gr = prob.gradient(gd["dv"])
    nrm, nfree = prob.cn_norm(gr)
    assert nrm <= OPTS.eps * np.sqrt(nfree) * (1 + 1e-6)
    assert prob.energy(gd["dv"]) < prob.energy(np.zeros_like(gd["dv"]))
    g.g2p()
    out = g.get_state()
    ref = O.g2p(sc, og, og.v + gd["dv"], prob.dt)
    assert rel(out["x"], ref.x) < 1e-12
    assert rel(out["v"], ref.v) < 1e-10
    assert rel(out["F"], ref.F) < 1e-12
    assert rel(out["C"], ref.C) < 1e-9


def test_fullsize_mixed_2m_converges_to_oracle_tolerance():
    """The 2,030,400-particle scene in mixed precision (FP32 hierarchy): one
    step reaches the same CN tolerance, judged by the FP64 oracle's gradient
    at the GPU's solution; its FP64 energy and G2P match the oracle's."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1911_07913_gb300 import hot
    sc = scenes.two_bars_2m_scene(seed=0)
    opts = scenes.SolverOptions(**{**OPTS.__dict__, "precision": 1})
    stream = torch.cuda.Stream()
    g = hot.HotScene(sc, opts, stream=stream.cuda_stream)
    g.p2g()
    st = g.solve()
    assert st["status"] == 0
    gd = g.grid()
    og = O.p2g(sc)
    assert np.array_equal(gd["coords"], og.coords.astype(np.int32))
    prob = O.Problem(sc, og, st["dt"])
    nrm, nfree = prob.cn_norm(prob.gradient(gd["dv"]))
    assert nrm <= opts.eps * np.sqrt(nfree) * (1 + 1e-6)
    assert abs(g.energy(gd["dv"]) - prob.energy(gd["dv"])) <= 1e-12 * abs(prob.energy(gd["dv"]))
    g.g2p()
    out = g.get_state()
    ref = O.g2p(sc, og, og.v + gd["dv"], prob.dt)
    assert rel(out["x"], ref.x) < 1e-12
    g.close()


@pytest.fixture(scope="module")
def later():
    """The benchmark scene twelve steps in (the trajectory bench.py times:
    HOT with the hierarchy refreshed every 5 iterations), stepped by the GPU
    from seed 0; the oracle gets the GPU's particle state."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1911_07913_gb300 import hot
    opts = scenes.SolverOptions(**{**OPTS.__dict__, "refresh_every": 5})
    sc = scenes.two_bars_scene(seed=0)
    stream = torch.cuda.Stream()
    g = hot.HotScene(sc, opts, stream=stream.cuda_stream)
    for _ in range(12):
        assert g.step()["status"] == 0
    st = g.get_state()
    sc12 = sc.copy()
    sc12.x, sc12.v, sc12.F, sc12.C = st["x"], st["v"], st["F"], st["C"]
    g.p2g()
    og = O.p2g(sc12)
    prob = O.Problem(sc12, og, O.step_dt(sc12, opts))
    yield sc12, g, og, prob, opts
    g.close()


def test_later_state_p2g_energy_gradient(later):
    """Twelve steps into the run: active nodes and Dirichlet flags bit-exact,
    m, v, xi, E and grad E at a random dv as tight as at step 0."""
    sc, g, og, prob, opts = later
    gd = g.grid()
    assert np.array_equal(gd["coords"], og.coords.astype(np.int32))
    assert np.array_equal(gd["fixed"], og.fixed)
    assert rel(gd["m"], og.m) < 1e-12 and rel(gd["v"], og.v) < 1e-12 and rel(gd["xi"], og.xi) < 1e-12
    rng = np.random.default_rng(15)
    dv = 0.01 * rng.normal(size=(prob.n, 3))
    dv[og.fixed] = 0.0
    assert abs(g.energy(dv) - prob.energy(dv)) <= 1e-12 * abs(prob.energy(dv))
    assert rel(g.gradient(dv), prob.gradient(dv)) < 1e-11


def test_later_state_vcycle_and_step(later):
    """At the same state: one V-cycle against the oracle's V-cycle on the
    GPU's hierarchy, then a solve whose result the oracle's CN test accepts."""
    sc, g, og, prob, opts = later
    g.build_hierarchy()
    mats = [g.hessian(m) for m in range(opts.levels)]
    levels = []
    for m, h in enumerate(mats):
        coords = h["coords"].astype(np.int64)
        Hm = gpu_level_matrix(h)
        R = O.restriction(coords, mats[m + 1]["coords"].astype(np.int64)) if m + 1 < len(mats) else None
        pat = sp.csr_matrix((np.ones(h["cols"].size), h["cols"], h["row_ptr"]), shape=(coords.shape[0],) * 2)
        levels.append(O.Level(coords=coords, H=Hm, pattern=pat, R=R, colors=O.node_colors(coords),
                              Dblk=O.diag_blocks(Hm, coords.shape[0])))
    b = np.random.default_rng(16).normal(size=(prob.n, 3))
    u, its = g.vcycle(b)
    vc = O.VCycle(levels, og.fixed, opts.eps, opts.max_coarse_cg)
    vc.forced = [its]
    assert rel(u, vc(b)) < 1e-9
    st = g.solve()
    assert st["status"] == 0
    gd = g.grid()
    nrm, nfree = prob.cn_norm(prob.gradient(gd["dv"]))
    assert nrm <= opts.eps * np.sqrt(nfree) * (1 + 1e-6)
    assert prob.energy(gd["dv"]) < prob.energy(np.zeros_like(gd["dv"]))
