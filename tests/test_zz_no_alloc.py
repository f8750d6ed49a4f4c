"""The allocation-free energy entry point (mpm_particle_energy_noalloc).

It serves callers that cannot allocate device memory when they need the
value -- loops that must avoid the implicit synchronisation of
cudaMalloc/cudaFree, hosts whose device memory is a fixed budget, code that
may not enter an allocator.  Checked through the C ABI against the
scene-based mpm_eval_energy on the same particles, twice in a row (the two
calls share the library's fixed scratch array), plus its edge cases: no
particles, no material ids, an id outside the table."""
import numpy as np
import pytest

from paper_1911_07913_gb300 import scenes

pytestmark = pytest.mark.gpu


def _scene(model):
    sc = scenes.tiny_scene(seed=11, res=32, cells=(6, 5, 4), lo=(12, 12, 12), ppc_axis=2,
                           model=model, E=3e5, F_jitter=0.15)
    sc.v[:] = 0.0     # zero grid velocity: F(dv = 0) is the particles' own F
    sc.C[:] = 0.0
    sc.bcs = []
    return sc


@pytest.mark.parametrize("model", [0, 1])
def test_noalloc_energy_matches_scene_energy_twice(model):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1911_07913_gb300 import hot
    sc = _scene(model)
    g = hot.HotScene(sc, scenes.SolverOptions(dt=1e-3))
    g.p2g()
    n_nodes = g.grid()["coords"].shape[0]
    e_ref = g.energy(np.zeros((n_nodes, 3)))
    g.close()
    dev = torch.device("cuda:0")
    F = torch.tensor(sc.F.reshape(-1, 9), dtype=torch.float64, device=dev)
    vol = torch.tensor(sc.vol, dtype=torch.float64, device=dev)
    mat = torch.tensor(sc.mat, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    for _ in range(2):
        e_host = hot.particle_energy_noalloc(F.data_ptr(), vol.data_ptr(), mat.data_ptr(), sc.materials, sc.n)
        assert abs(e_host - e_ref) <= 1e-12 * abs(e_ref)
        hot.particle_energy_noalloc(F.data_ptr(), vol.data_ptr(), mat.data_ptr(), sc.materials, sc.n,
                                    out_dev=out.data_ptr())
        torch.cuda.synchronize()
        assert abs(out.item() - e_ref) <= 1e-12 * abs(e_ref)


def test_noalloc_rejects_oversized_input():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1911_07913_gb300 import hot
    mats = [scenes.Material(1e5, 0.3, 1000.0)]
    with pytest.raises(hot.HotError) as e:
        hot.particle_energy_noalloc(0, 0, 0, mats, 134_217_729)
    assert e.value.code == 1 and "limit" in str(e.value)


def test_noalloc_edge_cases():
    """n = 0 gives 0 (only the total kernel runs, over zero partials); NULL
    material ids mean material 0; an id outside the table makes the sum NaN."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1911_07913_gb300 import hot
    sc = _scene(0)
    dev = torch.device("cuda:0")
    F = torch.tensor(sc.F.reshape(-1, 9), dtype=torch.float64, device=dev)
    vol = torch.tensor(sc.vol, dtype=torch.float64, device=dev)
    mat = torch.zeros(sc.n, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    assert hot.particle_energy_noalloc(F.data_ptr(), vol.data_ptr(), mat.data_ptr(), sc.materials, 0) == 0.0
    with_ids = hot.particle_energy_noalloc(F.data_ptr(), vol.data_ptr(), mat.data_ptr(), sc.materials, sc.n)
    no_ids = hot.particle_energy_noalloc(F.data_ptr(), vol.data_ptr(), 0, sc.materials, sc.n)
    assert no_ids == with_ids and with_ids > 0.0
    mat[sc.n // 2] = 5            # one material in the table
    torch.cuda.synchronize()
    assert np.isnan(hot.particle_energy_noalloc(F.data_ptr(), vol.data_ptr(), mat.data_ptr(), sc.materials, sc.n))
