"""CPU checks of the seeded input recipes (paper_1911_07913_gb300/scenes.py)
against the configurations they stand in for: grid spacing, body sizes,
particles per cell and their placement in sub-cells, materials, held regions,
per-scene distributions of the batch and the served set, and seeded
reproducibility."""
import numpy as np
import pytest

from paper_1911_07913_gb300 import scenes


def _cells(sc):
    return np.floor((sc.x - sc.origin) / sc.dx).astype(np.int64)


def _one_particle_per_subcell(sc, sel):
    sub = np.floor((sc.x[sel] - sc.origin) / (0.5 * sc.dx)).astype(np.int64)
    return len(np.unique(sub, axis=0)) == len(sub)


def _check_bars(sc, res, width, length, gap):
    assert sc.dx == 1.0 / res and tuple(sc.grid_dims) == (res, res, res)
    cells = _cells(sc)
    for b in (0, 1):
        cb = cells[sc.mat == b]
        assert len(cb) == width * width * length * 8
        assert tuple(cb.max(0) - cb.min(0) + 1) == (width, width, length)
        _, counts = np.unique(cb, axis=0, return_counts=True)
        assert counts.min() == 8 and counts.max() == 8          # 8 particles in every cell
        assert _one_particle_per_subcell(sc, sc.mat == b)       # one in each 2x2x2 sub-cell
    assert cells[sc.mat == 1][:, 0].min() - cells[sc.mat == 0][:, 0].max() - 1 == gap
    m = sc.materials
    assert (m[0].E, m[1].E) == (1e5, 1e9)
    assert all(mm.nu == 0.4 and mm.rho == 2000.0 and mm.model == scenes.MODEL_NH for mm in m)
    assert np.allclose(sc.vol, sc.dx ** 3 / 8) and np.allclose(sc.mass, 2000.0 * sc.dx ** 3 / 8)
    assert np.all(sc.F == np.eye(3)) and np.all(sc.C == 0.0) and np.all(sc.v == 0.0)
    # two rotating holds per bar about z, +1 rad/s at the low end and -1 at the high end; each a
    # cylinder 2 cells wider than the bar's half diagonal, short of the other bar's stencil nodes
    assert len(sc.bcs) == 4
    reach = gap + 0.5 * width - 1.0
    for k, bc in enumerate(sc.bcs):
        assert bc.type == scenes.BC_ROTATE and tuple(bc.axis) == (0.0, 0.0, 1.0)
        assert bc.omega == (1.0 if k % 2 == 0 else -1.0)
        r = bc.radius / sc.dx
        assert r == pytest.approx(min(np.sqrt(0.5) * width + 2.0, reach - 0.5))
        assert np.sqrt(0.5) * width < r < reach
        # the held slab covers the 4 end cell layers of its bar
        b = k // 2
        cz = cells[sc.mat == b][:, 2]
        if k % 2 == 0:
            assert bc.hi[2] / sc.dx == pytest.approx(cz.min() + 4.5)
        else:
            assert bc.lo[2] / sc.dx == pytest.approx(cz.max() + 1 - 4.5)


def test_two_bars_600k_recipe():
    sc = scenes.two_bars_scene()
    assert sc.n == 601_600
    _check_bars(sc, 256, 20, 94, 14)


def test_two_bars_2m_recipe():
    sc = scenes.two_bars_2m_scene()
    assert sc.n == 2_030_400
    _check_bars(sc, 384, 30, 141, 18)


def test_cube_8k_recipe():
    sc = scenes.cube_scene()
    assert sc.n == 8000 and sc.dx == 1.0 / 32
    cells = _cells(sc)
    assert tuple(cells.min(0)) == (11, 4, 11) and tuple(cells.max(0)) == (20, 13, 20)
    assert _one_particle_per_subcell(sc, slice(None))
    m = sc.materials[0]
    assert (m.E, m.nu, m.rho, m.model) == (1e5, 0.3, 1000.0, scenes.MODEL_FCR)
    assert np.all(np.abs(sc.v) <= 0.5) and np.abs(sc.v).max() > 0.45
    assert tuple(sc.gravity) == (0.0, -9.8, 0.0)


def test_three_material_bar_recipe():
    sc = scenes.three_material_bar_scene(E_mid=1e9)
    assert sc.n == 10 * 10 * 48 * 8
    z = _cells(sc)[:, 2]
    z0 = z.min()
    mid = (z - z0 >= 16) & (z - z0 < 32)
    assert np.all(sc.mat[mid] == 1) and np.all(sc.mat[~mid] == 0)
    assert (sc.materials[0].E, sc.materials[1].E) == (1e5, 1e9)
    assert all(m.model == scenes.MODEL_FCR for m in sc.materials)


def test_scenes_are_seeded():
    a, b, c = scenes.cube_scene(seed=3), scenes.cube_scene(seed=3), scenes.cube_scene(seed=4)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.v, b.v)
    assert not np.array_equal(a.x, c.x)


def test_batch_recipe():
    """64 boxes: particle counts log-uniform in [5k, 200k] (8 per cell), grids
    64^3 / 96^3 / 128^3, FCR with E log-uniform in [1e4, 1e8], every second
    scene von Mises with yield 1e4 Pa, bodies clear of the grid walls."""
    scs = scenes.batch_scenes(seed=0, count=64)
    assert len(scs) == 64
    n = np.array([s.n for s in scs])
    assert n.min() >= 4000 and n.max() <= 240_000
    ln = np.log(n)
    # log-uniform: the mean of log n sits near the middle of [log 5k, log 200k]
    assert abs(ln.mean() - 0.5 * (np.log(5000) + np.log(200_000))) < 0.5
    for k, s in enumerate(scs):
        res = int(s.grid_dims[0])
        assert res in (64, 96, 128) and s.dx == 1.0 / res
        cells = _cells(s)
        assert cells.min() >= 4 and cells.max() < res - 4
        _, counts = np.unique(cells, axis=0, return_counts=True)
        assert counts.min() == 8 and counts.max() == 8
        m = s.materials[0]
        assert 1e4 <= m.E <= 1e8 and m.model == scenes.MODEL_FCR and m.nu == 0.3
        assert (m.plasticity, m.yield_stress) == ((1, 1e4) if k % 2 else (0, 0.0))


def test_serving_recipe():
    """Served scenes: particle counts lognormal around a 50k median (sigma 1,
    at most 1M), E log-uniform in [1e4, 1e9], FCR or Neo-Hookean, every third
    scene von Mises (a subset of the 256, generated the same way)."""
    scs = scenes.serving_scenes(seed=0, count=24)
    n = np.array([s.n for s in scs])
    assert n.max() <= 1_000_000 * 1.1
    assert 15_000 < np.median(n) < 160_000
    models = set()
    for k, s in enumerate(scs):
        m = s.materials[0]
        assert 1e4 <= m.E <= 1e9
        models.add(m.model)
        assert m.plasticity == (1 if k % 3 == 0 else 0)
    assert models == {scenes.MODEL_FCR, scenes.MODEL_NH}
