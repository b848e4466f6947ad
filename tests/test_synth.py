"""The seeded generators are deterministic and shaped like the workloads they stand for."""
import numpy as np

import synth


def test_tile_deterministic_and_in_range():
    a = synth.tile(1)
    b = synth.tile(1)
    assert np.array_equal(a.x_cm, b.x_cm) and np.array_equal(a.z_m, b.z_m)
    assert a.x_cm.dtype == np.int32 and a.z_m.dtype == np.float32
    assert a.x_cm.size == 20_000 and a.x_cm.min() >= 0 and a.x_cm.max() < 51_200
    assert a.grid == synth.GridSpec(0, 0, 200, 256, 256)
    assert 3300 < float(a.z_m.min()) and float(a.z_m.max()) < 3700
    assert not np.array_equal(synth.tile(2).x_cm, a.x_cm)


def test_swath_shape_small():
    w = synth.swath(seed=2, lines=2, pings=50, beams=32)
    assert w.x_cm.size == 2 * 50 * 32
    # across-track half width of a +-60 deg fan at 100 m altitude
    assert abs(w.params["line_spacing_m"] - 500.0) < 1e-9
    y_m = w.y_cm / 100.0
    assert y_m.min() > -1.01 and y_m.max() < 2 * 173.21 + 500 + 1.01
    assert w.grid.nx == 50 and w.grid.cell_cm == 50


def test_full_swath_geometry_constants():
    # 4 lines x 20,000 pings x 256 beams = 20.48M soundings; grid 20,000 x 3,692 at 0.5 m
    import math
    half = 100 * math.tan(math.radians(60))
    width = 2 * half + 3 * 500
    assert int(math.floor(width * 100 / 50)) == 3692


def test_batched_tiles_mix():
    tiles = synth.batched_tiles(seed=3, count=6, scale=0.01)
    assert len(tiles) == 6 and all(m in (0, 1) for _, m in tiles)


def test_hole_grid_partitions_the_nodes():
    h = synth.hole_grid(seed=31, nx=50, ny=40, cell_cm=200, frac=0.07)
    h2 = synth.hole_grid(seed=31, nx=50, ny=40, cell_cm=200, frac=0.07)
    assert np.array_equal(h.z_full, h2.z_full) and np.array_equal(h.holes, h2.holes)
    assert h.holes.size == round(0.07 * 2000)
    assert np.all(np.diff(h.holes) > 0)
    kept = h.kept()
    assert kept.size + h.holes.size == 2000 and np.intersect1d(kept, h.holes).size == 0
    s = h.soundings()
    qx, qy = h.queries()
    # node centres of a 2 m lattice: odd metres in cm
    assert np.all((s.x_cm - 100) % 200 == 0) and np.all((qy - 100) % 200 == 0)
    assert np.array_equal(s.z_m, h.z_full[kept]) and np.array_equal(h.truth(), h.z_full[h.holes])
    src = h.source()
    assert np.isnan(src[h.holes]).all() and not np.isnan(src[kept]).any()
    assert 3300 < h.z_full.min() and h.z_full.max() < 3700


def test_row_midpoints_and_random_points():
    g = synth.GridSpec(1000, 2000, 200, 4, 3)
    qx, qy = synth.row_midpoints(g)
    assert qx.size == 4 * 2
    assert set(np.unique(qy)) == {2200, 2400}
    assert set(np.unique(qx)) == {1100, 1300, 1500, 1700}
    rx, ry = synth.random_points(5, g, 1000, margin_cells=1)
    assert rx.min() >= 1100 - 200 and rx.max() <= 1700 + 200
    assert ry.min() >= 2100 - 200 and ry.max() <= 2500 + 200
