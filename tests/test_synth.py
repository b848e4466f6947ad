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
