"""Batched gridding (bg_batch_*): uneven tiles in one graph of persistent kernels.

Every tile's grids must equal the per-grid calls bit for bit, on the first
(captured) run and on replays, across cell targets, and against the oracle.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_idw, assert_okrige

pytestmark = pytest.mark.gpu

VGM = (0, 0.25, 100.0, 50.0)


# k per tile, cycled by tile index: every batched system size (K = 4, 8, 16,
# 32 for kriging; the IDW k-NN at K = 4, 8, 16) and k below its K
IDW_KS = (16, 4, 8, 12)
OK_KS = (32, 4, 8, 16, 5, 24)


def _mk(bg, torch, tiles_np, cycle_k=False):
    dev = torch.device("cuda:0")
    tiles = []
    for i, (w, m) in enumerate(tiles_np):
        g = w.grid
        t = dict(x_cm=torch.from_numpy(w.x_cm).to(dev), y_cm=torch.from_numpy(w.y_cm).to(dev),
                 z_m=torch.from_numpy(w.z_m).to(dev),
                 grid_spec=(g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny), method=m,
                 k=(IDW_KS[i % len(IDW_KS)] if m == 0 else OK_KS[i % len(OK_KS)]) if cycle_k
                 else (16 if m == 0 else 32), power=2.0, vgm=bg.variogram(*VGM),
                 depth_out=torch.full((g.m,), -1.0, device=dev),
                 var_out=torch.full((g.m,), -1.0, device=dev) if m == 1 else None)
        tiles.append(t)
    return tiles


def _direct(bg, torch, ctx, t):
    nx, ny = t["grid_spec"][3], t["grid_spec"][4]
    grid = bg.grid_create(ctx, *t["grid_spec"])
    s = bg.soundings_upload(ctx, t["x_cm"], t["y_cm"], t["z_m"])
    d = torch.empty(nx * ny, device=t["x_cm"].device)
    v = torch.empty(nx * ny, device=t["x_cm"].device)
    if t["method"] == 0:
        bg.interp_idw(s, grid, t["k"], 2.0, d)
    else:
        bg.interp_okrige(s, grid, t["k"], t["vgm"], d, v)
    torch.cuda.synchronize()
    bg.soundings_destroy(s)
    bg.grid_destroy(grid)
    return d.cpu().numpy(), v.cpu().numpy()


def _same(a, b):
    return np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_batch_equals_per_grid_calls_and_replays():
    import torch

    import paper_2505_22675_gb300 as bg
    tiles_np = synth.batched_tiles(seed=3, count=24, scale=0.05)
    ctx = bg.ctx_create(0)
    try:
        tiles = _mk(bg, torch, tiles_np, cycle_k=True)
        used = {(t["method"], t["k"]) for t in tiles}
        assert {(1, 4), (1, 8), (1, 16), (1, 32), (0, 4), (0, 8), (0, 16)} <= used
        ref = [_direct(bg, torch, ctx, t) for t in tiles]
        b = bg.batch_create(ctx, tiles)
        for run in range(3):  # capture, then replays
            for t in tiles:
                t["depth_out"].fill_(-1.0)
                if t["var_out"] is not None:
                    t["var_out"].fill_(-1.0)
            bg.batch_run(b)
            torch.cuda.synchronize()
            for t, (rd, rv) in zip(tiles, ref):
                assert _same(t["depth_out"].cpu().numpy(), rd), run
                if t["method"] == 1:
                    assert _same(t["var_out"].cpu().numpy(), rv), run
        assert bg.batch_status(b) == 0
        # a different cell target records a new graph; results do not change
        bg.batch_set_cell_target(b, 5.0)
        bg.batch_run(b)
        torch.cuda.synchronize()
        for t, (rd, rv) in zip(tiles, ref):
            assert _same(t["depth_out"].cpu().numpy(), rd)
        # every launch shape (k-NN strip, solve item size) gives the same grids
        for strip in (1, 2, 4):
            for item in (1, 4, 16):
                bg.batch_set_shape(b, strip, item)
                for t in tiles:
                    t["depth_out"].fill_(-1.0)
                    if t["var_out"] is not None:
                        t["var_out"].fill_(-1.0)
                bg.batch_run(b)
                torch.cuda.synchronize()
                for t, (rd, rv) in zip(tiles, ref):
                    assert _same(t["depth_out"].cpu().numpy(), rd), (strip, item)
                    if t["method"] == 1:
                        assert _same(t["var_out"].cpu().numpy(), rv), (strip, item)
        with pytest.raises(bg.BGError):
            bg.batch_set_shape(b, 3, 8)
        best = bg.batch_tune(b)
        cfg = bg.batch_config(b)
        assert best in (1.0, 2.0, 3.0, 5.0) and cfg["soundings_per_cell"] == best
        assert cfg["knn_strip"] in (1, 2, 4) and cfg["solve_item"] in (2, 4, 8, 16)
        bg.batch_run(b)
        torch.cuda.synchronize()
        for t, (rd, rv) in zip(tiles, ref):
            assert _same(t["depth_out"].cpu().numpy(), rd)
        bg.batch_destroy(b)
    finally:
        bg.ctx_destroy(ctx)


def test_batch_matches_oracle_and_handles_empty_tiles():
    import torch

    import paper_2505_22675_gb300 as bg
    tiles_np = synth.batched_tiles(seed=8, count=8, scale=0.01)
    empty = synth.tile(seed=1, n=50, side_cm=3000, cell_cm=200)
    empty.z_m[:] = np.nan
    tiles_np.append((empty, 1))
    none = synth.tile(seed=2, n=0, side_cm=3000, cell_cm=200)
    tiles_np.append((none, 0))
    ctx = bg.ctx_create(0)
    try:
        tiles = _mk(bg, torch, tiles_np)
        b = bg.batch_create(ctx, tiles)
        bg.batch_run(b)
        torch.cuda.synchronize()
        for t, (w, m) in zip(tiles, tiles_np):
            g = w.grid
            qx, qy = oracle.grid_nodes(g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
            d = t["depth_out"].cpu().numpy()
            if m == 0:
                assert_idw(d, oracle.idw(w.x_cm, w.y_cm, w.z_m, qx, qy, 16, 2.0))
            else:
                rd, rv = oracle.okrige(w.x_cm, w.y_cm, w.z_m, qx, qy, 32, *VGM)
                assert_okrige(d, t["var_out"].cpu().numpy(), rd, rv, VGM[1])
        bg.batch_destroy(b)
    finally:
        bg.ctx_destroy(ctx)
