"""The allocation-free IDW entry point gives the same grids as the regular one.

bg_interp_idw_noalloc serves callers that cannot call cudaMalloc — code that
runs inside host callbacks or driver-owned threads, runtimes whose allocator
policy forbids device allocation, or processes that reserve all device memory
up front. It keeps its work space in one fixed device array, so a second call
must not see anything left over from the first: two calls in a row, on
different inputs, are each compared with bg_soundings_upload + bg_interp_idw.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import synth
from gpu_util import assert_idw

pytestmark = pytest.mark.gpu


def _regular(bg, torch, w, k, power):
    g = w.grid
    dev = torch.device("cuda:0")
    ctx = bg.ctx_create(0)
    grid = bg.grid_create(ctx, g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
    s = bg.soundings_upload(ctx, *(torch.from_numpy(a).to(dev) for a in (w.x_cm, w.y_cm, w.z_m)))
    d = torch.empty(g.m, device=dev)
    nb = torch.empty(g.m * k, dtype=torch.int32, device=dev)
    bg.interp_idw(s, grid, k, power, d, nb)
    torch.cuda.synchronize()
    out = d.cpu().numpy(), nb.cpu().numpy()
    bg.soundings_destroy(s)
    bg.grid_destroy(grid)
    bg.ctx_destroy(ctx)
    return out


def _noalloc(bg, torch, w, k, power):
    g = w.grid
    dev = torch.device("cuda:0")
    x, y, z = (torch.from_numpy(a).to(dev) for a in (w.x_cm, w.y_cm, w.z_m))
    d = torch.full((g.m,), -1.0, device=dev)
    nb = torch.full((g.m * k,), -7, dtype=torch.int32, device=dev)
    bg.interp_idw_noalloc(x, y, z, (g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny), k, power, d, nb)
    torch.cuda.synchronize()
    return d.cpu().numpy(), nb.cpu().numpy()


def test_noalloc_matches_regular_entry_point_twice_in_a_row():
    import torch

    import paper_2505_22675_gb300 as bg
    first = synth.tile(seed=21, n=20_000)                      # 512 m tile, 256 x 256 nodes
    second = synth.tile(seed=22, n=3_000, side_cm=15_000, cell_cm=300, x0_cm=-40_000)
    second.z_m[::17] = np.nan                                  # some invalid soundings
    for w, k, p in ((first, 16, 2.0), (second, 8, 1.5)):
        ref_d, ref_nb = _regular(bg, torch, w, k, p)
        d, nb = _noalloc(bg, torch, w, k, p)
        assert np.array_equal(nb, ref_nb)
        assert_idw(d, ref_d.astype(np.float64))


def test_noalloc_rejects_too_many_soundings():
    import torch

    import paper_2505_22675_gb300 as bg
    n = 262_145
    dev = torch.device("cuda:0")
    x = torch.zeros(n, dtype=torch.int32, device=dev)
    z = torch.zeros(n, dtype=torch.float32, device=dev)
    d = torch.empty(4, device=dev)
    with pytest.raises(bg.BGError) as e:
        bg.interp_idw_noalloc(x, x, z, (0, 0, 2, 2, 2), 8, 2.0, d)
    assert e.value.status == -1 and "262144" in str(e.value)
