"""The allocation-free IDW entry point gives bitwise the grids of the regular one.

bg_interp_idw_noalloc serves callers that cannot call cudaMalloc: processes
that reserve all device memory up front, runtimes whose allocator policy
forbids device allocation on their worker threads, and driver-owned threads
that must not allocate. It keeps its work space in one fixed device array, so
a call must not see anything left over from the one before: calls in a row,
on different inputs, are each compared bit for bit with bg_soundings_upload +
bg_interp_idw (depths and neighbour ids), including a call with no valid
sounding and one at the array's 262,144-sounding limit whose extent forces
the hash to widen its cells to fit the array's cell tables.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_idw

pytestmark = pytest.mark.gpu

MAX_SOUNDINGS = 262_144
MAX_CELLS = 262_144


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


def _bitwise(a, b):
    return np.array_equal(np.asarray(a, np.float32).view(np.uint32),
                          np.asarray(b, np.float32).view(np.uint32))


def _cap_line():
    """262,144 soundings on a 2e9 cm x 100 cm strip. At about four soundings
    per cell the first cell side is ~2 km, which would need over a million
    cells along the strip: more than the array's tables hold, so the hash
    must widen its cells before it fits."""
    grid = synth.GridSpec(-1_000_000_000, -244_091, 488_282, 4096, 2)  # first row on the strip
    w = synth.rect(31, MAX_SOUNDINGS, -1_000_000_000, 0, 2_000_000_000, 100, grid)
    W = int(w.x_cm.max()) - int(w.x_cm.min()) + 1
    H = int(w.y_cm.max()) - int(w.y_cm.min()) + 1
    cs = math.ceil(math.sqrt(4.0 * W * H / MAX_SOUNDINGS))
    assert math.ceil(W / cs) * math.ceil(H / cs) > MAX_CELLS  # the widening loop must run
    return w


def test_noalloc_matches_regular_entry_point_bitwise_on_calls_in_a_row():
    import torch

    import paper_2505_22675_gb300 as bg
    first = synth.tile(seed=21, n=20_000)                      # 512 m tile, 256 x 256 nodes
    second = synth.tile(seed=22, n=3_000, side_cm=15_000, cell_cm=300, x0_cm=-40_000)
    second.z_m[::17] = np.nan                                  # some invalid soundings
    no_valid = synth.tile(seed=23, n=500, side_cm=4_000, cell_cm=200)
    no_valid.z_m[:] = np.nan                                   # every depth invalid
    empty = synth.tile(seed=24, n=0, side_cm=4_000, cell_cm=200)
    cap = _cap_line()
    cases = ((first, 16, 2.0), (second, 8, 1.5), (no_valid, 8, 2.0), (empty, 4, 2.0),
             (cap, 16, 2.0), (first, 32, 3.0))
    for w, k, p in cases:
        ref_d, ref_nb = _regular(bg, torch, w, k, p)
        d, nb = _noalloc(bg, torch, w, k, p)
        assert np.array_equal(nb, ref_nb), (w.name, k)
        assert _bitwise(d, ref_d), (w.name, k)
        if w is no_valid or w is empty:
            assert np.isnan(d).all() and (nb == -1).all()
        if w is cap:
            # the widened hash still finds the exact neighbours (oracle, FP64)
            g = w.grid
            qx, qy = oracle.grid_nodes(g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
            rd, ri = oracle.idw(w.x_cm, w.y_cm, w.z_m, qx, qy, k, p, want_idx=True)
            assert np.array_equal(nb.reshape(-1, k), ri)
            assert_idw(d, rd)


def test_noalloc_rejects_too_many_soundings():
    import torch

    import paper_2505_22675_gb300 as bg
    n = MAX_SOUNDINGS + 1
    dev = torch.device("cuda:0")
    x = torch.zeros(n, dtype=torch.int32, device=dev)
    z = torch.zeros(n, dtype=torch.float32, device=dev)
    d = torch.empty(4, device=dev)
    with pytest.raises(bg.BGError) as e:
        bg.interp_idw_noalloc(x, x, z, (0, 0, 2, 2, 2), 8, 2.0, d)
    assert e.value.status == -1 and "262144" in str(e.value)
