"""Parity on a grid of about a million nodes (1021 x 1019 at 0.5 m over a
random tile of 240,000 soundings): the size at which the grid k-NN kernels
take strips of two nodes per thread (tiles take one, the survey swath four).
IDW k=16 and kriging k=32 with their neighbour ids, against the oracle's 2-d
tree at 20,000 random nodes and every node of the grid's border; the fused
pass and the kriging without id output (ids in the library's scratch
buffer) bitwise against the separate, id-writing calls.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_idw, assert_okrige

pytestmark = pytest.mark.gpu

VGM = (0, 0.25, 100.0, 50.0)


@pytest.fixture(scope="module")
def medium_run():
    import torch

    import paper_2505_22675_gb300 as bg
    w = synth.tile(seed=61, n=240_000, side_cm=51_100, cell_cm=50)
    g = synth.GridSpec(w.grid.x0_cm, w.grid.y0_cm, 50, 1021, 1019)
    assert (1 << 19) <= g.nx * g.ny < (1 << 21)
    dev = torch.device("cuda:0")
    ctx = bg.ctx_create(0)
    grid = bg.grid_create(ctx, g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
    s = bg.soundings_upload(ctx, *(torch.from_numpy(a).to(dev) for a in (w.x_cm, w.y_cm, w.z_m)))
    m = g.nx * g.ny
    rng = np.random.default_rng(13)
    sel = np.unique(np.concatenate([
        rng.choice(m, 20_000, replace=False),
        np.arange(g.nx), (g.ny - 1) * g.nx + np.arange(g.nx),
        np.arange(g.ny) * g.nx, np.arange(g.ny) * g.nx + g.nx - 1,
    ]).astype(np.int64))
    sel_t = torch.from_numpy(sel).to(dev)
    vgm = bg.variogram(*VGM)
    out = {}
    di = torch.empty(m, device=dev)
    nbi = torch.empty(m * 16, dtype=torch.int32, device=dev)
    bg.interp_idw(s, grid, 16, 2.0, di, nbi)
    dk = torch.empty(m, device=dev)
    vk = torch.empty(m, device=dev)
    nbk = torch.empty(m * 32, dtype=torch.int32, device=dev)
    bg.interp_okrige(s, grid, 32, vgm, dk, vk, nbk)
    dk2 = torch.empty(m, device=dev)
    vk2 = torch.empty(m, device=dev)
    bg.interp_okrige(s, grid, 32, vgm, dk2, vk2)
    fused = [torch.empty(m, device=dev) for _ in range(3)]
    bg.interp_idw_okrige(s, grid, 16, 2.0, 32, vgm, *fused)
    torch.cuda.synchronize()
    bits = lambda t: t.cpu().numpy().view(np.uint32)
    out["idw"] = (di[sel_t].cpu().numpy(), nbi.view(m, 16)[sel_t].cpu().numpy())
    out["ok"] = (dk[sel_t].cpu().numpy(), vk[sel_t].cpu().numpy(), nbk.view(m, 32)[sel_t].cpu().numpy())
    out["scratch_same"] = (np.array_equal(bits(dk), bits(dk2)) and np.array_equal(bits(vk), bits(vk2)))
    out["fused_same"] = (np.array_equal(bits(di), bits(fused[0]))
                         and np.array_equal(bits(dk), bits(fused[1]))
                         and np.array_equal(bits(vk), bits(fused[2])))
    bg.soundings_destroy(s)
    bg.grid_destroy(grid)
    bg.ctx_destroy(ctx)
    qx = (g.x0_cm + (sel % g.nx) * g.cell_cm + g.cell_cm // 2).astype(np.int32)
    qy = (g.y0_cm + (sel // g.nx) * g.cell_cm + g.cell_cm // 2).astype(np.int32)
    out["tree"] = oracle.Tree(w.x_cm, w.y_cm, w.z_m)
    return w, qx, qy, out


def test_medium_grid_idw_k16(medium_run):
    w, qx, qy, out = medium_run
    d, nb = out["idw"]
    ref, ridx = oracle.idw(w.x_cm, w.y_cm, w.z_m, qx, qy, 16, 2.0, want_idx=True, tree=out["tree"])
    assert np.array_equal(nb, ridx)
    assert_idw(d, ref)


def test_medium_grid_okrige_k32(medium_run):
    w, qx, qy, out = medium_run
    d, v, nb = out["ok"]
    rd, rv, ridx = oracle.okrige(w.x_cm, w.y_cm, w.z_m, qx, qy, 32, *VGM, want_idx=True,
                                 tree=out["tree"])
    assert np.array_equal(nb, ridx)
    assert_okrige(d, v, rd, rv, VGM[1])


def test_medium_grid_fused_and_scratch_id_passes_are_bitwise_equal(medium_run):
    out = medium_run[3]
    assert out["scratch_same"]
    assert out["fused_same"]
