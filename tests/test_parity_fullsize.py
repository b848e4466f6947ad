"""Parity at the benchmark's full size: the 4-line survey swath (20.48M
soundings, 20,000 x 3,692 nodes at 0.5 m), IDW k=16 and kriging k=32, in the
launch configuration bench.py times. The GPU grids every node; the oracle
recomputes about 290,000 of them one by one (200,000 anywhere, every node of
the grid's border, nodes along the edges of each survey line's coverage and
in the gaps between lines), with its 2-d tree k-NN over all 20.48M soundings.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_idw, assert_okrige

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def swath_run():
    import torch

    import paper_2505_22675_gb300 as bg
    w = synth.swath()
    g = w.grid
    dev = torch.device("cuda:0")
    ctx = bg.ctx_create(0)
    grid = bg.grid_create(ctx, g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
    x, y, z = (torch.from_numpy(a).to(dev) for a in (w.x_cm, w.y_cm, w.z_m))
    s = bg.soundings_upload(ctx, x, y, z)
    rng = np.random.default_rng(11)
    # survey geometry of the generator: line l covers y in [500 l, 500 l + 346.4] m
    spacing_m, width_m = w.params["line_spacing_m"], 2 * 100.0 * math.tan(math.radians(60.0))
    rows_per_m = 100.0 / g.cell_cm
    edge_rows = [int(round((spacing_m * l + e) * rows_per_m)) + dj
                 for l in range(w.params["lines"]) for e in (0.0, width_m) for dj in (-2, 0, 2)]
    edge_rows = [j for j in edge_rows if 0 <= j < g.ny]
    gap_lo, gap_hi = int((width_m + 2) * rows_per_m), int((spacing_m - 2) * rows_per_m)
    sel = np.unique(np.concatenate([
        rng.choice(g.m, 200_000, replace=False),                     # anywhere
        np.arange(g.nx),                                              # first row (grid border)
        (g.ny - 1) * g.nx + np.arange(g.nx),                          # last row
        np.arange(g.ny) * g.nx, np.arange(g.ny) * g.nx + g.nx - 1,    # first and last columns
        (rng.integers(0, g.nx, (len(edge_rows), 1500))
         + g.nx * np.array(edge_rows)[:, None]).ravel(),              # along the coverage edges
        rng.integers(0, g.nx, 20_000) + g.nx * rng.integers(gap_lo, gap_hi, 20_000),  # gaps
    ]).astype(np.int64))
    assert sel.size >= 250_000
    sel_t = torch.from_numpy(sel).to(dev)
    out = {}
    d = torch.empty(g.m, device=dev)
    nb = torch.empty(g.m * 16, dtype=torch.int32, device=dev)
    bg.interp_idw(s, grid, 16, 2.0, d, nb)
    out["idw"] = (d[sel_t].cpu().numpy(), nb.view(g.m, 16)[sel_t].cpu().numpy(),
                  int(torch.isnan(d).sum()))
    del d, nb
    d = torch.empty(g.m, device=dev)
    v = torch.empty(g.m, device=dev)
    nb = torch.empty(g.m * 32, dtype=torch.int32, device=dev)
    bg.interp_okrige(s, grid, 32, bg.variogram(0, 0.25, 100.0, 50.0), d, v, nb)
    out["ok"] = (d[sel_t].cpu().numpy(), v[sel_t].cpu().numpy(),
                 nb.view(g.m, 32)[sel_t].cpu().numpy(), int(torch.isnan(d).sum()),
                 float(v.min()))
    del nb
    # without nbr_out the grid runs in row chunks of about 1 GiB of ids (nine
    # here) instead of one pass over all ids; every node must come out
    # bitwise the same
    d2 = torch.empty(g.m, device=dev)
    v2 = torch.empty(g.m, device=dev)
    bg.interp_okrige(s, grid, 32, bg.variogram(0, 0.25, 100.0, 50.0), d2, v2)
    torch.cuda.synchronize()
    out["ok_same_without_nbr"] = bool(torch.equal(d.view(torch.int32), d2.view(torch.int32))
                                      and torch.equal(v.view(torch.int32), v2.view(torch.int32)))
    # the fused pass (one k-NN for both methods) gives bitwise the same grids
    fi, fd, fv = (torch.empty(g.m, device=dev) for _ in range(3))
    bg.interp_idw_okrige(s, grid, 16, 2.0, 32, bg.variogram(0, 0.25, 100.0, 50.0), fi, fd, fv)
    di = torch.empty(g.m, device=dev)
    bg.interp_idw(s, grid, 16, 2.0, di)
    torch.cuda.synchronize()
    out["fused_same"] = bool(torch.equal(fi.view(torch.int32), di.view(torch.int32))
                             and torch.equal(fd.view(torch.int32), d.view(torch.int32))
                             and torch.equal(fv.view(torch.int32), v.view(torch.int32)))
    # the same pass delivering the grids to pinned host memory chunk by chunk
    # (copies overlapped with the later chunks) gives bitwise the device grids
    hi, hd, hv = (torch.full((g.m,), -7.0, pin_memory=True) for _ in range(3))
    gi, gd, gv = (torch.empty(g.m, device=dev) for _ in range(3))
    bg.interp_idw_okrige_host(s, grid, 16, 2.0, 32, bg.variogram(0, 0.25, 100.0, 50.0),
                              gi, gd, gv, hi, hd, hv)
    torch.cuda.current_stream().synchronize()
    out["host_same"] = bool(all(torch.equal(h.view(torch.int32), a.cpu().view(torch.int32))
                                for h, a in ((hi, fi), (hd, fd), (hv, fv))))
    del d, v, d2, v2, fi, fd, fv, di, gi, gd, gv, hi, hd, hv
    torch.cuda.synchronize()
    bg.soundings_destroy(s)
    bg.grid_destroy(grid)
    bg.ctx_destroy(ctx)
    qx = (g.x0_cm + (sel % g.nx) * g.cell_cm + g.cell_cm // 2).astype(np.int32)
    qy = (g.y0_cm + (sel // g.nx) * g.cell_cm + g.cell_cm // 2).astype(np.int32)
    out["tree"] = oracle.Tree(w.x_cm, w.y_cm, w.z_m)
    return w, qx, qy, out


def test_swath_idw_k16(swath_run):
    w, qx, qy, out = swath_run
    d, nb, n_nan = out["idw"]
    assert n_nan == 0
    ref, ridx = oracle.idw(w.x_cm, w.y_cm, w.z_m, qx, qy, 16, 2.0, want_idx=True, tree=out["tree"])
    assert np.array_equal(nb, ridx)
    assert_idw(d, ref)


def test_swath_okrige_k32(swath_run):
    w, qx, qy, out = swath_run
    d, v, nb, n_nan, vmin = out["ok"]
    assert n_nan == 0 and vmin >= -1e-3
    rd, rv, ridx = oracle.okrige(w.x_cm, w.y_cm, w.z_m, qx, qy, 32, 0, 0.25, 100.0, 50.0,
                                 want_idx=True, tree=out["tree"])
    assert np.array_equal(nb, ridx)
    assert_okrige(d, v, rd, rv, 0.25)


def test_swath_okrige_row_chunks_match_one_pass(swath_run):
    assert swath_run[3]["ok_same_without_nbr"]


def test_swath_fused_pass_matches_separate_calls(swath_run):
    assert swath_run[3]["fused_same"]


def test_swath_grids_delivered_to_host_match_device(swath_run):
    assert swath_run[3]["host_same"]
