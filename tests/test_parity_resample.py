"""Gridded input (bg_resample_points / bg_resample_grid): bilinear and
Catmull-Rom against the oracle, element by element.

Values within the IDW tolerance (1e-4 m + half an fp32 ulp of the oracle
value), NaN pattern and the how-code (method / bilinear fallback / no value)
bit-exact. Cases: random points over and around a grid with missing nodes
(several blocks and a ragged tail), the nodes themselves, the row midpoints
of the paper's row-filling tests (Sec. IV Grid A) as an output grid, a finer
output grid that overhangs the source, a 2 x 2 source, and empty lists.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_idw

pytestmark = pytest.mark.gpu

METHODS = (0, 1)


def _dev(a, dtype=None):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a if dtype is None else a.astype(dtype))).to("cuda:0")


def _points(bg, src, spec, method, qx, qy):
    import torch
    m = len(qx)
    out = torch.full((m,), -7.0, device="cuda:0")
    how = torch.full((m,), 9, dtype=torch.int8, device="cuda:0")
    bg.resample_points(_dev(src), spec, method, _dev(qx, np.int32), _dev(qy, np.int32), out, how)
    torch.cuda.synchronize()
    return out.cpu().numpy(), how.cpu().numpy()


def _compare(got, ghow, ref, rhow):
    assert np.array_equal(ghow, rhow), f"{(ghow != rhow).sum()} how-codes differ"
    assert_idw(got, ref)


@pytest.mark.parametrize("method", METHODS)
def test_points_over_a_grid_with_holes(method):
    import paper_2505_22675_gb300 as bg
    h = synth.hole_grid(seed=41, nx=150, ny=110, cell_cm=200, frac=0.05)
    src = h.source()
    g = h.grid
    spec = (g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
    rx, ry = synth.random_points(42, g, 20_001, margin_cells=2)  # ragged tail
    nx_, ny_ = oracle.grid_nodes(*spec)
    qx = np.concatenate([rx, nx_])
    qy = np.concatenate([ry, ny_])
    got, how = _points(bg, src, spec, method, qx, qy)
    ref, rhow = oracle.resample(src, spec, qx, qy, method)
    _compare(got, how, ref, rhow)
    if method == 1:
        assert (rhow == 1).any() and (rhow == 0).any() and (rhow == 2).any()


@pytest.mark.parametrize("method", METHODS)
def test_row_midpoints_and_finer_overhanging_grid(method):
    import torch

    import paper_2505_22675_gb300 as bg
    h = synth.hole_grid(seed=43, nx=333, ny=97, cell_cm=400, frac=0.02, x0_cm=-20_000, y0_cm=50_000)
    src = h.source()
    g = h.grid
    spec = (g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
    # row midpoints: the source lattice shifted by half a cell in y, one row fewer
    mid = (g.x0_cm, g.y0_cm + g.cell_cm // 2, g.cell_cm, g.nx, g.ny - 1)
    # a grid at a quarter of the spacing that overhangs the source by a few cells
    fine = (g.x0_cm - 3 * g.cell_cm, g.y0_cm - 2 * g.cell_cm, g.cell_cm // 4, 4 * g.nx + 20,
            4 * g.ny + 13)
    for out_spec in (mid, fine):
        m = out_spec[3] * out_spec[4]
        out = torch.full((m,), -7.0, device="cuda:0")
        how = torch.full((m,), 9, dtype=torch.int8, device="cuda:0")
        bg.resample_grid(_dev(src), spec, method, out_spec, out, how)
        torch.cuda.synchronize()
        qx, qy = oracle.grid_nodes(*out_spec)
        ref, rhow = oracle.resample(src, spec, qx, qy, method)
        _compare(out.cpu().numpy(), how.cpu().numpy(), ref, rhow)
    mx, my = synth.row_midpoints(g)
    got, ghow = _points(bg, src, spec, method, mx, my)
    ref, rhow = oracle.resample(src, spec, mx, my, method)
    _compare(got, ghow, ref, rhow)


def test_two_by_two_source_and_empty_lists():
    import torch

    import paper_2505_22675_gb300 as bg
    src = np.array([3500.0, 3510.0, 3520.0, np.nan], dtype=np.float32)
    spec = (0, 0, 200, 2, 2)
    qx = np.array([100, 300, 150, 200, 100, 299, 301, 99])
    qy = np.array([100, 100, 100, 300, 300, 299, 100, 100])
    for method in METHODS:
        got, how = _points(bg, src, spec, method, qx, qy)
        ref, rhow = oracle.resample(src, spec, qx, qy, method)
        _compare(got, how, ref, rhow)
        out = torch.empty(0, device="cuda:0")
        bg.resample_points(_dev(src), spec, method, _dev(np.zeros(0, np.int32)),
                           _dev(np.zeros(0, np.int32)), out)
    with pytest.raises(bg.BGError):
        bg.resample_points(_dev(src), (0, 0, 201, 2, 2), 0, _dev(qx, np.int32), _dev(qy, np.int32),
                           torch.empty(qx.size, device="cuda:0"))


@pytest.mark.parametrize("method", METHODS)
def test_output_grids_of_every_shape(method):
    """Output grids off the source lattice at the same cell, at half and at
    three times the cell (stencils that skip source columns), one wholly
    outside the hull, and a 2 x 2 source gridded at a quarter cell."""
    import torch

    import paper_2505_22675_gb300 as bg
    h = synth.hole_grid(seed=47, nx=301, ny=75, cell_cm=400, frac=0.03, x0_cm=10_000, y0_cm=-8_000)
    src = h.source()
    g = h.grid
    spec = (g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
    cases = [
        (src, spec, (g.x0_cm + 150, g.y0_cm + 66, g.cell_cm, g.nx - 1, g.ny - 1)),
        (src, spec, (g.x0_cm - 1_000, g.y0_cm + 250, g.cell_cm // 2, 2 * g.nx + 9, 2 * g.ny + 3)),
        (src, spec, (g.x0_cm + 37 * 2, g.y0_cm - 100, 3 * g.cell_cm + 2, g.nx // 3 + 2, g.ny // 3 + 2)),
        (src, spec, (g.x0_cm + 10_000_000, g.y0_cm, g.cell_cm, 50, 40)),
        (np.array([3500.0, 3510.0, 3520.0, np.nan], np.float32), (0, 0, 200, 2, 2),
         (-100, -50, 50, 13, 11)),
    ]
    for s_arr, s_spec, out_spec in cases:
        m = out_spec[3] * out_spec[4]
        out = torch.full((m,), -7.0, device="cuda:0")
        how = torch.full((m,), 9, dtype=torch.int8, device="cuda:0")
        bg.resample_grid(_dev(s_arr), s_spec, method, out_spec, out, how)
        torch.cuda.synchronize()
        qx, qy = oracle.grid_nodes(*out_spec)
        ref, rhow = oracle.resample(s_arr, s_spec, qx, qy, method)
        _compare(out.cpu().numpy(), how.cpu().numpy(), ref, rhow)


@pytest.mark.parametrize("method", METHODS)
def test_row_filling_in_vectors(method):
    """Output grids at the source's own spacing on its node columns, rows a
    multiple of 4 long: the 16-byte vector path. Row midpoints, a grid shifted
    by 8 columns that overhangs both ends (whole vectors outside the hull) and
    rows above and below, the last source column (remainder = cell), and the
    same without how-codes (values bitwise equal)."""
    import torch

    import paper_2505_22675_gb300 as bg
    h = synth.hole_grid(seed=53, nx=256, ny=61, cell_cm=400, frac=0.04, x0_cm=-3_000, y0_cm=7_000)
    src = h.source()
    g = h.grid
    c = g.cell_cm
    spec = (g.x0_cm, g.y0_cm, c, g.nx, g.ny)
    cases = [
        (g.x0_cm, g.y0_cm + c // 2, c, g.nx, g.ny - 1),
        (g.x0_cm - 8 * c, g.y0_cm - 3 * c // 2, c, g.nx + 16, g.ny + 5),
        (g.x0_cm + 4 * c, g.y0_cm + 130, c, 2048 + 8, 9),
    ]
    dsrc = _dev(src)
    for out_spec in cases:
        m = out_spec[3] * out_spec[4]
        out = torch.full((m,), -7.0, device="cuda:0")
        how = torch.full((m,), 9, dtype=torch.int8, device="cuda:0")
        bg.resample_grid(dsrc, spec, method, out_spec, out, how)
        out2 = torch.full((m,), -7.0, device="cuda:0")
        bg.resample_grid(dsrc, spec, method, out_spec, out2)
        torch.cuda.synchronize()
        qx, qy = oracle.grid_nodes(*out_spec)
        ref, rhow = oracle.resample(src, spec, qx, qy, method)
        _compare(out.cpu().numpy(), how.cpu().numpy(), ref, rhow)
        a, b = out.cpu().numpy(), out2.cpu().numpy()
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
        assert (rhow == 2).any() and (rhow != 2).any()
