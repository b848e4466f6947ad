"""bg_interp_idw_okrige: IDW and kriging of one grid from a single k-NN pass.

Every output must be bitwise what bg_interp_idw and bg_interp_okrige give when
called one after the other (the fused IDW repeats idw_from's operations in the
same order over the first k_idw of the kriging's sorted neighbours), and so
also within the oracle's tolerances. Cases: several (k_idw, k_okrige) pairs,
powers 1, 2 and 3, both variogram models, duplicated positions, NaN depths,
fewer soundings than k, and no valid sounding at all.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_idw, assert_okrige

pytestmark = pytest.mark.gpu

SPH = (0, 0.25, 100.0, 50.0)
EXP = (1, 0.0, 100.0, 50.0)


def _run(w, k_idw, power, k_ok, vgm):
    import torch

    import paper_2505_22675_gb300 as bg
    g = w.grid
    dev = torch.device("cuda:0")
    ctx = bg.ctx_create(0)
    try:
        grid = bg.grid_create(ctx, g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
        s = bg.soundings_upload(ctx, *(torch.from_numpy(np.ascontiguousarray(a)).to(dev)
                                       for a in (w.x_cm, w.y_cm, w.z_m)))
        v = bg.variogram(*vgm)
        sep = [torch.empty(g.m, device=dev) for _ in range(3)]
        bg.interp_idw(s, grid, k_idw, power, sep[0])
        bg.interp_okrige(s, grid, k_ok, v, sep[1], sep[2])
        fused = [torch.full((g.m,), -7.0, device=dev) for _ in range(3)]
        bg.interp_idw_okrige(s, grid, k_idw, power, k_ok, v, *fused)
        torch.cuda.synchronize()
        out = [a.cpu().numpy() for a in sep], [a.cpu().numpy() for a in fused]
        bg.soundings_destroy(s)
        bg.grid_destroy(grid)
        return out
    finally:
        bg.ctx_destroy(ctx)


def _bitwise(a, b):
    return np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("k_idw,power,k_ok,vgm", [
    (16, 2.0, 32, SPH), (8, 2.0, 16, SPH), (5, 1.0, 20, EXP), (1, 2.0, 4, SPH),
    (16, 3.0, 16, SPH), (3, 2.0, 3, EXP), (32, 2.0, 32, SPH)])
def test_fused_equals_separate_calls(k_idw, power, k_ok, vgm):
    w = synth.tile(seed=51, n=6000, side_cm=30_000, cell_cm=200)
    sep, fused = _run(w, k_idw, power, k_ok, vgm)
    for a, b in zip(sep, fused):
        assert _bitwise(a, b)
    g = w.grid
    qx, qy = oracle.grid_nodes(g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
    assert_idw(fused[0], oracle.idw(w.x_cm, w.y_cm, w.z_m, qx, qy, k_idw, power))
    rd, rv = oracle.okrige(w.x_cm, w.y_cm, w.z_m, qx, qy, k_ok, *vgm)
    assert_okrige(fused[1], fused[2], rd, rv, vgm[1])


def test_fused_duplicates_nan_and_sparse_data():
    rng = np.random.default_rng(52)
    xs = rng.integers(0, 40, 900) * 100 + 50
    ys = rng.integers(0, 40, 900) * 100 + 50
    x = np.concatenate([xs, xs[:100]]).astype(np.int32)
    y = np.concatenate([ys, ys[:100]]).astype(np.int32)
    z = (3500 + 0.01 * x / 100 + rng.normal(0, 0.5, x.size)).astype(np.float32)
    z[rng.random(x.size) < 0.1] = np.nan
    cases = [synth.Workload(x, y, z, synth.GridSpec(0, 0, 100, 40, 40), "dup", {}),
             synth.Workload(np.array([0, 500, 900], np.int32), np.array([0, 100, 800], np.int32),
                            np.array([3500, 3510, np.nan], np.float32),
                            synth.GridSpec(-500, -500, 200, 9, 7), "sparse", {}),
             synth.Workload(np.array([0, 1], np.int32), np.array([0, 1], np.int32),
                            np.array([np.nan, np.nan], np.float32),
                            synth.GridSpec(0, 0, 100, 5, 3), "none", {})]
    for w in cases:
        sep, fused = _run(w, 8, 2.0, 16, SPH)
        for a, b in zip(sep, fused):
            assert _bitwise(a, b)
    assert np.isnan(fused[0]).all() and np.isnan(fused[1]).all()  # no valid sounding


def test_fused_rejects_k_idw_above_k_okrige():
    import torch

    import paper_2505_22675_gb300 as bg
    w = synth.tile(seed=53, n=500, side_cm=5_000, cell_cm=500)
    g = w.grid
    ctx = bg.ctx_create(0)
    try:
        grid = bg.grid_create(ctx, g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
        s = bg.soundings_upload(ctx, w.x_cm, w.y_cm, w.z_m)
        out = [torch.empty(g.m, device="cuda:0") for _ in range(3)]
        with pytest.raises(bg.BGError) as e:
            bg.interp_idw_okrige(s, grid, 17, 2.0, 16, bg.variogram(*SPH), *out)
        assert e.value.status == -1
        bg.soundings_destroy(s)
        bg.grid_destroy(grid)
    finally:
        bg.ctx_destroy(ctx)


@pytest.mark.parametrize("k_idw,k_ok,with_var", [(16, 32, True), (8, 16, True), (4, 32, False)])
def test_grids_delivered_to_host(k_idw, k_ok, with_var):
    """bg_interp_idw_okrige_host: the host arrays (pinned or pageable) hold
    bitwise the device grids once the stream is synchronized; K = 16 takes the
    separate IDW pass and copies the whole IDW grid first."""
    import torch

    import paper_2505_22675_gb300 as bg
    w = synth.tile(seed=57, n=6000, side_cm=30_000, cell_cm=200)
    g = w.grid
    dev = torch.device("cuda:0")
    ctx = bg.ctx_create(0)
    try:
        grid = bg.grid_create(ctx, g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
        s = bg.soundings_upload(ctx, *(torch.from_numpy(np.ascontiguousarray(a)).to(dev)
                                       for a in (w.x_cm, w.y_cm, w.z_m)))
        v = bg.variogram(*SPH)
        for pinned in (True, False):
            dv = [torch.empty(g.m, device=dev) for _ in range(3)]
            hv = [torch.full((g.m,), -7.0, pin_memory=pinned) for _ in range(3)]
            bg.interp_idw_okrige_host(s, grid, k_idw, 2.0, k_ok, v, dv[0], dv[1],
                                      dv[2] if with_var else None, hv[0], hv[1],
                                      hv[2] if with_var else None)
            torch.cuda.current_stream().synchronize()
            for i in range(3 if with_var else 2):
                assert _bitwise(hv[i].numpy(), dv[i].cpu().numpy())
            if not with_var:
                assert (hv[2].numpy() == -7.0).all()
            ref = [torch.empty(g.m, device=dev) for _ in range(3)]
            bg.interp_idw_okrige(s, grid, k_idw, 2.0, k_ok, v, *ref)
            torch.cuda.synchronize()
            assert _bitwise(hv[1].numpy(), ref[1].cpu().numpy())
        with pytest.raises(bg.BGError):  # var_host without var_out
            bg.interp_idw_okrige_host(s, grid, k_idw, 2.0, k_ok, v, dv[0], dv[1], None,
                                      hv[0], hv[1], hv[2])
        bg.soundings_destroy(s)
        bg.grid_destroy(grid)
    finally:
        bg.ctx_destroy(ctx)
