"""Serving (bg_submit / bg_poll / bg_wait / bg_cancel): continuous batching.

Each request's grids must be bitwise the same whether it runs alone, in a mix
of overlapping requests, or through the direct API; admission must respect the
context's HBM budget; queued tickets can be cancelled and waits time out.
"""
import time

import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_idw, assert_okrige

pytestmark = pytest.mark.gpu

VGM = (0, 0.25, 100.0, 50.0)


def _tiles(count, seed=3, scale=0.03):
    return synth.batched_tiles(seed=seed, count=count, scale=scale)


def _k(method):
    return 16 if method == 0 else 32


def _submit(bg, ctx, w, method):
    g = w.grid
    d = np.full(g.m, -1.0, np.float32)
    v = np.full(g.m, -1.0, np.float32) if method == 1 else None
    t = bg.submit(ctx, w.x_cm, w.y_cm, w.z_m, (g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny), method,
                  _k(method), d, v, power=2.0, vgm=bg.variogram(*VGM))
    return t, d, v


def _direct(bg, torch, ctx, w, method):
    g = w.grid
    dev = torch.device("cuda:0")
    grid = bg.grid_create(ctx, g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
    s = bg.soundings_upload(ctx, *(torch.from_numpy(a).to(dev) for a in (w.x_cm, w.y_cm, w.z_m)))
    d = torch.empty(g.m, device=dev)
    v = torch.empty(g.m, device=dev)
    if method == 0:
        bg.interp_idw(s, grid, 16, 2.0, d)
    else:
        bg.interp_okrige(s, grid, 32, bg.variogram(*VGM), d, v)
    torch.cuda.synchronize()
    out = d.cpu().numpy(), (v.cpu().numpy() if method == 1 else None)
    bg.soundings_destroy(s)
    bg.grid_destroy(grid)
    return out


def test_mix_alone_and_direct_are_bitwise_equal():
    import torch

    import paper_2505_22675_gb300 as bg
    tiles = _tiles(16)
    ctx = bg.ctx_create(0)
    try:
        alone = []
        for w, m in tiles:
            t, d, v = _submit(bg, ctx, w, m)
            res = bg.wait(ctx, t, 60_000)
            assert res.status == 0 and res.nodes == w.grid.m
            assert res.t_submit_us <= res.t_start_us <= res.t_done_us
            alone.append((d, v))
        mix = [_submit(bg, ctx, w, m) for w, m in tiles]
        for (t, d, v), (ad, av), (w, m) in zip(mix, alone, tiles):
            res = bg.wait(ctx, t, 60_000)
            assert res.status == 0
            assert np.array_equal(d.view(np.uint32), ad.view(np.uint32))
            if m == 1:
                assert np.array_equal(v.view(np.uint32), av.view(np.uint32))
            dd, dv = _direct(bg, torch, ctx, w, m)
            assert np.array_equal(d.view(np.uint32), dd.view(np.uint32))
            if m == 1:
                assert np.array_equal(v.view(np.uint32), dv.view(np.uint32))
    finally:
        bg.ctx_destroy(ctx)


def test_large_grids_copied_out_in_shares_are_bitwise_equal():
    """Grids of 256 KB and more leave pinned staging in four shares (the
    completion thread and three helpers): 301 x 301 and 517 x 517 nodes (odd
    sizes, so the last share takes a remainder), IDW and kriging, submitted
    one at a time and then all at once, against the direct API."""
    import torch

    import paper_2505_22675_gb300 as bg
    tiles = [(synth.tile(seed=31, n=20_000, side_cm=60_200, cell_cm=200), 0),
             (synth.tile(seed=32, n=30_000, side_cm=60_200, cell_cm=200), 1),
             (synth.tile(seed=33, n=40_000, side_cm=103_400, cell_cm=200), 1),
             (synth.tile(seed=34, n=25_000, side_cm=103_400, cell_cm=200), 0)]
    assert all(w.grid.m * 4 >= 256 << 10 for w, _ in tiles)
    ctx = bg.ctx_create(0)
    try:
        alone = []
        for w, m in tiles:
            t, d, v = _submit(bg, ctx, w, m)
            assert bg.wait(ctx, t, 60_000).status == 0
            alone.append((d, v))
        mix = [_submit(bg, ctx, w, m) for w, m in tiles]
        for (t, d, v), (ad, av), (w, m) in zip(mix, alone, tiles):
            assert bg.wait(ctx, t, 60_000).status == 0
            dd, dv = _direct(bg, torch, ctx, w, m)
            for got in (d, ad):
                assert np.array_equal(got.view(np.uint32), dd.view(np.uint32))
            if m == 1:
                for got in (v, av):
                    assert np.array_equal(got.view(np.uint32), dv.view(np.uint32))
    finally:
        bg.ctx_destroy(ctx)


def test_served_results_match_the_oracle():
    import paper_2505_22675_gb300 as bg
    tiles = [t for t in _tiles(10, seed=5, scale=0.01)][:6]
    ctx = bg.ctx_create(0)
    try:
        subs = [_submit(bg, ctx, w, m) for w, m in tiles]
        for (t, d, v), (w, m) in zip(subs, tiles):
            assert bg.wait(ctx, t, 60_000).status == 0
            g = w.grid
            qx, qy = oracle.grid_nodes(g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
            if m == 0:
                assert_idw(d, oracle.idw(w.x_cm, w.y_cm, w.z_m, qx, qy, 16, 2.0))
            else:
                rd, rv = oracle.okrige(w.x_cm, w.y_cm, w.z_m, qx, qy, 32, *VGM)
                assert_okrige(d, v, rd, rv, VGM[1])
    finally:
        bg.ctx_destroy(ctx)


def test_admission_respects_a_small_budget():
    import paper_2505_22675_gb300 as bg
    budget = 64 << 20
    ctx = bg.ctx_create(0, budget)
    try:
        tiles = [synth.tile(seed=100 + i, n=60_000, side_cm=60_000, cell_cm=100) for i in range(12)]
        subs = [_submit(bg, ctx, w, 1) for w in tiles]
        seen_running, peak = 0, 0
        pending = {t for t, _, _ in subs}
        deadline = time.time() + 120
        while pending and time.time() < deadline:
            q, r, b = bg.serve_stats(ctx)
            seen_running = max(seen_running, r)
            peak = max(peak, b)
            for t in list(pending):
                res = bg.poll(ctx, t)
                if res is not None:
                    assert res.status == 0
                    pending.discard(t)
        assert not pending
        assert 0 < peak <= budget
        assert bg.ctx_device_bytes(ctx) <= budget
        # a request that cannot fit alone is refused up front
        big = synth.tile(seed=7, n=2_000_000, side_cm=200_000, cell_cm=100)
        with pytest.raises(bg.BGError) as e:
            _submit(bg, ctx, big, 1)
        assert e.value.status == -2
    finally:
        bg.ctx_destroy(ctx)


def test_cancel_queued_and_wait_timeout():
    import paper_2505_22675_gb300 as bg
    w = synth.tile(seed=9, n=60_000, side_cm=60_000, cell_cm=100)
    ctx = bg.ctx_create(0, 64 << 20)  # room for one such kriging request (~53 MB) at a time
    try:
        subs = [_submit(bg, ctx, w, 1) for _ in range(6)]
        last = subs[-1][0]
        bg.cancel(ctx, last)
        with pytest.raises(bg.BGError) as e:
            bg.wait(ctx, subs[-2][0], 0)
        assert e.value.status == -4  # still queued or running: timed out
        for t, _, _ in subs[:-1]:
            assert bg.wait(ctx, t, 120_000).status == 0
        assert bg.wait(ctx, last, 1000).status == -5
        with pytest.raises(bg.BGError) as e:
            bg.poll(ctx, last)  # released by the wait above
        assert e.value.status == -7
    finally:
        bg.ctx_destroy(ctx)


def test_invalid_requests_are_rejected():
    import paper_2505_22675_gb300 as bg
    ctx = bg.ctx_create(0)
    try:
        w = synth.tile(seed=1, n=100, side_cm=1000, cell_cm=100)
        d = np.empty(w.grid.m, np.float32)
        g = w.grid
        for kw in (dict(method=2, k=8), dict(method=0, k=0), dict(method=0, k=40)):
            with pytest.raises(bg.BGError) as e:
                bg.submit(ctx, w.x_cm, w.y_cm, w.z_m, (0, 0, 100, g.nx, g.ny), kw["method"], kw["k"], d)
            assert e.value.status == -1
        with pytest.raises(bg.BGError):
            bg.submit(ctx, w.x_cm, w.y_cm, w.z_m, (0, 0, 101, g.nx, g.ny), 0, 8, d)  # odd cell
    finally:
        bg.ctx_destroy(ctx)
