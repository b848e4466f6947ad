"""Multi-GPU partitioning logic, run as CPU ranks over gloo (world size 2).

The per-rank compute is the FP64 oracle here, so the test checks only the
partitioning, the broadcast of the soundings and the gather of the slabs or
tiles: the assembled grids must equal the oracle's single-process grids.
"""
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_2505_22675_gb300 import distributed as D


def oracle_compute(x, y, z, spec, method, k, power, vgm):
    qx, qy = oracle.grid_nodes(*spec)
    if method == D.IDW:
        return oracle.idw(x, y, z, qx, qy, k, power, nthreads=1).astype(np.float32), None
    d, v = oracle.okrige(x, y, z, qx, qy, k, *vgm, nthreads=1)
    return d.astype(np.float32), v.astype(np.float32)


def test_slab_rows_cover_the_grid():
    for ny in (1, 7, 100, 3692):
        for world in (1, 2, 3, 8):
            rows = [D.slab_rows(ny, world, r) for r in range(world)]
            assert rows[0][0] == 0 and rows[-1][1] == ny
            assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
            sizes = [b - a for a, b in rows]
            assert max(sizes) - min(sizes) <= 1
    assert D.slab_spec((100, 200, 50, 10, 20), 5, 12) == (100, 450, 50, 10, 7)


def test_assign_tiles_balances_and_is_deterministic():
    rng = np.random.default_rng(0)
    costs = list(rng.lognormal(10, 1, 200))
    a = D.assign_tiles(costs, 4)
    assert a == D.assign_tiles(costs, 4)
    loads = np.zeros(4)
    for c, r in zip(costs, a):
        loads[r] += c
    assert loads.max() - loads.min() <= max(costs)  # LPT bound


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = synth.swath(seed=2, lines=2, pings=40, beams=32)
        g = w.grid
        spec = (g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
        src = (w.x_cm, w.y_cm, w.z_m) if rank == 0 else (None, None, None)
        d, _ = D.grid_swath(*src, spec, D.IDW, 8, compute=oracle_compute)
        dk, vk = D.grid_swath(*src, spec, D.OKRIGE, 8, compute=oracle_compute)
        tiles = []
        for t, (tw, m) in enumerate(synth.batched_tiles(seed=4, count=7, scale=0.005)):
            tg = tw.grid
            tiles.append(dict(x_cm=tw.x_cm, y_cm=tw.y_cm, z_m=tw.z_m, method=m, k=8,
                              grid_spec=(tg.x0_cm, tg.y0_cm, tg.cell_cm, tg.nx, tg.ny)))
        res = D.grid_tiles(tiles, compute=oracle_compute)
        if rank == 0:
            np.save(os.path.join(out_dir, "idw.npy"), d)
            np.save(os.path.join(out_dir, "okd.npy"), dk)
            np.save(os.path.join(out_dir, "okv.npy"), vk)
            for i, (td, tv) in enumerate(res):
                np.save(os.path.join(out_dir, f"tile{i}_d.npy"), td)
                if tv is not None:
                    np.save(os.path.join(out_dir, f"tile{i}_v.npy"), tv)
        else:
            assert d is None and res is None
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_single_process(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    w = synth.swath(seed=2, lines=2, pings=40, beams=32)
    g = w.grid
    spec = (g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
    d, _ = oracle_compute(w.x_cm, w.y_cm, w.z_m, spec, D.IDW, 8, 2.0, None)
    assert np.array_equal(np.load(tmp_path / "idw.npy"), d)
    dk, vk = oracle_compute(w.x_cm, w.y_cm, w.z_m, spec, D.OKRIGE, 8, 2.0, (0, 0.25, 100.0, 50.0))
    assert np.array_equal(np.load(tmp_path / "okd.npy"), dk)
    assert np.array_equal(np.load(tmp_path / "okv.npy"), vk)
    for i, (tw, m) in enumerate(synth.batched_tiles(seed=4, count=7, scale=0.005)):
        tg = tw.grid
        rd, rv = oracle_compute(tw.x_cm, tw.y_cm, tw.z_m, (tg.x0_cm, tg.y0_cm, tg.cell_cm, tg.nx, tg.ny),
                                m, 8, 2.0, (0, 0.25, 100.0, 50.0))
        assert np.array_equal(np.load(tmp_path / f"tile{i}_d.npy"), rd)
        if m == D.OKRIGE:
            assert np.array_equal(np.load(tmp_path / f"tile{i}_v.npy"), rv)


@pytest.mark.gpu
def test_slabs_on_one_gpu_equal_the_unsplit_grid():
    """The slabs a multi-GPU run would compute, run one after another on one
    GPU, assemble into exactly the single-GPU grid."""
    w = synth.swath(seed=2, lines=2, pings=300, beams=256)
    g = w.grid
    spec = (g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
    run = D.library_compute(0)
    for method, k in ((D.IDW, 16), (D.OKRIGE, 32)):
        full_d, full_v = run(w.x_cm, w.y_cm, w.z_m, spec, method, k, 2.0, (0, 0.25, 100.0, 50.0))
        for world in (2, 3):
            parts = [run(w.x_cm, w.y_cm, w.z_m, D.slab_spec(spec, *D.slab_rows(g.ny, world, r)),
                         method, k, 2.0, (0, 0.25, 100.0, 50.0)) for r in range(world)]
            d = np.concatenate([p[0] for p in parts])
            assert np.array_equal(d.view(np.uint32), full_d.view(np.uint32))
            if method == D.OKRIGE:
                v = np.concatenate([p[1] for p in parts])
                assert np.array_equal(v.view(np.uint32), full_v.view(np.uint32))


def _nccl_rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["NCCL_NVLS_ENABLE"] = "0"
    torch.cuda.set_device(rank)
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        w = synth.swath(seed=2, lines=2, pings=300, beams=256)
        g = w.grid
        spec = (g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
        d, _ = D.grid_swath(w.x_cm, w.y_cm, w.z_m, spec, D.IDW, 16)
        dk, vk = D.grid_swath(w.x_cm, w.y_cm, w.z_m, spec, D.OKRIGE, 32)
        tiles = []
        for tw, m in synth.batched_tiles(seed=4, count=5, scale=0.02):
            tg = tw.grid
            tiles.append(dict(x_cm=tw.x_cm, y_cm=tw.y_cm, z_m=tw.z_m, method=m, k=16 if m == 0 else 32,
                              grid_spec=(tg.x0_cm, tg.y0_cm, tg.cell_cm, tg.nx, tg.ny)))
        res = D.grid_tiles(tiles)
        if rank == 0:
            np.save(os.path.join(out_dir, "idw.npy"), d)
            np.save(os.path.join(out_dir, "okd.npy"), dk)
            np.save(os.path.join(out_dir, "okv.npy"), vk)
            for i, (td, tv) in enumerate(res):
                np.save(os.path.join(out_dir, f"tile{i}_d.npy"), td)
                if tv is not None:
                    np.save(os.path.join(out_dir, f"tile{i}_v.npy"), tv)
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
def test_nccl_group_runs_the_partitioned_paths(tmp_path):
    """grid_swath and grid_tiles on an NCCL process group (one rank on this
    GPU: the collectives' buffers must be device tensors) give bitwise the
    single-GPU grids."""
    import torch.multiprocessing as mp
    mp.spawn(_nccl_rank_main, args=(1, _free_port(), str(tmp_path)), nprocs=1, join=True)
    w = synth.swath(seed=2, lines=2, pings=300, beams=256)
    g = w.grid
    spec = (g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
    run = D.library_compute(0)
    vgm = (0, 0.25, 100.0, 50.0)
    same = lambda a, b: np.array_equal(np.asarray(a, np.float32).view(np.uint32),
                                       np.asarray(b, np.float32).view(np.uint32))
    d, _ = run(w.x_cm, w.y_cm, w.z_m, spec, D.IDW, 16, 2.0, vgm)
    assert same(np.load(tmp_path / "idw.npy"), d)
    dk, vk = run(w.x_cm, w.y_cm, w.z_m, spec, D.OKRIGE, 32, 2.0, vgm)
    assert same(np.load(tmp_path / "okd.npy"), dk) and same(np.load(tmp_path / "okv.npy"), vk)
    for i, (tw, m) in enumerate(synth.batched_tiles(seed=4, count=5, scale=0.02)):
        tg = tw.grid
        rd, rv = run(tw.x_cm, tw.y_cm, tw.z_m, (tg.x0_cm, tg.y0_cm, tg.cell_cm, tg.nx, tg.ny), m,
                     16 if m == 0 else 32, 2.0, vgm)
        assert same(np.load(tmp_path / f"tile{i}_d.npy"), rd)
        if m == D.OKRIGE:
            assert same(np.load(tmp_path / f"tile{i}_v.npy"), rv)


def _rank_leaves(rank, world, port, out_dir):
    import datetime

    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    if rank == 1:
        os._exit(0)  # leaves between steps: none of its collectives is in flight
    w = synth.swath(seed=2, lines=2, pings=40, beams=32)
    g = w.grid
    outcome = "no error"
    try:
        D.grid_swath(w.x_cm, w.y_cm, w.z_m, (g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny), D.IDW, 8,
                     compute=oracle_compute)
    except D.RankFailure:
        outcome = "rank failure"
    with open(os.path.join(out_dir, "rank0.txt"), "w") as f:
        f.write(outcome)
    os._exit(0)  # the group is broken: no orderly teardown


def test_a_rank_that_leaves_is_reported_not_waited_for(tmp_path):
    import time

    import torch.multiprocessing as mp
    t0 = time.time()
    mp.spawn(_rank_leaves, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    assert (tmp_path / "rank0.txt").read_text() == "rank failure"
    assert time.time() - t0 < 120
