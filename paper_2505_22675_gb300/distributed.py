"""Multi-GPU partitioning of the gridding path (one process per GPU).

Two ways to split the work, both without any exchange inside the path:

- A large swath is split into slabs of consecutive grid rows. Every rank
  holds all soundings (one broadcast from rank 0), so each slab's exact
  k-NN needs no halo; a slab is itself a regular grid whose node
  coordinates equal those rows of the full grid, and results are per node
  and canonical, so the assembled grid equals the single-GPU grid bit for
  bit. Slabs are gathered to rank 0.
- Independent tiles (batches, serving) are assigned to ranks longest-first
  to the least-loaded rank, by an estimated cost; results are gathered to
  rank 0.

`compute` is the per-rank gridding function; by default it is the CUDA
library on the rank's device. The collective calls use torch.distributed on
whatever backend the process group was created with: their buffers live on
the rank's current CUDA device when the group's backend is NCCL (which takes
device tensors only), on the host for gloo.
"""
from __future__ import annotations

import heapq
from typing import Callable, Sequence

import numpy as np

IDW = 0
OKRIGE = 1


class RankFailure(RuntimeError):
    """A collective of the partitioning failed: a rank left the group, timed
    out or raised. Ranks leave only between steps (no kernel of theirs is in
    flight); the others learn of it here, at their next collective, within
    the process group's timeout."""

# relative cost per node of the two methods (kriging k=32 vs IDW k=16, measured
# on one GB300: about 10x); used only to balance tile assignments
METHOD_COST = {IDW: 1.0, OKRIGE: 10.0}


def slab_rows(ny: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [j0, j1) of rank `rank` when ny rows are split into `world`
    contiguous slabs whose sizes differ by at most one row."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(ny, world)
    j0 = rank * base + min(rank, extra)
    return j0, j0 + base + (1 if rank < extra else 0)


def slab_spec(grid_spec, j0: int, j1: int):
    """The sub-grid holding rows [j0, j1) of grid_spec = (x0, y0, cell, nx, ny)."""
    x0, y0, cell, nx, ny = grid_spec
    if not 0 <= j0 <= j1 <= ny:
        raise ValueError("rows out of range")
    return (x0, y0 + j0 * cell, cell, nx, j1 - j0)


def tile_cost(n_soundings: int, nx: int, ny: int, method: int) -> float:
    """Estimated work of a tile: nodes times the method's cost per node, plus
    a small term for the hash build."""
    return nx * ny * METHOD_COST[method] + 0.05 * n_soundings


def assign_tiles(costs: Sequence[float], world: int) -> list[int]:
    """Rank of each tile: longest processing time first onto the least-loaded
    rank (ties to the lower rank). Deterministic."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    out = [0] * len(costs)
    for i in order:
        load, r = heapq.heappop(heap)
        out[i] = r
        heapq.heappush(heap, (load + costs[i], r))
    return out


# --------------------------------------------------------------- collectives

def _collective(fn, *args, **kwargs):
    try:
        return fn(*args, **kwargs)
    except Exception as e:  # the backend's own error types differ
        raise RankFailure(f"collective {getattr(fn, '__name__', fn)} failed: {e}") from e


def _comm_device(dist, group):
    """Where the collectives' buffers live: the current CUDA device for an
    NCCL group, the host otherwise."""
    import torch
    if str(dist.get_backend(group)).lower() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def _broadcast_array(dist, arr, src, group, dtype):
    import torch
    dev = _comm_device(dist, group)
    n = torch.tensor([0 if arr is None else arr.size], dtype=torch.int64, device=dev)
    _collective(dist.broadcast, n, src, group=group)
    if arr is not None and dist.get_rank(group) == src:
        t = torch.from_numpy(np.ascontiguousarray(arr)).to(dev)
    else:
        t = torch.empty(int(n.item()), dtype=dtype, device=dev)
    _collective(dist.broadcast, t, src, group=group)
    return t.cpu().numpy()


def _all_sizes(dist, size: int, group):
    """Every rank's `size`, in rank order."""
    import torch
    dev = _comm_device(dist, group)
    world = dist.get_world_size(group)
    n = torch.tensor([size], dtype=torch.int64, device=dev)
    sizes = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    _collective(dist.all_gather, sizes, n, group=group)
    return [int(s.item()) for s in sizes]


def _gather_to_root(dist, piece: np.ndarray, group, root=0):
    """Concatenate equal-dtype 1-D pieces of varying lengths on `root`."""
    import torch
    dev = _comm_device(dist, group)
    world = dist.get_world_size(group)
    sizes = _all_sizes(dist, piece.size, group)
    m = max(sizes)
    buf = torch.zeros(m, dtype=torch.from_numpy(piece[:0]).dtype, device=dev)
    buf[:piece.size] = torch.from_numpy(piece).to(dev)
    parts = [torch.zeros_like(buf) for _ in range(world)]
    _collective(dist.all_gather, parts, buf, group=group)
    if dist.get_rank(group) != root:
        return None
    return np.concatenate([p[:s].cpu().numpy() for p, s in zip(parts, sizes)])


# ------------------------------------------------------------------- default

def library_compute(device: int = 0):
    """compute(x, y, z, grid_spec, method, k, power, vgm) on the CUDA library."""
    def run(x, y, z, spec, method, k, power, vgm):
        import torch

        import paper_2505_22675_gb300 as bg
        dev = torch.device("cuda", device)
        ctx = bg.ctx_create(device)
        try:
            grid = bg.grid_create(ctx, *spec)
            s = bg.soundings_upload(ctx, *(torch.from_numpy(np.ascontiguousarray(a)).to(dev)
                                           for a in (x, y, z)))
            m = spec[3] * spec[4]
            d = torch.empty(m, device=dev)
            v = torch.empty(m, device=dev)
            if method == IDW:
                bg.interp_idw(s, grid, k, power, d)
                out = (d.cpu().numpy(), None)
            else:
                bg.interp_okrige(s, grid, k, bg.variogram(*vgm), d, v)
                out = (d.cpu().numpy(), v.cpu().numpy())
            bg.soundings_destroy(s)
            bg.grid_destroy(grid)
            return out
        finally:
            bg.ctx_destroy(ctx)
    return run


# --------------------------------------------------------------------- paths

def grid_swath(x, y, z, grid_spec, method: int, k: int, power: float = 2.0,
               vgm=(0, 0.25, 100.0, 50.0), group=None, compute: Callable | None = None,
               src: int = 0):
    """Grid one swath over all ranks of `group` by row slabs.

    x, y, z are needed on rank `src` only (others may pass None). Returns
    (depth, var) for the full grid on rank `src` (var is None for IDW), and
    (None, None) elsewhere.
    """
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    x = _broadcast_array(dist, x, src, group, torch.int32)
    y = _broadcast_array(dist, y, src, group, torch.int32)
    z = _broadcast_array(dist, z, src, group, torch.float32)
    j0, j1 = slab_rows(grid_spec[4], world, rank)
    compute = compute or library_compute(torch.cuda.current_device() if torch.cuda.is_available() else 0)
    if j1 > j0:
        d, v = compute(x, y, z, slab_spec(grid_spec, j0, j1), method, k, power, vgm)
    else:
        d, v = np.zeros(0, np.float32), (np.zeros(0, np.float32) if method == OKRIGE else None)
    depth = _gather_to_root(dist, np.asarray(d, np.float32), group, src)
    var = _gather_to_root(dist, np.asarray(v, np.float32), group, src) if method == OKRIGE else None
    return depth, var


def grid_tiles(tiles, group=None, compute: Callable | None = None, root: int = 0):
    """Grid independent tiles over the ranks of `group`.

    tiles: the same list on every rank, of dicts with x_cm, y_cm, z_m (numpy),
    grid_spec, method, k, power, vgm. Returns on `root` a list of (depth, var)
    in tile order; None elsewhere.
    """
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    costs = [tile_cost(t["x_cm"].size, t["grid_spec"][3], t["grid_spec"][4], t["method"])
             for t in tiles]
    owner = assign_tiles(costs, world)
    compute = compute or library_compute(torch.cuda.current_device() if torch.cuda.is_available() else 0)
    mine = [i for i in range(len(tiles)) if owner[i] == rank]
    pieces = []
    for i in mine:
        t = tiles[i]
        d, v = compute(t["x_cm"], t["y_cm"], t["z_m"], t["grid_spec"], t["method"], t["k"],
                       t.get("power", 2.0), t.get("vgm", (0, 0.25, 100.0, 50.0)))
        pieces.append(np.asarray(d, np.float32))
        if t["method"] == OKRIGE:
            pieces.append(np.asarray(v, np.float32))
    flat = np.concatenate(pieces) if pieces else np.zeros(0, np.float32)
    allflat = _gather_to_root(dist, flat, group, root)
    # every rank knows every owner, so rank-major order is reproducible on root
    if rank != root:
        return None
    out = [None] * len(tiles)
    at = 0
    for r in range(world):
        for i in (j for j in range(len(tiles)) if owner[j] == r):
            m = tiles[i]["grid_spec"][3] * tiles[i]["grid_spec"][4]
            d = allflat[at:at + m]
            at += m
            v = None
            if tiles[i]["method"] == OKRIGE:
                v = allflat[at:at + m]
                at += m
            out[i] = (d, v)
    return out
