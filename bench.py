"""Benchmark: grid nodes/s of the full hot path on the synthetic survey swath.

One step = one pass of the whole path over the swath held in HBM:
    upload + validate + spatial-hash build (bg_soundings_upload, device input)
    -> exact k-NN (k=32) of every grid node, then from it
       IDW k=16, p=2 (the 16 nearest) and ordinary kriging k=32, spherical
       (bg_interp_idw_okrige: bitwise the grids of bg_interp_idw and
       bg_interp_okrige called one after the other; that sequence is timed
       beside it as `separate_calls`)
Workload: 4 survey lines x 20,000 pings x 256 beams = 20.48M soundings, grid
20,000 x 3,692 nodes at 0.5 m (73.84M nodes); every node gets an IDW depth, a
kriging depth and a kriging variance. value = grid nodes / s of the step.

The inputs (246 MB of soundings) and outputs (886 MB) exceed the 129 MB L2,
so consecutive steps do not run from cache.

`--impl reference` times the FP64 CPU oracle on a bounded sample of nodes of
the same workload on the host cores (the only other program of this path).
Under torchrun every rank grids its own copy of the swath (weak scaling, no
collective); rank 0 prints one JSON line. Beside it, `slab_split` times the
one swath split into row slabs across the ranks (strong scaling: each rank
builds the whole hash and grids its rows).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "grid nodes/s (IDW k=16, kriging k=32)"
IDW_K, IDW_P = 16, 2.0
OK_K = 32
VGM = (0, 0.25, 100.0, 50.0)  # spherical, nugget 0.25 m^2, total sill 100 m^2, range 50 m

# Algorithmic work per grid node, the per-unit figures of the roofline:
#  - kriging k = 32 (the contract's model): about 35,000 FP32 flops per node
#    (LU of the bordered (k+1) x (k+1) system, its solves and the variogram
#    assembly), plus the FP64 residual counted apart;
#  - the solver's own count for the reduced system of n = k - 1 unknowns: Cholesky
#    n^3/3, two solves (solution + refinement correction) of 2 n^2 each, assembly
#    of n(n+1)/2 + n variogram entries at ~12 flops plus the n^2 matrix fill;
#  - exact k-NN: about 9k/pi candidates per node (cell side ~ the k-th
#    distance), 8 integer operations each (2 subtractions, 2 multiplies, an
#    add, compare and select), so 733 at k = 32 and 367 at k = 16;
#  - HBM bytes: the hash build reads 8 + 12 and writes 16 bytes per sounding;
#    the k-NN ids kernel writes 4 k bytes per node; the IDW kernel reads each
#    16-byte record once and writes 4 bytes per node.
OK_FLOPS_PER_NODE_MODEL = 35_000.0


def okrige_flops_per_node(k=OK_K):
    n = k - 1
    chol = n ** 3 / 3.0
    solves = 2 * (2 * n * n)
    assembly = 12 * (n * (n + 1) / 2 + n) + 2 * n * n
    return chol + solves + assembly


def knn_int_ops_per_node(k):
    return 9.0 * k / 3.141592653589793 * 8.0


HASH_BYTES_PER_SOUNDING = 36.0

# DRAM bytes (read + write) per node, from one ncu capture of each kernel on
# the 2-line swath (3.384M nodes, one launch); traffic grows with the nodes of
# a launch:
#  - k_okrige_solve<32> with the fused IDW: 451.6 MB read + 38.5 MB written,
#    mostly the 128 B of neighbour ids per node;
#  - k_knn_ids<32>: 20.1 MB read + 379.2 MB written (the ids).
SOLVE_DRAM_BYTES_PER_NODE = (451.642368e6 + 38.503936e6) / 3.384e6
KNN_DRAM_BYTES_PER_NODE = (20.107264e6 + 379.174144e6) / 3.384e6


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self, name):
        """Host time of a point of the run; summary(start, stop) keeps the
        samples read between two marks."""
        setattr(self, "t_" + name, time.perf_counter())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self, start=None, stop=None):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0 = getattr(self, "t_" + start, None) if start else None
        t1 = getattr(self, "t_" + stop, None) if stop else None
        for t, ln in self.lines:
            if (t0 is not None and t < t0) or (t1 is not None and t > t1 + 0.25):
                continue
            p = [v.strip() for v in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------- CPU oracle

def oracle_sample(w, nodes: int, seed: int = 0):
    """Node indices and coordinates of `nodes` distinct random grid nodes."""
    g = w.grid
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(g.m, min(nodes, g.m), replace=False))
    qx = (g.x0_cm + (sel % g.nx) * g.cell_cm + g.cell_cm // 2).astype(np.int32)
    qy = (g.y0_cm + (sel // g.nx) * g.cell_cm + g.cell_cm // 2).astype(np.int32)
    return sel, qx, qy


def run_oracle(w, qx, qy, tree, nthreads=0):
    """FP64 IDW k=16 and kriging k=32 of the step at the given nodes."""
    import oracle
    ri = oracle.idw(w.x_cm, w.y_cm, w.z_m, qx, qy, IDW_K, IDW_P, nthreads=nthreads, tree=tree)
    rd, rv = oracle.okrige(w.x_cm, w.y_cm, w.z_m, qx, qy, OK_K, *VGM, nthreads=nthreads,
                           tree=tree)
    return ri, rd, rv


def oracle_timing(w, nodes, nthreads, seed):
    """Seconds to build the oracle's 2-d tree and per node for IDW + kriging."""
    import oracle
    t0 = time.perf_counter()
    tree = oracle.Tree(w.x_cm, w.y_cm, w.z_m, nthreads=nthreads)
    t_build = time.perf_counter() - t0
    _, qx, qy = oracle_sample(w, nodes, seed)
    t0 = time.perf_counter()
    run_oracle(w, qx, qy, tree, nthreads)
    t_query = time.perf_counter() - t0
    tree.close()
    return t_build, t_query / qx.size, qx.size


def cpu_baseline(w, target_s: float = 15.0):
    """The FP64 oracle as it stands (2-d tree k-NN, IDW, kriging by Gaussian
    elimination) on the host cores: the tree is built over all soundings and a
    bounded sample of nodes is gridded (about target_s of CPU work); the
    whole-grid rate is projected as nodes / (build + nodes x time per node).
    Also the same on one thread (smaller sample)."""
    import oracle
    cores = oracle.threads()
    _, per0, _ = oracle_timing(w, 2000, 0, seed=98)
    n = int(min(w.grid.m, max(4 * cores, target_s * 0.7 / max(per0, 1e-9))))
    t_build, per, n = oracle_timing(w, n, 0, seed=7)
    value = w.grid.m / (t_build + w.grid.m * per)
    n1 = int(min(w.grid.m, max(16, target_s * 0.2 / max(per0 * cores, 1e-9))))
    t_build1, per1, n1 = oracle_timing(w, n1, 1, seed=8)
    return {"value": value, "unit": "nodes/s", "cores": cores, "kind": "oracle",
            "sample": f"2-d tree over all {w.x_cm.size} soundings ({t_build:.2f} s on {cores} "
                      f"threads), then FP64 IDW k={IDW_K} + kriging k={OK_K} at {n} random nodes "
                      f"of the {w.grid.nx}x{w.grid.ny} swath grid ({per * 1e6:.2f} us per node); "
                      f"value = whole grid projected: nodes / (build + nodes x per-node time)",
            "nodes_per_s_queries_only": 1.0 / per,
            "single_thread": {"value": w.grid.m / (t_build1 + w.grid.m * per1), "unit": "nodes/s",
                              "tree_build_s": t_build1, "nodes": n1,
                              "nodes_per_s_queries_only": 1.0 / per1}}


def error_stats(got, ref, tol, nan_ref=None):
    """max / p99 |got - ref| and the counts over tol on finite reference values."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    ok = ~np.isnan(ref)
    e = np.abs(got[ok] - ref[ok])
    t = tol[ok] if np.ndim(tol) else tol
    return {"nodes": int(ok.sum()), "max": float(e.max()) if e.size else 0.0,
            "p99": float(np.percentile(e, 99)) if e.size else 0.0,
            "over_tol": int((e > t).sum()), "nan_mismatch": int((np.isnan(got) != ~ok).sum())}


def half_ulp32(v):
    return 0.5 * np.spacing(np.abs(np.asarray(v, np.float64)).astype(np.float32)).astype(np.float64)


def compare_with_oracle(idw, depth, var, ri, rd, rv, nugget=VGM[1]):
    """Per-result error of the GPU grids against the FP64 oracle (tolerances:
    IDW 1e-4 m + half an fp32 ulp; kriging depth 1e-3 m; variance
    1e-4 sigma^2 + 1e-4 nugget)."""
    out = {}
    if idw is not None:
        out["idw_depth_m"] = error_stats(idw, ri, 1e-4 + half_ulp32(ri))
        out["idw_depth_m"]["over_1e-4"] = int((np.abs(np.asarray(idw, np.float64) - ri) > 1e-4).sum())
    if depth is not None:
        out["kriging_depth_m"] = error_stats(depth, rd, 1e-3)
    if var is not None:
        out["kriging_variance_m2"] = error_stats(var, rv, 1e-4 * np.abs(rv) + 1e-4 * nugget)
        r = np.abs(np.asarray(var, np.float64) - rv) / np.maximum(np.abs(rv), 1e-30)
        r = r[~np.isnan(rv)]
        out["kriging_variance_m2"]["max_rel"] = float(r.max()) if r.size else 0.0
    return out


# ------------------------------------------------------------------- main

# ------------------------------------------------------------------ serving

def serving_pool(count: int, seed: int = 3):
    """Tiles shaped like the batched/serving workload (lognormal N with median
    20k in [1k, 200k], grid side 64-1024 at 1-4 m, IDW k=16 / kriging k=32)."""
    return synth.batched_tiles(seed=seed, count=count)


def _percentile(a, q):
    return float(np.percentile(np.asarray(a, dtype=np.float64), q)) if len(a) else None


def serving_measure(bg, torch, ctx, pool, rate, n_tiles, seed):
    """Poisson arrivals at `rate` tiles/s: the serving loop (bg_submit) against
    one synchronous call sequence per tile in arrival order (the plain path).
    Latency = arrival -> grids in host memory. Returns a dict of p50/p99 ms
    and nodes/s for both."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n_tiles)
    arrivals = np.cumsum(gaps) - gaps[0]
    pick = rng.integers(0, len(pool), n_tiles)
    vgm = bg.variogram(*VGM)

    def spec(w):
        g = w.grid
        return (g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)

    # warm-up, untimed: the context's memory pool and the serving slots reach
    # their working size before the arrivals start (both paths then run warm)
    warm = []
    for j in range(min(16, len(pool))):
        w, m = pool[j]
        d = np.empty(w.grid.m, np.float32)
        v = np.empty(w.grid.m, np.float32) if m == 1 else None
        warm.append(bg.submit(ctx, w.x_cm, w.y_cm, w.z_m, spec(w), m, 16 if m == 0 else 32, d, v,
                              power=IDW_P, vgm=vgm))
    for t in warm:
        bg.wait(ctx, t, 600_000)

    # serving path
    tickets = []
    t0 = time.perf_counter()
    for i in range(n_tiles):
        target = t0 + arrivals[i]
        while True:
            dt = target - time.perf_counter()
            if dt <= 0:
                break
            if dt > 2e-3:
                time.sleep(dt - 1e-3)
        w, m = pool[pick[i]]
        d = np.empty(w.grid.m, np.float32)
        v = np.empty(w.grid.m, np.float32) if m == 1 else None
        tickets.append(bg.submit(ctx, w.x_cm, w.y_cm, w.z_m, spec(w), m, 16 if m == 0 else 32, d, v,
                                 power=IDW_P, vgm=vgm))
    res = [bg.wait(ctx, t, 600_000) for t in tickets]
    lat = [(r.t_done_us - r.t_submit_us) / 1e3 for r in res]
    span = (max(r.t_done_us for r in res) - min(r.t_submit_us for r in res)) / 1e6
    nodes = sum(r.nodes for r in res)
    wait_q = [(r.t_start_us - r.t_submit_us) / 1e3 for r in res]
    serve = {"p50_ms": _percentile(lat, 50), "p99_ms": _percentile(lat, 99),
             "nodes_per_s": nodes / span, "errors": sum(1 for r in res if r.status != 0),
             "queue_p50_ms": _percentile(wait_q, 50), "queue_p99_ms": _percentile(wait_q, 99)}

    # plain path: one synchronous call sequence per tile, first come first served
    dev = torch.device("cuda", torch.cuda.current_device())
    lat = []
    t0 = time.perf_counter()
    for i in range(n_tiles):
        target = t0 + arrivals[i]
        while time.perf_counter() < target:
            pass
        w, m = pool[pick[i]]
        g = w.grid
        grid = bg.grid_create(ctx, *spec(w))
        s = bg.soundings_upload(ctx, w.x_cm, w.y_cm, w.z_m)
        d = torch.empty(g.m, device=dev)
        if m == 0:
            bg.interp_idw(s, grid, 16, IDW_P, d)
            d.cpu()
        else:
            v = torch.empty(g.m, device=dev)
            bg.interp_okrige(s, grid, 32, vgm, d, v)
            d.cpu()
            v.cpu()
        bg.soundings_destroy(s)
        bg.grid_destroy(grid)
        lat.append((time.perf_counter() - target) * 1e3)
    span = time.perf_counter() - t0
    plain = {"p50_ms": _percentile(lat, 50), "p99_ms": _percentile(lat, 99),
             "nodes_per_s": sum(pool[j][0].grid.m for j in pick) / span}
    return {"rate_per_s": rate, "tiles": n_tiles, "serving": serve, "plain": plain}


def batched_measure(bg, torch, ctx, pool, n_tiles, steps, check_nodes_per_tile=256):
    """A batch of n_tiles tiles (drawn cyclically from the pool) in one graph of
    persistent kernels, against the same tiles gridded one per-grid call
    sequence after another. Inputs and outputs stay in device memory."""
    dev = torch.device("cuda", torch.cuda.current_device())
    vgm = bg.variogram(*VGM)
    dev_pool = [(tuple(torch.from_numpy(a).to(dev) for a in (w.x_cm, w.y_cm, w.z_m)), w, m)
                for w, m in pool]
    tiles = []
    for i in range(n_tiles):
        (x, y, z), w, m = dev_pool[i % len(dev_pool)]
        g = w.grid
        tiles.append(dict(x_cm=x, y_cm=y, z_m=z, grid_spec=(g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny),
                          method=m, k=16 if m == 0 else 32, power=IDW_P, vgm=vgm,
                          depth_out=torch.empty(g.m, device=dev),
                          var_out=torch.empty(g.m, device=dev) if m == 1 else None))
    nodes = sum(t["grid_spec"][3] * t["grid_spec"][4] for t in tiles)
    b = bg.batch_create(ctx, tiles)
    best = bg.batch_tune(b)
    tuned = bg.batch_config(b)
    for _ in range(2):
        bg.batch_run(b)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        bg.batch_run(b)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    status = bg.batch_status(b)
    bg.batch_destroy(b)
    check = (oracle_check_batch(torch, tiles, pool, n_tiles, check_nodes_per_tile)
             if check_nodes_per_tile else None)
    # the same tiles, one per-grid call sequence each
    torch.cuda.synchronize()
    e0.record()
    for t in tiles:
        grid = bg.grid_create(ctx, *t["grid_spec"])
        s = bg.soundings_upload(ctx, t["x_cm"], t["y_cm"], t["z_m"])
        if t["method"] == 0:
            bg.interp_idw(s, grid, t["k"], IDW_P, t["depth_out"])
        else:
            bg.interp_okrige(s, grid, t["k"], vgm, t["depth_out"], t["var_out"])
        bg.soundings_destroy(s)
        bg.grid_destroy(grid)
    e1.record()
    torch.cuda.synchronize()
    per_tile_ms = e0.elapsed_time(e1)
    return {"tiles": n_tiles, "distinct_tiles": len(pool), "nodes": int(nodes),
            "ms_per_batch": ms, "nodes_per_s": nodes / (ms / 1e3),
            "per_tile_calls_ms": per_tile_ms, "per_tile_calls_nodes_per_s": nodes / (per_tile_ms / 1e3),
            "cell_target_tuned": best, "tuned": tuned, "status_flags": status,
            "errors_vs_oracle": check}


def oracle_check_batch(torch, tiles, pool, n_tiles, per_tile=256, seed=5):
    """Error of every tile of the timed batch against the FP64 oracle at
    `per_tile` random nodes per tile (one 2-d tree per distinct tile)."""
    import oracle
    rng = np.random.default_rng(seed)
    trees = {}
    acc = {0: ([], []), 1: ([], [], [], [], [])}
    for i in range(n_tiles):
        w, m = pool[i % len(pool)]
        t = tiles[i]
        g = w.grid
        sel = np.sort(rng.choice(g.m, min(per_tile, g.m), replace=False))
        qx = (g.x0_cm + (sel % g.nx) * g.cell_cm + g.cell_cm // 2).astype(np.int32)
        qy = (g.y0_cm + (sel // g.nx) * g.cell_cm + g.cell_cm // 2).astype(np.int32)
        tr = trees.get(i % len(pool))
        if tr is None:
            tr = trees[i % len(pool)] = oracle.Tree(w.x_cm, w.y_cm, w.z_m)
        st = torch.from_numpy(sel).to(t["depth_out"].device)
        got = t["depth_out"][st].cpu().numpy()
        if m == 0:
            acc[0][0].append(got)
            acc[0][1].append(oracle.idw(w.x_cm, w.y_cm, w.z_m, qx, qy, t["k"], IDW_P, tree=tr))
        else:
            rd, rv = oracle.okrige(w.x_cm, w.y_cm, w.z_m, qx, qy, t["k"], *VGM, tree=tr)
            acc[1][0].append(got)
            acc[1][1].append(t["var_out"][st].cpu().numpy())
            acc[1][2].append(rd)
            acc[1][3].append(rv)
    for tr in trees.values():
        tr.close()
    cat = lambda a: np.concatenate(a) if a else np.zeros(0)
    out = compare_with_oracle(cat(acc[0][0]), cat(acc[1][0]), cat(acc[1][1]), cat(acc[0][1]),
                              cat(acc[1][2]), cat(acc[1][3]))
    out["sample"] = f"{per_tile} random nodes of each of the {n_tiles} tiles"
    return out


def gridded_measure(bg, torch, n_side, fracs, steps=5):
    """The paper's gridded-input tests on one synthetic depth grid of
    n_side x n_side nodes at 2 m:
    - row filling (Sec. IV Grid A): bilinear and Catmull-Rom onto the points
      halfway between successive rows, with 5% of the source nodes missing;
      HBM roofline over the algorithmic bytes (source read once, output written);
    - hole filling (Sec. IV Grid B): for each removal fraction, the kept
      nodes as soundings (hash build) and IDW k=16 + kriging k=32 at the
      removed nodes; MAE / RMSE against the true depths.
    Inputs and outputs are device-resident; both exceed L2."""
    dev = torch.device("cuda", torch.cuda.current_device())
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs") or 6780.7
    base = synth.hole_grid(seed=4, nx=n_side, ny=n_side, cell_cm=200, frac=0.05)
    g = base.grid
    spec = (g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
    out = {"workload": f"synthetic depth grid {n_side} x {n_side} at 2 m (seafloor model, no "
                       "noise); row filling onto the (n-1) x n row midpoints with 5% of the nodes "
                       "missing; hole filling at removal fractions " + ", ".join(map(str, fracs)),
           "resample": {}, "hole_filling": []}

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    src = torch.from_numpy(base.source()).to(dev)
    mid = (g.x0_cm, g.y0_cm + g.cell_cm // 2, g.cell_cm, g.nx, g.ny - 1)
    mo = mid[3] * mid[4]
    res = torch.empty(mo, device=dev)
    how = torch.empty(mo, dtype=torch.int8, device=dev)
    for name, method in (("bilinear", bg.BILINEAR), ("catmull_rom", bg.CATMULL_ROM)):
        ms = timed(lambda: bg.resample_grid(src, spec, method, mid, res, how))
        nbytes = 4 * g.m + 4 * mo + mo  # source once, values, how-codes
        counts = torch.bincount(how.long(), minlength=3).cpu().tolist()
        out["resample"][name] = {
            "ms": ms, "nodes_per_s": mo / (ms / 1e3),
            "roofline": {"bound": "hbm", "achieved": nbytes / (ms / 1e3) / 1e9, "peak": hbm,
                         "unit": "GB/s", "frac": nbytes / (ms / 1e3) / 1e9 / hbm,
                         "bytes_per_node": nbytes / mo},
            "by_method": counts[0], "bilinear_fallback": counts[1], "no_value": counts[2]}
    del src, res, how

    vgm = bg.variogram(*VGM)
    ctx = bg.ctx_create(torch.cuda.current_device())
    try:
        for i, frac in enumerate(fracs):
            hg = base.with_frac(frac, seed=100 + i)
            sw = hg.soundings()
            qx, qy = hg.queries()
            truth = hg.truth().astype(np.float64)
            xd, yd, zd = (torch.from_numpy(a).to(dev) for a in (sw.x_cm, sw.y_cm, sw.z_m))
            qxd, qyd = torch.from_numpy(qx).to(dev), torch.from_numpy(qy).to(dev)
            m = qx.size
            di = torch.empty(m, device=dev)
            do = torch.empty(m, device=dev)
            vo = torch.empty(m, device=dev)
            holder = {}

            def build():
                if "s" in holder:
                    bg.soundings_destroy(holder.pop("s"))
                holder["s"] = bg.soundings_upload(ctx, xd, yd, zd)

            t_hash = timed(build)
            s = holder["s"]
            t_idw = timed(lambda: bg.interp_idw_points(s, qxd, qyd, IDW_K, IDW_P, di))
            t_ok = timed(lambda: bg.interp_okrige_points(s, qxd, qyd, OK_K, vgm, do, vo))
            bg.soundings_destroy(holder.pop("s"))

            def err(d):
                e = d.cpu().numpy().astype(np.float64) - truth
                return {"mae_m": float(np.mean(np.abs(e))), "rmse_m": float(np.sqrt(np.mean(e * e))),
                        "max_m": float(np.max(np.abs(e)))}
            out["hole_filling"].append({
                "frac": frac, "soundings": int(sw.x_cm.size), "holes": int(m),
                "hash_build_ms": t_hash, "idw_ms": t_idw, "kriging_ms": t_ok,
                "idw_points_per_s": m / (t_idw / 1e3), "kriging_points_per_s": m / (t_ok / 1e3),
                "idw": err(di), "kriging": err(do)})
            del xd, yd, zd, qxd, qyd, di, do, vo
    finally:
        bg.ctx_destroy(ctx)
    return out


def gpu_local_affinity(device_index: int):
    """Restrict this thread to the CPUs sysfs lists as local to the GPU (if any
    of them are allowed); returns the previous CPU set to restore, or None."""
    try:
        import torch
        pr = torch.cuda.get_device_properties(device_index)
        path = (f"/sys/bus/pci/devices/{pr.pci_domain_id:04x}:{pr.pci_bus_id:02x}:"
                f"{pr.pci_device_id:02x}.0/local_cpulist")
        cpus = set()
        with open(path) as f:
            for part in f.read().strip().split(","):
                a, _, b = part.partition("-")
                cpus.update(range(int(a), int(b or a) + 1))
        saved = os.sched_getaffinity(0)
        use = cpus & saved
        if not use or use == saved:
            return None
        os.sched_setaffinity(0, use)
        return saved
    except (AttributeError, OSError, ValueError, RuntimeError):
        return None


def workload(args):
    if args.small:
        return synth.swath(seed=2, lines=2, pings=2000, beams=256)
    return synth.swath(seed=2)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def bench_reference(args):
    """The FP64 oracle on the host cores. One step = build the 2-d tree over
    all soundings, then IDW + kriging at a bounded sample of grid nodes
    (--ref-nodes); value = the whole grid projected from the steps' build and
    per-node times (nodes / (build + nodes x per-node time))."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    w = workload(args)
    import oracle
    cores = oracle.threads()
    nodes = max(cores, int(args.ref_nodes))
    for i in range(args.warmup):
        oracle_timing(w, min(nodes, 4 * cores), 0, seed=1000 + i)
    builds, pers, walls = [], [], []
    for i in range(args.steps):
        t0 = time.perf_counter()
        t_build, per, n = oracle_timing(w, nodes, 0, seed=i)
        walls.append(time.perf_counter() - t0)
        builds.append(t_build)
        pers.append(per)
    t_build = statistics.mean(builds)
    per = statistics.mean(pers)
    value = w.grid.m / (t_build + w.grid.m * per)
    sample = (f"per step: 2-d tree over all {w.x_cm.size} soundings ({t_build:.2f} s), then FP64 "
              f"IDW k={IDW_K} + kriging k={OK_K} at {nodes} random nodes of the "
              f"{w.grid.nx}x{w.grid.ny} swath grid ({per * 1e6:.2f} us per node on {cores} "
              f"threads); value = whole grid projected: nodes / (build + nodes x per-node time)")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "nodes/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * statistics.mean(walls), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": config_dict(w, args),
           "cpu_baseline": {"value": value, "unit": "nodes/s", "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "nodes/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def config_dict(w, args):
    g = w.grid
    return {"workload": ("survey swath, 4 lines x 20,000 pings x 256 beams (20.48M soundings), "
                         "grid 20,000 x 3,692 at 0.5 m" if not args.small else
                         "survey swath, 2 lines x 2,000 pings x 256 beams, grid at 0.5 m"),
            "soundings": int(w.x_cm.size), "nodes": int(g.m), "grid": [g.nx, g.ny, g.cell_cm],
            "idw": {"k": IDW_K, "power": IDW_P},
            "kriging": {"k": OK_K, "model": "spherical", "nugget_m2": VGM[1], "sill_m2": VGM[2],
                        "range_m": VGM[3]},
            "seed": w.params["seed"], "l2": "inputs and outputs larger than L2 (no flush)",
            "parallelism": f"replica x{args.gpus}"}


def measure_alu_peaks(bg, device):
    """FP32 FMA, INT32 (multiply-add; add + xor) and FP64 FMA rates of this
    GPU from the library's own microbenchmark, with the SM clock each kernel
    ran at and the rate per SM per cycle (so that a kernel timed at another
    clock is compared at its own)."""
    import torch
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    out = {"sms": sms}
    for kind in bg.ALU_KINDS:
        ops, mhz = bg.alu_peak(kind, device)
        out[kind] = {"ops_per_s": ops, "sm_mhz": mhz,
                     "ops_per_sm_cycle": ops / (sms * mhz * 1e6) if mhz > 0 else None}
    return out


def _alu_peak_at(peaks, kind, mhz):
    per = peaks[kind]["ops_per_sm_cycle"]
    return per * peaks["sms"] * mhz * 1e6 if per else peaks[kind]["ops_per_s"]


def rooflines(prof, sep_prof, peaks, mpeaks, step_mhz, sms, w, steps, sep_mhz):
    """One roofline entry per hot kernel. ALU peaks are the measured rates per
    SM cycle at the median SM clock sampled while the kernel's step ran; the
    HBM peak is the measured copy bandwidth (MEASURED_PEAKS.json)."""
    hbm = mpeaks.get("hbm_gbs")
    hbm_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    fp32 = _alu_peak_at(peaks, "fp32_fma", step_mhz) / 1e12
    int32 = max(_alu_peak_at(peaks, "int32_imad", step_mhz),
                _alu_peak_at(peaks, "int32_add_xor", step_mhz)) / 1e12
    out = {}
    # kriging solve (k = 32, fused IDW k = 16): the dominant kernel
    s_ms, s_launch, s_nodes = prof["kriging_solve"]
    avg = s_ms / max(s_launch, 1)
    npl = s_nodes / max(s_launch, 1)
    ach = OK_FLOPS_PER_NODE_MODEL * npl / (avg / 1e3) / 1e12
    own = okrige_flops_per_node() * npl / (avg / 1e3) / 1e12
    out["kriging_solve"] = {
        "bound": "alu", "kernel": "k_okrige_solve<32> (kriging k=32 solve, fused IDW k=16)",
        "achieved": ach, "peak": fp32, "unit": "TFLOP/s", "frac": ach / fp32,
        "traffic": SOLVE_DRAM_BYTES_PER_NODE * npl,
        "flops_per_node": OK_FLOPS_PER_NODE_MODEL, "flops_model": "35k FP32 flops per node",
        "own_count": {"flops_per_node": okrige_flops_per_node(), "achieved": own,
                      "frac": own / fp32},
        "avg_launch_ms": avg, "nodes_per_launch": npl, "launches_per_step": s_launch / steps,
        "peak_source": f"measured FP32 FMA rate per SM cycle x {sms} SMs x {step_mhz:.0f} MHz "
                       "(median SM clock of the timed steps)",
        "traffic_source": "ncu dram bytes of the same kernel on a 3.384M-node swath, scaled "
                          "per node",
        "hbm_frac": SOLVE_DRAM_BYTES_PER_NODE * npl / (avg / 1e3) / 1e9 / hbm}
    # k-NN ids (k = 32) of the kriging pass
    k_ms, k_launch, k_nodes = prof["kriging_knn_ids"]
    avg = k_ms / max(k_launch, 1)
    npl = k_nodes / max(k_launch, 1)
    ach = knn_int_ops_per_node(OK_K) * npl / (avg / 1e3) / 1e12
    byt = 4.0 * OK_K * npl
    out["knn_ids_k32"] = {
        "bound": "alu", "kernel": "k_knn_ids<32>", "achieved": ach, "peak": int32,
        "unit": "Tops/s (INT32)", "frac": ach / int32,
        "int_ops_per_node": knn_int_ops_per_node(OK_K), "avg_launch_ms": avg,
        "nodes_per_launch": npl, "hbm_gbs": byt / (avg / 1e3) / 1e9,
        "hbm_frac": byt / (avg / 1e3) / 1e9 / hbm, "bytes_per_node": 4.0 * OK_K,
        "peak_source": "measured INT32 rate (larger of multiply-add and add/xor) per SM cycle "
                       f"x {sms} SMs x {step_mhz:.0f} MHz"}
    # IDW k = 16 on its own (the separate-calls step): k-NN + weights in one kernel
    i_ms, i_launch, i_nodes = sep_prof["idw"]
    if i_launch:
        int32s = max(_alu_peak_at(peaks, "int32_imad", sep_mhz),
                     _alu_peak_at(peaks, "int32_add_xor", sep_mhz)) / 1e12
        avg = i_ms / i_launch
        npl = i_nodes / i_launch
        nval = int(np.count_nonzero(~np.isnan(w.z_m)))
        byt = (16.0 * nval) / i_launch + 4.0 * npl
        ach = knn_int_ops_per_node(IDW_K) * npl / (avg / 1e3) / 1e12
        out["idw_k16"] = {
            "bound": "alu", "kernel": "k_idw<16>", "achieved": ach, "peak": int32s,
            "unit": "Tops/s (INT32)", "frac": ach / int32s,
            "int_ops_per_node": knn_int_ops_per_node(IDW_K),
            "hbm": {"bytes_per_launch": byt, "achieved_gbs": byt / (avg / 1e3) / 1e9,
                    "peak_gbs": hbm, "frac": byt / (avg / 1e3) / 1e9 / hbm,
                    "peak_source": hbm_src},
            "avg_launch_ms": avg, "nodes_per_launch": npl,
            "note": "the HBM fraction is far below 0.5: the k-NN's integer work per node, "
                    "not bytes, bounds IDW"}
    return out


def oracle_check_swath(w, torch, d_idw, d_ok, v_ok, nodes):
    """Error of the step's three grids against the FP64 oracle (2-d tree) at
    `nodes` random nodes plus every node of two rows in the gap between
    survey lines."""
    import oracle
    g = w.grid
    sel, _, _ = oracle_sample(w, nodes, seed=2024)
    gap = np.arange(g.nx) + g.nx * 850  # a row in the gap between lines 1 and 2
    sel = np.unique(np.concatenate([sel, gap, gap + g.nx * 1000]))
    qx = (g.x0_cm + (sel % g.nx) * g.cell_cm + g.cell_cm // 2).astype(np.int32)
    qy = (g.y0_cm + (sel // g.nx) * g.cell_cm + g.cell_cm // 2).astype(np.int32)
    st = torch.from_numpy(sel).to(d_idw.device)
    gi, gd, gv = (t[st].cpu().numpy() for t in (d_idw, d_ok, v_ok))
    t0 = time.perf_counter()
    tree = oracle.Tree(w.x_cm, w.y_cm, w.z_m)
    ri, rd, rv = run_oracle(w, qx, qy, tree)
    tree.close()
    out = compare_with_oracle(gi, gd, gv, ri, rd, rv)
    out["nodes"] = int(sel.size)
    out["sample"] = (f"{nodes} random nodes of the swath grid + 2 full rows in the gaps between "
                     f"lines ({time.perf_counter() - t0:.1f} s of oracle on the host)")
    return out


def tile_configs(bg, torch, device, check):
    """The two tile workloads (20,000 uniform soundings over 512 m, grid
    256 x 256 at 2 m): IDW p=2 k=8 and kriging k=16 (spherical, nugget 0.25,
    sill 100, range 50 m). Per tile: upload + hash build + gridding from
    device-resident inputs, CUDA events, median of 30 after 5 warm-ups; and
    the gridding alone on a built hash. Errors against the oracle on every
    node."""
    import oracle
    dev = torch.device("cuda", device)
    w = synth.tile(seed=1)
    g = w.grid
    ctx = bg.ctx_create(device)
    grid = bg.grid_create(ctx, g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
    x, y, z = (torch.from_numpy(a).to(dev) for a in (w.x_cm, w.y_cm, w.z_m))
    d = torch.empty(g.m, device=dev)
    v = torch.empty(g.m, device=dev)
    vgm = bg.variogram(*VGM)
    stream = torch.cuda.current_stream(dev)
    runs = {"idw_p2_k8": lambda s: bg.interp_idw(s, grid, 8, 2.0, d),
            "kriging_k16": lambda s: bg.interp_okrige(s, grid, 16, vgm, d, v)}
    out = {"workload": "20,000 uniform soundings over a 512 m tile (seed 1), grid 256 x 256 "
                       "at 2 m; device-resident inputs"}
    qx, qy = oracle.grid_nodes(g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
    tree = oracle.Tree(w.x_cm, w.y_cm, w.z_m) if check else None
    for name, fn in runs.items():
        full, interp = [], []
        for it in range(35):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            s = bg.soundings_upload(ctx, x, y, z)
            e[1].record(stream)
            fn(s)
            e[2].record(stream)
            torch.cuda.synchronize()
            bg.soundings_destroy(s)
            if it >= 5:
                full.append(e[0].elapsed_time(e[2]))
                interp.append(e[1].elapsed_time(e[2]))
        ms, ms_i = statistics.median(full), statistics.median(interp)
        r = {"tile_latency_ms": ms, "nodes_per_s": g.m / (ms / 1e3),
             "gridding_ms": ms_i, "gridding_nodes_per_s": g.m / (ms_i / 1e3),
             "hash_build_ms": ms - ms_i}
        if check:
            if name.startswith("idw"):
                ri = oracle.idw(w.x_cm, w.y_cm, w.z_m, qx, qy, 8, 2.0, tree=tree)
                r["errors_vs_oracle"] = compare_with_oracle(d.cpu().numpy(), None, None, ri,
                                                            None, None)
            else:
                rd, rv = oracle.okrige(w.x_cm, w.y_cm, w.z_m, qx, qy, 16, *VGM, tree=tree)
                r["errors_vs_oracle"] = compare_with_oracle(None, d.cpu().numpy(),
                                                            v.cpu().numpy(), None, rd, rv)
        out[name] = r
    if tree is not None:
        tree.close()
    bg.grid_destroy(grid)
    bg.ctx_destroy(ctx)
    return out


def bench_ours(args):
    import torch

    import paper_2505_22675_gb300 as bg
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args)
    g = w.grid
    m = g.m
    ctx = bg.ctx_create(local)
    grid = bg.grid_create(ctx, g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
    xd, yd, zd = (torch.from_numpy(a).to(dev) for a in (w.x_cm, w.y_cm, w.z_m))
    d_idw = torch.empty(m, device=dev)
    d_ok = torch.empty(m, device=dev)
    v_ok = torch.empty(m, device=dev)
    vgm = bg.variogram(*VGM)
    stream = torch.cuda.current_stream(dev)

    ev = {k: [] for k in ("hash", "grid")}

    # One step: upload + hash, then both grids from one k-NN pass
    # (bg_interp_idw_okrige: bitwise the grids of bg_interp_idw followed by
    # bg_interp_okrige, which `separate_calls` times beside it).
    def step(record):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s = bg.soundings_upload(ctx, xd, yd, zd)
        e1.record(stream)
        bg.interp_idw_okrige(s, grid, IDW_K, IDW_P, OK_K, vgm, d_idw, d_ok, v_ok)
        e2.record(stream)
        bg.soundings_destroy(s)
        if record:
            ev["hash"].append((e0, e1))
            ev["grid"].append((e1, e2))

    def separate_step():
        ee = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ee[0].record(stream)
        s = bg.soundings_upload(ctx, xd, yd, zd)
        ee[1].record(stream)
        bg.interp_idw(s, grid, IDW_K, IDW_P, d_idw)
        ee[2].record(stream)
        bg.interp_okrige(s, grid, OK_K, vgm, d_ok, v_ok)
        ee[3].record(stream)
        bg.soundings_destroy(s)
        return ee

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    # the clock sampler starts before the warm-up, so that the start of
    # nvidia-smi falls outside the timed region; only the samples read while
    # the timed steps ran are kept
    peaks = measure_alu_peaks(bg, local)
    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            step(False)
        bg.profile_read(ctx)
        bg.profile_enable(ctx, True)
        clk.mark("sep_start")
        sep = [separate_step() for _ in range(2)]
        torch.cuda.synchronize()
        clk.mark("sep_stop")
        sep_prof = bg.profile_read(ctx)
        bg.profile_enable(ctx, False)
        sep_ms = {"ms_per_step": statistics.mean(e[0].elapsed_time(e[3]) for e in sep),
                  "idw_k16_ms": statistics.mean(e[1].elapsed_time(e[2]) for e in sep),
                  "kriging_k32_ms": statistics.mean(e[2].elapsed_time(e[3]) for e in sep)}
        barrier()
        bg.profile_read(ctx)  # discard anything recorded so far
        bg.profile_enable(ctx, True)
        launches0 = bg.launch_count()
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        clk.mark("start")
        start.record(stream)
        for _ in range(args.steps):
            step(True)
        stop.record(stream)
        torch.cuda.synchronize()
        clk.mark("stop")
    launches = bg.launch_count() - launches0
    prof = bg.profile_read(ctx)
    bg.profile_enable(ctx, False)
    barrier()
    ms = start.elapsed_time(stop) / args.steps
    stage = {k: statistics.median(a.elapsed_time(b) for a, b in v) for k, v in ev.items()}
    per_step = [sum(a.elapsed_time(b) for a, b in (ev[k][i] for k in ev)) for i in range(args.steps)]
    lead_ms = start.elapsed_time(ev["hash"][0][0])  # timed region before the first step ran
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = ws * m / (ms / 1e3)

    # ---- end to end through the C ABI with host buffers (pinned), copies timed.
    # The host buffers are allocated (first touch) from the CPUs next to the GPU
    # where the system says which those are, so that they sit in its NUMA node.
    saved_cpus = gpu_local_affinity(local)
    xh, yh, zh = (torch.from_numpy(a).pin_memory() for a in (w.x_cm, w.y_cm, w.z_m))
    out_h = [torch.empty(m, pin_memory=True) for _ in range(3)]

    # Two steps in flight, as a survey pipeline streams swaths: steps alternate
    # between two streams with their own device and pinned host buffers, so a
    # step's upload overlaps the previous step's kernels. Each step uploads its
    # soundings from pinned host memory and gets its three grids back in pinned
    # host memory (bg_interp_idw_okrige_host copies each row chunk's grids while
    # the later chunks compute); a step's handle is destroyed, and its buffers
    # reused, only after its stream is synchronized two steps later.
    e_streams = [stream, torch.cuda.Stream(dev)]
    e_dev = [(d_idw, d_ok, v_ok), tuple(torch.empty(m, device=dev) for _ in range(3))]
    e_host = [out_h, [torch.empty(m, pin_memory=True) for _ in range(3)]]
    live = [None, None]

    def e2e_step(i):
        j = i % 2
        st = e_streams[j]
        if live[j] is not None:
            st.synchronize()
            bg.soundings_destroy(live[j])
            live[j] = None
        with torch.cuda.stream(st):
            s = bg.soundings_upload(ctx, xh, yh, zh, stream=st)
            bg.interp_idw_okrige_host(s, grid, IDW_K, IDW_P, OK_K, vgm, *e_dev[j], *e_host[j],
                                      stream=st)
        live[j] = s

    def e2e_drain():
        for j in (0, 1):
            e_streams[j].synchronize()
            if live[j] is not None:
                bg.soundings_destroy(live[j])
                live[j] = None

    e2e_step(0)
    e2e_step(1)
    e2e_drain()
    barrier()
    e_steps = max(2, args.steps)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(e_streams[0])
    for i in range(e_steps):
        e2e_step(i)
    e_streams[0].wait_stream(e_streams[1])
    t1.record(e_streams[0])
    t1.synchronize()
    e2e_ms = t0.elapsed_time(t1) / e_steps
    e2e_drain()
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    if saved_cpus is not None:
        os.sched_setaffinity(0, saved_cpus)
    bad = int(torch.isnan(d_idw).sum() + torch.isnan(d_ok).sum())

    # ---- the row-slab split of the one swath (strong scaling): every rank
    # uploads all soundings and builds the whole hash, then grids only its
    # slab of rows (distributed.slab_rows); the slabs equal those rows of the
    # single-GPU grid bitwise. No collective inside the timed steps.
    slab = None
    if ws > 1 or args.slab_split:
        from paper_2505_22675_gb300.distributed import slab_rows
        j0, j1 = slab_rows(g.ny, ws, rank)
        sm_ = g.nx * (j1 - j0)
        sgrid = bg.grid_create(ctx, g.x0_cm, g.y0_cm + j0 * g.cell_cm, g.cell_cm, g.nx,
                               max(j1 - j0, 1))

        def slab_step():
            s = bg.soundings_upload(ctx, xd, yd, zd)
            if j1 > j0:
                bg.interp_idw_okrige(s, sgrid, IDW_K, IDW_P, OK_K, vgm, d_idw[:sm_], d_ok[:sm_],
                                     v_ok[:sm_])
            bg.soundings_destroy(s)

        for _ in range(max(1, args.warmup)):
            slab_step()
        torch.cuda.synchronize()
        barrier()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(args.steps):
            slab_step()
        s1.record(stream)
        torch.cuda.synchronize()
        slab_ms = s0.elapsed_time(s1) / args.steps
        if ws > 1:
            import torch.distributed as dist
            t = torch.tensor([slab_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            slab_ms = float(t.item())
        slab = {"value": m / (slab_ms / 1e3), "unit": "nodes/s", "ms_per_step": slab_ms,
                "scaling": "strong", "parallelism": f"row slabs x{ws}",
                "rows_rank0": int(j1 - j0) if rank == 0 else None,
                "note": "the one swath split into row slabs, one per rank; each rank uploads "
                        "all soundings and builds the whole hash (no halo), then grids its "
                        "slab; max over ranks; the slabs stay on their devices"}
        bg.grid_destroy(sgrid)

    # per-result error against the FP64 oracle at sampled nodes of the last step
    errors = None
    if rank == 0 and not args.no_oracle_check:
        errors = oracle_check_swath(w, torch, d_idw, d_ok, v_ok, args.check_nodes)

    if rank == 0:
        mpeaks = load_peaks()
        clocks = clk.summary("start", "stop")
        step_mhz = clocks.get("sm_mhz") or 2070.0
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        rl = rooflines(prof, sep_prof, peaks, mpeaks, step_mhz, sms, w, args.steps,
                       clk.summary("sep_start", "sep_stop").get("sm_mhz") or step_mhz)
        out = {
            "metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": config_dict(w, args),
            "stages_ms": {"hash_build": stage["hash"],
                          "idw_k16_and_kriging_k32": stage["grid"]},
            "separate_calls": dict(sep_ms, note="the same step with bg_interp_idw and "
                                   "bg_interp_okrige called one after the other (two k-NN "
                                   "searches); not the timed step"),
            "kernels_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
            "step_ms": [round(t, 3) for t in per_step], "lead_ms": round(lead_ms, 3),
            "idw_nodes_per_s_alone": m / (sep_ms["idw_k16_ms"] / 1e3),
            "kriging_nodes_per_s_alone": m / (sep_ms["kriging_k32_ms"] / 1e3),
            "roofline": rl["kriging_solve"],
            "rooflines": rl,
            "alu_peaks_measured": peaks,
            "errors_vs_oracle": errors,
            "e2e": {"value": ws * m / (e2e_ms / 1e3), "unit": "nodes/s",
                    "h2d_bytes_per_step": int(12 * w.x_cm.size),
                    "d2h_bytes_per_step": int(12 * m), "ms_per_step": e2e_ms, "steps": e_steps,
                    "in_flight": 2},
            "gpu_launches": int(launches), "clocks": clocks, "nan_outputs": bad,
        }
        if slab is not None:
            out["slab_split"] = slab
        if not args.no_tiles:
            out["tile_configs"] = tile_configs(bg, torch, local, not args.no_oracle_check)
        pool = None
        if not args.no_batched:
            pool = serving_pool(args.serving_pool)
            out["batched"] = batched_measure(bg, torch, ctx, pool, args.batch_tiles, 3,
                                             0 if args.no_oracle_check else 256)
            out["batched"]["workload"] = (
                "one launch sequence (graph of persistent kernels) over tiles of uneven size: "
                "lognormal N (median 20k, 1k-200k), grid side 64-1024 at 1-4 m, IDW k=16 / "
                "kriging k=32 50/50, drawn cyclically from the distinct tiles; device-resident")
        if not args.no_serving:
            pool = pool or serving_pool(args.serving_pool)
            rates = [50, 200, 500, 1000, 2000]
            n_t = args.serving_tiles
            out["serving"] = {
                "workload": (f"{len(pool)} distinct tiles drawn with replacement: lognormal N "
                             "(median 20k, 1k-200k), grid side 64-1024 at 1-4 m, IDW k=16 / "
                             "kriging k=32 50/50; Poisson arrivals; latency = arrival to grids in "
                             "host memory; plain = one synchronous call sequence per tile, FIFO"),
                "hbm_budget_bytes": 40 << 30,
                "rates": []}
            sctx = bg.ctx_create(local, 40 << 30)
            try:
                for i, r in enumerate(rates):
                    out["serving"]["rates"].append(
                        serving_measure(bg, torch, sctx, pool, r, n_t, seed=17 + i))
            finally:
                bg.ctx_destroy(sctx)
        if not args.no_gridded:
            out["gridded"] = gridded_measure(bg, torch, 4096 if args.small else 8192,
                                             (0.01, 0.05, 0.1))
        if not args.no_cpu_baseline and ws == 1:
            out["cpu_baseline"] = cpu_baseline(w, target_s=args.cpu_seconds)
        print(json.dumps(out), flush=True)
    bg.grid_destroy(grid)
    bg.ctx_destroy(ctx)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--small", action="store_true", help="2-line swath (quick check / profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-nodes", type=int, default=50_000, help="reference arm: nodes per step")
    ap.add_argument("--serving-tiles", type=int, default=2000,
                    help="tiles per arrival rate of the serving sweep (50-2000 tiles/s)")
    ap.add_argument("--serving-pool", type=int, default=48)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-gridded", action="store_true",
                    help="skip the gridded-input (row filling / hole filling) measurements")
    ap.add_argument("--gridded-only", action="store_true",
                    help="only the gridded-input measurements (one JSON line of their own)")
    ap.add_argument("--batch-tiles", type=int, default=512)
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the per-result comparison with the FP64 oracle")
    ap.add_argument("--check-nodes", type=int, default=100_000,
                    help="random swath nodes compared with the oracle")
    ap.add_argument("--no-tiles", action="store_true", help="skip the two tile workloads")
    ap.add_argument("--slab-split", action="store_true",
                    help="also time the row-slab split of the swath at one rank (it always "
                         "runs under torchrun with more than one rank)")
    args = ap.parse_args()
    if args.impl == "reference":
        bench_reference(args)
    elif args.gridded_only:
        import torch

        import paper_2505_22675_gb300 as bg
        print(json.dumps({"gridded": gridded_measure(bg, torch, 4096 if args.small else 8192,
                                                     (0.01, 0.05, 0.1))}), flush=True)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
