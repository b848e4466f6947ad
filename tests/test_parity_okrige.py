"""GPU parity of the fused k-NN + ordinary-kriging path against the FP64 oracle.

Depth within 1e-3 m, variance within 1e-4 relative (+ 1e-4 * nugget), and the
neighbour lists bit-exact; see tests/gpu_util.py for where the bounds come from.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import Lib, assert_okrige

pytestmark = pytest.mark.gpu

SPH = dict(model=0, nugget=0.25, sill=100.0, range_m=50.0)


def _run(w, k, cell_hint=0, **vp):
    lib = Lib(w.x_cm, w.y_cm, w.z_m, w.grid, cell_hint=cell_hint)
    try:
        return lib.okrige(k, **vp)
    finally:
        lib.close()


def _oracle_nodes(w, qx, qy, k, model, nugget, sill, range_m):
    return oracle.okrige(w.x_cm, w.y_cm, w.z_m, qx, qy, k, model, nugget, sill, range_m,
                         want_idx=True)


def _oracle(w, k, **vp):
    g = w.grid
    qx, qy = oracle.grid_nodes(g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
    return _oracle_nodes(w, qx, qy, k, vp["model"], vp["nugget"], vp["sill"], vp["range_m"])


def test_tile_20k_k16_spherical_full_grid():
    """The 20,000-sounding 512 m tile, 256 x 256 nodes, spherical nugget 0.25 / sill 100 / range 50 m."""
    w = synth.tile(seed=1)
    d, v, nb = _run(w, 16, **SPH)
    rd, rv, ridx = _oracle(w, 16, **SPH)
    assert np.array_equal(nb, ridx)
    ed, ev = assert_okrige(d, v, rd, rv, SPH["nugget"])
    print(f"kriging k=16: max |dz| {ed:.2e} m, max |dvar| {ev:.2e} m^2")


@pytest.mark.parametrize("k,model", [(32, 0), (8, 0), (16, 1), (32, 1), (3, 0), (1, 0), (2, 1)])
def test_tile_other_k_and_models(k, model):
    w = synth.tile(seed=8, n=5000, side_cm=25_000, cell_cm=250)
    vp = dict(SPH, model=model)
    d, v, nb = _run(w, k, **vp)
    rd, rv, ridx = _oracle(w, k, **vp)
    assert np.array_equal(nb, ridx)
    assert_okrige(d, v, rd, rv, vp["nugget"])


def test_paper_exponential_model_without_nugget():
    # the variogram printed in Sec. III-C: C0 (1 - exp(-h/a)), no nugget; soundings
    # well spread (no duplicates), so the system stays non-singular
    w = synth.tile(seed=9, n=1500, side_cm=30_000, cell_cm=600)
    vp = dict(model=1, nugget=0.0, sill=100.0, range_m=50.0)
    d, v, nb = _run(w, 8, **vp)
    rd, rv, ridx = _oracle(w, 8, **vp)
    assert np.array_equal(nb, ridx)
    assert_okrige(d, v, rd, rv, 1e-3)


def test_cell_size_invariance_bitwise():
    w = synth.tile(seed=10, n=4000, side_cm=20_000, cell_cm=250)
    d0, v0, n0 = _run(w, 32, **SPH)
    for hint in (45, 333, 2500):
        d, v, nb = _run(w, 32, cell_hint=hint, **SPH)
        assert np.array_equal(nb, n0)
        assert np.array_equal(d.view(np.uint32), d0.view(np.uint32))
        assert np.array_equal(v.view(np.uint32), v0.view(np.uint32))


def test_coincident_nodes_duplicates_and_nan():
    rng = np.random.default_rng(4)
    # soundings on the node lattice (coincident nodes), duplicated positions, NaN depths
    xs = rng.integers(0, 40, 900) * 100 + 50
    ys = rng.integers(0, 40, 900) * 100 + 50
    x = np.concatenate([xs, xs[:100]]).astype(np.int32)
    y = np.concatenate([ys, ys[:100]]).astype(np.int32)
    z = (3500 + 0.01 * x / 100 + rng.normal(0, 0.5, x.size)).astype(np.float32)
    z[rng.random(x.size) < 0.1] = np.nan
    w = synth.Workload(x, y, z, synth.GridSpec(0, 0, 100, 40, 40), "coinc", {})
    for k in (4, 16, 32):
        d, v, nb = _run(w, k, **SPH)
        rd, rv, ridx = _oracle(w, k, **SPH)
        assert np.array_equal(nb, ridx)
        assert_okrige(d, v, rd, rv, SPH["nugget"])
    # nodes on a unique sounding reproduce it with zero variance
    d, v, nb = _run(w, 16, **SPH)
    qx, qy = oracle.grid_nodes(0, 0, 100, 40, 40)
    valid = ~np.isnan(z)
    pos = {}
    for i in np.flatnonzero(valid):
        pos.setdefault((int(x[i]), int(y[i])), []).append(i)
    hits = [(m, p[0]) for m, key in enumerate(zip(qx.tolist(), qy.tolist()))
            if len(p := pos.get(key, [])) == 1]
    assert len(hits) > 100
    for m, i in hits:
        assert abs(float(d[m]) - float(z[i])) <= 1e-3 and abs(float(v[m])) <= 2.5e-5


def _lattice_with_duplicates(seed):
    rng = np.random.default_rng(seed)
    xs = rng.integers(0, 40, 900) * 100 + 50
    ys = rng.integers(0, 40, 900) * 100 + 50
    x = np.concatenate([xs, xs[:100]]).astype(np.int32)
    y = np.concatenate([ys, ys[:100]]).astype(np.int32)
    z = (3500 + 0.01 * x / 100 + rng.normal(0, 0.5, x.size)).astype(np.float32)
    z[rng.random(x.size) < 0.1] = np.nan
    return synth.Workload(x, y, z, synth.GridSpec(0, 0, 100, 40, 40), "coinc", {})


@pytest.mark.parametrize("k", [32, 16, 5, 1])
def test_without_neighbour_output_the_solve_orders_the_ids(k):
    # without nbr_out the k-NN hands the ids over unsorted and the solve puts
    # them in (d2, index) order itself: results bitwise those with nbr_out
    for w in (synth.tile(seed=12, n=8000, side_cm=30_000, cell_cm=200),
              _lattice_with_duplicates(13)):
        lib = Lib(w.x_cm, w.y_cm, w.z_m, w.grid)
        try:
            d1, v1, _ = lib.okrige(k, **SPH, want_nbr=True)
            d2, v2, _ = lib.okrige(k, **SPH, want_nbr=False)
        finally:
            lib.close()
        assert np.array_equal(d1.view(np.uint32), d2.view(np.uint32))
        assert np.array_equal(v1.view(np.uint32), v2.view(np.uint32))
        rd, rv, _ = _oracle(w, k, **SPH)
        assert_okrige(d2, v2, rd, rv, SPH["nugget"])


def test_fewer_soundings_than_k_and_none_valid():
    x = np.array([0, 500, 900, 40], np.int32)
    y = np.array([0, 200, -300, 700], np.int32)
    z = np.array([3500.0, np.nan, 3510.0, 3490.0], np.float32)
    w = synth.Workload(x, y, z, synth.GridSpec(-1000, -1000, 200, 11, 9), "tiny", {})
    d, v, nb = _run(w, 16, **SPH)
    rd, rv, ridx = _oracle(w, 16, **SPH)
    assert np.array_equal(nb, ridx)
    assert_okrige(d, v, rd, rv, SPH["nugget"])
    w.z_m = np.full(4, np.nan, np.float32)
    d, v, nb = _run(w, 16, **SPH)
    assert np.all(np.isnan(d)) and np.all(np.isnan(v)) and np.all(nb == -1)


def test_wide_key_path():
    rng = np.random.default_rng(5)
    n = 1 << 20
    x = rng.integers(-(1 << 28), 1 << 28, n).astype(np.int32)
    y = rng.integers(-(1 << 28), 1 << 28, n).astype(np.int32)
    z = np.full(n, np.nan, np.float32)
    keep = rng.choice(n, 50, replace=False)
    z[keep] = rng.normal(3500, 20, 50).astype(np.float32)
    w = synth.Workload(x, y, z, synth.GridSpec(-(1 << 28), -(1 << 28), 1 << 23, 64, 64), "far", {})
    d, v, nb = _run(w, 8, **SPH)
    rd, rv, ridx = _oracle(w, 8, **SPH)
    assert np.array_equal(nb, ridx)
    assert_okrige(d, v, rd, rv, SPH["nugget"])


def test_small_swath_k32_sampled_nodes_including_gaps():
    w = synth.swath(seed=2, lines=2, pings=600, beams=256)
    d, v, nb = _run(w, 32, **SPH)
    g = w.grid
    rng = np.random.default_rng(2)
    sel = rng.choice(g.m, 1500, replace=False)
    qx = (g.x0_cm + (sel % g.nx) * g.cell_cm + g.cell_cm // 2).astype(np.int32)
    qy = (g.y0_cm + (sel // g.nx) * g.cell_cm + g.cell_cm // 2).astype(np.int32)
    assert ((qy > 36_000) & (qy < 48_000)).sum() > 100
    rd, rv, ridx = _oracle_nodes(w, qx, qy, 32, **{"model": 0, "nugget": 0.25, "sill": 100.0,
                                                   "range_m": 50.0})
    assert np.array_equal(nb[sel], ridx)
    assert_okrige(d[sel], v[sel], rd, rv, SPH["nugget"])


@pytest.mark.parametrize("k", [32, 16])
def test_neighbour_output_at_an_unaligned_address(k):
    """nbr_out 4 bytes past a 16-byte boundary: the k-NN kernels store ids four
    at a time only into aligned buffers, so here they fall back to one at a
    time; ids and grids equal those of an aligned buffer (IDW and kriging)."""
    import torch

    import paper_2505_22675_gb300 as bg
    w = synth.tile(seed=8, n=5000, side_cm=25_000, cell_cm=250)
    lib = Lib(w.x_cm, w.y_cm, w.z_m, w.grid)
    try:
        m = w.grid.nx * w.grid.ny
        d_al, v_al, nb_al = lib.okrige(k)
        i_al, ib_al = lib.idw(k, 2.0)
        raw = torch.full((m * k + 4,), -9, dtype=torch.int32, device=lib.dev)
        nb = raw[1:1 + m * k]
        assert nb.data_ptr() % 16 == 4
        d = torch.empty(m, device=lib.dev)
        v = torch.empty(m, device=lib.dev)
        bg.interp_okrige(lib.s, lib.grid, k, bg.variogram(0, 0.25, 100.0, 50.0), d, v, nb)
        torch.cuda.synchronize()
        assert np.array_equal(nb.cpu().numpy().reshape(m, k), nb_al)
        assert np.array_equal(d.cpu().numpy().view(np.uint32), d_al.view(np.uint32))
        assert np.array_equal(v.cpu().numpy().view(np.uint32), v_al.view(np.uint32))
        assert raw[0].item() == -9 and raw[1 + m * k].item() == -9
        raw.fill_(-9)
        bg.interp_idw(lib.s, lib.grid, k, 2.0, d, nb)
        torch.cuda.synchronize()
        assert np.array_equal(nb.cpu().numpy().reshape(m, k), ib_al)
        assert np.array_equal(d.cpu().numpy().view(np.uint32), i_al.view(np.uint32))
        assert raw[0].item() == -9 and raw[1 + m * k].item() == -9
    finally:
        lib.close()
