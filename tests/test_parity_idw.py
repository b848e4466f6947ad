"""GPU parity of the fused k-NN + IDW path against the FP64 oracle (C ABI).

Neighbour lists must match bit-exactly, depths within the IDW tolerance of
tests/gpu_util.py. Sizes span many 16 x 8 node patches and ragged edges.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import Lib, assert_idw

pytestmark = pytest.mark.gpu


def _run(w, k, power, cell_hint=0, on_device=True):
    lib = Lib(w.x_cm, w.y_cm, w.z_m, w.grid, cell_hint=cell_hint, on_device=on_device)
    try:
        d, nb = lib.idw(k, power)
    finally:
        lib.close()
    return d, nb


def _oracle(w, k, power):
    g = w.grid
    qx, qy = oracle.grid_nodes(g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
    return oracle.idw(w.x_cm, w.y_cm, w.z_m, qx, qy, k, power, want_idx=True)


def test_tile_20k_k8_p2_full_grid():
    """The 20,000-sounding 512 m tile, 256 x 256 nodes at 2 m, IDW p=2 k=8."""
    w = synth.tile(seed=1)
    d, nb = _run(w, 8, 2.0)
    ref, ridx = _oracle(w, 8, 2.0)
    assert np.array_equal(nb, ridx)
    assert_idw(d, ref)


@pytest.mark.parametrize("k,power", [(16, 2.0), (16, 1.0), (5, 3.0), (32, 2.0), (1, 2.0)])
def test_tile_other_k_and_powers(k, power):
    w = synth.tile(seed=4, n=6000, side_cm=30_000, cell_cm=300)
    d, nb = _run(w, k, power)
    ref, ridx = _oracle(w, k, power)
    assert np.array_equal(nb, ridx)
    assert_idw(d, ref)


def test_results_do_not_depend_on_cell_size():
    w = synth.tile(seed=5, n=5000, side_cm=25_000, cell_cm=250)
    base_d, base_nb = _run(w, 16, 2.0)
    for hint in (37, 180, 900, 7000):
        d, nb = _run(w, 16, 2.0, cell_hint=hint)
        assert np.array_equal(nb, base_nb), hint
        assert np.array_equal(d.view(np.uint32), base_d.view(np.uint32)), hint


def test_host_and_device_upload_agree():
    w = synth.tile(seed=6, n=3000, side_cm=20_000, cell_cm=400)
    d1, n1 = _run(w, 8, 2.0, on_device=True)
    d2, n2 = _run(w, 8, 2.0, on_device=False)
    assert np.array_equal(n1, n2) and np.array_equal(d1.view(np.uint32), d2.view(np.uint32))


def test_ragged_grid_outside_and_around_the_data():
    # grid larger than the data extent, not a multiple of the 16 x 8 patch
    w = synth.tile(seed=7, n=2500, side_cm=20_000, cell_cm=400)
    w.grid = synth.GridSpec(-3_000, -1_500, 600, 37, 43)
    d, nb = _run(w, 8, 2.0)
    ref, ridx = _oracle(w, 8, 2.0)
    assert np.array_equal(nb, ridx)
    assert_idw(d, ref)


def test_lattice_ties_duplicates_and_nan():
    # integer lattice: many exactly equidistant soundings; duplicates; NaN depths
    xs, ys = np.meshgrid(np.arange(30) * 100, np.arange(30) * 100)
    x = np.concatenate([xs.ravel(), xs.ravel()[:200]]).astype(np.int32)
    y = np.concatenate([ys.ravel(), ys.ravel()[:200]]).astype(np.int32)
    rng = np.random.default_rng(0)
    perm = rng.permutation(x.size)
    x, y = x[perm], y[perm]
    z = (3500 + rng.normal(size=x.size)).astype(np.float32)
    z[rng.random(x.size) < 0.15] = np.nan
    w = synth.Workload(x, y, z, synth.GridSpec(-100, -100, 50, 70, 66), "lattice", {})
    for k in (4, 12, 32):
        d, nb = _run(w, k, 2.0, cell_hint=100)
        ref, ridx = _oracle(w, k, 2.0)
        assert np.array_equal(nb, ridx), k
        assert_idw(d, ref)


def test_fewer_soundings_than_k_and_none_valid():
    x = np.array([0, 500, 900], np.int32)
    y = np.array([0, 200, -300], np.int32)
    z = np.array([3500.0, np.nan, 3510.0], np.float32)
    w = synth.Workload(x, y, z, synth.GridSpec(-1000, -1000, 200, 11, 9), "tiny", {})
    d, nb = _run(w, 8, 2.0)
    ref, ridx = _oracle(w, 8, 2.0)
    assert np.array_equal(nb, ridx)
    assert_idw(d, ref)
    w.z_m = np.full(3, np.nan, np.float32)
    d, nb = _run(w, 8, 2.0)
    assert np.all(np.isnan(d)) and np.all(nb == -1)
    w.x_cm = w.x_cm[:0]
    w.y_cm = w.y_cm[:0]
    w.z_m = w.z_m[:0]
    d, nb = _run(w, 3, 2.0)
    assert np.all(np.isnan(d)) and np.all(nb == -1)


def test_one_node_grid_and_coincident_node():
    x = np.array([100, 100, 300, 700], np.int32)
    y = np.array([100, 100, 300, 900], np.int32)
    z = np.array([3400.5, 3401.0, 3402.0, 3403.0], np.float32)
    w = synth.Workload(x, y, z, synth.GridSpec(0, 0, 200, 1, 1), "one", {})  # node at (100, 100)
    d, nb = _run(w, 3, 2.0)
    assert d[0] == np.float32(3400.5) and list(nb[0]) == [0, 1, 2]


def test_wide_key_path_far_apart_soundings():
    # 2^20 uploaded soundings (20 index bits) of which 60 are valid and lie
    # thousands of km apart: d2 needs more than 44 bits, so the wide-key pass
    # handles every node.
    rng = np.random.default_rng(3)
    n = 1 << 20
    x = rng.integers(-(1 << 29), 1 << 29, n).astype(np.int32)
    y = rng.integers(-(1 << 29), 1 << 29, n).astype(np.int32)
    z = np.full(n, np.nan, np.float32)
    keep = rng.choice(n, 60, replace=False)
    z[keep] = rng.normal(3500, 20, 60).astype(np.float32)
    w = synth.Workload(x, y, z, synth.GridSpec(-(1 << 29), -(1 << 29), 1 << 24, 64, 64), "far", {})
    d, nb = _run(w, 8, 2.0)
    ref, ridx = _oracle(w, 8, 2.0)
    assert np.array_equal(nb, ridx)
    assert_idw(d, ref)


def test_small_swath_sampled_nodes_including_gaps():
    """Two survey lines with the inter-line gap; nodes sampled across swath, edges and gap."""
    w = synth.swath(seed=2, lines=2, pings=600, beams=256)
    lib = Lib(w.x_cm, w.y_cm, w.z_m, w.grid)
    try:
        d, nb = lib.idw(16, 2.0)
    finally:
        lib.close()
    g = w.grid
    rng = np.random.default_rng(1)
    sel = rng.choice(g.m, 2500, replace=False)
    qx = (g.x0_cm + (sel % g.nx) * g.cell_cm + g.cell_cm // 2).astype(np.int32)
    qy = (g.y0_cm + (sel // g.nx) * g.cell_cm + g.cell_cm // 2).astype(np.int32)
    gap = (qy > 36_000) & (qy < 48_000)
    assert gap.sum() > 200  # the gap between the swaths is exercised
    ref, ridx = oracle.idw(w.x_cm, w.y_cm, w.z_m, qx, qy, 16, 2.0, want_idx=True)
    assert np.array_equal(nb[sel], ridx)
    assert_idw(d[sel], ref)
