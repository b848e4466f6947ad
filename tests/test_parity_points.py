"""Point queries (bg_interp_idw_points / bg_interp_okrige_points) against the
oracle, and against the grid entry points on the same nodes.

The oracle takes arbitrary query points, so every case compares element by
element: neighbour ids bit-exact, depths and variances within the shared
tolerances. Cases: random points over and around a tile (several blocks and
a ragged tail), the holes of a gridded product in scan order (the paper's
hole filling, Sec. IV Grid B), grid nodes passed as points (bitwise equal to
the grid call), shuffled order (results do not depend on the chain bound),
points outside the coordinate range, far from the data (wide keys), and an
empty list.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_idw, assert_okrige

pytestmark = pytest.mark.gpu

VGM = (0, 0.25, 100.0, 50.0)


class PLib:
    def __init__(self, x, y, z):
        import torch

        import paper_2505_22675_gb300 as bg
        self.bg, self.torch = bg, torch
        self.dev = torch.device("cuda:0")
        self.ctx = bg.ctx_create(0)
        self.s = bg.soundings_upload(self.ctx, *(torch.from_numpy(np.ascontiguousarray(a)).to(self.dev)
                                                 for a in (x, y, z)))

    def _q(self, qx, qy):
        t = self.torch
        return (t.from_numpy(np.ascontiguousarray(qx, dtype=np.int32)).to(self.dev),
                t.from_numpy(np.ascontiguousarray(qy, dtype=np.int32)).to(self.dev))

    def idw(self, qx, qy, k, power=2.0):
        t = self.torch
        m = len(qx)
        dx, dy = self._q(qx, qy)
        d = t.full((m,), -7.0, device=self.dev)
        nb = t.full((m * k,), -9, dtype=t.int32, device=self.dev)
        self.bg.interp_idw_points(self.s, dx, dy, k, power, d, nb)
        t.cuda.synchronize()
        return d.cpu().numpy(), nb.cpu().numpy().reshape(m, k)

    def okrige(self, qx, qy, k, vgm=VGM, want_nbr=True):
        t = self.torch
        m = len(qx)
        dx, dy = self._q(qx, qy)
        d = t.full((m,), -7.0, device=self.dev)
        v = t.full((m,), -7.0, device=self.dev)
        nb = t.full((m * k,), -9, dtype=t.int32, device=self.dev) if want_nbr else None
        self.bg.interp_okrige_points(self.s, dx, dy, k, self.bg.variogram(*vgm), d, v, nb)
        t.cuda.synchronize()
        return d.cpu().numpy(), v.cpu().numpy(), (nb.cpu().numpy().reshape(m, k) if want_nbr else None)

    def close(self):
        self.bg.soundings_destroy(self.s)
        self.bg.ctx_destroy(self.ctx)


def _check(lib, x, y, z, qx, qy, k_idw=16, k_ok=32, vgm=VGM):
    d, nb = lib.idw(qx, qy, k_idw)
    ref_i = oracle.knn(x, y, z, qx, qy, k_idw)[0]
    assert np.array_equal(nb, ref_i)
    assert_idw(d, oracle.idw(x, y, z, qx, qy, k_idw, 2.0))
    od, ov, onb = lib.okrige(qx, qy, k_ok, vgm)
    assert np.array_equal(onb, oracle.knn(x, y, z, qx, qy, k_ok)[0])
    rd, rv = oracle.okrige(x, y, z, qx, qy, k_ok, *vgm)
    assert_okrige(od, ov, rd, rv, vgm[1])
    return d, od, ov


def test_random_points_over_and_around_a_tile():
    w = synth.tile(seed=21, n=6000, side_cm=30_000, cell_cm=200)
    qx, qy = synth.random_points(22, w.grid, 3001, margin_cells=8)  # ragged: 3001 = 5 blocks + tail
    lib = PLib(w.x_cm, w.y_cm, w.z_m)
    try:
        _check(lib, w.x_cm, w.y_cm, w.z_m, qx, qy)
    finally:
        lib.close()


def test_hole_filling_in_scan_order_and_shuffled():
    h = synth.hole_grid(seed=23, nx=96, ny=80, cell_cm=200, frac=0.1)
    s = h.soundings()
    qx, qy = h.queries()
    lib = PLib(s.x_cm, s.y_cm, s.z_m)
    try:
        d, od, ov = _check(lib, s.x_cm, s.y_cm, s.z_m, qx, qy)
        perm = np.random.default_rng(0).permutation(qx.size)
        d2, _ = lib.idw(qx[perm], qy[perm], 16)
        od2, ov2, _ = lib.okrige(qx[perm], qy[perm], 32, want_nbr=False)  # ids unsorted
        assert np.array_equal(d2.view(np.uint32), d[perm].view(np.uint32))
        assert np.array_equal(od2.view(np.uint32), od[perm].view(np.uint32))
        assert np.array_equal(ov2.view(np.uint32), ov[perm].view(np.uint32))
        # kriging fills the holes of a smooth surface far better than the trend alone
        err = np.abs(od.astype(np.float64) - h.truth())
        assert np.sqrt(np.mean(err ** 2)) < 0.5
    finally:
        lib.close()


def test_grid_nodes_as_points_equal_the_grid_call():
    import torch

    import paper_2505_22675_gb300 as bg
    w = synth.tile(seed=24, n=5000, side_cm=25_600, cell_cm=200)
    g = w.grid
    qx, qy = oracle.grid_nodes(g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
    lib = PLib(w.x_cm, w.y_cm, w.z_m)
    try:
        grid = bg.grid_create(lib.ctx, g.x0_cm, g.y0_cm, g.cell_cm, g.nx, g.ny)
        dev = lib.dev
        gd = torch.empty(g.m, device=dev)
        bg.interp_idw(lib.s, grid, 16, 2.0, gd)
        gok = torch.empty(g.m, device=dev)
        gov = torch.empty(g.m, device=dev)
        bg.interp_okrige(lib.s, grid, 32, bg.variogram(*VGM), gok, gov)
        torch.cuda.synchronize()
        bg.grid_destroy(grid)
        d, _ = lib.idw(qx, qy, 16)
        od, ov, _ = lib.okrige(qx, qy, 32)
        assert np.array_equal(d.view(np.uint32), gd.cpu().numpy().view(np.uint32))
        assert np.array_equal(od.view(np.uint32), gok.cpu().numpy().view(np.uint32))
        assert np.array_equal(ov.view(np.uint32), gov.cpu().numpy().view(np.uint32))
    finally:
        lib.close()


def test_out_of_range_far_coincident_duplicate_and_empty():
    w = synth.tile(seed=25, n=3000, side_cm=20_000, cell_cm=200)
    lim = 1 << 30
    qx = np.array([w.x_cm[0], w.x_cm[0], 5000, -lim, lim - 1, 0, lim - 2, -(lim - 2), 7000],
                  dtype=np.int64)
    qy = np.array([w.y_cm[0], w.y_cm[0], 5000, 0, 0, lim, lim - 2, -(lim - 2), 7000],
                  dtype=np.int64)
    bad = (np.abs(qx) >= lim) | (np.abs(qy) >= lim)
    qx32, qy32 = qx.astype(np.int32), qy.astype(np.int32)
    lib = PLib(w.x_cm, w.y_cm, w.z_m)
    try:
        d, nb = lib.idw(qx32, qy32, 8)
        od, ov, onb = lib.okrige(qx32, qy32, 16)
        assert np.isnan(d[bad]).all() and np.isnan(od[bad]).all() and np.isnan(ov[bad]).all()
        assert (nb[bad] == -1).all() and (onb[bad] == -1).all()
        ok = ~bad
        ref_i = oracle.knn(w.x_cm, w.y_cm, w.z_m, qx32[ok], qy32[ok], 8)[0]
        assert np.array_equal(nb[ok], ref_i)
        assert_idw(d[ok], oracle.idw(w.x_cm, w.y_cm, w.z_m, qx32[ok], qy32[ok], 8, 2.0))
        rd, rv = oracle.okrige(w.x_cm, w.y_cm, w.z_m, qx32[ok], qy32[ok], 16, *VGM)
        assert_okrige(od[ok], ov[ok], rd, rv, VGM[1])
        # a query on a sounding returns its depth with zero variance
        assert d[0] == w.z_m[0] and od[0] == w.z_m[0] and ov[0] == 0.0
        # an empty list is a no-op
        e, _ = lib.idw(np.zeros(0, np.int32), np.zeros(0, np.int32), 8)
        assert e.size == 0
    finally:
        lib.close()
