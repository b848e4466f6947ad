"""Helpers for the GPU parity tests: run the library through its C ABI and
compare with the FP64 oracle under the tolerances the tests share.

Tolerances (derived from the arithmetic; the paper states none):
  - neighbour sets: bit-exact, including order;
  - IDW depth: |gpu - oracle| <= 1e-4 m + half an fp32 ulp of the oracle value
    (an fp32 output cannot hold 1e-4 m at 2048-4096 m, where half an ulp is
    1.22e-4 m);
  - kriging depth: <= 1e-3 m absolute;
  - kriging variance: <= 1e-4 * sigma^2_oracle + 1e-4 * nugget (a relative
    bound alone is undefined at sigma^2 = 0, a node on a sounding).
"""
from __future__ import annotations

import numpy as np

IDW_ABS = 1e-4
OK_DEPTH_ABS = 1e-3
OK_VAR_REL = 1e-4


def half_ulp32(v):
    return 0.5 * np.spacing(np.abs(np.asarray(v, dtype=np.float64)).astype(np.float32)).astype(np.float64)


def idw_tol(ref):
    return IDW_ABS + half_ulp32(ref)


def var_tol(ref_var, nugget):
    return OK_VAR_REL * np.abs(ref_var) + OK_VAR_REL * nugget


class Lib:
    """One context, device-resident soundings and a grid, for a test."""

    def __init__(self, x_cm, y_cm, z_m, grid, cell_hint=0, on_device=True):
        import torch

        import paper_2505_22675_gb300 as bg
        self.bg = bg
        self.torch = torch
        self.dev = torch.device("cuda:0")
        self.ctx = bg.ctx_create(0)
        self.g = grid
        self.grid = bg.grid_create(self.ctx, grid.x0_cm, grid.y0_cm, grid.cell_cm, grid.nx, grid.ny)
        if on_device:
            xs = [torch.from_numpy(np.ascontiguousarray(a)).to(self.dev) for a in (x_cm, y_cm, z_m)]
        else:
            xs = [np.ascontiguousarray(a) for a in (x_cm, y_cm, z_m)]
        self.s = bg.soundings_upload(self.ctx, *xs, cell_cm_hint=cell_hint)
        self.info = bg.soundings_info(self.s)

    def idw(self, k, power, want_nbr=True):
        t = self.torch
        m = self.g.nx * self.g.ny
        d = t.empty(m, device=self.dev)
        nb = t.empty(m * k, dtype=t.int32, device=self.dev) if want_nbr else None
        self.bg.interp_idw(self.s, self.grid, k, power, d, nb)
        t.cuda.synchronize()
        return d.cpu().numpy(), (nb.cpu().numpy().reshape(m, k) if want_nbr else None)

    def okrige(self, k, model=0, nugget=0.25, sill=100.0, range_m=50.0, want_nbr=True):
        t = self.torch
        m = self.g.nx * self.g.ny
        d = t.empty(m, device=self.dev)
        v = t.empty(m, device=self.dev)
        nb = t.empty(m * k, dtype=t.int32, device=self.dev) if want_nbr else None
        self.bg.interp_okrige(self.s, self.grid, k, self.bg.variogram(model, nugget, sill, range_m),
                              d, v, nb)
        t.cuda.synchronize()
        return d.cpu().numpy(), v.cpu().numpy(), (nb.cpu().numpy().reshape(m, k) if want_nbr else None)

    def close(self):
        self.bg.soundings_destroy(self.s)
        self.bg.grid_destroy(self.grid)
        self.bg.ctx_destroy(self.ctx)


def assert_idw(got, ref):
    got = np.asarray(got, dtype=np.float64)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan), "NaN pattern differs"
    err = np.abs(got[~nan] - ref[~nan])
    bad = err > idw_tol(ref[~nan])
    assert not bad.any(), f"{bad.sum()} IDW depths over tolerance; max err {err.max():.3e} m"
    return float(err.max()) if err.size else 0.0


def assert_okrige(gd, gv, rd, rv, nugget):
    gd = np.asarray(gd, dtype=np.float64)
    gv = np.asarray(gv, dtype=np.float64)
    nan = np.isnan(rd)
    assert np.array_equal(np.isnan(gd), nan), "NaN pattern differs (depth)"
    ed = np.abs(gd[~nan] - rd[~nan])
    ev = np.abs(gv[~nan] - rv[~nan])
    assert not (ed > OK_DEPTH_ABS).any(), \
        f"{(ed > OK_DEPTH_ABS).sum()} kriging depths over 1e-3 m; max {ed.max():.3e}"
    badv = ev > var_tol(rv[~nan], nugget)
    assert not badv.any(), f"{badv.sum()} kriging variances over tolerance; worst rel " \
        f"{np.max(ev / np.maximum(np.abs(rv[~nan]), 1e-30)):.3e}"
    return (float(ed.max()) if ed.size else 0.0, float(ev.max()) if ev.size else 0.0)
