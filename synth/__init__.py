"""Seeded synthetic sounding workloads shared by the oracle tests and the GPU path.

This module only draws inputs: positions, depths and grid descriptions. It
holds none of the gridding arithmetic (no neighbour search, no weights, no
variogram), so both sides of a parity test can read the same inputs without
sharing any of the method.

Every generator takes an integer seed and uses numpy's PCG64 bit generator.
Coordinates are int32 centimetres rounded as floor(v * 100 + 0.5) from
metres; depths are float32 metres, positive down.

Seafloor model (all workloads): depth = 3500 + 0.01 * x
+ sum_b A_b * exp(-r_b^2 / (2 sigma_b^2)) + N(0, 0.5^2), with x, y in metres,
A_b ~ U(-30, 30) m, sigma_b ~ U(10, 60) m and bump centres uniform over the
extent. The paper evaluates on GEBCO bathymetry grids that are not available
here; these seeded surfaces stand in for them (same depth range, relief
scales of tens of metres, sounding-level noise).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "GridSpec", "Workload", "HoleGrid", "bumps", "seafloor", "to_cm", "tile", "rect", "swath",
    "batched_tiles", "hole_grid", "row_midpoints", "random_points",
]

BUMP_DENSITY_PER_M2 = 40.0 / (512.0 * 512.0)


@dataclasses.dataclass(frozen=True)
class GridSpec:
    """Regular output grid: node (i, j) sits at (x0 + i*cell + cell/2, y0 + j*cell + cell/2) cm."""
    x0_cm: int
    y0_cm: int
    cell_cm: int
    nx: int
    ny: int

    @property
    def m(self) -> int:
        return self.nx * self.ny


@dataclasses.dataclass
class Workload:
    x_cm: np.ndarray      # int32[N]
    y_cm: np.ndarray      # int32[N]
    z_m: np.ndarray       # float32[N]
    grid: GridSpec
    name: str
    params: dict


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def to_cm(v_m: np.ndarray) -> np.ndarray:
    """Round metres to int32 centimetres as floor(v*100 + 0.5)."""
    return np.floor(np.asarray(v_m, dtype=np.float64) * 100.0 + 0.5).astype(np.int32)


def bumps(rng: np.random.Generator, x_lo: float, x_hi: float, y_lo: float, y_hi: float,
          count: int | None = None) -> np.ndarray:
    """Gaussian bump table [count, 4] = (cx_m, cy_m, amp_m, sigma_m)."""
    if count is None:
        count = max(1, int(round(BUMP_DENSITY_PER_M2 * (x_hi - x_lo) * (y_hi - y_lo))))
    cx = rng.uniform(x_lo, x_hi, count)
    cy = rng.uniform(y_lo, y_hi, count)
    amp = rng.uniform(-30.0, 30.0, count)
    sig = rng.uniform(10.0, 60.0, count)
    return np.stack([cx, cy, amp, sig], axis=1)


def _bump_field_direct(x_m, y_m, table):
    out = np.zeros_like(x_m, dtype=np.float64)
    for cx, cy, a, s in table:
        r2 = (x_m - cx) ** 2 + (y_m - cy) ** 2
        out += a * np.exp(-r2 / (2.0 * s * s))
    return out


def _bump_field_raster(x_m, y_m, table, res_m=1.0, cut_sigmas=5.0):
    """Bump field sampled on a res_m raster (bumps cut at cut_sigmas) and read bilinearly.

    Used for the large swath, where evaluating every bump at every sounding
    would take minutes in numpy. The cut leaves a step below 4e-6 * |A_b|.
    """
    x_lo, x_hi = float(x_m.min()) - 2 * res_m, float(x_m.max()) + 2 * res_m
    y_lo, y_hi = float(y_m.min()) - 2 * res_m, float(y_m.max()) + 2 * res_m
    nxr = int(math.ceil((x_hi - x_lo) / res_m)) + 2
    nyr = int(math.ceil((y_hi - y_lo) / res_m)) + 2
    field = np.zeros((nyr, nxr), dtype=np.float64)
    for cx, cy, a, s in table:
        rad = cut_sigmas * s
        i0 = max(0, int(math.floor((cx - rad - x_lo) / res_m)))
        i1 = min(nxr, int(math.ceil((cx + rad - x_lo) / res_m)) + 1)
        j0 = max(0, int(math.floor((cy - rad - y_lo) / res_m)))
        j1 = min(nyr, int(math.ceil((cy + rad - y_lo) / res_m)) + 1)
        if i0 >= i1 or j0 >= j1:
            continue
        gx = x_lo + res_m * np.arange(i0, i1)
        gy = y_lo + res_m * np.arange(j0, j1)
        ex = np.exp(-((gx - cx) ** 2) / (2 * s * s))
        ey = np.exp(-((gy - cy) ** 2) / (2 * s * s))
        field[j0:j1, i0:i1] += a * np.outer(ey, ex)
    fx = (x_m - x_lo) / res_m
    fy = (y_m - y_lo) / res_m
    ix = np.clip(np.floor(fx).astype(np.int64), 0, nxr - 2)
    iy = np.clip(np.floor(fy).astype(np.int64), 0, nyr - 2)
    tx = fx - ix
    ty = fy - iy
    f00 = field[iy, ix]
    f10 = field[iy, ix + 1]
    f01 = field[iy + 1, ix]
    f11 = field[iy + 1, ix + 1]
    return (f00 * (1 - tx) * (1 - ty) + f10 * tx * (1 - ty)
            + f01 * (1 - tx) * ty + f11 * tx * ty)


def seafloor(x_m: np.ndarray, y_m: np.ndarray, table: np.ndarray,
             rng: np.random.Generator | None = None, noise_m: float = 0.5) -> np.ndarray:
    """Depth in metres (float64) of the synthetic seafloor at (x_m, y_m), plus noise."""
    x_m = np.asarray(x_m, dtype=np.float64)
    y_m = np.asarray(y_m, dtype=np.float64)
    if x_m.size * len(table) <= 4e7:
        field = _bump_field_direct(x_m, y_m, table)
    else:
        field = _bump_field_raster(x_m, y_m, table)
    d = 3500.0 + 0.01 * x_m + field
    if rng is not None and noise_m > 0:
        d = d + rng.normal(0.0, noise_m, x_m.shape)
    return d


def tile(seed: int = 1, n: int = 20_000, side_cm: int = 51_200, cell_cm: int = 200,
         n_bumps: int = 40, x0_cm: int = 0, y0_cm: int = 0) -> Workload:
    """Uniform soundings over a square tile [x0, x0+side) x [y0, y0+side) cm.

    Defaults: the 20,000-sounding 512 m tile with 40 bumps, gridded 256 x 256
    at 2 m.
    """
    rng = _rng(seed)
    x = rng.integers(0, side_cm, n, dtype=np.int64) + x0_cm
    y = rng.integers(0, side_cm, n, dtype=np.int64) + y0_cm
    table = bumps(rng, x0_cm / 100.0, (x0_cm + side_cm) / 100.0,
                  y0_cm / 100.0, (y0_cm + side_cm) / 100.0, count=n_bumps)
    z = seafloor(x / 100.0, y / 100.0, table, rng)
    nx = side_cm // cell_cm
    grid = GridSpec(x0_cm, y0_cm, cell_cm, nx, nx)
    return Workload(x.astype(np.int32), y.astype(np.int32), z.astype(np.float32), grid,
                    f"tile{n}", dict(seed=seed, n=n, side_cm=side_cm, cell_cm=cell_cm))


def rect(seed: int, n: int, x0_cm: int, y0_cm: int, w_cm: int, h_cm: int, grid: GridSpec,
         n_bumps: int = 40) -> Workload:
    """Uniform soundings over the rectangle [x0, x0+w) x [y0, y0+h) cm with
    the seafloor model (n_bumps bumps over the rectangle), gridded on `grid`.
    Long thin rectangles give the extreme aspect ratios that stress a hash's
    cell-size choice."""
    rng = _rng(seed)
    x = rng.integers(0, w_cm, n, dtype=np.int64) + x0_cm
    y = rng.integers(0, h_cm, n, dtype=np.int64) + y0_cm
    table = bumps(rng, x0_cm / 100.0, (x0_cm + w_cm) / 100.0,
                  y0_cm / 100.0, (y0_cm + h_cm) / 100.0, count=n_bumps)
    z = seafloor(x / 100.0, y / 100.0, table, rng)
    return Workload(x.astype(np.int32), y.astype(np.int32), z.astype(np.float32), grid, "rect",
                    dict(seed=seed, n=n, x0_cm=x0_cm, y0_cm=y0_cm, w_cm=w_cm, h_cm=h_cm))


def swath(seed: int = 2, lines: int = 4, pings: int = 20_000, beams: int = 256,
          altitude_m: float = 100.0, fan_deg: float = 60.0, ping_step_m: float = 0.5,
          line_spacing_m: float = 500.0, jitter_m: float = 1.0, cell_cm: int = 50) -> Workload:
    """Multibeam survey: `lines` parallel tracks along +x, `pings` pings each.

    Beam b of a ping points at theta_b, equiangular over [-fan, +fan]; its
    across-track offset is altitude * tan(theta_b). Every sounding gets an
    independent uniform +-jitter in x and y. Line l runs at
    y = half_width + l * line_spacing, so the first swath starts at y ~ 0.
    The output grid is the nominal coverage box (track length x
    (2*half_width + (lines-1)*spacing)) at `cell_cm`.
    Soundings are ordered line-major, then ping, then beam, as logged.
    """
    rng = _rng(seed)
    theta = np.deg2rad(np.linspace(-fan_deg, fan_deg, beams))
    across = altitude_m * np.tan(theta)
    half_w = float(across.max())
    xs = []
    ys = []
    for line in range(lines):
        yc = half_w + line * line_spacing_m
        px = np.arange(pings, dtype=np.float64) * ping_step_m
        x = np.repeat(px, beams)
        y = np.tile(yc + across, pings)
        x = x + rng.uniform(-jitter_m, jitter_m, x.size)
        y = y + rng.uniform(-jitter_m, jitter_m, y.size)
        xs.append(x)
        ys.append(y)
    x = np.concatenate(xs)
    y = np.concatenate(ys)
    length_m = pings * ping_step_m
    width_m = 2 * half_w + (lines - 1) * line_spacing_m
    table = bumps(rng, 0.0, length_m, 0.0, width_m)
    x_cm = to_cm(x)
    y_cm = to_cm(y)
    z = seafloor(x_cm / 100.0, y_cm / 100.0, table, rng)
    nx = int(round(length_m * 100)) // cell_cm
    ny = int(math.floor(width_m * 100 / cell_cm))
    grid = GridSpec(0, 0, cell_cm, nx, ny)
    return Workload(x_cm, y_cm, z.astype(np.float32), grid,
                    f"swath{lines}x{pings}x{beams}",
                    dict(seed=seed, lines=lines, pings=pings, beams=beams, cell_cm=cell_cm,
                         line_spacing_m=line_spacing_m))


def batched_tiles(seed: int = 3, count: int = 512, median_n: int = 20_000, sigma_ln: float = 1.0,
                  n_min: int = 1_000, n_max: int = 200_000,
                  sides=(64, 128, 256, 512, 1024), cells_m=(1, 2, 3, 4),
                  scale: float = 1.0):
    """Tiles of uneven size for batched and serving runs.

    N ~ lognormal(median, sigma_ln) clipped to [n_min, n_max]; grid side from
    `sides`, cell from `cells_m`, extent = side * cell; soundings uniform over
    the extent; method alternates by a fair coin (0 = IDW k=16, 1 = kriging
    k=32). `scale` < 1 shrinks N and the grid side for quick tests.
    Returns a list of (Workload, method).
    """
    rng = _rng(seed)
    out = []
    for t in range(count):
        n = int(np.clip(round(median_n * math.exp(sigma_ln * rng.standard_normal())), n_min, n_max))
        side = int(rng.choice(sides))
        cell_m = int(rng.choice(cells_m))
        method = int(rng.integers(0, 2))
        tseed = int(rng.integers(0, 2**31 - 1))
        if scale != 1.0:
            n = max(16, int(n * scale))
            side = max(8, int(side * math.sqrt(scale)))
        w = tile(seed=tseed, n=n, side_cm=side * cell_m * 100, cell_cm=cell_m * 100,
                 n_bumps=max(1, int(round(BUMP_DENSITY_PER_M2 * (side * cell_m) ** 2))))
        w.name = f"batch{t}"
        out.append((w, method))
    return out


# ------------------------------------------------------- gridded workloads

@dataclasses.dataclass
class HoleGrid:
    """A regular depth grid with a random fraction of its nodes removed.

    grid: the node lattice; z_full: float32 [ny * nx] true depths, row-major;
    holes: sorted int64 indices of the removed nodes.
    """
    grid: GridSpec
    z_full: np.ndarray
    holes: np.ndarray
    frac: float
    seed: int

    def node_xy(self, idx: np.ndarray):
        g = self.grid
        i = idx % g.nx
        j = idx // g.nx
        return ((g.x0_cm + i * g.cell_cm + g.cell_cm // 2).astype(np.int32),
                (g.y0_cm + j * g.cell_cm + g.cell_cm // 2).astype(np.int32))

    def kept(self) -> np.ndarray:
        mask = np.ones(self.grid.m, dtype=bool)
        mask[self.holes] = False
        return np.flatnonzero(mask)

    def soundings(self) -> Workload:
        """The kept nodes as soundings (row-major order)."""
        idx = self.kept()
        x, y = self.node_xy(idx)
        return Workload(x, y, self.z_full[idx].copy(), self.grid, f"holes{self.frac}",
                        dict(seed=self.seed, frac=self.frac))

    def queries(self):
        """(qx_cm, qy_cm) of the removed nodes, in row-major order."""
        return self.node_xy(self.holes)

    def truth(self) -> np.ndarray:
        return self.z_full[self.holes]

    def source(self) -> np.ndarray:
        """The grid as float32 [ny * nx] with NaN at the removed nodes."""
        z = self.z_full.copy()
        z[self.holes] = np.nan
        return z

    def with_frac(self, frac: float, seed: int) -> "HoleGrid":
        """The same depths with another random removal (seeded)."""
        m = self.grid.m
        holes = np.sort(_rng(seed).choice(m, size=int(round(frac * m)), replace=False))
        return HoleGrid(self.grid, self.z_full, holes.astype(np.int64), frac, seed)


def _lattice_field(x_m: np.ndarray, y_m: np.ndarray, table: np.ndarray, cut_sigmas=5.0):
    """Bump field on the lattice x_m (columns) by y_m (rows), both ascending and
    evenly spaced: each Gaussian is separable, so it is added as an outer
    product over the window of nodes within cut_sigmas of its centre."""
    field = np.zeros((y_m.size, x_m.size), dtype=np.float64)
    dx = x_m[1] - x_m[0] if x_m.size > 1 else 1.0
    dy = y_m[1] - y_m[0] if y_m.size > 1 else 1.0
    for cx, cy, a, s in table:
        rad = cut_sigmas * s
        i0 = max(0, int(math.floor((cx - rad - x_m[0]) / dx)))
        i1 = min(x_m.size, int(math.ceil((cx + rad - x_m[0]) / dx)) + 1)
        j0 = max(0, int(math.floor((cy - rad - y_m[0]) / dy)))
        j1 = min(y_m.size, int(math.ceil((cy + rad - y_m[0]) / dy)) + 1)
        if i0 >= i1 or j0 >= j1:
            continue
        ex = np.exp(-((x_m[i0:i1] - cx) ** 2) / (2 * s * s))
        ey = np.exp(-((y_m[j0:j1] - cy) ** 2) / (2 * s * s))
        field[j0:j1, i0:i1] += a * np.outer(ey, ex)
    return field


def hole_grid(seed: int = 4, nx: int = 4096, ny: int = 4096, cell_cm: int = 200,
              frac: float = 0.05, x0_cm: int = 0, y0_cm: int = 0,
              noise_m: float = 0.0) -> HoleGrid:
    """A gridded bathymetry product with round(frac * nx * ny) nodes removed at
    random (the shape of the paper's hole-filling tests, Sec. IV Grid B).

    The depth of node (i, j) is the shared seafloor model at its centre (bumps
    cut at 5 sigma), plus N(0, noise_m^2) if noise_m > 0. The removed nodes are
    drawn without replacement from the same seeded generator.
    """
    if not 0.0 <= frac < 1.0:
        raise ValueError("frac must be in [0, 1)")
    rng = _rng(seed)
    xs = (x0_cm + np.arange(nx) * cell_cm + cell_cm // 2) / 100.0
    ys = (y0_cm + np.arange(ny) * cell_cm + cell_cm // 2) / 100.0
    table = bumps(rng, x0_cm / 100.0, (x0_cm + nx * cell_cm) / 100.0,
                  y0_cm / 100.0, (y0_cm + ny * cell_cm) / 100.0)
    field = _lattice_field(xs, ys, table)
    z = 3500.0 + 0.01 * xs[None, :] + field
    if noise_m > 0:
        z = z + rng.normal(0.0, noise_m, z.shape)
    m = nx * ny
    holes = np.sort(rng.choice(m, size=int(round(frac * m)), replace=False)).astype(np.int64)
    return HoleGrid(GridSpec(x0_cm, y0_cm, cell_cm, nx, ny), z.astype(np.float32).ravel(),
                    holes, frac, seed)


def row_midpoints(grid: GridSpec):
    """Query points halfway between successive grid rows, on every node column:
    the shape of the paper's row-filling tests (Sec. IV Grid A, latitudes added
    between existing ones). Returns (qx_cm, qy_cm), (ny - 1) * nx points, row-major.
    """
    i = np.arange(grid.nx)
    j = np.arange(grid.ny - 1)
    qx = grid.x0_cm + i * grid.cell_cm + grid.cell_cm // 2
    qy = grid.y0_cm + (j + 1) * grid.cell_cm
    X, Y = np.meshgrid(qx, qy)
    return X.ravel().astype(np.int32), Y.ravel().astype(np.int32)


def random_points(seed: int, grid: GridSpec, m: int, margin_cells: float = 0.0):
    """m uniform query points (int32 cm) over the grid's node hull, widened by
    margin_cells on every side."""
    rng = _rng(seed)
    c = grid.cell_cm
    lo_x = grid.x0_cm + c // 2 - margin_cells * c
    hi_x = grid.x0_cm + (grid.nx - 1) * c + c // 2 + margin_cells * c
    lo_y = grid.y0_cm + c // 2 - margin_cells * c
    hi_y = grid.y0_cm + (grid.ny - 1) * c + c // 2 + margin_cells * c
    qx = np.floor(rng.uniform(lo_x, hi_x + 1, m)).astype(np.int32)
    qy = np.floor(rng.uniform(lo_y, hi_y + 1, m)).astype(np.int32)
    return qx, qy
