"""FP64 CPU oracle for exact k-NN, IDW, ordinary kriging and gridded
bilinear / Catmull-Rom resampling (ctypes over oracle.c).

The k-NN is brute force by default; `Tree` builds a 2-d tree over the same
soundings that gives the same (d2, index)-ordered neighbours far faster on
large inputs (pass it as `tree=` to knn, idw and okrige).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of the benchmark may import this package; the library under
paper_2505_22675_gb300/ never does, and shares no code with it.

The C source (oracle.c) states the definitions it follows. `build()` compiles
it with gcc; importing the package builds it on first use if the shared
object is missing or older than the source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

SPHERICAL = 0
EXPONENTIAL = 1

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, -O2, IEEE arithmetic)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.oracle_grid_nodes.argtypes = [i32, i32, i32, i32, i32, P, P]
    lib.oracle_grid_nodes.restype = None
    lib.oracle_knn.argtypes = [P, P, P, i64, P, P, i64, ctypes.c_int, P, P, P, ctypes.c_int, P]
    lib.oracle_knn.restype = ctypes.c_int
    lib.oracle_idw.argtypes = [P, P, P, i64, P, P, i64, ctypes.c_int, dbl, P, P, ctypes.c_int, P]
    lib.oracle_idw.restype = ctypes.c_int
    lib.oracle_okrige.argtypes = [P, P, P, i64, P, P, i64, ctypes.c_int, ctypes.c_int,
                                  dbl, dbl, dbl, P, P, P, P, P, ctypes.c_int, P]
    lib.oracle_okrige.restype = ctypes.c_int
    lib.oracle_variogram.argtypes = [ctypes.c_int, dbl, dbl, dbl, dbl]
    lib.oracle_variogram.restype = dbl
    lib.oracle_solve.argtypes = [ctypes.c_int, P, P, P]
    lib.oracle_solve.restype = ctypes.c_int
    lib.oracle_resample.argtypes = [P, i32, i32, i32, i32, i32, ctypes.c_int, P, P, i64, P, P]
    lib.oracle_resample.restype = ctypes.c_int
    lib.oracle_tree_build.argtypes = [P, P, P, i64, ctypes.c_int]
    lib.oracle_tree_build.restype = P
    lib.oracle_tree_free.argtypes = [P]
    lib.oracle_tree_free.restype = None
    lib.oracle_threads.argtypes = [ctypes.c_int]
    lib.oracle_threads.restype = ctypes.c_int
    _lib = lib
    return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _inputs(x, y, z, qx, qy):
    x = np.ascontiguousarray(x, dtype=np.int32)
    y = np.ascontiguousarray(y, dtype=np.int32)
    z = np.ascontiguousarray(z, dtype=np.float32)
    qx = np.ascontiguousarray(qx, dtype=np.int32)
    qy = np.ascontiguousarray(qy, dtype=np.int32)
    if not (x.shape == y.shape == z.shape) or qx.shape != qy.shape:
        raise ValueError("shape mismatch")
    return x, y, z, qx, qy


class Tree:
    """2-d tree over the valid soundings of (x, y, z), for knn / idw / okrige
    on large inputs. It keeps references to the arrays it was built from;
    pass the same x, y, z to the queries."""

    def __init__(self, x, y, z, nthreads: int = 0):
        self.x = np.ascontiguousarray(x, dtype=np.int32)
        self.y = np.ascontiguousarray(y, dtype=np.int32)
        self.z = np.ascontiguousarray(z, dtype=np.float32)
        if not (self.x.shape == self.y.shape == self.z.shape):
            raise ValueError("shape mismatch")
        self._h = _load().oracle_tree_build(_p(self.x), _p(self.y), _p(self.z), self.x.size,
                                            nthreads)
        if not self._h:
            raise MemoryError("oracle_tree_build")

    def handle(self, x, y, z):
        """The tree's handle, after checking it was built from these arrays."""
        for a, b in ((x, self.x), (y, self.y), (z, self.z)):
            a = np.asarray(a)
            if a.shape != b.shape or not (a is b or np.array_equal(a, b, equal_nan=True)):
                raise ValueError("the tree was built from other soundings")
        return ctypes.c_void_p(self._h)

    def close(self):
        if self._h:
            _load().oracle_tree_free(ctypes.c_void_p(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _tree(tree, x, y, z):
    return None if tree is None else tree.handle(x, y, z)


def threads(requested: int = 0) -> int:
    """Threads the oracle uses for `requested` (0 = every online core)."""
    return int(_load().oracle_threads(requested))


def grid_nodes(x0_cm: int, y0_cm: int, cell_cm: int, nx: int, ny: int):
    """Node coordinates (int32 cm) of a grid, row-major j*nx + i."""
    qx = np.empty(nx * ny, dtype=np.int32)
    qy = np.empty(nx * ny, dtype=np.int32)
    _load().oracle_grid_nodes(x0_cm, y0_cm, cell_cm, nx, ny, _p(qx), _p(qy))
    return qx, qy


def knn(x, y, z, qx, qy, k: int, nthreads: int = 0, tree: Tree | None = None):
    """Exact k-NN (brute force, or `tree`): (idx int32[m,k], d2 int64[m,k], keff int32[m]); -1 pads."""
    x, y, z, qx, qy = _inputs(x, y, z, qx, qy)
    m = qx.size
    idx = np.empty((m, k), dtype=np.int32)
    d2 = np.empty((m, k), dtype=np.int64)
    keff = np.empty(m, dtype=np.int32)
    rc = _load().oracle_knn(_p(x), _p(y), _p(z), x.size, _p(qx), _p(qy), m, k,
                            _p(idx), _p(d2), _p(keff), nthreads, _tree(tree, x, y, z))
    if rc != 0:
        raise ValueError("oracle_knn: bad arguments")
    return idx, d2, keff


def idw(x, y, z, qx, qy, k: int, power: float = 2.0, nthreads: int = 0, want_idx: bool = False,
        tree: Tree | None = None):
    """FP64 IDW depth per node (NaN where no valid sounding exists)."""
    x, y, z, qx, qy = _inputs(x, y, z, qx, qy)
    m = qx.size
    depth = np.empty(m, dtype=np.float64)
    idx = np.empty((m, k), dtype=np.int32) if want_idx else None
    rc = _load().oracle_idw(_p(x), _p(y), _p(z), x.size, _p(qx), _p(qy), m, k, float(power),
                            _p(depth), _p(idx), nthreads, _tree(tree, x, y, z))
    if rc != 0:
        raise ValueError("oracle_idw: bad arguments")
    return (depth, idx) if want_idx else depth


def okrige(x, y, z, qx, qy, k: int, model: int = SPHERICAL, nugget: float = 0.25,
           sill: float = 100.0, range_m: float = 50.0, nthreads: int = 0,
           want_weights: bool = False, want_idx: bool = False, tree: Tree | None = None):
    """FP64 ordinary kriging: (depth, variance[, lambda[m,k], mu[m]][, idx])."""
    x, y, z, qx, qy = _inputs(x, y, z, qx, qy)
    m = qx.size
    depth = np.empty(m, dtype=np.float64)
    var = np.empty(m, dtype=np.float64)
    lam = np.empty((m, k), dtype=np.float64) if want_weights else None
    mu = np.empty(m, dtype=np.float64) if want_weights else None
    idx = np.empty((m, k), dtype=np.int32) if want_idx else None
    rc = _load().oracle_okrige(_p(x), _p(y), _p(z), x.size, _p(qx), _p(qy), m, k, int(model),
                               float(nugget), float(sill), float(range_m), _p(depth), _p(var),
                               _p(lam), _p(mu), _p(idx), nthreads, _tree(tree, x, y, z))
    if rc != 0:
        raise ValueError("oracle_okrige: bad arguments")
    out = [depth, var]
    if want_weights:
        out += [lam, mu]
    if want_idx:
        out.append(idx)
    return tuple(out)


def variogram(model: int, nugget: float, sill: float, range_m: float, h_m: float) -> float:
    """gamma(h) for h > 0 metres."""
    return float(_load().oracle_variogram(int(model), nugget, sill, range_m, float(h_m)))


def solve(A, b):
    """Solve A x = b by the oracle's Gaussian elimination with partial pivoting."""
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    b = np.array(b, dtype=np.float64, copy=True)
    n = b.size
    x = np.empty(n, dtype=np.float64)
    if _load().oracle_solve(n, _p(A), _p(b), _p(x)) != 0:
        raise np.linalg.LinAlgError("zero pivot")
    return x


BILINEAR = 0
CATMULL_ROM = 1


def resample(src, grid_spec, qx, qy, method: int):
    """Bilinear (method 0) or Catmull-Rom (1) of a regular grid at query points.

    src: float32 [ny * nx] row-major node values (NaN = missing); grid_spec =
    (x0_cm, y0_cm, cell_cm, nx, ny). Returns (values float64[m], how int8[m]):
    how = 0 by the method itself, 1 by the bilinear fallback, 2 no value (NaN).
    """
    x0, y0, cell, nx, ny = (int(v) for v in grid_spec)
    src = np.ascontiguousarray(src, dtype=np.float32)
    if src.size != nx * ny:
        raise ValueError("src must hold nx * ny values")
    qx = np.ascontiguousarray(qx, dtype=np.int32)
    qy = np.ascontiguousarray(qy, dtype=np.int32)
    m = qx.size
    out = np.empty(m, dtype=np.float64)
    how = np.empty(m, dtype=np.int8)
    rc = _load().oracle_resample(_p(src), x0, y0, cell, nx, ny, int(method), _p(qx), _p(qy), m,
                                 _p(out), _p(how))
    if rc != 0:
        raise ValueError("oracle_resample: bad arguments")
    return out, how
