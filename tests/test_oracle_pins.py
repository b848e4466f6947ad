"""Pins for the FP64 oracle against facts that do not come from the oracle itself.

Each test checks a closed form, an invariant, a hand-worked value
(tests/golden/hand_worked.txt), a brute force written differently (Python
sort) or a library routine (numpy.linalg.solve, scipy's k-d tree). The
cases are chosen so that a dropped term, a wrong sign or index, or a swapped
operand in the oracle fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_worked.txt")

SPH = dict(model=oracle.SPHERICAL, nugget=0.25, sill=100.0, range_m=50.0)


def _golden():
    cases = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, pts, node, params, expected = [s.strip() for s in line.split("|")]
            num, den = expected.split("/")
            cases[name] = dict(
                pts=None if pts == "-" else [tuple(float(v) for v in p.split(":")) for p in pts.split(",")],
                node=None if node == "-" else tuple(int(v) for v in node.split(":")),
                params={kv.split("=")[0]: float(kv.split("=")[1]) for kv in params.split()},
                expected=float(num) / float(den))
    return cases


def _arrays(pts):
    x = np.array([p[0] for p in pts], dtype=np.int32)
    y = np.array([p[1] for p in pts], dtype=np.int32)
    z = np.array([p[2] for p in pts], dtype=np.float32)
    return x, y, z


def _py_knn(x, y, z, qx, qy, k):
    """Reference k-NN: Python sort of (d2, index) over valid soundings."""
    keys = sorted(((int(x[p]) - qx) ** 2 + (int(y[p]) - qy) ** 2, p)
                  for p in range(len(x)) if not math.isnan(float(z[p])))
    return keys[:k]


# ------------------------------------------------------------------- kNN

@pytest.mark.parametrize("seed", range(6))
def test_knn_matches_python_sort(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 160))
    span = int(rng.choice([5, 40, 3000]))  # small spans force many exact ties and duplicates
    x = rng.integers(-span, span, n).astype(np.int32)
    y = rng.integers(-span, span, n).astype(np.int32)
    z = rng.normal(size=n).astype(np.float32)
    z[rng.random(n) < 0.1] = np.nan
    m = 40
    qx = rng.integers(-span - 3, span + 3, m).astype(np.int32)
    qy = rng.integers(-span - 3, span + 3, m).astype(np.int32)
    for k in (1, 3, 8, 17):
        idx, d2, keff = oracle.knn(x, y, z, qx, qy, k, nthreads=2)
        for q in range(m):
            ref = _py_knn(x, y, z, int(qx[q]), int(qy[q]), k)
            assert keff[q] == len(ref)
            assert [(int(d2[q, i]), int(idx[q, i])) for i in range(keff[q])] == ref
            assert np.all(idx[q, keff[q]:] == -1)


@pytest.mark.parametrize("seed", range(8))
def test_tree_knn_equals_brute_force(seed):
    # the 2-d tree must return the brute force's (d2, index) lists exactly: ties,
    # duplicate positions, NaN depths, N < k, and spans from a few cm to km
    rng = np.random.default_rng(100 + seed)
    n = int(rng.choice([1, 7, 9, 40, 300, 5000]))
    span = int(rng.choice([3, 50, 4000, 10**8]))
    x = rng.integers(-span, span, n).astype(np.int32)
    y = rng.integers(-span, span, n).astype(np.int32)
    if seed % 2:
        x[: n // 3] = x[0]  # a column of equal x (median splits through equal keys)
    z = rng.normal(size=n).astype(np.float32)
    z[rng.random(n) < 0.15] = np.nan
    m = 300
    qx = rng.integers(-span - 5, span + 5, m).astype(np.int32)
    qy = rng.integers(-span - 5, span + 5, m).astype(np.int32)
    tree = oracle.Tree(x, y, z)
    for k in (1, 4, 16, 33):
        ref = oracle.knn(x, y, z, qx, qy, k, nthreads=2)
        got = oracle.knn(x, y, z, qx, qy, k, nthreads=2, tree=tree)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)


def test_tree_knn_lattice_duplicates_and_empty():
    xs, ys = np.meshgrid(np.arange(40) * 100, np.arange(30) * 100)
    x = np.concatenate([xs.ravel(), xs.ravel()[::7]]).astype(np.int32)  # every 7th point twice
    y = np.concatenate([ys.ravel(), ys.ravel()[::7]]).astype(np.int32)
    z = np.arange(x.size, dtype=np.float32)
    qx, qy = oracle.grid_nodes(-150, -150, 100, 44, 34)  # nodes on cell centres, ties everywhere
    qx = np.concatenate([qx, x[::13]])                    # and nodes on soundings
    qy = np.concatenate([qy, y[::13]])
    tree = oracle.Tree(x, y, z)
    for k in (4, 8, 32):
        ref = oracle.knn(x, y, z, qx, qy, k)
        got = oracle.knn(x, y, z, qx, qy, k, tree=tree)
        assert all(np.array_equal(a, b) for a, b in zip(ref, got))
        # IDW and kriging take the same neighbours, so the same values bit for bit
        assert np.array_equal(oracle.idw(x, y, z, qx, qy, k, tree=tree), oracle.idw(x, y, z, qx, qy, k))
        a = oracle.okrige(x, y, z, qx[:200], qy[:200], k, tree=tree)
        b = oracle.okrige(x, y, z, qx[:200], qy[:200], k)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # no valid sounding, and no sounding at all
    for xx, yy, zz in ((x[:5], y[:5], np.full(5, np.nan, np.float32)),
                       (x[:0], y[:0], z[:0])):
        t = oracle.Tree(xx, yy, zz)
        idx, d2, keff = oracle.knn(xx, yy, zz, qx[:10], qy[:10], 4, tree=t)
        assert (keff == 0).all() and (idx == -1).all() and (d2 == -1).all()
    with pytest.raises(ValueError):
        oracle.knn(x[:-1], y[:-1], z[:-1], qx, qy, 4, tree=tree)  # built from other soundings


def test_knn_lattice_ties_break_by_index():
    # node at the centre of a 2 x 2 cell of a unit lattice: four soundings tie at every ring
    xs, ys = np.meshgrid(np.arange(6) * 100, np.arange(6) * 100)
    x = xs.ravel().astype(np.int32)
    y = ys.ravel().astype(np.int32)
    perm = np.random.default_rng(0).permutation(x.size)
    x, y = x[perm], y[perm]
    z = np.zeros(x.size, np.float32)
    idx, d2, _ = oracle.knn(x, y, z, [250], [250], 12)
    assert list(d2[0, :4]) == [5000] * 4 and list(d2[0, 4:12]) == [25000] * 8
    assert list(idx[0, :4]) == sorted(idx[0, :4]) and list(idx[0, 4:12]) == sorted(idx[0, 4:12])


def test_knn_matches_kdtree_on_distinct_distances():
    scipy_spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(7)
    x = rng.integers(0, 10**6, 3000).astype(np.int32)
    y = rng.integers(0, 10**6, 3000).astype(np.int32)
    z = np.zeros(3000, np.float32)
    qx = rng.integers(0, 10**6, 200).astype(np.int32)
    qy = rng.integers(0, 10**6, 200).astype(np.int32)
    idx, d2, _ = oracle.knn(x, y, z, qx, qy, 10)
    tree = scipy_spatial.cKDTree(np.stack([x, y], 1).astype(np.float64))
    dist, ref = tree.query(np.stack([qx, qy], 1).astype(np.float64), k=10)
    ok = np.all(np.diff(dist, axis=1) > 1e-6, axis=1)  # rows without ties
    assert ok.sum() > 150
    assert np.array_equal(idx[ok], ref[ok])


def test_knn_fewer_than_k_and_none_valid():
    x = np.array([0, 10, 20], np.int32)
    y = np.zeros(3, np.int32)
    z = np.array([1.0, np.nan, 3.0], np.float32)
    idx, d2, keff = oracle.knn(x, y, z, [9], [0], 5)
    assert keff[0] == 2 and list(idx[0]) == [0, 2, -1, -1, -1] and list(d2[0, :2]) == [81, 121]
    z[:] = np.nan
    _, _, keff = oracle.knn(x, y, z, [9], [0], 5)
    assert keff[0] == 0


def test_grid_nodes_are_pixel_centres():
    qx, qy = oracle.grid_nodes(-100, 300, 50, 3, 2)
    assert list(qx) == [-75, -25, 25, -75, -25, 25]
    assert list(qy) == [325, 325, 325, 375, 375, 375]


# ------------------------------------------------------------------- IDW

def test_idw_hand_worked():
    g = _golden()
    for name in ("idw_p2_123", "idw_p1_123", "idw_p2_k2"):
        c = g[name]
        x, y, z = _arrays(c["pts"])
        d = oracle.idw(x, y, z, [c["node"][0]], [c["node"][1]], int(c["params"]["k"]),
                       c["params"]["p"])
        assert d[0] == pytest.approx(c["expected"], abs=1e-14), name


def test_idw_constant_field_exact():
    rng = np.random.default_rng(1)
    x = rng.integers(0, 5000, 300).astype(np.int32)
    y = rng.integers(0, 5000, 300).astype(np.int32)
    qx = rng.integers(0, 5000, 100).astype(np.int32)
    qy = rng.integers(0, 5000, 100).astype(np.int32)
    for p in (1.0, 2.0, 3.0):
        # a power-of-two depth scales every product exactly: the ratio is exact
        d = oracle.idw(x, y, np.full(300, 2048.0, np.float32), qx, qy, 8, p)
        assert np.all(d == 2048.0)
        d = oracle.idw(x, y, np.full(300, 3500.25, np.float32), qx, qy, 8, p)
        assert np.max(np.abs(d - 3500.25)) <= 4 * np.spacing(3500.25)


def test_idw_coincident_node_returns_lowest_index_sounding():
    x = np.array([500, 0, 500, 900], np.int32)
    y = np.array([500, 0, 500, 100], np.int32)
    z = np.array([7.0, 1.0, 9.0, 2.0], np.float32)
    d, idx = oracle.idw(x, y, z, [500], [500], 3, 2.0, want_idx=True)
    assert d[0] == 7.0 and list(idx[0]) == [0, 2, 3]


def test_idw_midpoint_is_mean():
    x = np.array([0, 1000, 5000], np.int32)
    y = np.array([0, 0, 5000], np.int32)
    z = np.array([10.0, 30.0, 99.0], np.float32)
    for p in (1.0, 2.0, 4.5):
        assert oracle.idw(x, y, z, [500], [0], 2, p)[0] == pytest.approx(20.0, abs=1e-12)


def _lattice(n_side=8, s=200, a=3500.0, bx=0.01, by=-0.02):
    xs, ys = np.meshgrid(np.arange(n_side) * s, np.arange(n_side) * s)
    x = xs.ravel().astype(np.int32)
    y = ys.ravel().astype(np.int32)
    z = (a + bx * x + by * y).astype(np.float32)
    return x, y, z


def test_idw_linear_surface_symmetric_patch():
    s = 200
    x, y, z = _lattice(s=s)
    qx, qy = 3 * s + s // 2, 3 * s + s // 2  # centre of a lattice cell inside the patch
    idx, d2, _ = oracle.knn(x, y, z, [qx], [qy], 16)
    assert sorted(set(d2[0].tolist())) == [s * s // 2, 5 * s * s // 2, 9 * s * s // 2]
    expect = 3500.0 + 0.01 * qx - 0.02 * qy
    zf = z.astype(np.float64)
    # exact linear target, evaluated from the float32 depths actually stored
    d = oracle.idw(x, y, z, [qx], [qy], 16, 2.0)[0]
    assert d == pytest.approx(np.mean(zf[idx[0]]), abs=1e-9)
    assert abs(d - expect) < 1e-3


# --------------------------------------------------------------- variogram

def test_variogram_closed_forms():
    g = _golden()
    for name in ("sph_half_range", "sph_fifth_range"):
        p = g[name]["params"]
        v = oracle.variogram(int(p["model"]), p["nugget"], p["sill"], p["range"], p["h"])
        assert v == pytest.approx(g[name]["expected"], abs=1e-12), name
    assert oracle.variogram(0, 0.25, 100, 50, 50.0) == 100.0
    assert oracle.variogram(0, 0.25, 100, 50, 80.0) == 100.0
    # continuity at the range and at 0+
    assert oracle.variogram(0, 0.25, 100, 50, 50 - 1e-9) == pytest.approx(100.0, abs=1e-6)
    assert oracle.variogram(0, 0.25, 100, 50, 1e-9) == pytest.approx(0.25, abs=1e-6)
    # exponential, the form printed in Sec. III-C: C0 (1 - exp(-h/a)) with no nugget
    assert oracle.variogram(1, 0.0, 100, 50, 50.0) == pytest.approx(100 * (1 - math.exp(-1)), abs=1e-12)
    assert oracle.variogram(1, 0.5, 10, 5, 10.0) == pytest.approx(0.5 + 9.5 * (1 - math.exp(-2)), abs=1e-12)


# ----------------------------------------------------------------- solver

def test_solver_matches_numpy():
    rng = np.random.default_rng(3)
    for n in (1, 2, 5, 17, 33):
        A = rng.normal(size=(n, n)) + n * np.eye(n) * rng.choice([0.0, 1.0])
        b = rng.normal(size=n)
        if abs(np.linalg.det(A)) < 1e-6:
            continue
        assert np.allclose(oracle.solve(A, b), np.linalg.solve(A, b), rtol=1e-9, atol=1e-9)


def test_solver_needs_pivoting():
    # the leading zero makes elimination without row exchanges fail
    A = np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
    b = np.array([2.0, 3.0, 4.0])
    assert np.allclose(oracle.solve(A, b), np.linalg.solve(A, b), atol=1e-14)
    # an exactly bordered kriging matrix: zero in the corner
    G = np.array([[0, 3, 1], [3, 0, 1], [1, 1, 0]], dtype=float)
    assert np.allclose(oracle.solve(G, [1, 2, 1]), np.linalg.solve(G, [1, 2, 1]), atol=1e-14)


# ---------------------------------------------------------------- kriging

def test_okrige_weights_sum_to_one_and_solve_the_system():
    rng = np.random.default_rng(5)
    x = rng.integers(0, 3000, 400).astype(np.int32)
    y = rng.integers(0, 3000, 400).astype(np.int32)
    z = (3500 + rng.normal(size=400)).astype(np.float32)
    qx = rng.integers(0, 3000, 60).astype(np.int32)
    qy = rng.integers(0, 3000, 60).astype(np.int32)
    for model in (oracle.SPHERICAL, oracle.EXPONENTIAL):
        for k in (1, 2, 5, 16, 32):
            d, v, lam, mu, idx = oracle.okrige(x, y, z, qx, qy, k, model, 0.25, 100.0, 50.0,
                                               want_weights=True, want_idx=True)
            assert np.all(np.abs(lam.sum(1) - 1.0) < 1e-12)
            # re-check the system rows directly from the variogram (no shared code with the solve)
            q = 7
            pts = idx[q]
            gam = lambda h: oracle.variogram(model, 0.25, 100.0, 50.0, h)
            for i in range(k):
                row = 0.0
                for j in range(k):
                    if i == j:
                        continue
                    h = math.hypot(int(x[pts[i]]) - int(x[pts[j]]), int(y[pts[i]]) - int(y[pts[j]])) / 100
                    row += lam[q, j] * (gam(h) if h > 0 else 0.25)
                h0 = math.hypot(int(x[pts[i]]) - int(qx[q]), int(y[pts[i]]) - int(qy[q])) / 100
                assert row + mu[q] == pytest.approx(gam(h0) if h0 > 0 else 0.0, abs=1e-9)
            assert d[q] == pytest.approx(float(np.dot(lam[q], z[pts].astype(np.float64))), abs=1e-9)


def test_okrige_k1_closed_form():
    x = np.array([0, 900], np.int32)
    y = np.array([0, 0], np.int32)
    z = np.array([12.5, 40.0], np.float32)
    d, v, lam, mu = oracle.okrige(x, y, z, [300], [400], 1, want_weights=True)
    g10 = oracle.variogram(0, 0.25, 100, 50, 5.0)
    assert lam[0, 0] == 1.0 and mu[0] == pytest.approx(g10, abs=1e-12)
    assert v[0] == pytest.approx(2 * g10, abs=1e-12) and d[0] == 12.5


def test_okrige_k2_hand_worked():
    c = _golden()["ok_k2_line"]
    x, y, z = _arrays(c["pts"])
    p = c["params"]
    d, v, lam, mu = oracle.okrige(x, y, z, [c["node"][0]], [c["node"][1]], 2, int(p["model"]),
                                  p["nugget"], p["sill"], p["range"], want_weights=True)
    assert lam[0, 0] == pytest.approx(c["expected"], abs=1e-12)
    assert d[0] == pytest.approx(10 * c["expected"] + 20 * (1 - c["expected"]), abs=1e-10)
    # mu from the first system row; variance = sum lambda gamma_0 + mu
    g = lambda h: 100 * (0.03 * h - 4e-6 * h ** 3)
    mu_ref = g(2) - g(10) * (1 - c["expected"])
    assert mu[0] == pytest.approx(mu_ref, abs=1e-10)
    assert v[0] == pytest.approx(c["expected"] * g(2) + (1 - c["expected"]) * g(8) + mu_ref, abs=1e-10)


def _ok_golden(name):
    c = _golden()[name]
    x, y, z = _arrays(c["pts"])
    p = c["params"]
    d, v, lam, mu, idx = oracle.okrige(x, y, z, [c["node"][0]], [c["node"][1]], int(p["k"]),
                                       int(p["model"]), p["nugget"], p["sill"], p["range"],
                                       want_weights=True, want_idx=True)
    return c, z, d[0], v[0], lam[0], mu[0], idx[0]


def test_okrige_colocated_pair_hand_worked():
    # two distinct soundings at one position take gamma = c0 (the h -> 0+ limit)
    c, z, d, v, lam, mu, idx = _ok_golden("ok_dup_k2_mu")
    assert list(idx) == [0, 1]
    assert np.allclose(lam, 0.5, atol=1e-13)
    assert d == pytest.approx(15.0, abs=1e-12)
    assert mu == pytest.approx(c["expected"], abs=1e-12)
    assert v == pytest.approx(_golden()["ok_dup_k2_var"]["expected"], abs=1e-12)


def test_okrige_colocated_pair_with_third_sounding_hand_worked():
    c, z, d, v, lam, mu, idx = _ok_golden("ok_dup_k3_lambda")
    a = c["expected"]
    assert list(idx) == [0, 1, 2]
    assert lam[0] == pytest.approx(a, abs=1e-13) and lam[1] == pytest.approx(a, abs=1e-13)
    assert lam[2] == pytest.approx(1 - 2 * a, abs=1e-13)
    assert d == pytest.approx(10 * a + 20 * a + 40 * (1 - 2 * a), abs=1e-11)
    assert mu == pytest.approx(_golden()["ok_dup_k3_mu"]["expected"], abs=1e-11)
    assert v == pytest.approx(_golden()["ok_dup_k3_var"]["expected"], abs=1e-11)


def test_okrige_node_on_colocated_pair_hand_worked():
    # the node on P: gamma_0 = 0 to P and P', but P and P' take c0 to each other
    c, z, d, v, lam, mu, idx = _ok_golden("ok_dup_node_lambda3")
    l3 = c["expected"]
    assert list(idx) == [0, 1, 2]
    assert lam[0] == pytest.approx((1 - l3) / 2, abs=1e-13)
    assert lam[1] == pytest.approx((1 - l3) / 2, abs=1e-13)
    assert lam[2] == pytest.approx(l3, abs=1e-13)
    assert d == pytest.approx(15 * (1 - l3) + 40 * l3, abs=1e-11)
    assert v == pytest.approx(_golden()["ok_dup_node_var"]["expected"], abs=1e-12)


def test_okrige_k2_general_closed_form():
    rng = np.random.default_rng(11)
    for _ in range(20):
        x = rng.integers(-4000, 4000, 2).astype(np.int32)
        y = rng.integers(-4000, 4000, 2).astype(np.int32)
        z = rng.normal(3500, 5, 2).astype(np.float32)
        qx, qy = rng.integers(-4000, 4000, 2)
        for model in (0, 1):
            d, v, lam, mu, idx = oracle.okrige(x, y, z, [qx], [qy], 2, model, 0.25, 100, 50,
                                               want_weights=True, want_idx=True)
            a, b = idx[0]
            gm = lambda h: oracle.variogram(model, 0.25, 100, 50, h) if h > 0 else 0.0
            g_a0 = gm(math.hypot(int(x[a]) - qx, int(y[a]) - qy) / 100)
            g_b0 = gm(math.hypot(int(x[b]) - qx, int(y[b]) - qy) / 100)
            g_ab = gm(math.hypot(int(x[a]) - int(x[b]), int(y[a]) - int(y[b])) / 100)
            la = 0.5 + (g_b0 - g_a0) / (2 * g_ab)
            assert lam[0, 0] == pytest.approx(la, abs=1e-10)
            assert mu[0] == pytest.approx(g_a0 - g_ab * (1 - la), abs=1e-9)
            assert v[0] == pytest.approx(la * g_a0 + (1 - la) * g_b0 + mu[0], abs=1e-9)


def test_okrige_pure_nugget():
    # every pairwise and node separation beyond the range: Gamma = sill off the diagonal
    x = (np.arange(5) * 10000).astype(np.int32)
    y = np.zeros(5, np.int32)
    z = np.array([1, 2, 3, 4, 5], np.float32)
    d, v, lam = oracle.okrige(x, y, z, [20000], [9000], 5, want_weights=True)[:3]
    assert np.allclose(lam[0], 0.2, atol=1e-14)
    assert d[0] == pytest.approx(3.0, abs=1e-12)
    assert v[0] == pytest.approx(100.0 * (1 + 1 / 5), abs=1e-10)


def test_okrige_coincident_node_is_exact():
    rng = np.random.default_rng(2)
    x = rng.integers(0, 3000, 50).astype(np.int32)
    y = rng.integers(0, 3000, 50).astype(np.int32)
    z = rng.normal(3500, 3, 50).astype(np.float32)
    for k in (4, 16):
        d, v, lam, mu, idx = oracle.okrige(x, y, z, [x[17]], [y[17]], k, want_weights=True,
                                           want_idx=True)
        assert idx[0, 0] == 17
        assert np.allclose(lam[0], np.eye(k)[0], atol=1e-12)
        assert d[0] == pytest.approx(float(z[17]), abs=1e-9) and abs(v[0]) < 1e-10


def test_okrige_square_symmetry_closed_form():
    # four soundings on a square around the node: lambda = 1/4, mu = g0 - rowsum/4
    a = 300
    x = np.array([-a, a, -a, a], np.int32)
    y = np.array([-a, -a, a, a], np.int32)
    z = np.array([1, 2, 3, 10], np.float32)
    for model in (0, 1):
        d, v, lam, mu = oracle.okrige(x, y, z, [0], [0], 4, model, 0.25, 100, 50, want_weights=True)
        gm = lambda h: oracle.variogram(model, 0.25, 100, 50, h)
        g0 = gm(math.sqrt(2) * a / 100)
        rowsum = 2 * gm(2 * a / 100) + gm(2 * math.sqrt(2) * a / 100)
        assert np.allclose(lam[0], 0.25, atol=1e-13)
        assert mu[0] == pytest.approx(g0 - rowsum / 4, abs=1e-10)
        assert v[0] == pytest.approx(2 * g0 - rowsum / 4, abs=1e-10)
        assert d[0] == pytest.approx(4.0, abs=1e-12)


def test_okrige_linear_surface_symmetric_patch():
    s = 200
    x, y, z = _lattice(s=s)
    qx, qy = 3 * s + s // 2, 3 * s + s // 2
    d, v = oracle.okrige(x, y, z, [qx], [qy], 16)
    _, idx, = oracle.idw(x, y, z, [qx], [qy], 16, want_idx=True)
    assert d[0] == pytest.approx(np.mean(z[idx[0]].astype(np.float64)), abs=1e-9)


def test_okrige_exchangeable_with_constant_field():
    # OK reproduces a constant field for any configuration (the weights sum to one)
    rng = np.random.default_rng(9)
    x = rng.integers(0, 2000, 200).astype(np.int32)
    y = rng.integers(0, 2000, 200).astype(np.int32)
    z = np.full(200, 2048.0, np.float32)
    qx = rng.integers(0, 2000, 30).astype(np.int32)
    qy = rng.integers(0, 2000, 30).astype(np.int32)
    d, v = oracle.okrige(x, y, z, qx, qy, 16)
    assert np.max(np.abs(d - 2048.0)) < 1e-9
    assert np.all(v >= 0.0)


def test_okrige_no_valid_soundings_is_nan():
    d, v = oracle.okrige([0, 1], [0, 1], [np.nan, np.nan], [0], [0], 4)
    assert math.isnan(d[0]) and math.isnan(v[0])


# ------------------------------------------------------- gridded input

RESAMPLE_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "resample_hand_worked.txt")


def _resample_golden():
    cases = []
    with open(RESAMPLE_GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, size, vals, q, method, expected, how = [s.strip() for s in line.split("|")]
            nx, ny = (int(v) for v in size.split())
            values = np.array([float(v) for v in vals.split(",")], dtype=np.float32)
            qx, qy = (int(v) for v in q.split())
            if expected == "nan":
                exp = math.nan
            else:
                num, den = expected.split("/")
                exp = float(num) / float(den)
            cases.append((name, nx, ny, values, qx, qy, int(method), exp, int(how)))
    return cases


@pytest.mark.parametrize("case", _resample_golden(), ids=lambda c: c[0])
def test_resample_hand_worked(case):
    name, nx, ny, values, qx, qy, method, exp, how = case
    out, h = oracle.resample(values, (0, 0, 200, nx, ny), [qx], [qy], method)
    if math.isnan(exp):
        assert math.isnan(out[0])
    else:
        assert out[0] == pytest.approx(exp, abs=1e-12)
    assert h[0] == how


def _node_values(nx, ny, cell, f, x0=0, y0=0):
    """Node values f(x_m, y_m) on the lattice, row-major."""
    xs = (x0 + np.arange(nx) * cell + cell // 2) / 100.0
    ys = (y0 + np.arange(ny) * cell + cell // 2) / 100.0
    X, Y = np.meshgrid(xs, ys)
    return f(X, Y).astype(np.float64).ravel()


@pytest.mark.parametrize("seed", range(3))
def test_bilinear_reproduces_bilinear_functions(seed):
    rng = np.random.default_rng(seed)
    nx, ny, cell = int(rng.integers(2, 9)), int(rng.integers(2, 9)), 2 * int(rng.integers(1, 200))
    a, b, c, d = rng.normal(size=4)
    f = lambda x, y: a + b * x + c * y + d * x * y  # noqa: E731
    src = _node_values(nx, ny, cell, f).astype(np.float32)
    # float32 nodes: compare with the function of the rounded nodes, i.e. the
    # bilinear interpolant of src itself, through exact corners only
    qx = rng.integers(cell // 2, cell // 2 + (nx - 1) * cell + 1, 400)
    qy = rng.integers(cell // 2, cell // 2 + (ny - 1) * cell + 1, 400)
    got, how = oracle.resample(src, (0, 0, cell, nx, ny), qx, qy, oracle.BILINEAR)
    exact = _node_values(nx, ny, cell, f)  # unrounded corner values
    ref = f(qx / 100.0, qy / 100.0)
    # rounding of the nodes to float32 moves a convex combination by at most their ulp
    assert np.all(how == 0)
    assert np.max(np.abs(got - ref)) <= 2 * np.max(np.abs(exact - src)) + 1e-12


@pytest.mark.parametrize("seed", range(3))
def test_catmull_rom_reproduces_separable_quadratics(seed):
    rng = np.random.default_rng(10 + seed)
    nx, ny, cell = 9, 8, 200
    p = rng.normal(size=3)
    q = rng.normal(size=3)
    f = lambda x, y: (p[0] + p[1] * x + p[2] * x * x) * (q[0] + q[1] * y + q[2] * y * y)  # noqa: E731
    src64 = _node_values(nx, ny, cell, f)
    src = src64.astype(np.float32)
    # interior cells only (the 4 x 4 stencil does not reach the edge)
    qx = rng.integers(100 + 200, 100 + 200 * (nx - 2) + 1, 300)
    qy = rng.integers(100 + 200, 100 + 200 * (ny - 2) + 1, 300)
    got, how = oracle.resample(src, (0, 0, cell, nx, ny), qx, qy, oracle.CATMULL_ROM)
    assert np.all(how == 0)
    # Catmull-Rom weights are bounded (sum |w| <= 1.25 per axis): node rounding moves
    # the result by at most 1.25^2 * the largest node rounding error
    bound = 1.25 ** 2 * np.max(np.abs(src64 - src)) + 1e-9
    assert np.max(np.abs(got - f(qx / 100.0, qy / 100.0))) <= bound


def test_gridded_methods_at_nodes_outside_and_last_node():
    nx, ny, cell = 5, 4, 200
    rng = np.random.default_rng(3)
    src = rng.normal(3500, 20, nx * ny).astype(np.float32)
    i, j = np.meshgrid(np.arange(nx), np.arange(ny))
    qx = (100 + 200 * i).ravel()
    qy = (100 + 200 * j).ravel()
    for method in (oracle.BILINEAR, oracle.CATMULL_ROM):
        got, how = oracle.resample(src, (0, 0, cell, nx, ny), qx, qy, method)
        assert np.array_equal(got, src.astype(np.float64)) and np.all(how == 0)
        out, how = oracle.resample(src, (0, 0, cell, nx, ny), [99, 100, 901, 500], [100, 99, 100, 701],
                                   method)
        assert np.isnan(out).all() and np.all(how == 2)


def test_catmull_rom_falls_back_exactly_to_bilinear():
    nx, ny, cell = 12, 10, 200
    rng = np.random.default_rng(4)
    src = rng.normal(3500, 20, nx * ny).astype(np.float32)
    src[rng.choice(nx * ny, 12, replace=False)] = np.nan
    qx = rng.integers(100, 100 + 200 * (nx - 1) + 1, 3000)
    qy = rng.integers(100, 100 + 200 * (ny - 1) + 1, 3000)
    cr, how = oracle.resample(src, (0, 0, cell, nx, ny), qx, qy, oracle.CATMULL_ROM)
    bl, bhow = oracle.resample(src, (0, 0, cell, nx, ny), qx, qy, oracle.BILINEAR)
    assert set(np.unique(how)) == {0, 1, 2}
    fb = how >= 1
    assert np.array_equal(np.isnan(cr[fb]), np.isnan(bl[fb]))
    assert np.array_equal(cr[how == 1], bl[how == 1])
    assert np.all(bhow[how == 2] == 2) and np.all(np.isnan(cr[how == 2]))
    assert not np.isnan(cr[how == 0]).any()
