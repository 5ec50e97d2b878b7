"""Pins for the CPU oracle, each against something other than the oracle itself:
closed forms, a different algorithm, a library routine, textbook values, or
values printed in the paper.  CPU only."""
import itertools
import json
import math
import os
from functools import lru_cache

import numpy as np
import pytest

import oracle
from paper_2510_14147_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def lattice(a: int) -> np.ndarray:
    g = np.arange(a + 1, dtype=np.float32)
    return np.array(list(itertools.product(g, g, g)), dtype=np.float32)


def lattice_degree_closed_form(pts: np.ndarray, a: int, max_nonzero: int) -> np.ndarray:
    """Neighbours of each lattice vertex by enumeration of offsets in {-1,0,1}^3
    with 1..max_nonzero non-zero components (no distance is evaluated)."""
    offs = [o for o in itertools.product((-1, 0, 1), repeat=3)
            if 0 < sum(1 for c in o if c) <= max_nonzero]
    deg = np.zeros(len(pts), dtype=np.int64)
    for i, p in enumerate(pts.astype(np.int64)):
        for o in offs:
            q = p + np.array(o)
            if np.all(q >= 0) and np.all(q <= a):
                deg[i] += 1
    return deg


# ---------------------------------------------------------------- L2 pins

def test_sq_l2_exact_small_values():
    assert oracle.sq_l2([0, 0, 0], [1, 2, 2]) == 9.0
    assert oracle.sq_l2([0.5], [0.25]) == 0.0625
    # symmetric: (x-y)^2 == (y-x)^2 exactly
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(128).astype(np.float32), rng.standard_normal(128).astype(np.float32)
    assert oracle.sq_l2(x, y) == oracle.sq_l2(y, x)


def test_sq_l2_is_sequential_fp64_sum():
    """The pinned sum is a left-to-right FP64 sum: with terms 1, 2^-53, 2^-53 the
    sequential order loses both small terms, a pairwise or reordered sum does not."""
    x = np.array([1.0, 2.0 ** -26.5 if False else 0.0, 0.0], dtype=np.float32)
    # t0^2 = 1, t1^2 = t2^2 = 2^-54 (t = 2^-27, exactly representable in fp32)
    x = np.array([1.0, 2.0 ** -27, 2.0 ** -27], dtype=np.float32)
    y = np.zeros(3, dtype=np.float32)
    assert oracle.sq_l2(x, y) == 1.0          # 1 + 2^-54 rounds to 1, twice
    assert oracle.sq_l2(x[::-1].copy(), y) == 1.0 + 2.0 ** -53  # 2^-54+2^-54 first


@pytest.mark.parametrize("a", [2, 3, 5])
def test_lattice_eps_one_closed_form(a):
    """Integer lattice {0..a}^3 with eps = 1: degree 6 interior, 5 face, 4 edge,
    3 corner; every edge lies exactly at distance eps (tests the closed ball)."""
    pts = lattice(a)
    sp = oracle.Space(points=pts)
    bf = oracle.brute_force(sp, 1.0)
    deg = np.diff(bf["row_ptr"])
    np.testing.assert_array_equal(deg, lattice_degree_closed_form(pts, a, 1))
    interior = np.all((pts > 0) & (pts < a), axis=1)
    if interior.any():
        assert np.all(deg[interior] == 6)
    corners = np.all((pts == 0) | (pts == a), axis=1)
    assert np.all(deg[corners] == 3)
    assert np.all(bf["dist"] == 1.0)
    tr = oracle.build_tree(sp, zeta=4)
    assert oracle.check_tree(sp, tr)[0] == 0
    assert oracle.csr_equal(bf, oracle.tree_query(sp, tr, 1.0))


def test_lattice_sqrt2_rounding():
    """eps = sqrt(2) rounded up to fp32 takes the 12 face diagonals (18 interior);
    rounded down it takes none of them (6 interior)."""
    a = 4
    pts = lattice(a)
    sp = oracle.Space(points=pts)
    down = float(np.float32(math.sqrt(2.0)))
    up = float(np.nextafter(np.float32(math.sqrt(2.0)), np.float32(np.inf)))
    assert down < math.sqrt(2.0) < up
    deg_up = np.diff(oracle.brute_force(sp, up)["row_ptr"])
    deg_dn = np.diff(oracle.brute_force(sp, down)["row_ptr"])
    np.testing.assert_array_equal(deg_up, lattice_degree_closed_form(pts, a, 2))
    np.testing.assert_array_equal(deg_dn, lattice_degree_closed_form(pts, a, 1))
    interior = np.all((pts > 0) & (pts < a), axis=1)
    assert np.all(deg_up[interior] == 18) and np.all(deg_dn[interior] == 6)
    tr = oracle.build_tree(sp, zeta=8)
    assert oracle.csr_equal(oracle.brute_force(sp, up), oracle.tree_query(sp, tr, up))


def test_complete_and_empty_graphs():
    x = I.uniform_cube(300, 5, seed=3)
    sp = oracle.Space(points=x)
    n = x.shape[0]
    full = oracle.brute_force(sp, 10.0)             # diameter of [0,1]^5 is sqrt(5)
    assert full["row_ptr"][-1] == n * (n - 1)
    assert oracle.brute_force(sp, 10.0, include_self=True)["row_ptr"][-1] == n * n
    # grid with spacing 1: eps = 0.5 is below the minimum separation
    g = lattice(3)
    assert oracle.brute_force(oracle.Space(points=g), 0.5)["row_ptr"][-1] == 0


def test_eps_zero_gives_duplicate_classes():
    rng = np.random.default_rng(7)
    distinct = rng.random((20, 4)).astype(np.float32)
    idx = rng.integers(0, 20, size=400)
    x = distinct[idx]
    sp = oracle.Space(points=x)
    bf = oracle.brute_force(sp, 0.0)
    counts = np.bincount(idx, minlength=20)
    assert bf["row_ptr"][-1] == int(np.sum(counts * (counts - 1)))
    for i in range(0, 400, 37):
        row = bf["col"][bf["row_ptr"][i]:bf["row_ptr"][i + 1]]
        np.testing.assert_array_equal(row, np.flatnonzero((idx == idx[i]) & (np.arange(400) != i)))
    # many duplicates (> zeta) become one radius-0 leaf block; the tree still agrees
    tr = oracle.build_tree(sp, zeta=4)
    assert oracle.check_tree(sp, tr)[0] == 0
    assert np.any((tr.radius == 0) & (tr.pts_count > 4))
    assert oracle.csr_equal(bf, oracle.tree_query(sp, tr, 0.0))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_one_dimensional_sorted_sweep(seed):
    """1-D: neighbours by sorting and a two-pointer sweep over the sorted order
    (a different algorithm); the predicate (x-y)^2 <= eps^2 in FP64."""
    rng = np.random.default_rng(seed)
    x = rng.random((1500, 1)).astype(np.float32)
    eps = 0.003
    bf = oracle.brute_force(oracle.Space(points=x), eps)
    v = x[:, 0].astype(np.float64)
    order = np.argsort(v, kind="stable")
    sv = v[order]
    eps2 = eps * eps
    rows = [[] for _ in range(v.size)]
    lo = 0
    for a in range(sv.size):
        while (sv[a] - sv[lo]) * (sv[a] - sv[lo]) > eps2:
            lo += 1
        for b in range(lo, a):
            t = sv[a] - sv[b]
            if t * t <= eps2:
                rows[order[a]].append(order[b])
                rows[order[b]].append(order[a])
    deg = np.array([len(r) for r in rows])
    np.testing.assert_array_equal(np.diff(bf["row_ptr"]), deg)
    for i in range(0, v.size, 97):
        np.testing.assert_array_equal(bf["col"][bf["row_ptr"][i]:bf["row_ptr"][i + 1]], sorted(rows[i]))


@pytest.mark.parametrize("dim", [2, 7, 32])
def test_against_torch_cdist_away_from_band(dim):
    """torch.cdist in float64 (a library routine with another op order) agrees on
    every pair farther than 1e-9*eps from the boundary."""
    torch = pytest.importorskip("torch")
    x = I.gmm_embedded(700, dim=dim, intrinsic=min(4, dim), n_centres=3, seed=dim)
    sp = oracle.Space(points=x)
    t = torch.from_numpy(x.astype(np.float64))
    d = torch.cdist(t, t).numpy()
    eps = float(np.quantile(d[np.triu_indices(700, 1)], 0.02))
    bf = oracle.brute_force(sp, eps)
    adj = np.zeros((700, 700), dtype=bool)
    rows = np.repeat(np.arange(700), np.diff(bf["row_ptr"]))
    adj[rows, bf["col"]] = True
    far = np.abs(d - eps) > 1e-9 * eps
    np.fill_diagonal(far, False)
    ref = d <= eps
    assert np.array_equal(adj[far], ref[far])
    np.testing.assert_allclose(bf["dist"], d[rows, bf["col"]], rtol=1e-12, atol=1e-12)


def test_table1_counts_both_directions():
    """Table I's 'Edges' equals points x average neighbours, i.e. each undirected
    edge is counted in both directions, which is the CSR nnz convention."""
    with open(os.path.join(GOLDEN, "table1_edges.json")) as f:
        rows = json.load(f)["rows"]
    for r in rows:
        est = r["points"] * r["avg"]
        digits = len(str(int(round(r["edges"] / 10 ** int(math.log10(r["edges"]) - 2)))))
        assert abs(est - r["edges"]) / r["edges"] < 0.035, r
    # and the oracle's nnz equals n x mean degree by construction
    x = I.uniform_cube(500, 3, seed=5)
    bf = oracle.brute_force(oracle.Space(points=x), 0.1)
    assert bf["row_ptr"][-1] == np.diff(bf["row_ptr"]).sum()
    assert oracle.csr_symmetric(bf)


# ------------------------------------------------------------- Levenshtein

def _lev_recursive(a: bytes, b: bytes) -> int:
    @lru_cache(maxsize=None)
    def f(i, j):
        if i == 0:
            return j
        if j == 0:
            return i
        return min(f(i - 1, j) + 1, f(i, j - 1) + 1, f(i - 1, j - 1) + (a[i - 1] != b[j - 1]))
    return f(len(a), len(b))


def test_levenshtein_textbook_values():
    with open(os.path.join(GOLDEN, "levenshtein_textbook.json")) as f:
        pairs = json.load(f)["pairs"]
    for a, b, d in pairs:
        assert oracle.lev(a.encode(), b.encode()) == d, (a, b)
        assert oracle.lev_banded(a.encode(), b.encode(), d) == d
        assert oracle.lev_banded(a.encode(), b.encode(), max(d - 1, 0)) == max(d - 1, 0) + 1 or d == 0


def test_levenshtein_against_recursive_definition():
    rng = np.random.default_rng(11)
    for _ in range(300):
        la, lb = rng.integers(0, 9, size=2)
        a = bytes(rng.choice(list(b"ACG"), size=la).tolist())
        b = bytes(rng.choice(list(b"ACG"), size=lb).tolist())
        assert oracle.lev(a, b) == _lev_recursive(a, b)


def test_levenshtein_banded_matches_full_and_properties():
    data, off = I.random_strings(120, 0, 40, seed=4)
    s = [bytes(data[off[i]:off[i + 1]]) for i in range(120)]
    rng = np.random.default_rng(5)
    for _ in range(2000):
        i, j = rng.integers(0, 120, size=2)
        k = int(rng.integers(0, 45))
        full = oracle.lev(s[i], s[j])
        band = oracle.lev_banded(s[i], s[j], k)
        assert band == (full if full <= k else k + 1)
        assert full == oracle.lev(s[j], s[i])
        assert full >= abs(len(s[i]) - len(s[j]))
    for _ in range(300):
        i, j, m = rng.integers(0, 120, size=3)
        assert oracle.lev(s[i], s[m]) <= oracle.lev(s[i], s[j]) + oracle.lev(s[j], s[m])
    # one substitution -> 1, identical -> 0
    a = bytearray(s[3]) or bytearray(b"A")
    b = bytearray(a)
    b[len(b) // 2] = ord("T") if b[len(b) // 2] != ord("T") else ord("A")
    assert oracle.lev(bytes(a), bytes(b)) == 1 and oracle.lev(bytes(a), bytes(a)) == 0


def test_levenshtein_brute_force_graph():
    data, off = I.dna_strings(n_seeds=6, per_seed=25, seed=2)
    sp = oracle.Space(strings=(data, off))
    n = off.size - 1
    bf = oracle.brute_force(sp, 8)
    s = [bytes(data[off[i]:off[i + 1]]) for i in range(n)]
    rng = np.random.default_rng(0)
    for i in rng.integers(0, n, size=10):
        want = [j for j in range(n) if j != i and oracle.lev(s[i], s[j]) <= 8]
        np.testing.assert_array_equal(bf["col"][bf["row_ptr"][i]:bf["row_ptr"][i + 1]], want)
    assert oracle.csr_symmetric(bf)


# ------------------------------------------------------------- cover tree

@pytest.mark.parametrize("dim,n,seed,zeta", [(1, 800, 0, 8), (2, 1500, 1, 16), (3, 2000, 0, 32),
                                              (8, 1200, 2, 32), (16, 1000, 3, 5), (5, 600, 4, 1)])
def test_tree_query_equals_brute_force(dim, n, seed, zeta):
    x = I.gmm_embedded(n, dim=dim, intrinsic=min(dim, 4), n_centres=4, seed=seed) \
        if dim > 3 else I.uniform_cube(n, dim, seed=seed)
    sp = oracle.Space(points=x)
    tr = oracle.build_tree(sp, zeta=zeta)
    assert oracle.check_tree(sp, tr) == (0, "")
    rng = np.random.default_rng(seed)
    bf_full = oracle.brute_force(sp, 1e9)
    d_sample = bf_full["dist"][rng.integers(0, bf_full["dist"].size, size=2000)]
    for q in (0.002, 0.02, 0.1):
        eps = float(np.quantile(d_sample, q))
        bf = oracle.brute_force(sp, eps)
        tq = oracle.tree_query(sp, tr, eps)
        assert oracle.csr_equal(bf, tq), (dim, eps)
        np.testing.assert_array_equal(bf["dist"], tq["dist"])
        assert oracle.csr_symmetric(tq)
        assert tq["dist_evals"] < bf["dist_evals"] or n < 1000


def test_tree_small_and_degenerate_sizes():
    for n in (0, 1, 2, 3):
        x = I.uniform_cube(n, 3, seed=n)
        sp = oracle.Space(points=x)
        tr = oracle.build_tree(sp, zeta=1)
        assert oracle.check_tree(sp, tr)[0] == 0
        for eps in (0.0, 0.5, 5.0):
            bf = oracle.brute_force(sp, eps)
            assert oracle.csr_equal(bf, oracle.tree_query(sp, tr, eps))
            assert bf["row_ptr"].size == n + 1
    # all points identical: one radius-0 leaf block of every point
    x = np.ones((100, 3), dtype=np.float32)
    sp = oracle.Space(points=x)
    tr = oracle.build_tree(sp, zeta=8)
    assert tr.n_nodes == 1 and tr.radius[0] == 0 and tr.pts_count[0] == 100
    assert oracle.tree_query(sp, tr, 0.0)["row_ptr"][-1] == 100 * 99


def test_tree_levenshtein_equals_brute_force():
    data, off = I.dna_strings(n_seeds=8, per_seed=30, seed=3)
    sp = oracle.Space(strings=(data, off))
    tr = oracle.build_tree(sp, zeta=8)
    assert oracle.check_tree(sp, tr) == (0, "")
    for eps in (0, 3, 8, 20):
        assert oracle.csr_equal(oracle.brute_force(sp, eps), oracle.tree_query(sp, tr, eps))


def test_tree_net_properties_by_direct_check():
    """Covering and separation recomputed here, outside the C checker."""
    x = I.uniform_cube(400, 2, seed=9)
    sp = oracle.Space(points=x)
    tr = oracle.build_tree(sp, zeta=4)
    X = x.astype(np.float64)
    for u in range(tr.n_nodes):
        nc = tr.child_count[u]
        if nc == 0:
            continue
        kids = tr.center[tr.child_begin[u]:tr.child_begin[u] + nc]
        assert kids[0] == tr.center[u]
        lvl = tr.level[u]
        dc = np.sqrt(((X[kids] - X[tr.center[u]]) ** 2).sum(1))
        assert np.all(dc <= 2.0 ** lvl * (1 + 1e-12))
        for a in range(nc):
            for b in range(a + 1, nc):
                assert np.sqrt(((X[kids[a]] - X[kids[b]]) ** 2).sum()) > 2.0 ** (lvl - 1) * (1 - 1e-12)


def _copy_tree(tr):
    return oracle.Tree(**{f: getattr(tr, f).copy() for f in oracle.Tree.FIELDS})


def test_checker_catches_planted_mistakes():
    """Plant one mistake at a time in an oracle tree; each check must fire."""
    x = I.uniform_cube(500, 3, seed=2)
    sp = oracle.Space(points=x)
    tr = oracle.build_tree(sp, zeta=8)
    assert oracle.check_tree(sp, tr)[0] == 0
    internal = np.flatnonzero(tr.child_count > 0)
    u = int(internal[-1])

    bad = _copy_tree(tr)                       # radius one ulp too small
    bad.radius[u] = np.nextafter(bad.radius[u], 0.0)
    code, msg = oracle.check_tree(sp, bad)
    assert code in (6, 7, 9) and code != 0

    bad = _copy_tree(tr)                       # radius too small by 10%
    leaf = int(np.flatnonzero((tr.child_count == 0) & (tr.pts_count > 2))[0])
    bad.radius[leaf] *= 0.9
    assert oracle.check_tree(sp, bad)[0] == 9

    bad = _copy_tree(tr)                       # nesting broken
    cb = bad.child_begin[u]
    bad.center[cb], bad.center[cb + 1] = bad.center[cb + 1], bad.center[cb]
    assert oracle.check_tree(sp, bad)[0] != 0

    bad = _copy_tree(tr)                       # a point in two leaf blocks
    bad.leaf_pts[1] = bad.leaf_pts[2]
    assert oracle.check_tree(sp, bad)[0] == 3

    bad = _copy_tree(tr)                       # separation violated: level too high
    bad.level[0] += 3
    code, _ = oracle.check_tree(sp, bad)
    assert code == 8


def test_tree_query_catches_planted_radius_error():
    """A tree whose radius underestimates a subtree loses edges: the brute-force
    comparison detects it (the pruning depends on the radius bound)."""
    x = I.uniform_cube(1500, 2, seed=6)
    sp = oracle.Space(points=x)
    tr = oracle.build_tree(sp, zeta=8)
    bad = _copy_tree(tr)
    bad.radius[1:] *= 0.5
    eps = 0.02
    assert not oracle.csr_equal(oracle.brute_force(sp, eps), oracle.tree_query(sp, bad, eps))
