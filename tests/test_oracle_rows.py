"""Pins of the oracle's row-restricted routines, ``brute_rows`` and
``tree_query_rows``: the checkers of every full-size parity test and the timed
CPU baseline.  Each is held against something other than itself -- the
whole-graph brute force (itself pinned by closed forms and library routines),
closed forms on the integer lattice, and an independent numpy evaluation of
the Sec. III definition.  CPU only."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2510_14147_gb300 import inputs as I


def rows_of(csr: dict, r: int):
    a, b = int(csr["row_ptr"][r]), int(csr["row_ptr"][r + 1])
    return np.asarray(csr["col"][a:b], np.int64), np.asarray(csr["dist"][a:b], np.float64)


def assert_rows_match(sub: dict, full: dict, rows):
    """Row k of `sub` must be row rows[k] of `full`, entry for entry."""
    assert sub["row_ptr"].size == len(rows) + 1
    for k, r in enumerate(rows):
        c1, d1 = rows_of(sub, k)
        c2, d2 = rows_of(full, int(r))
        np.testing.assert_array_equal(c1, c2, err_msg="row %d (point %d)" % (k, r))
        np.testing.assert_array_equal(d1, d2, err_msg="row %d (point %d)" % (k, r))


def row_lists(n: int, rng):
    """Row lists that catch an index mix-up: unsorted, repeated, reversed, the
    first and last point, a single row and the empty list."""
    perm = rng.permutation(n)
    return [perm[: min(n, 37)],                       # unsorted
            np.array([n - 1, 0, n - 1, 3 % n]),        # repeated, ends of the range
            np.arange(n)[::-1][: min(n, 20)],          # descending
            np.array([n // 2]),
            np.array([], dtype=np.int64)]


@pytest.mark.parametrize("dim,seed,include_self", [(2, 0, False), (3, 1, True), (8, 2, False), (16, 3, True)])
def test_brute_rows_equal_rows_of_brute_force(dim, seed, include_self):
    rng = np.random.default_rng(seed)
    x = I.uniform_cube(400, dim, seed=seed)
    # a few duplicates: distance-0 pairs with distinct indices are edges
    x[5] = x[17]
    x[200] = x[17]
    sp = oracle.Space(points=x)
    eps = float(np.float32(0.35 if dim <= 3 else 0.8))
    full = oracle.brute_force(sp, eps, include_self=include_self)
    for rows in row_lists(x.shape[0], rng):
        sub = oracle.brute_rows(sp, eps, rows, include_self=include_self)
        assert_rows_match(sub, full, rows)
        assert sub["dist_evals"] == len(rows) * x.shape[0]


@pytest.mark.parametrize("dim,seed,zeta,include_self", [(2, 4, 4, False), (3, 5, 32, True),
                                                        (8, 6, 1, False), (16, 7, 8, True)])
def test_tree_query_rows_equal_rows_of_tree_query_and_brute_force(dim, seed, zeta, include_self):
    rng = np.random.default_rng(seed)
    x = I.gmm_embedded(500, dim=dim, n_centres=5, intrinsic=min(4, dim), centre_sd=2.0, seed=seed)
    sp = oracle.Space(points=x)
    eps = float(np.float32(0.9))
    tree = oracle.build_tree(sp, zeta=zeta)
    full_tree = oracle.tree_query(sp, tree, eps, include_self=include_self)
    full_bf = oracle.brute_force(sp, eps, include_self=include_self)
    for rows in row_lists(x.shape[0], rng):
        sub = oracle.tree_query_rows(sp, tree, eps, rows, include_self=include_self)
        assert_rows_match(sub, full_tree, rows)
        assert_rows_match(sub, full_bf, rows)


def test_row_routines_on_edit_distance():
    data, off = I.dna_strings(n_seeds=6, per_seed=12, seed_len=40, min_len=30, max_len=50, seed=3)
    sp = oracle.Space(strings=(data, off))
    full = oracle.brute_force(sp, 6)
    tree = oracle.build_tree(sp, zeta=4)
    rows = np.array([71, 0, 13, 13, 40])
    assert_rows_match(oracle.brute_rows(sp, 6, rows), full, rows)
    assert_rows_match(oracle.tree_query_rows(sp, tree, 6, rows), full, rows)


def test_rows_on_the_lattice_closed_form():
    """{0..a}^3 at eps = 1: a vertex's neighbours are exactly its lattice
    neighbours one unit away along an axis (enumerated, no distance taken)."""
    a = 4
    g = np.arange(a + 1, dtype=np.float32)
    pts = np.array(list(itertools.product(g, g, g)), dtype=np.float32)
    index = {tuple(p.astype(int)): i for i, p in enumerate(pts)}
    sp = oracle.Space(points=pts)
    tree = oracle.build_tree(sp, zeta=3)
    rows = np.array([124, 0, 62, 31, 7])
    for fn in (lambda: oracle.brute_rows(sp, 1.0, rows),
               lambda: oracle.tree_query_rows(sp, tree, 1.0, rows)):
        sub = fn()
        for k, r in enumerate(rows):
            p = pts[r].astype(int)
            want = []
            for ax, s in itertools.product(range(3), (-1, 1)):
                q = p.copy()
                q[ax] += s
                if np.all(q >= 0) and np.all(q <= a):
                    want.append(index[tuple(q)])
            c, d = rows_of(sub, k)
            np.testing.assert_array_equal(c, np.sort(want))
            assert np.all(d == 1.0)


def test_brute_rows_against_numpy_definition():
    """Independent evaluation of Sec. III's set for sampled rows: numpy FP64
    squared distances compared with eps^2, away from the boundary (a pair whose
    squared distance is within 1e-9 relative of eps^2 is skipped)."""
    x = I.gmm_embedded(3000, dim=32, n_centres=10, intrinsic=8, seed=9)
    sp = oracle.Space(points=x)
    eps = float(np.float32(2.5))
    rng = np.random.default_rng(10)
    rows = rng.choice(x.shape[0], size=64, replace=False)
    sub = oracle.brute_rows(sp, eps, rows)
    xd = x.astype(np.float64)
    for k, r in enumerate(rows):
        s = np.sum((xd - xd[r]) ** 2, axis=1)
        near = np.abs(s - eps * eps) <= 1e-9 * eps * eps
        want = np.flatnonzero((s <= eps * eps) & (np.arange(x.shape[0]) != r))
        c, d = rows_of(sub, k)
        assert set(c.tolist()) ^ set(want.tolist()) <= set(np.flatnonzero(near).tolist())
        np.testing.assert_allclose(d, np.sqrt(s[c]), rtol=1e-12)
