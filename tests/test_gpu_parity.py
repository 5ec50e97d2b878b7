"""Parity of the CUDA path (through the C-ABI) with the CPU oracle: exact
row_ptr/col, dist within 1e-6 relative of FP64, GPU-built trees checked by
the oracle's invariant checker."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2510_14147_gb300 import inputs as I
from helpers import assert_csr_matches, gpu_graph, tree_from_export

pytestmark = pytest.mark.gpu

# fp32-built trees: relative tolerance of the net properties.  The build
# decides every split on fp32 distances whose relative error is below 2^-17
# (sums of at most 4096 squared differences in lane-split fp32), and its
# triangle-inequality skip never changes a decision (a point is skipped only
# when the computed distance could not have been smaller, with a 2^-12
# margin against errors of that size), so covering and separation hold
# within 2^-17 in FP64.  A vertex's level is ceil(log2 r) of its fp32 radius
# r, and the radius is stored rounded up to r (1 + 2^-16) so that the query's
# pruning bound stays safe: the stored radius may exceed 2^l by 2^-16.
# Together: 2^-16 + 2^-17 < 2.5e-5.
TREE_TOL = 2.5e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_14147_gb300 import build
    build.build()
    oracle.build()


def _check_tree(space, out):
    code, msg = oracle.check_tree(space, tree_from_export(out["tree"]), TREE_TOL)
    assert code == 0, msg


def test_small_3d_workload_exact():
    """n=2000 uniform [0,1]^3, eps=0.08, zeta=32 (the small configuration)."""
    x = I.uniform_cube(2000, 3, seed=0)
    sp = oracle.Space(points=x)
    ref = oracle.brute_force(sp, 0.08)
    out = gpu_graph(points=x, eps=0.08, export=True)
    assert_csr_matches(out, ref)
    _check_tree(sp, out)
    assert out["stats"]["leaf_pairs"] > 0 and out["stats"]["traversal_evals"] > 0


@pytest.mark.parametrize("dim,n,zeta,seed", [
    (1, 1500, 8, 0), (2, 2500, 16, 1), (3, 3000, 32, 2), (5, 2000, 32, 3), (8, 2600, 32, 4),
    (16, 2200, 17, 5), (33, 1800, 32, 6), (64, 2100, 32, 7), (128, 2300, 32, 8),
    (130, 1200, 32, 9), (300, 900, 24, 10), (7, 2000, 1, 11), (12, 1000, 100, 12)])
def test_parity_dims_and_leaf_sizes(dim, n, zeta, seed):
    """Several tiles per group and candidate, ragged tails (n, dim, zeta not
    multiples of the tile sizes), K-chunked rows above 128 floats."""
    x = I.gmm_embedded(n, dim=dim, intrinsic=min(dim, 6), n_centres=5, seed=seed) if dim > 3 \
        else I.uniform_cube(n, dim, seed=seed)
    sp = oracle.Space(points=x)
    rng = np.random.default_rng(seed)
    sample = oracle.brute_rows(sp, 1e30, rng.integers(0, n, size=8))["dist"]
    for q in (0.003, 0.03, 0.15):
        eps = float(np.float32(np.quantile(sample, q)))
        ref = oracle.brute_force(sp, eps)
        out = gpu_graph(points=x, eps=eps, leaf_size=zeta, export=(q == 0.03))
        assert_csr_matches(out, ref)
        if q == 0.03:
            _check_tree(sp, out)


@pytest.mark.parametrize("precision", [0, 1])
def test_flat_split_in_high_dimension(precision):
    """Uniform points in 64-D: every pairwise distance lies above the split
    threshold of the second level, so farthest-first splitting would make
    every point its own child.  The split stops after its first centres and
    their cells become leaf blocks larger than zeta (still a valid net with
    exact stored radii); the graph stays exact."""
    x = I.uniform_cube(6000, 64, seed=21)
    sp = oracle.Space(points=x)
    rng = np.random.default_rng(21)
    sample = oracle.brute_rows(sp, 1e30, rng.integers(0, 6000, size=8))["dist"]
    for q in (0.001, 0.02):
        eps = float(np.float32(np.quantile(sample, q)))
        out = gpu_graph(points=x, eps=eps, precision=precision, export=True)
        assert_csr_matches(out, oracle.brute_force(sp, eps))
        _check_tree(sp, out)
        tr = out["tree"]
        leaf = np.asarray(tr["child_count"]) == 0
        big = leaf & (np.asarray(tr["pts_count"]) > 32) & (np.asarray(tr["radius"]) > 0)
        assert big.any(), "no flat split happened"


def test_degenerate_sizes():
    for n in (0, 1, 2, 3, 33):
        x = I.uniform_cube(n, 3, seed=n)
        sp = oracle.Space(points=x)
        for eps in (0.0, 0.3, 10.0):
            out = gpu_graph(points=x, eps=eps, export=True)
            assert_csr_matches(out, oracle.brute_force(sp, eps))
            if n:
                _check_tree(sp, out)
            else:
                assert out["row_ptr"].tolist() == [0]


def test_duplicates_above_leaf_size_and_eps_zero():
    rng = np.random.default_rng(3)
    distinct = rng.random((40, 6)).astype(np.float32)
    x = distinct[rng.integers(0, 40, size=3000)]
    x[:200] = x[0]                      # one class far above zeta
    sp = oracle.Space(points=x)
    for eps in (0.0, 0.05, 0.4):
        out = gpu_graph(points=x, eps=eps, leaf_size=16, export=True)
        assert_csr_matches(out, oracle.brute_force(sp, eps))
    _check_tree(sp, out)


def test_eps_zero_with_tiny_coordinates():
    """eps = 0: only exact duplicates are neighbours, also where the fp32
    square of a nonzero difference underflows to zero (|x - y| < 2^-75)."""
    rng = np.random.default_rng(8)
    base = (rng.random((300, 3)) * 1e-30).astype(np.float32)
    base[:10, 0] = np.float32(3e-39)                # subnormal coordinates
    base[10:20] = 0.0
    base[20:30, 1] = np.float32(1e-38)
    x = np.concatenate([base, base[:60]])          # duplicates of the first 60
    x = x[rng.permutation(x.shape[0])]
    sp = oracle.Space(points=x)
    for precision in (0, 1):
        out = gpu_graph(points=x, eps=0.0, leaf_size=8, precision=precision)
        assert_csr_matches(out, oracle.brute_force(sp, 0.0))


def test_row_lengths_in_every_sort_class():
    """Tight clusters of 20..5000 points give rows in the row sort's classes
    (<= 32, 128, 512, 1024, 4096, longer)."""
    rng = np.random.default_rng(12)
    parts = []
    for k, size in enumerate((20, 100, 400, 900, 3000, 5000)):
        centre = rng.random(4) * 100.0
        parts.append(centre + rng.random((size, 4)) * 0.1)
    x = np.concatenate(parts).astype(np.float32)
    x = x[rng.permutation(x.shape[0])]
    sp = oracle.Space(points=x)
    for precision in (0, 1):
        out = gpu_graph(points=x, eps=0.5, precision=precision)
        assert_csr_matches(out, oracle.brute_force(sp, 0.5))
        deg = np.diff(out["row_ptr"])
        assert sorted(set(deg.tolist())) == [19, 99, 399, 899, 2999, 4999]


def test_row_lengths_at_sort_class_boundaries():
    """Rows one below, at and one above each length boundary of the row sort
    (32, 64, 128, 256, 512, 1024, 2048, 4096), and rows of 3 and 6 runs of
    512 (1500, 2600: a run left without a partner in a merge round, a partial
    last run): the sorted rows equal brute force's."""
    rng = np.random.default_rng(5)
    degrees = (2, 31, 32, 33, 63, 64, 65, 127, 128, 129, 200, 255, 256, 257, 511, 512, 513, 1023, 1024, 1025,
               1500, 2047, 2048, 2049, 2600, 4095, 4096, 4097)
    parts = [rng.random(4) * 100.0 + rng.random((d + 1, 4)) * 0.1 for d in degrees]
    x = np.concatenate(parts).astype(np.float32)
    x = x[rng.permutation(x.shape[0])]
    ref = oracle.brute_force(oracle.Space(points=x), 0.5)
    for precision in (0, 1):
        out = gpu_graph(points=x, eps=0.5, precision=precision)
        assert_csr_matches(out, ref)
        assert sorted(set(np.diff(out["row_ptr"]).tolist())) == list(degrees)


def test_row_sort_past_the_packed_keys():
    """1.1M points: more columns than the row sort's packed keys (column << 12
    | position, 32 bits) hold, so rows sort as (column, distance) pairs.
    Tight clusters of 40..5000 points give rows in every length class;
    sampled rows of every cluster and of the background equal brute force's,
    and every row is strictly increasing."""
    rng = np.random.default_rng(21)
    sizes = (40, 70, 140, 300, 600, 1500, 3000, 5000)
    n = 1_100_000
    assert n > 1 << 20
    parts = [rng.random(3) * 1000.0 + rng.random((s, 3)) * 0.2 for s in sizes]
    parts.append(rng.random((n - sum(sizes), 3)) * 1000.0)
    perm = rng.permutation(n)
    x = np.concatenate(parts).astype(np.float32)[perm]
    where = np.argsort(perm)                     # original index -> row
    out = gpu_graph(points=x, eps=0.5)
    rows, start = [], 0
    for s in sizes:
        rows += list(where[start + rng.choice(s, size=3, replace=False)])
        start += s
    rows += list(rng.choice(n, size=40, replace=False))
    rows = np.unique(np.asarray(rows, np.int64))
    ref = oracle.brute_rows(oracle.Space(points=x), 0.5, rows)
    rp, col, dist = out["row_ptr"], out["col"], out["dist"]
    deg = np.diff(rp)
    for s in sizes:
        assert (deg == s - 1).any() or (deg == s).any()
    for k, r in enumerate(rows):
        a, b = int(rp[r]), int(rp[r + 1])
        ra, rb = int(ref["row_ptr"][k]), int(ref["row_ptr"][k + 1])
        np.testing.assert_array_equal(np.asarray(col[a:b], np.int64), ref["col"][ra:rb], err_msg="row %d" % r)
        rd = ref["dist"][ra:rb]
        assert np.all(np.abs(np.asarray(dist[a:b], np.float64) - rd) <= 1e-6 * np.abs(rd)), "row %d" % r
    step = np.diff(np.asarray(col, np.int64))
    inner = np.ones(step.size, bool)
    starts = rp[1:-1][(rp[1:-1] > 0) & (rp[1:-1] < col.size)] - 1
    inner[starts] = False
    assert np.all(step[inner] > 0)


def test_complete_graph_and_include_self():
    x = I.uniform_cube(700, 4, seed=1)
    sp = oracle.Space(points=x)
    out = gpu_graph(points=x, eps=5.0)
    assert out["row_ptr"][-1] == 700 * 699
    assert_csr_matches(out, oracle.brute_force(sp, 5.0))
    out = gpu_graph(points=x, eps=0.2, include_self=True)
    assert_csr_matches(out, oracle.brute_force(sp, 0.2, include_self=True))


def test_lattice_ties_exactly_at_eps():
    """Every edge of the lattice lies exactly at eps (or at sqrt 2 rounded to
    fp32 either way): the decision at the boundary is the FP64 one."""
    g = np.arange(9, dtype=np.float32)
    x = np.array(list(itertools.product(g, g, g)), dtype=np.float32)
    sp = oracle.Space(points=x)
    up = float(np.nextafter(np.float32(math.sqrt(2)), np.float32(np.inf)))
    dn = float(np.float32(math.sqrt(2)))
    for eps in (1.0, up, dn, math.sqrt(3)):
        out = gpu_graph(points=x, eps=eps, leaf_size=8)
        ref = oracle.brute_force(sp, eps)
        assert_csr_matches(out, ref)
        assert out["stats"]["guard_fp64"] > 0 or eps == math.sqrt(3)


def test_large_offsets_no_cancellation():
    """Points far from the origin with small separations: direct differences
    keep full relative accuracy."""
    base = I.uniform_cube(2500, 16, seed=4).astype(np.float64)
    x = (base + 3000.0).astype(np.float32)      # |x|^2 ~ 1.4e8 against d^2 ~ 1
    sp = oracle.Space(points=x)
    sample = oracle.brute_rows(sp, 1e30, [0, 1, 2])["dist"]
    eps = float(np.quantile(sample[sample > 0], 0.02))
    assert_csr_matches(gpu_graph(points=x, eps=eps), oracle.brute_force(sp, eps))


def test_root_choice_does_not_change_output():
    x = I.uniform_cube(1500, 5, seed=8)
    a = gpu_graph(points=x, eps=0.2, root=0)
    b = gpu_graph(points=x, eps=0.2, root=777)
    assert np.array_equal(a["row_ptr"], b["row_ptr"]) and np.array_equal(a["col"], b["col"])


def test_near_boundary_pairs_random():
    """Pairs placed at eps * (1 +- 1e-7 .. 1e-3): inside the guard band the FP64
    decision must match the oracle bit for bit."""
    rng = np.random.default_rng(0)
    n, dim, eps = 1200, 24, 0.75
    a = rng.standard_normal((n // 2, dim)).astype(np.float32) * 3
    u = rng.standard_normal((n // 2, dim))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    scale = eps * (1 + rng.choice([-1, 1], n // 2) * 10 ** rng.uniform(-7.5, -3, n // 2))
    b = (a + u * scale[:, None]).astype(np.float32)
    x = np.concatenate([a, b])
    sp = oracle.Space(points=x)
    out = gpu_graph(points=x, eps=eps)
    assert_csr_matches(out, oracle.brute_force(sp, eps))
    assert out["stats"]["guard_fp64"] >= n // 4


# ------------------------------------------------------------ edit distance

@pytest.mark.parametrize("eps", [0, 3, 8, 15])
def test_levenshtein_dna(eps):
    data, off = I.dna_strings(n_seeds=12, per_seed=60, seed=5)
    sp = oracle.Space(strings=(data, off))
    out = gpu_graph(strings=(data, off), eps=eps, leaf_size=16, export=(eps == 8))
    assert_csr_matches(out, oracle.brute_force(sp, eps), integer_dist=True)
    if eps == 8:
        code, msg = oracle.check_tree(sp, tree_from_export(out["tree"]), 0.0)
        assert code == 0, msg


def test_levenshtein_mixed_lengths_and_alphabet():
    d1, o1 = I.random_strings(500, 0, 150, alphabet=b"ACGTN", seed=1)
    d2, o2 = I.random_strings(300, 60, 70, alphabet=bytes(range(32, 127)), seed=2)
    data = np.concatenate([d1, d2])
    off = np.concatenate([o1, o2[1:] + o1[-1]])
    # a few near-duplicates so that some edges exist
    sp = oracle.Space(strings=(data, off))
    for eps in (2, 40, 300):
        out = gpu_graph(strings=(data, off), eps=eps, leaf_size=8)
        assert_csr_matches(out, oracle.brute_force(sp, eps), integer_dist=True)


def test_levenshtein_long_strings_multiword():
    data, off = I.dna_strings(n_seeds=4, per_seed=40, seed_len=700, min_len=600, max_len=800, seed=9)
    sp = oracle.Space(strings=(data, off))
    out = gpu_graph(strings=(data, off), eps=60, leaf_size=8)
    assert_csr_matches(out, oracle.brute_force(sp, 60), integer_dist=True)


# ------------------------------------------------------------ full size

@pytest.mark.parametrize("key", ["gmm_1m_k70"])
def test_full_size_sampled_rows(key):
    """1M x 128 points at the calibrated eps: sampled rows equal the oracle's
    brute force; the whole output is symmetric with sorted rows."""
    wl = I.load_workloads()[key]
    x = I.gmm_embedded(wl["n"], dim=wl["dim"], seed=wl["seed"])
    out = gpu_graph(points=x, eps=wl["eps"])
    rp, col = out["row_ptr"], out["col"].astype(np.int64)
    n = x.shape[0]
    mean_deg = rp[-1] / n
    assert 0.5 * wl["target_degree"] < mean_deg < 2.0 * wl["target_degree"]
    rows_ok = np.all((np.diff(col) > 0) | (np.diff(np.repeat(np.arange(n), np.diff(rp))) != 0))
    assert rows_ok
    assert oracle.csr_symmetric({"row_ptr": rp, "col": col})
    rng = np.random.default_rng(1)
    rows = np.sort(rng.choice(n, size=48, replace=False))
    sp = oracle.Space(points=x)
    ref = oracle.brute_rows(sp, wl["eps"], rows)
    sub = {"row_ptr": np.concatenate([[0], np.cumsum(rp[rows + 1] - rp[rows])]),
           "col": np.concatenate([col[rp[r]:rp[r + 1]] for r in rows]),
           "dist": np.concatenate([out["dist"][rp[r]:rp[r + 1]] for r in rows])}
    assert_csr_matches(sub, ref)
