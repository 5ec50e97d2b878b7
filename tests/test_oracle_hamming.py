"""Pins of the oracle's Hamming metric (the binary datasets of Sec. V-A,
Table I: sift-hamming, word2bits) against things other than itself: numpy's
bit unpacking, closed forms on the hypercube, and brute force.  CPU only."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2510_14147_gb300 import inputs as I


def unpack(rows, dim):
    return np.unpackbits(np.asarray(rows, np.uint8), axis=1, bitorder="little")[:, :dim]


def pack(bits):
    return np.packbits(np.asarray(bits, bool), axis=1, bitorder="little")


@pytest.mark.parametrize("dim", [1, 7, 8, 13, 63, 64, 65, 256, 800])
def test_hamming_against_numpy_bits(dim):
    rng = np.random.default_rng(dim)
    b = rng.random((40, dim)) < 0.5
    rows = pack(b)
    for i, j in itertools.combinations(range(12), 2):
        assert oracle.hamming(rows[i], rows[j], dim) == int(np.sum(b[i] != b[j]))


@pytest.mark.parametrize("dim", [5, 13, 64, 100])
def test_hamming_closed_forms(dim):
    zero = np.zeros((1, dim), bool)
    rows0 = pack(zero)[0]
    for j in range(dim):              # one set bit at position j (catches a reversed bit order)
        e = zero.copy()
        e[0, j] = True
        assert oracle.hamming(rows0, pack(e)[0], dim) == 1
    rng = np.random.default_rng(1)
    x = rng.random((1, dim)) < 0.5
    assert oracle.hamming(pack(x)[0], pack(x)[0], dim) == 0
    assert oracle.hamming(pack(x)[0], pack(~x)[0], dim) == dim       # complement: every bit
    # bits past dim in the last byte do not count
    raw = pack(x)[0].copy()
    if dim % 8:
        raw2 = raw.copy()
        raw2[-1] |= np.uint8(0xFF << (dim % 8) & 0xFF)
        assert oracle.hamming(raw, raw2, dim) == 0


def test_hypercube_degrees_closed_form():
    """{0,1}^k: every vertex has sum_{j=1..r} C(k, j) vertices within Hamming
    distance r; eps = r + 0.7 gives the same graph (integer distances)."""
    k = 10
    cube = np.array(list(itertools.product([0, 1], repeat=k)), bool)
    sp = oracle.Space(bits=(pack(cube), k))
    for r in (0, 1, 2, 4, k):
        want = sum(math.comb(k, j) for j in range(1, r + 1))
        for eps in (float(r), r + 0.7):
            bf = oracle.brute_force(sp, eps)
            assert np.all(np.diff(bf["row_ptr"]) == want)
        assert np.all(bf["dist"] <= r) and np.all(bf["dist"] == np.round(bf["dist"]))
    assert oracle.csr_symmetric(oracle.brute_force(sp, 3))


@pytest.mark.parametrize("dim,n,zeta,seed", [(32, 1500, 8, 0), (256, 2000, 32, 1), (800, 1200, 16, 2),
                                             (13, 900, 4, 3)])
def test_tree_query_equals_brute_force_and_invariants(dim, n, zeta, seed):
    rows = I.binary_codes(n, dim, n_centres=12, flip=0.06, seed=seed)
    sp = oracle.Space(bits=(rows, dim))
    tree = oracle.build_tree(sp, zeta=zeta)
    assert oracle.check_tree(sp, tree)[0] == 0
    b = unpack(rows, dim)
    for eps in (0, 2, 0.12 * dim, 0.3 * dim):
        bf = oracle.brute_force(sp, eps)
        assert oracle.csr_equal(bf, oracle.tree_query(sp, tree, eps))
        # spot-check rows against numpy's bits
        for i in (0, n // 2, n - 1):
            a, e = int(bf["row_ptr"][i]), int(bf["row_ptr"][i + 1])
            d = np.sum(b != b[i], axis=1)
            want = np.flatnonzero((d <= math.floor(eps)) & (np.arange(n) != i))
            np.testing.assert_array_equal(bf["col"][a:e], want)
            np.testing.assert_array_equal(bf["dist"][a:e], d[want])


def test_triangle_inequality_and_symmetry():
    rows = I.binary_codes(60, 77, n_centres=3, flip=0.2, seed=4)
    h = lambda i, j: oracle.hamming(rows[i], rows[j], 77)
    for i, j, k in itertools.combinations(range(0, 60, 4), 3):
        assert h(i, j) == h(j, i)
        assert h(i, k) <= h(i, j) + h(j, k)
