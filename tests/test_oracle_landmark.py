"""Pins of the oracle's landmark construction (Sec. IV-D): Voronoi cells of
random centres, ε-ghosts by Lemma 1, rows by brute force inside each cell and
its ghosts.  Held against numpy's distances, the whole-graph brute force and
the lemma itself; a ghost bound below Lemma 1's (d(p, C) + eps instead of +
2 eps) must lose edges on some input, so that the pin notices a wrong
bound.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_2510_14147_gb300 import inputs as I


def _centres(n, m, seed):
    return np.random.default_rng(seed).choice(n, size=m, replace=False)


@pytest.mark.parametrize("dim,m", [(2, 1), (3, 7), (8, 20), (16, 60)])
def test_voronoi_matches_numpy(dim, m):
    x = I.gmm_embedded(900, dim=dim, intrinsic=min(dim, 4), n_centres=4, seed=dim) if dim > 2 else \
        I.uniform_cube(900, dim, seed=dim)
    c = _centres(900, m, m)
    cell, dmin = oracle.voronoi(oracle.Space(points=x), c)
    d = np.sqrt(((x[:, None, :].astype(np.float64) - x[c][None, :, :]) ** 2).sum(-1))
    np.testing.assert_allclose(dmin, d.min(1), rtol=1e-12)
    # the nearest centre, the lowest index among (numerically) equal ones
    assert np.all(d[np.arange(900), cell] <= d.min(1) * (1 + 1e-12))


@pytest.mark.parametrize("dim,m,q", [(2, 5, 0.01), (3, 30, 0.03), (8, 60, 0.02), (16, 10, 0.05), (8, 900, 0.02)])
def test_lemma1_and_landmark_graph_equal_brute_force(dim, m, q):
    x = I.gmm_embedded(900, dim=dim, intrinsic=min(dim, 4), n_centres=4, seed=3) if dim > 2 else \
        I.uniform_cube(900, dim, seed=3)
    sp = oracle.Space(points=x)
    eps = float(np.float32(np.quantile(oracle.brute_rows(sp, 1e30, [0, 1, 2])["dist"], q)))
    c = _centres(900, m, 11)
    bf = oracle.brute_force(sp, eps)
    # Lemma 1 on every edge between two cells, with numpy's FP64 distances
    cell, dmin = oracle.voronoi(sp, c)
    xd = x.astype(np.float64)
    rows = np.repeat(np.arange(900), np.diff(bf["row_ptr"]))
    cols = bf["col"]
    cross = cell[rows] != cell[cols]
    dpc = np.sqrt(((xd[rows[cross]] - xd[c[cell[cols[cross]]]]) ** 2).sum(-1))
    assert np.all(dpc <= dmin[rows[cross]] + 2 * eps + 1e-12)
    assert oracle.csr_equal(oracle.landmark_graph(sp, c, eps), bf)
    assert oracle.csr_equal(oracle.landmark_graph(sp, c, eps, include_self=True),
                            oracle.brute_force(sp, eps, include_self=True))


def test_landmark_graph_other_metrics():
    data, off = I.dna_strings(n_seeds=6, per_seed=25, seed=2)
    sp = oracle.Space(strings=(data, off))
    c = _centres(off.size - 1, 12, 4)
    assert oracle.csr_equal(oracle.landmark_graph(sp, c, 8), oracle.brute_force(sp, 8))
    rows = I.binary_codes(700, 128, n_centres=8, flip=0.08, seed=5)
    sb = oracle.Space(bits=(rows, 128))
    c = _centres(700, 25, 6)
    assert oracle.csr_equal(oracle.landmark_graph(sb, c, 20), oracle.brute_force(sb, 20))


def test_smaller_ghost_bound_loses_edges():
    """With ghosts only up to d(p, C) + eps some cross-cell edges are missed:
    the factor 2 of Lemma 1 is what the construction needs."""
    lost = 0
    for seed in range(4):
        x = I.uniform_cube(800, 2, seed=seed)
        sp = oracle.Space(points=x)
        c = _centres(800, 40, seed)
        bf = oracle.brute_force(sp, 0.08)
        weak = oracle.landmark_graph(sp, c, 0.08, factor=1.0)
        assert weak["row_ptr"][-1] <= bf["row_ptr"][-1]
        lost += int(bf["row_ptr"][-1] - weak["row_ptr"][-1])
        assert oracle.csr_equal(oracle.landmark_graph(sp, c, 0.08), bf)
    assert lost > 0
