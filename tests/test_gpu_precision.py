"""Precision form (precision=1): tensor-core filter (fp16 rows), FP32 recheck, FP64
guard band.  Same edge set as the oracle (and as precision 0), bit for bit."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2510_14147_gb300 import inputs as I
from helpers import assert_csr_matches, gpu_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_14147_gb300 import build
    build.build()
    oracle.build()


def test_small_3d_precision1():
    x = I.uniform_cube(2000, 3, seed=0)
    out = gpu_graph(points=x, eps=0.08, precision=1)
    assert_csr_matches(out, oracle.brute_force(oracle.Space(points=x), 0.08))
    assert out["stats"]["recheck_fp32"] >= out["row_ptr"][-1]


@pytest.mark.parametrize("dim,n,zeta,seed", [(2, 2500, 16, 1), (16, 2200, 17, 5), (33, 1800, 32, 6),
                                              (64, 2100, 32, 7), (128, 2300, 32, 8), (130, 1200, 32, 9),
                                              (7, 2000, 1, 11), (12, 1000, 100, 12)])
def test_precision1_dims(dim, n, zeta, seed):
    x = I.gmm_embedded(n, dim=dim, intrinsic=min(dim, 6), n_centres=5, seed=seed) if dim > 3 \
        else I.uniform_cube(n, dim, seed=seed)
    sp = oracle.Space(points=x)
    rng = np.random.default_rng(seed)
    sample = oracle.brute_rows(sp, 1e30, rng.integers(0, n, size=8))["dist"]
    for q in (0.003, 0.05):
        eps = float(np.float32(np.quantile(sample, q)))
        assert_csr_matches(gpu_graph(points=x, eps=eps, leaf_size=zeta, precision=1),
                           oracle.brute_force(sp, eps))


def test_precision1_lattice_ties_and_boundary():
    g = np.arange(8, dtype=np.float32)
    x = np.array(list(itertools.product(g, g, g)), dtype=np.float32)
    sp = oracle.Space(points=x)
    up = float(np.nextafter(np.float32(math.sqrt(2)), np.float32(np.inf)))
    for eps in (1.0, up, float(np.float32(math.sqrt(2)))):
        assert_csr_matches(gpu_graph(points=x, eps=eps, leaf_size=8, precision=1), oracle.brute_force(sp, eps))
    rng = np.random.default_rng(0)
    n, dim, eps = 1200, 24, 0.75
    a = rng.standard_normal((n // 2, dim)).astype(np.float32) * 3
    u = rng.standard_normal((n // 2, dim))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    scale = eps * (1 + rng.choice([-1, 1], n // 2) * 10 ** rng.uniform(-7.5, -3, n // 2))
    x = np.concatenate([a, (a + u * scale[:, None]).astype(np.float32)])
    assert_csr_matches(gpu_graph(points=x, eps=eps, precision=1), oracle.brute_force(oracle.Space(points=x), eps))


def test_precision1_offsets_duplicates_complete():
    base = I.uniform_cube(2500, 16, seed=4).astype(np.float64)
    x = (base + 3000.0).astype(np.float32)
    sp = oracle.Space(points=x)
    sample = oracle.brute_rows(sp, 1e30, [0, 1, 2])["dist"]
    eps = float(np.quantile(sample[sample > 0], 0.02))
    assert_csr_matches(gpu_graph(points=x, eps=eps, precision=1), oracle.brute_force(sp, eps))
    rng = np.random.default_rng(3)
    distinct = rng.random((40, 6)).astype(np.float32)
    x = distinct[rng.integers(0, 40, size=3000)]
    x[:200] = x[0]
    sp = oracle.Space(points=x)
    for eps in (0.0, 0.4):
        assert_csr_matches(gpu_graph(points=x, eps=eps, leaf_size=16, precision=1), oracle.brute_force(sp, eps))
    x = I.uniform_cube(700, 4, seed=1)
    out = gpu_graph(points=x, eps=5.0, precision=1, include_self=True)
    assert out["row_ptr"][-1] == 700 * 700


@pytest.mark.parametrize("key", ["gmm_1m_k500"])
def test_precision1_full_size_sampled(key):
    """1M x 128, eps for ~500 neighbours: sampled rows equal brute force; the
    whole CSR equals the FP32 path's."""
    wl = I.load_workloads()[key]
    x = I.gmm_embedded(wl["n"], dim=wl["dim"], seed=wl["seed"])
    out = gpu_graph(points=x, eps=wl["eps"], precision=1)
    plain = gpu_graph(points=x, eps=wl["eps"], precision=0)
    assert np.array_equal(out["row_ptr"], plain["row_ptr"]) and np.array_equal(out["col"], plain["col"])
    assert np.array_equal(out["dist"], plain["dist"])
    rp, col = out["row_ptr"], out["col"].astype(np.int64)
    n = x.shape[0]
    assert 0.5 * wl["target_degree"] < rp[-1] / n < 2.0 * wl["target_degree"]
    rng = np.random.default_rng(2)
    rows = np.sort(rng.choice(n, size=24, replace=False))
    ref = oracle.brute_rows(oracle.Space(points=x), wl["eps"], rows)
    sub = {"row_ptr": np.concatenate([[0], np.cumsum(rp[rows + 1] - rp[rows])]),
           "col": np.concatenate([col[rp[r]:rp[r + 1]] for r in rows]),
           "dist": np.concatenate([out["dist"][rp[r]:rp[r + 1]] for r in rows])}
    assert_csr_matches(sub, ref)
    assert out["stats"]["recheck_fp32"] < out["stats"]["leaf_pairs"] // 4


@pytest.mark.parametrize("scale", [1e-12, 1.0, 1e12])
def test_precision1_coordinate_scales(scale):
    """The fp16 rows are centred on the column means and scaled by a power of
    two chosen from the root radius and eps: tiny and huge coordinates give
    the oracle's graph."""
    base = I.gmm_embedded(1500, dim=40, intrinsic=5, n_centres=3, seed=21).astype(np.float64)
    x = (base * scale + 7.0 * scale).astype(np.float32)
    sp = oracle.Space(points=x)
    sample = oracle.brute_rows(sp, 1e30, [0, 1, 2])["dist"]
    eps = float(np.float32(np.quantile(sample[sample > 0], 0.03)))
    assert_csr_matches(gpu_graph(points=x, eps=eps, precision=1), oracle.brute_force(sp, eps))


def test_precision1_wide_extent():
    """Points spread far beyond eps from the column means (the fp16 filter's
    slack grows with |x - m| / eps): the filter keeps more pairs, the graph is
    still the oracle's."""
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.uniform(-2000, 2000, (1500, 32)),
                        rng.standard_normal((1500, 32)) * 0.05 + 1500.0]).astype(np.float32)
    sp = oracle.Space(points=x)
    for eps in (0.4, 2.0):
        out = gpu_graph(points=x, eps=eps, precision=1)
        assert_csr_matches(out, oracle.brute_force(sp, eps))
        assert out["row_ptr"][-1] > 0
