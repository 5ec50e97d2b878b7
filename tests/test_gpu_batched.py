"""Many-cloud batch (eps_graph_query_batched): clouds of different sizes,
dimensions and radii share every launch; each output equals the single-cloud
query's and the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2510_14147_gb300 import inputs as I
from helpers import assert_csr_matches

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_14147_gb300 import build
    build.build()
    oracle.build()


def _cg():
    from paper_2510_14147_gb300 import ctgraph as cg
    return cg


def _tree(points=None, strings=None, leaf_size=32):
    import torch
    cg = _cg()
    if points is not None:
        return cg.ct_build(points=torch.from_numpy(np.ascontiguousarray(points, np.float32)).cuda(),
                           leaf_size=leaf_size)
    data, off = strings
    return cg.ct_build(strings=(torch.from_numpy(np.ascontiguousarray(data, np.uint8)).cuda(),
                                torch.from_numpy(np.ascontiguousarray(off, np.int64)).cuda()),
                       leaf_size=leaf_size)


def _np(csr):
    out = csr.to_numpy()
    out["stats"] = csr.stats()
    return out


def _eps_for(x, q):
    if x.shape[0] < 2:
        return 0.5
    d = oracle.brute_rows(oracle.Space(points=x), 1e30, [0, min(1, x.shape[0] - 1)])["dist"]
    return float(np.float32(np.quantile(d[d > 0], q))) if (d > 0).any() else 0.5


def _clouds(seed):
    rng = np.random.default_rng(seed)
    shapes = [(1500, 3, "u"), (0, 3, "u"), (1, 16, "u"), (2, 16, "u"), (900, 16, "g"), (1200, 64, "g"),
              (700, 64, "u"), (33, 5, "u"), (2000, 3, "g"), (64, 12, "g")]
    xs, eps = [], []
    for i, (n, d, k) in enumerate(shapes):
        if n == 0:
            x = np.zeros((0, d), np.float32)
        elif k == "u":
            x = I.uniform_cube(n, d, seed=seed * 100 + i)
        else:
            x = I.gmm_embedded(n, dim=d, intrinsic=min(d, 6), n_centres=3, seed=seed * 100 + i)
        xs.append(x)
        eps.append(_eps_for(x, rng.uniform(0.005, 0.05)))
    return xs, eps


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_single_queries_and_oracle(precision):
    cg = _cg()
    xs, eps = _clouds(1)
    trees = [_tree(points=x, leaf_size=16) for x in xs]
    outs = cg.eps_graph_query_batched(trees, eps, precision=precision)
    for x, t, e, o in zip(xs, trees, eps, outs):
        got = _np(o)
        single = cg.eps_graph_query(t, e, precision=precision).to_numpy()
        for k in ("row_ptr", "col", "dist"):
            assert np.array_equal(got[k], single[k]), k
        assert_csr_matches(got, oracle.brute_force(oracle.Space(points=x), e))
    # release in scrambled order: the views stay valid until the last release
    last = outs[3]
    keep = last.to_numpy()
    for i in (7, 0, 9, 2, 5, 1, 8, 6, 4):
        outs[i].free()
    again = last.to_numpy()
    for k in ("row_ptr", "col", "dist"):
        assert np.array_equal(keep[k], again[k])
    last.free()
    for t in trees:
        t.free()


def test_batch_above_64_clouds_and_wide_rows():
    """70 clouds (two batches); one cloud of 130-D rows sends its batch to the
    FP32 tiles in precision 1."""
    cg = _cg()
    xs, eps = [], []
    for i in range(70):
        d = 130 if i == 5 else (3 if i % 2 else 8)
        x = I.uniform_cube(40 + 13 * i, d, seed=500 + i)
        xs.append(x)
        eps.append(_eps_for(x, 0.05))
    trees = [_tree(points=x) for x in xs]
    for precision in (0, 1):
        outs = cg.eps_graph_query_batched(trees, eps, precision=precision)
        for x, e, o in zip(xs, eps, outs):
            assert_csr_matches(_np(o), oracle.brute_force(oracle.Space(points=x), e))
            o.free()
    for t in trees:
        t.free()


def test_batch_mixes_edit_distance_clouds():
    cg = _cg()
    data, off = I.dna_strings(n_seeds=6, per_seed=50, seed=9)
    x0 = I.uniform_cube(800, 3, seed=3)
    x1 = I.gmm_embedded(600, dim=16, intrinsic=5, n_centres=2, seed=4)
    trees = [_tree(points=x0), _tree(strings=(data, off)), _tree(points=x1)]
    eps = [0.07, 8.0, _eps_for(x1, 0.02)]
    outs = cg.eps_graph_query_batched(trees, eps)
    assert_csr_matches(_np(outs[0]), oracle.brute_force(oracle.Space(points=x0), eps[0]))
    assert_csr_matches(_np(outs[1]), oracle.brute_force(oracle.Space(strings=(data, off)), 8.0), integer_dist=True)
    assert_csr_matches(_np(outs[2]), oracle.brute_force(oracle.Space(points=x1), eps[2]))
    for o in outs:
        o.free()
    for t in trees:
        t.free()


def test_learned_batch_equals_two_pass():
    cg = _cg()
    xs, eps = _clouds(2)
    trees = [_tree(points=x, leaf_size=16) for x in xs]
    p = cg.ct_predictor_create(seed=1)
    cg.ct_predictor_fit(p, trees[8], eps[8], steps=200, batch=1024, seed=2)
    for precision in (0, 1):
        two = cg.eps_graph_query_batched(trees, eps, precision=precision)
        one = cg.eps_graph_query_batched(trees, eps, precision=precision, use_predictor=True, predictor=p)
        for a, b in zip(one, two):
            na, nb = a.to_numpy(), b.to_numpy()
            for k in ("row_ptr", "col", "dist"):
                assert np.array_equal(na[k], nb[k]), k
        for o in one + two:
            o.free()
    p.free()
    for t in trees:
        t.free()


def test_many_cloud_workload_sample():
    """The four smallest clouds of the 64-cloud workload, with their
    calibrated eps, against brute force."""
    cg = _cg()
    specs = sorted(I.load_workloads()["clouds_64"]["specs"], key=lambda sp: sp["n"])[:4]
    xs = [I.cloud_points(sp) for sp in specs]
    trees = [_tree(points=x) for x in xs]
    outs = cg.eps_graph_query_batched(trees, [sp["eps"] for sp in specs], precision=1)
    for x, sp, o in zip(xs, specs, outs):
        got = _np(o)
        assert_csr_matches(got, oracle.brute_force(oracle.Space(points=x), sp["eps"]))
        deg = got["row_ptr"][-1] / x.shape[0]
        assert 0.5 * sp["target_degree"] < deg < 2.0 * sp["target_degree"]
        o.free()
    for t in trees:
        t.free()


def test_autotuned_precision_keeps_the_output():
    """precision 2 before and after tuning, on a batch spanning four row-length
    classes, equals precision 0 cloud by cloud."""
    cg = _cg()
    cg.ct_autotune_reset()
    xs, eps = _clouds(3)
    trees = [_tree(points=x, leaf_size=16) for x in xs]
    ref = [o.to_numpy() for o in cg.eps_graph_query_batched(trees, eps, precision=0)]
    before = cg.eps_graph_query_batched(trees, eps, precision=2)
    choices = cg.ct_autotune(trees, eps)
    assert len(choices) == len(trees) and set(choices) <= {0, 1}
    after = cg.eps_graph_query_batched(trees, eps, precision=2)
    for r, a, b in zip(ref, before, after):
        for out in (a.to_numpy(), b.to_numpy()):
            for k in ("row_ptr", "col", "dist"):
                assert np.array_equal(out[k], r[k]), k
    for o in before + after:
        o.free()
    single = cg.eps_graph_query(trees[0], eps[0], precision=2).to_numpy()
    assert np.array_equal(single["col"], ref[0]["col"])
    cg.ct_autotune_reset()
    for t in trees:
        t.free()
