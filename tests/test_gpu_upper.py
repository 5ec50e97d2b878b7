"""The upper-triangle form (ct_query_opts.upper_triangle): a pair of points
from two different query groups is evaluated once, from the group that comes
first in tree order, and written into both rows (the symmetry d(p, q) =
d(q, p) of Sec. III that the paper's ring uses to halve its rounds,
Sec. IV-C).  Its CSR must equal the full query's bit for bit and the
oracle's brute force, in every leaf kernel, emit form and driver, with
about half the leaf pairs."""
import numpy as np
import pytest

import oracle
from paper_2510_14147_gb300 import inputs as I
from helpers import assert_csr_matches

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_14147_gb300 import build
    build.build()
    oracle.build()


def _cg():
    from paper_2510_14147_gb300 import ctgraph as cg
    return cg


def _same(a, b):
    import torch
    assert a.nnz == b.nnz
    assert torch.equal(a.row_ptr, b.row_ptr)
    assert torch.equal(a.col, b.col)
    assert torch.equal(a.dist.view(torch.int32), b.dist.view(torch.int32))


def _eps(x, q, seed=0):
    rng = np.random.default_rng(seed)
    d = oracle.brute_rows(oracle.Space(points=x), 1e30, rng.integers(0, x.shape[0], size=6))["dist"]
    return float(np.float32(np.quantile(d, q)))


@pytest.mark.parametrize("dim,precision", [(3, 0), (16, 1), (64, 1), (128, 0), (130, 0), (96, 2)])
def test_upper_triangle_equals_full_query(dim, precision):
    import torch
    cg = _cg()
    x = I.uniform_cube(4000, dim, seed=dim) if dim <= 3 else \
        I.gmm_embedded(4000, dim=dim, intrinsic=min(dim, 6), n_centres=5, seed=dim)
    x[100:150] = x[3]                     # a duplicate class above the leaf size (a cut leaf block)
    t = cg.ct_build(points=torch.from_numpy(x).cuda())
    sp = oracle.Space(points=x)
    for q in (0.005, 0.05):
        eps = _eps(x, q, dim)
        for inc in (False, True):
            full = cg.eps_graph_query(t, eps, precision=precision, include_self=inc)
            half = cg.eps_graph_query(t, eps, precision=precision, include_self=inc, upper_triangle=True)
            _same(half, full)
            if not inc:
                assert_csr_matches(half.to_numpy(), oracle.brute_force(sp, eps))
                pf, ph = full.stats()["leaf_pairs"], half.stats()["leaf_pairs"]
                assert ph < 0.75 * pf, (ph, pf)
            full.free()
            half.free()
    t.free()


def test_upper_triangle_learned_one_pass_and_forced_overflow():
    """The one-pass emit writes mirrored entries into other rows' capacities;
    with no capacity and no arena every row is emitted again, and a row can
    only be rebuilt with the mirrored entries of other groups' queries."""
    import torch
    cg = _cg()
    x = I.gmm_embedded(3000, dim=24, intrinsic=6, n_centres=5, seed=9)
    eps = _eps(x, 0.03, 9)
    t = cg.ct_build(points=torch.from_numpy(x).cuda())
    p = cg.ct_predictor_create(seed=3)
    cg.ct_predictor_fit(p, t, eps, steps=100, seed=4)
    full = cg.eps_graph_query(t, eps)
    deg = np.diff(full.row_ptr.cpu().numpy())
    for prec in (0, 1):
        for cap in (dict(), dict(margin=-1.0, pad=0, arena_frac=0.0, arena_min=int(deg.sum()) + 10),
                    dict(margin=-1.0, pad=0, arena_frac=0.0, arena_min=0),
                    dict(margin=-1.0, pad=2, arena_frac=0.0, arena_min=500)):
            cg.ct_predictor_set_capacity(p, **cap)
            one = cg.eps_graph_query(t, eps, precision=prec, use_predictor=True, predictor=p, upper_triangle=True)
            _same(one, full)
            one.free()
    cg.ct_predictor_set_capacity(p)
    full.free()
    t.free()


def test_upper_triangle_integer_metrics():
    import torch
    cg = _cg()
    data, off = I.dna_strings(n_seeds=12, per_seed=60, seed=5)
    ts = cg.ct_build(strings=(torch.from_numpy(data).cuda(), torch.from_numpy(off).cuda()))
    rows = I.binary_codes(3000, 256, n_centres=30, flip=0.05, seed=6)
    tb = cg.ct_build(bits=(torch.from_numpy(rows).cuda(), 256))
    pred = cg.ct_predictor_create(seed=2)
    cg.ct_predictor_fit(pred, tb, 20, steps=100, seed=3)
    for t, eps, sp in ((ts, 8, oracle.Space(strings=(data, off))), (tb, 20, oracle.Space(bits=(rows, 256)))):
        full = cg.eps_graph_query(t, eps)
        half = cg.eps_graph_query(t, eps, upper_triangle=True)
        _same(half, full)
        assert_csr_matches(half.to_numpy(), oracle.brute_force(sp, eps), integer_dist=True)
        assert half.stats()["leaf_pairs"] < 0.75 * full.stats()["leaf_pairs"]
        half.free()
        if t is tb:
            cg.ct_predictor_set_capacity(pred, margin=-1.0, pad=0, arena_frac=0.0, arena_min=0)
            one = cg.eps_graph_query(t, eps, use_predictor=True, predictor=pred, upper_triangle=True)
            _same(one, full)
            one.free()
        full.free()
    ts.free()
    tb.free()


def test_upper_triangle_batched_sweep_and_plan():
    import torch
    cg = _cg()
    xs = [I.uniform_cube(2500, 3, seed=1), I.gmm_embedded(3000, dim=16, intrinsic=4, n_centres=3, seed=2),
          I.gmm_embedded(2000, dim=64, intrinsic=6, n_centres=3, seed=3)]
    eps = [_eps(x, 0.02, i) for i, x in enumerate(xs)]
    trees = [cg.ct_build(points=torch.from_numpy(x).cuda()) for x in xs]
    full = cg.eps_graph_query_batched(trees, eps)
    half = cg.eps_graph_query_batched(trees, eps, upper_triangle=True, precision=1)
    for a, b in zip(half, full):
        _same(a, b)
    sw = cg.eps_graph_query_sweep(trees[1], [eps[1], eps[1] * 0.7], upper_triangle=True)
    ref = cg.eps_graph_query(trees[1], eps[1] * 0.7)
    _same(sw[1], ref)
    plan = cg.ct_plan_create(trees, eps, upper_triangle=True)
    cg.ct_plan_launch(plan)
    outs = cg.ct_plan_result(plan)
    for a, b in zip(outs, full):
        _same(a, b)
    plan.free()
    for c in full + half + sw + [ref]:
        c.free()
    for t in trees:
        t.free()
