"""Plans (ct_plan_*): a batch of L2 clouds with every buffer allocated once,
run without host read-back -- the leaf stage one persistent launch over a
device work queue of (cloud, group) items -- and replayed from a CUDA graph.
Each run's CSRs must equal the batched and single-cloud queries bit for bit
and the oracle's brute force; a work-queue wait whose producer is withheld
(on the host: the producers publish nothing, no TMA or MMA is involved) must
run out and report CT_ETIMEOUT, leaving the context usable."""
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


def _same(a, b):
    import torch
    assert a.nnz == b.nnz
    assert torch.equal(a.row_ptr, b.row_ptr)
    assert torch.equal(a.col, b.col)
    assert torch.equal(a.dist.view(torch.int32), b.dist.view(torch.int32))


def _clouds(seed):
    rng = np.random.default_rng(seed)
    shapes = [(2500, 3, "u"), (1, 16, "u"), (1800, 16, "g"), (3000, 64, "g"), (1400, 64, "u"),
              (40, 5, "u"), (4000, 3, "g"), (6000, 64, "u")]
    xs, eps = [], []
    for i, (n, d, k) in enumerate(shapes):
        x = I.uniform_cube(n, d, seed=seed * 100 + i) if k == "u" else \
            I.gmm_embedded(n, dim=d, intrinsic=min(d, 6), n_centres=3, seed=seed * 100 + i)
        xs.append(x)
        if n < 2:
            eps.append(0.5)
            continue
        dd = oracle.brute_rows(oracle.Space(points=x), 1e30, [0, 1, 2])["dist"]
        eps.append(float(np.float32(np.quantile(dd, rng.uniform(0.005, 0.04)))))
    return xs, eps


def _trees(xs):
    import torch
    cg = _cg()
    return [cg.ct_build(points=torch.from_numpy(x).cuda(), leaf_size=32) for x in xs]


@pytest.mark.parametrize("use_graph", [True, False])
def test_plan_runs_equal_batched_query_and_oracle(use_graph):
    cg = _cg()
    xs, eps = _clouds(3)
    trees = _trees(xs)
    ref = cg.eps_graph_query_batched(trees, eps)
    plan = cg.ct_plan_create(trees, eps, use_graph=use_graph)
    for run in range(3):            # replays reuse the plan's buffers
        cg.ct_plan_launch(plan)
        outs = cg.ct_plan_result(plan)
        for x, e, o, r in zip(xs, eps, outs, ref):
            _same(o, r)
            if run == 0:
                assert_csr_matches(o.to_numpy(), oracle.brute_force(oracle.Space(points=x), e))
    st = outs[0].stats()
    assert st["leaf_pairs"] == ref[0].stats()["leaf_pairs"] and st["kernel_launches"] >= 0
    for c in ref:
        c.free()
    plan.free()
    for t in trees:
        t.free()


def test_plan_with_predictor_order_and_tuned_items():
    cg = _cg()
    xs, eps = _clouds(4)
    trees = _trees(xs)
    pred = cg.ct_predictor_create(seed=5)
    cg.ct_predictor_fit(pred, trees[3], eps[3], steps=200, seed=6)
    cg.ct_autotune(trees, eps)
    try:
        plan = cg.ct_plan_create(trees, eps, precision=2, use_predictor=True, predictor=pred, margin=0.0)
        cg.ct_plan_launch(plan)
        outs = cg.ct_plan_result(plan)
        for t, e, o in zip(trees, eps, outs):
            single = cg.eps_graph_query(t, e)
            _same(o, single)
            single.free()
        plan.free()
    finally:
        cg.ct_autotune_reset()
    for t in trees:
        t.free()


def test_withheld_producer_times_out_and_context_survives():
    cg = _cg()
    xs, eps = _clouds(5)
    trees = _trees(xs)
    ref = cg.eps_graph_query_batched(trees, eps)
    plan = cg.ct_plan_create(trees, eps, use_graph=True)
    cg.ct_plan_set_wait(plan, withhold_producers=True, max_polls=2000)
    cg.ct_plan_launch(plan)
    with pytest.raises(cg.CtError) as e:
        cg.ct_plan_result(plan)
    assert e.value.status == cg.CT_ETIMEOUT
    # the context is intact: the same graph with the producers released
    cg.ct_plan_set_wait(plan, withhold_producers=False)
    cg.ct_plan_launch(plan)
    outs = cg.ct_plan_result(plan)
    for o, r in zip(outs, ref):
        _same(o, r)
    for c in ref:
        c.free()
    plan.free()
    for t in trees:
        t.free()


def test_plan_rejects_bad_arguments():
    import torch
    cg = _cg()
    x = I.uniform_cube(500, 3, seed=1)
    t = cg.ct_build(points=torch.from_numpy(x).cuda())
    with pytest.raises(cg.CtError) as e:
        cg.ct_plan_create([t], [-1.0])
    assert e.value.status == cg.CT_EINVAL
    with pytest.raises(cg.CtError) as e:
        cg.ct_plan_create([t], [0.1], margin=-1.0)
    assert e.value.status == cg.CT_EINVAL
    data, off = I.dna_strings(n_seeds=2, per_seed=5, seed=1)
    st = cg.ct_build(strings=(torch.from_numpy(data).cuda(), torch.from_numpy(off).cuda()))
    with pytest.raises(cg.CtError) as e:
        cg.ct_plan_create([st], [2.0])
    assert e.value.status == cg.CT_EINVAL
    st.free()
    t.free()


def test_plan_rows_longer_than_the_in_place_sorts():
    """A duplicate class of 5000 points makes rows of 4999 entries, above the
    4096 the in-place sorts take: the plan sorts them by its radix pass."""
    cg = _cg()
    x = I.uniform_cube(9000, 3, seed=11)
    x[:5000] = x[0]
    y = I.gmm_embedded(3000, dim=16, intrinsic=4, n_centres=3, seed=12)
    xs, eps = [x, y], [0.05, 1.0]
    trees = _trees(xs)
    plan = cg.ct_plan_create(trees, eps, use_graph=True)
    for _ in range(2):
        cg.ct_plan_launch(plan)
        outs = cg.ct_plan_result(plan)
        for xx, e, o in zip(xs, eps, outs):
            assert_csr_matches(o.to_numpy(), oracle.brute_force(oracle.Space(points=xx), e))
    assert int((outs[0].row_ptr[1:] - outs[0].row_ptr[:-1]).max()) > 4096
    plan.free()
    for t in trees:
        t.free()
