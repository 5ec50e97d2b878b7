"""Learned form: the degree/work predictor's kernels against the FP64
reference (oracle/mlp.py), and the one-pass emit into predicted capacities --
whatever the predictions, the CSR equals the two-pass form's and the oracle's."""
import numpy as np
import pytest

import oracle
from oracle import mlp
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


def _query(t, eps, **kw):
    csr = _cg().eps_graph_query(t, eps, **kw)
    out = csr.to_numpy()
    out["stats"] = csr.stats()
    csr.free()
    return out


def _same(a, b):
    assert np.array_equal(a["row_ptr"], b["row_ptr"])
    assert np.array_equal(a["col"], b["col"])
    assert np.array_equal(a["dist"], b["dist"])


# ------------------------------------------------------------ the perceptron

@pytest.mark.parametrize("n", [1, 63, 64, 1000, 4096])
def test_mlp_loss_and_gradient_match_fp64(n):
    import torch
    rng = np.random.default_rng(n)
    theta = rng.normal(0.0, 0.25, mlp.N_PARAMS)
    x = rng.normal(0.0, 1.0, (n, mlp.N_IN))
    t = rng.normal(0.0, 1.0, (n, mlp.N_OUT))
    loss_ref, g_ref = mlp.loss_grad(theta, x, t)
    loss, g = _cg().ct_mlp_loss_grad(torch.tensor(theta, dtype=torch.float32).cuda(),
                                     torch.tensor(x, dtype=torch.float32).cuda(),
                                     torch.tensor(t, dtype=torch.float32).cuda())
    # inputs rounded to fp32, fp32 sums over at most 64 terms per block
    assert abs(loss - loss_ref) <= 1e-5 * max(1.0, abs(loss_ref))
    g = g.cpu().numpy().astype(np.float64)
    scale = np.abs(g_ref).max()
    assert np.abs(g - g_ref).max() <= 2e-5 * scale + 1e-7


def test_mlp_forward_f16_matches_fp64_of_rounded_weights():
    import torch
    rng = np.random.default_rng(7)
    theta = rng.normal(0.0, 0.25, mlp.N_PARAMS)
    x = rng.normal(0.0, 1.0, (3000, mlp.N_IN)).astype(np.float32)
    y = _cg().ct_mlp_forward_f16(torch.tensor(theta, dtype=torch.float32).cuda(), torch.from_numpy(x).cuda())
    th16 = theta.astype(np.float32).astype(np.float16).astype(np.float64)
    ref, _ = mlp.forward(th16, x.astype(np.float64))
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max())


# ------------------------------------------------------------ features

@pytest.mark.parametrize("dim,eps_q", [(3, 0.02), (16, 0.05)])
def test_features_match_definition(dim, eps_q):
    cg = _cg()
    x = I.uniform_cube(1500, 3, seed=2) if dim == 3 else I.gmm_embedded(1500, dim=dim, intrinsic=5,
                                                                         n_centres=4, seed=3)
    sample = oracle.brute_rows(oracle.Space(points=x), 1e30, [0, 1, 2])["dist"]
    eps = float(np.float32(np.quantile(sample, eps_q)))
    t = _tree(points=x, leaf_size=8)
    f = cg.ct_predictor_features(t, eps).cpu().numpy().astype(np.float64)
    ex = cg.ct_tree_export(t)
    t.free()
    ref = mlp.features(ex, x, eps)
    assert f.shape == ref.shape
    err = np.abs(f - ref)
    assert err.max() <= 1e-4, np.unravel_index(np.argmax(err), err.shape)


# ------------------------------------------------------------ one-pass emit

def _fit(t, eps, steps=300, **kw):
    cg = _cg()
    p = cg.ct_predictor_create(seed=1)
    loss = cg.ct_predictor_fit(p, t, eps, steps=steps, batch=2048, seed=3, **kw)
    assert np.isfinite(loss)
    return p


@pytest.mark.parametrize("kind", ["cube3", "gmm16", "gmm128", "dups"])
def test_learned_equals_two_pass_and_oracle(kind):
    rng = np.random.default_rng(0)
    if kind == "cube3":
        x, eps, zeta = I.uniform_cube(3000, 3, seed=5), 0.08, 32
    elif kind == "gmm16":
        x, zeta = I.gmm_embedded(2500, dim=16, intrinsic=6, n_centres=5, seed=6), 17
        eps = float(np.float32(np.quantile(oracle.brute_rows(oracle.Space(points=x), 1e30, [0, 1])["dist"], 0.04)))
    elif kind == "gmm128":
        x, zeta = I.gmm_embedded(2200, dim=128, intrinsic=8, n_centres=5, seed=7), 32
        eps = float(np.float32(np.quantile(oracle.brute_rows(oracle.Space(points=x), 1e30, [0, 1])["dist"], 0.03)))
    else:
        d = rng.random((40, 6)).astype(np.float32)
        x, eps, zeta = d[rng.integers(0, 40, size=2500)], 0.4, 16
    t = _tree(points=x, leaf_size=zeta)
    p = _fit(t, eps)
    ref = oracle.brute_force(oracle.Space(points=x), eps)
    for prec in (0, 1):
        two = _query(t, eps, precision=prec)
        one = _query(t, eps, precision=prec, use_predictor=True, predictor=p)
        _same(one, two)
        assert_csr_matches(one, ref)
    p.free()
    t.free()


def test_learned_forced_overflow_paths():
    """Capacities of zero: every entry goes through the arena; an empty arena:
    every row with an edge is lost and emitted again; a tiny arena: a mix."""
    cg = _cg()
    x = I.gmm_embedded(3000, dim=24, intrinsic=6, n_centres=5, seed=9)
    eps = float(np.float32(np.quantile(oracle.brute_rows(oracle.Space(points=x), 1e30, [0, 1])["dist"], 0.03)))
    t = _tree(points=x)
    p = _fit(t, eps, steps=100)
    two = _query(t, eps)
    deg = np.diff(two["row_ptr"])
    rows_with_edges = int((deg > 0).sum())
    for prec in (0, 1):
        cg.ct_predictor_set_capacity(p, margin=-1.0, pad=0, arena_frac=0.0, arena_min=int(deg.sum()) + 10)
        one = _query(t, eps, precision=prec, use_predictor=True, predictor=p)
        _same(one, two)
        assert one["stats"]["overflow_rows"] == rows_with_edges and one["stats"]["reemit_rows"] == 0
        cg.ct_predictor_set_capacity(p, margin=-1.0, pad=0, arena_frac=0.0, arena_min=0)
        one = _query(t, eps, precision=prec, use_predictor=True, predictor=p)
        _same(one, two)
        assert one["stats"]["reemit_rows"] == rows_with_edges
        cg.ct_predictor_set_capacity(p, margin=-1.0, pad=2, arena_frac=0.0, arena_min=500)
        one = _query(t, eps, precision=prec, use_predictor=True, predictor=p)
        _same(one, two)
        assert 0 < one["stats"]["reemit_rows"] < rows_with_edges
    cg.ct_predictor_set_capacity(p)
    t.free()


def test_learned_edit_distance():
    data, off = I.dna_strings(n_seeds=15, per_seed=100, seed=4)
    t = _tree(strings=(data, off))
    p = _fit(t, 8.0, steps=100)
    two = _query(t, 8.0)
    one = _query(t, 8.0, use_predictor=True, predictor=p)
    _same(one, two)
    _cg().ct_predictor_set_capacity(p, margin=-1.0, pad=0, arena_frac=0.0, arena_min=0)
    one = _query(t, 8.0, use_predictor=True, predictor=p)
    _same(one, two)
    ref = oracle.brute_force(oracle.Space(strings=(data, off)), 8.0)
    assert_csr_matches(one, ref, integer_dist=True)


def test_predictor_generalises_and_roundtrips():
    """Fitted on one draw, the predicted degrees of another draw of the same
    recipe beat the best constant guess; parameters survive get/set."""
    cg = _cg()
    wl = dict(n=60000, dim=32, intrinsic=8, n_centres=12)
    xa = I.gmm_embedded(wl["n"], dim=wl["dim"], intrinsic=wl["intrinsic"], n_centres=wl["n_centres"], seed=21)
    xb = I.gmm_embedded(wl["n"], dim=wl["dim"], intrinsic=wl["intrinsic"], n_centres=wl["n_centres"], seed=22)
    d = oracle.brute_rows(oracle.Space(points=xa), 1e30, [0, 1, 2, 3])["dist"]
    eps = float(np.float32(np.quantile(d, 40.0 / wl["n"])))
    ta, tb = _tree(points=xa), _tree(points=xb)
    p = _fit(ta, eps, steps=1500)
    deg = np.diff(_query(tb, eps)["row_ptr"])
    pred, _ = cg.ct_predictor_predict(p, tb, eps)
    ld = np.log1p(deg)
    err = np.median(np.abs(np.log1p(pred.cpu().numpy()) - ld))
    const = np.median(np.abs(ld - np.median(ld)))
    assert err < 0.8 * const, (err, const)
    params, norm = cg.ct_predictor_get_params(p)
    q = cg.ct_predictor_create(seed=99)
    cg.ct_predictor_set_params(q, params, norm)
    pred2, _ = cg.ct_predictor_predict(q, tb, eps)
    assert np.array_equal(pred.cpu().numpy(), pred2.cpu().numpy())
    one = _query(tb, eps, use_predictor=True, predictor=q)
    assert np.array_equal(np.diff(one["row_ptr"]), deg)
    assert one["stats"]["overflow_rows"] < 0.5 * wl["n"]
    for h in (p, q, ta, tb):
        h.free()


def test_learned_form_gains_over_two_pass():
    """What the trained network buys: the one-pass emit evaluates no pair a
    second time (the two-pass emit re-evaluates every edge-bearing block),
    re-emits no row, and ordering the walks by predicted length keeps the
    edge set."""
    cg = _cg()
    x = I.gmm_embedded(200000, dim=64, intrinsic=8, n_centres=40, seed=31)
    xf = I.gmm_embedded(200000, dim=64, intrinsic=8, n_centres=40, seed=32)
    d = oracle.brute_rows(oracle.Space(points=x), 1e30, [0, 1, 2, 3])["dist"]
    eps = float(np.float32(np.quantile(d, 60.0 / 200000)))
    t, tf = _tree(points=x), _tree(points=xf)
    p = _fit(tf, eps, steps=1500)
    two = _query(t, eps)
    one = _query(t, eps, use_predictor=True, predictor=p)
    _same(one, two)
    assert two["stats"]["emit_pairs"] > 0
    assert one["stats"]["emit_pairs"] == 0 and one["stats"]["reemit_rows"] == 0
    cg.ct_predictor_set_order(p, False)
    _same(_query(t, eps, use_predictor=True, predictor=p), two)
    for h in (p, t, tf):
        h.free()


def test_learned_form_is_faster_than_two_pass():
    """The network's gain in time: on a fixed 300k x 64 mixture (eps for about
    60 neighbours, tensor-core filter), the one-pass emit's stages -- the
    count pass writing the edges, the predictor's forward pass and the
    compaction -- take less device time than the two-pass form's count and
    emit passes.  Stage times are CUDA events around each stage's launches
    (the library's stage timer), the median of five alternating runs of
    each form, whose CSRs are equal."""
    cg = _cg()
    x = I.gmm_embedded(300000, dim=64, intrinsic=8, n_centres=60, seed=41)
    xf = I.gmm_embedded(300000, dim=64, intrinsic=8, n_centres=60, seed=42)
    d = oracle.brute_rows(oracle.Space(points=x), 1e30, [0, 1, 2, 3])["dist"]
    eps = float(np.float32(np.quantile(d, 60.0 / 300000)))
    t, tf = _tree(points=x), _tree(points=xf)
    p = _fit(tf, eps, steps=1500)
    one_stages = ("leaf_count_tc", "predict", "compact", "reemit")
    two_stages = ("leaf_count_tc", "leaf_emit")
    times = {True: [], False: []}
    ref = None
    try:
        for rep in range(6):
            for learned in (False, True):
                cg.ct_profile_reset()
                cg.ct_profile_enable(True)
                try:
                    got = _query(t, eps, precision=1, use_predictor=learned, predictor=p if learned else None)
                finally:
                    cg.ct_profile_enable(False)
                prof = cg.ct_profile_read()
                if ref is None:
                    ref = got
                _same(got, ref)
                if rep:                                      # the first run of each form warms up
                    times[learned].append(sum(prof.get(k, (0.0, 0))[0]
                                              for k in (one_stages if learned else two_stages)))
    finally:
        cg.ct_profile_enable(False)
    one, two = float(np.median(times[True])), float(np.median(times[False]))
    assert one < two, "learned %.3f ms, two-pass %.3f ms" % (one, two)
    for h in (p, t, tf):
        h.free()


def test_one_pass_under_a_memory_budget():
    """The one-pass buffers under a memory budget below what the predicted
    capacities ask for: the capacities are scaled down to the budget, entries
    past them go to the overflow arena and rows past the arena are emitted
    again exactly -- the CSR equals the two-pass form's, with the re-emit
    taken when the budget is far too small.  A budget below the arena's
    minimum takes the two-pass emit (the same CSR)."""
    cg = _cg()
    x = I.gmm_embedded(20000, dim=32, intrinsic=6, n_centres=8, seed=51)
    d = oracle.brute_rows(oracle.Space(points=x), 1e30, [0, 1, 2, 3])["dist"]
    eps = float(np.float32(np.quantile(d, 60.0 / 20000)))
    t = _tree(points=x)
    p = _fit(t, eps, steps=300)
    two = _query(t, eps)
    nnz = int(two["row_ptr"][-1])
    arena_min_bytes = 65536 * 16
    try:
        # room for about the whole graph: scaled capacities, the arena takes the rest
        cg.ct_debug_capacity_budget(arena_min_bytes + 12 * nnz)
        one = _query(t, eps, use_predictor=True, predictor=p)
        _same(one, two)
        # room for an eighth of it: most rows lose entries and are emitted again
        cg.ct_debug_capacity_budget(arena_min_bytes + 12 * (nnz // 8))
        one = _query(t, eps, use_predictor=True, predictor=p)
        _same(one, two)
        assert one["stats"]["reemit_rows"] > 0
        # below the arena's minimum: the two-pass emit
        cg.ct_debug_capacity_budget(arena_min_bytes // 2)
        one = _query(t, eps, use_predictor=True, predictor=p)
        _same(one, two)
        assert one["stats"]["emit_pairs"] > 0
    finally:
        cg.ct_debug_capacity_budget(0)
    for h in (p, t):
        h.free()


def test_unfitted_predictor_is_rejected():
    cg = _cg()
    t = _tree(points=I.uniform_cube(100, 3, seed=0))
    p = cg.ct_predictor_create(seed=0)
    with pytest.raises(cg.CtError) as e:
        cg.eps_graph_query(t, 0.1, use_predictor=True, predictor=p)
    assert e.value.status == cg.CT_EINVAL
    p.free()
    t.free()


@pytest.mark.parametrize("key", ["gmm_1m_k70"])
def test_learned_full_size(key):
    """1M x 128 at ~70 neighbours: predictor fitted on another draw of the
    same recipe; the one-pass CSR equals the two-pass CSR."""
    wl = I.load_workloads()[key]
    x = I.gmm_embedded(wl["n"], dim=wl["dim"], seed=wl["seed"])
    xt = I.gmm_embedded(wl["n"], dim=wl["dim"], seed=wl["seed"] + 1)
    t, tt = _tree(points=x), _tree(points=xt)
    p = _fit(tt, wl["eps"], steps=1500)
    tt.free()
    for prec in (0, 1):
        two = _query(t, wl["eps"], precision=prec)
        one = _query(t, wl["eps"], precision=prec, use_predictor=True, predictor=p)
        _same(one, two)
        assert one["stats"]["reemit_rows"] < 0.01 * wl["n"]
    p.free()
    t.free()
