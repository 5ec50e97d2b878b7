"""Parity at the benchmark's own sizes, for the forms the benchmark times.

- 1M x 128 mixture, eps for ~70 neighbours: the timed form (tensor-core
  filter, learned one-pass emit, upper triangle) equals the plain FP32
  two-pass query over the whole CSR, bit for bit, and the oracle's brute
  force (the Sec. III definition) on 512 random rows plus every row that
  holds a pair decided by the FP64 sum (the pairs nearest eps, recorded by
  the library's diagnostic hook).
- 50,000 DNA strings, edit distance 8: the timed form equals the plain one
  and sampled rows equal the oracle's banded brute force; the graph is
  symmetric.
- the 64 clouds: every cloud's CSR from the batched timed form equals the
  plain form's and sampled rows of every cloud equal the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2510_14147_gb300 import inputs as I

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


def _rows_match(csr, rows, ref, rtol=1e-6, integer=False):
    rp = csr.row_ptr.cpu().numpy()
    col = csr.col
    dist = csr.dist
    for k, r in enumerate(rows):
        a, b = int(rp[r]), int(rp[r + 1])
        c = col[a:b].cpu().numpy().astype(np.int64)
        d = dist[a:b].cpu().numpy().astype(np.float64)
        ra, rb = int(ref["row_ptr"][k]), int(ref["row_ptr"][k + 1])
        np.testing.assert_array_equal(c, ref["col"][ra:rb], err_msg="row %d" % r)
        if integer:
            np.testing.assert_array_equal(d, ref["dist"][ra:rb])
        else:
            rd = ref["dist"][ra:rb]
            assert np.all(np.abs(d - rd) <= rtol * np.abs(rd)), "row %d dist" % r


def _fit(cg, tree, eps, steps=300):
    p = cg.ct_predictor_create(seed=1)
    cg.ct_predictor_fit(p, tree, eps, steps=steps, seed=2)
    return p


def test_timed_form_at_full_size_gmm_1m_k70():
    import torch
    cg = _cg()
    wl = I.load_workloads()["gmm_1m_k70"]
    x = I.gmm_embedded(wl["n"], dim=wl["dim"], seed=wl["seed"])
    eps = wl["eps"]
    xf = I.gmm_embedded(wl["n"], dim=wl["dim"], seed=wl["seed"] + 1)   # the predictor's own draw
    tf = cg.ct_build(points=torch.from_numpy(xf).cuda())
    pred = _fit(cg, tf, eps)
    tf.free()
    del xf
    t = cg.ct_build(points=torch.from_numpy(x).cuda())
    ref = cg.eps_graph_query(t, eps, precision=0)
    cap = 1 << 16
    rows_dev = torch.zeros(cap, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    cg.ct_debug_guard_rows(rows_dev, count)
    try:
        timed = cg.eps_graph_query(t, eps, precision=1, use_predictor=True, predictor=pred, upper_triangle=True)
    finally:
        cg.ct_debug_guard_rows(None)
    _same(timed, ref)
    st = timed.stats()
    n_guard = int(count.item())
    assert n_guard == 2 * st["guard_fp64"] and 0 < n_guard <= cap
    guard_rows = np.unique(rows_dev[:n_guard].cpu().numpy())
    rng = np.random.default_rng(70)
    assert guard_rows.size <= 4096       # every one of them is checked below
    rows = np.unique(np.concatenate([rng.choice(wl["n"], size=512, replace=False), guard_rows]))
    refo = oracle.brute_rows(oracle.Space(points=x), eps, rows)
    _rows_match(timed, rows, refo)
    timed.free()
    ref.free()
    t.free()


def test_timed_form_at_full_size_dna_50k():
    import torch
    cg = _cg()
    wl = I.load_workloads()["dna_50k"]
    data, off = I.dna_strings(n_seeds=wl["n_seeds"], per_seed=wl["per_seed"], seed_len=wl["seed_len"],
                              seed=wl["seed"])
    t = cg.ct_build(strings=(torch.from_numpy(data).cuda(), torch.from_numpy(off).cuda()))
    pred = _fit(cg, t, wl["eps"], steps=200)
    ref = cg.eps_graph_query(t, wl["eps"])
    timed = cg.eps_graph_query(t, wl["eps"], use_predictor=True, predictor=pred, upper_triangle=True)
    _same(timed, ref)
    n = off.size - 1
    rows = np.sort(np.random.default_rng(50).choice(n, size=300, replace=False))
    refo = oracle.brute_rows(oracle.Space(strings=(data, off)), wl["eps"], rows)
    _rows_match(timed, rows, refo, integer=True)
    assert oracle.csr_symmetric({"row_ptr": timed.row_ptr.cpu().numpy(), "col": timed.col.cpu().numpy()})
    timed.free()
    ref.free()
    t.free()


def test_timed_form_every_cloud_of_clouds_64():
    import torch
    cg = _cg()
    specs = I.load_workloads()["clouds_64"]["specs"]
    xs = [I.cloud_points(sp) for sp in specs]
    eps = [sp["eps"] for sp in specs]
    trees = [cg.ct_build(points=torch.from_numpy(x).cuda()) for x in xs]
    pred = _fit(cg, trees[1], eps[1], steps=200)
    ref = cg.eps_graph_query_batched(trees, eps, precision=0)
    timed = cg.eps_graph_query_batched(trees, eps, precision=1, use_predictor=True, predictor=pred,
                                       upper_triangle=True)
    rng = np.random.default_rng(64)
    for x, e, a, b in zip(xs, eps, timed, ref):
        _same(a, b)
        rows = np.sort(rng.choice(x.shape[0], size=12, replace=False))
        _rows_match(a, rows, oracle.brute_rows(oracle.Space(points=x), e, rows))
    for c in timed + ref:
        c.free()
    for t in trees:
        t.free()
