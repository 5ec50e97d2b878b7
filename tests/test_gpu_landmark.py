"""The landmark form (eps_graph_query_landmark; Sec. IV-D and Lemma 1 on one
GPU): Voronoi cells of random centres, Lemma 1 ghosts, a tree per cell, one
batched query.  Its CSR must equal eps_graph_query's on the whole set bit
for bit, and the oracle's landmark and brute-force graphs."""
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


@pytest.mark.parametrize("dim,m,precision,upper", [(3, 10, 0, False), (16, 60, 1, True), (64, 7, 1, False),
                                                   (128, 60, 0, True), (8, 1, 0, False), (5, 1500, 0, False)])
def test_landmark_equals_query_and_oracle(dim, m, precision, upper):
    import torch
    cg = _cg()
    n = 4000 if m < 1500 else 1500
    x = I.uniform_cube(n, dim, seed=dim) if dim <= 3 else \
        I.gmm_embedded(n, dim=dim, intrinsic=min(dim, 6), n_centres=6, seed=dim)
    x[10:60] = x[5]                                        # duplicates across the cells
    xd = torch.from_numpy(x).cuda()
    sp = oracle.Space(points=x)
    eps = float(np.float32(np.quantile(oracle.brute_rows(sp, 1e30, [0, 1, 2])["dist"], 0.02)))
    centres = np.random.default_rng(m).choice(n, size=m, replace=False)
    t = cg.ct_build(points=xd)
    ref = cg.eps_graph_query(t, eps, precision=precision, upper_triangle=upper)
    got, info = cg.eps_graph_query_landmark(centres, eps, points=xd, precision=precision, upper_triangle=upper)
    _same(got, ref)
    assert info["cells"] == m and info["members"] == n + info["ghosts"] and info["ghosts"] >= 0
    out = got.to_numpy()
    assert_csr_matches(out, oracle.brute_force(sp, eps))
    assert oracle.csr_equal(out, oracle.landmark_graph(sp, centres, eps))
    got.free()
    ref.free()
    t.free()


def test_landmark_hamming_include_self_and_learned():
    import torch
    cg = _cg()
    rows = I.binary_codes(3000, 256, n_centres=20, flip=0.06, seed=4)
    rd = torch.from_numpy(rows).cuda()
    sp = oracle.Space(bits=(rows, 256))
    centres = np.random.default_rng(5).choice(3000, size=30, replace=False)
    for inc in (False, True):
        got, info = cg.eps_graph_query_landmark(centres, 20, bits=(rd, 256), include_self=inc)
        assert_csr_matches(got.to_numpy(), oracle.brute_force(sp, 20, include_self=inc), integer_dist=True)
        got.free()
    x = I.gmm_embedded(3000, dim=32, intrinsic=6, n_centres=4, seed=6)
    xd = torch.from_numpy(x).cuda()
    eps = float(np.float32(np.quantile(oracle.brute_rows(oracle.Space(points=x), 1e30, [0])["dist"], 0.03)))
    t = cg.ct_build(points=xd)
    pred = cg.ct_predictor_create(seed=1)
    cg.ct_predictor_fit(pred, t, eps, steps=100, seed=2)
    ref = cg.eps_graph_query(t, eps)
    got, _ = cg.eps_graph_query_landmark(np.arange(0, 3000, 100), eps, points=xd, use_predictor=True,
                                         predictor=pred, upper_triangle=True)
    _same(got, ref)
    got.free()
    ref.free()
    t.free()


def test_landmark_rejects_bad_arguments():
    import torch
    cg = _cg()
    xd = torch.from_numpy(I.uniform_cube(100, 3, seed=1)).cuda()
    for centres in ([], [100], [-1, 3]):
        with pytest.raises(cg.CtError) as e:
            cg.eps_graph_query_landmark(np.array(centres, np.int64), 0.1, points=xd)
        assert e.value.status == cg.CT_EINVAL
    empty = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    got, info = cg.eps_graph_query_landmark([0], 0.1, points=empty)      # n = 0: the empty graph
    assert got.nnz == 0 and got.row_ptr.cpu().tolist() == [0]
    got.free()


def test_landmark_with_stage_timing_enabled():
    """The landmark form's stages contain whole builds and queries (scopes
    that nest): timing them must work and leave the results unchanged."""
    import torch
    cg = _cg()
    x = I.gmm_embedded(3000, dim=16, intrinsic=4, n_centres=3, seed=8)
    xd = torch.from_numpy(x).cuda()
    eps = float(np.float32(np.quantile(oracle.brute_rows(oracle.Space(points=x), 1e30, [0])["dist"], 0.03)))
    cg.ct_profile_reset()
    cg.ct_profile_enable(True)
    try:
        for _ in range(2):
            got, _ = cg.eps_graph_query_landmark(np.arange(0, 3000, 150), eps, points=xd)
            got.free()
    finally:
        cg.ct_profile_enable(False)
    prof = cg.ct_profile_read()
    assert prof["landmark_build"][1] == 2 and prof["landmark_query"][1] == 2 and prof["build"][1] == 40
    t = cg.ct_build(points=xd)
    ref = cg.eps_graph_query(t, eps)
    got, _ = cg.eps_graph_query_landmark(np.arange(0, 3000, 150), eps, points=xd)
    _same(got, ref)
    got.free()
    ref.free()
    t.free()
