"""Several radii over one tree (eps_graph_query_sweep) and trees written to a
file and read back (ct_tree_save / ct_tree_load), through the C-ABI.

The paper queries each dataset at three radii (Table I).  The sweep derives
every smaller radius from the CSR of the next larger one; its outputs must be
the CSRs eps_graph_query returns at each radius, bit for bit, and the oracle's
brute force (the Sec. III definition) entry for entry."""
import os

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


def _radii(x, qs, seed):
    sp = oracle.Space(points=x)
    rng = np.random.default_rng(seed)
    d = oracle.brute_rows(sp, 1e30, rng.integers(0, x.shape[0], size=8))["dist"]
    return [float(np.float32(np.quantile(d, q))) for q in qs]


@pytest.mark.parametrize("dim,precision,learned", [(3, 0, False), (16, 1, False), (128, 1, True),
                                                   (130, 0, False), (64, 2, False)])
def test_sweep_equals_independent_queries_and_oracle(dim, precision, learned):
    import torch
    cg = _cg()
    n = 3000
    x = I.uniform_cube(n, dim, seed=dim) if dim <= 3 else \
        I.gmm_embedded(n, dim=dim, intrinsic=min(dim, 6), n_centres=6, seed=dim)
    r = _radii(x, (0.004, 0.02, 0.06), dim)
    # two radii one part in 10^5 apart: their guard bands overlap almost whole
    eps = [r[1], r[2], r[0], r[1] * (1 + 1e-5), 0.0]
    tree = cg.ct_build(points=torch.from_numpy(x).cuda())
    pred = None
    if learned:
        pred = cg.ct_predictor_create(seed=3)
        cg.ct_predictor_fit(pred, tree, r[2], steps=200, seed=4)
    sw = cg.eps_graph_query_sweep(tree, eps, precision=precision, use_predictor=learned, predictor=pred)
    sp = oracle.Space(points=x)
    for e, c in zip(eps, sw):
        ind = cg.eps_graph_query(tree, e, precision=precision, use_predictor=learned, predictor=pred)
        _same(c, ind)
        ind.free()
        assert_csr_matches(c.to_numpy(), oracle.brute_force(sp, e))
        c.free()
    tree.free()


def test_sweep_include_self_duplicates_and_order():
    import torch
    cg = _cg()
    x = I.uniform_cube(1500, 4, seed=5)
    x[100:160] = x[7]      # a duplicate class above the leaf size
    eps = [0.05, 0.0, 0.2, 0.1]
    tree = cg.ct_build(points=torch.from_numpy(x).cuda())
    sw = cg.eps_graph_query_sweep(tree, eps, include_self=True)
    sp = oracle.Space(points=x)
    for e, c in zip(eps, sw):
        assert_csr_matches(c.to_numpy(), oracle.brute_force(sp, e, include_self=True))
        c.free()
    assert cg.eps_graph_query_sweep(tree, []) == []
    tree.free()


def test_sweep_edit_distance():
    import torch
    cg = _cg()
    data, off = I.dna_strings(n_seeds=8, per_seed=40, seed=6)
    tree = cg.ct_build(strings=(torch.from_numpy(data).cuda(), torch.from_numpy(off).cuda()))
    eps = [3, 8, 5.5, 0]
    sw = cg.eps_graph_query_sweep(tree, eps)
    sp = oracle.Space(strings=(data, off))
    for e, c in zip(eps, sw):
        ind = cg.eps_graph_query(tree, e)
        _same(c, ind)
        ind.free()
        assert_csr_matches(c.to_numpy(), oracle.brute_force(sp, e), integer_dist=True)
        c.free()
    tree.free()


def test_tree_save_load_round_trip(tmp_path):
    import torch
    cg = _cg()
    x = I.gmm_embedded(5000, dim=32, intrinsic=6, n_centres=5, seed=8)
    eps = _radii(x, (0.02,), 8)[0]
    tree = cg.ct_build(points=torch.from_numpy(x).cuda())
    path = str(tmp_path / "gmm.cttree")
    cg.ct_tree_save(tree, path)
    t2 = cg.ct_tree_load(path)
    a, b = cg.ct_tree_export(tree), cg.ct_tree_export(t2)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    for prec in (0, 1):
        c1, c2 = cg.eps_graph_query(tree, eps, precision=prec), cg.eps_graph_query(t2, eps, precision=prec)
        _same(c1, c2)
        c1.free()
        c2.free()
    t2.free()
    # strings
    data, off = I.dna_strings(n_seeds=4, per_seed=30, seed=9)
    st = cg.ct_build(strings=(torch.from_numpy(data).cuda(), torch.from_numpy(off).cuda()))
    spath = str(tmp_path / "dna.cttree")
    cg.ct_tree_save(st, spath)
    st2 = cg.ct_tree_load(spath)
    c1, c2 = cg.eps_graph_query(st, 6), cg.eps_graph_query(st2, 6)
    _same(c1, c2)
    c1.free()
    c2.free()
    st.free()
    st2.free()
    # an empty tree
    et = cg.ct_build(points=torch.zeros((0, 3), dtype=torch.float32, device="cuda"))
    epath = str(tmp_path / "empty.cttree")
    cg.ct_tree_save(et, epath)
    et2 = cg.ct_tree_load(epath)
    c = cg.eps_graph_query(et2, 1.0)
    assert c.nnz == 0 and c.row_ptr.cpu().tolist() == [0]
    c.free()
    et.free()
    et2.free()
    tree.free()


def test_tree_load_rejects_damaged_files(tmp_path):
    import torch
    cg = _cg()
    x = I.uniform_cube(800, 3, seed=10)
    tree = cg.ct_build(points=torch.from_numpy(x).cuda())
    path = str(tmp_path / "t.cttree")
    cg.ct_tree_save(tree, path)
    tree.free()
    raw = open(path, "rb").read()
    cases = {"flipped": raw[:200] + bytes([raw[200] ^ 1]) + raw[201:],
             "truncated": raw[:-9], "trailing": raw + b"\0", "magic": b"XX" + raw[2:]}
    for name, blob in cases.items():
        p = str(tmp_path / (name + ".cttree"))
        with open(p, "wb") as f:
            f.write(blob)
        with pytest.raises(cg.CtError) as e:
            cg.ct_tree_load(p)
        assert e.value.status == cg.CT_EINVAL, name
    with pytest.raises(cg.CtError) as e:
        cg.ct_tree_load(str(tmp_path / "missing.cttree"))
    assert e.value.status == cg.CT_EINVAL
    assert not os.path.exists(str(tmp_path / "missing.cttree"))
